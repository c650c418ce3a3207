// sort.cu -- SortByKeys (Algorithm 1): stable LSD radix sort of u32 keys with
// u32 values, 8-bit digits, three kernels per digit and no device-side waits:
//
//   k_radix_hist     per sort tile (kSortTile keys): the 256-bin digit
//                    histogram, stored per tile and summed into its group of
//                    kGroupTiles tiles;
//   k_radix_groups   one block: exclusive scan of the group sums down the tiles
//                    (per digit) and of the digit totals (the digit bases);
//   k_radix_scatter  per sort tile: stable warp-level ranking (peer masks from a
//                    per-warp shared atomicOr of lane bits), the tile's offset per digit =
//                    digit base + group prefix + sum over the earlier tiles of
//                    its group, reordering by digit in shared memory and
//                    contiguous writes of each digit run.
//
// The key count stays on the device: both per-tile kernels launch one block per
// tile of the workspace capacity and the blocks past the count exit at once.
#include <algorithm>

#include "geer_internal.cuh"

namespace geer {
namespace {

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t key_count(const uint32_t *misc, int count_slot, int check_capacity) {
    if (check_capacity && (misc[kMiscStatus] & kStatusCapacity)) return 0u;
    return misc[count_slot];
}

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t *__restrict__ kin,
                                                             const uint32_t *__restrict__ misc, int count_slot,
                                                             int check_capacity, int shift,
                                                             uint32_t *__restrict__ tile_hist,
                                                             uint32_t *__restrict__ group_sum) {
    constexpr int W = kSortThreads / 32;
    __shared__ uint32_t s_h[W][kRadix];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n = key_count(misc, count_slot, check_capacity);
    const uint32_t tile = blockIdx.x;
    if ((uint64_t)tile * kSortTile >= n) return;
    for (int i = tid; i < W * kRadix; i += kSortThreads) (&s_h[0][0])[i] = 0u;
    const uint64_t base = (uint64_t)tile * kSortTile + (uint64_t)warp * 32 * kSortItems + lane;
    uint32_t key[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const uint64_t i = base + (uint64_t)k * 32;
        key[k] = i < n ? kin[i] : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSortItems; ++k)
        if (base + (uint64_t)k * 32 < n) atomicAdd(&s_h[warp][(key[k] >> shift) & 0xffu], 1u);
    __syncthreads();
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) c += s_h[w][tid];
    tile_hist[(uint64_t)tile * kRadix + tid] = c;
    if (c) atomicAdd(&group_sum[(uint64_t)(tile / kGroupTiles) * kRadix + tid], c);
}

// 1024 threads = 4 quarters x 256 digits: exclusive prefix of the group sums
// down the groups (into group_excl; the sums are cleared for the next pass),
// then the digit bases (exclusive scan of the digit totals).
__global__ void __launch_bounds__(1024) k_radix_groups(const uint32_t *__restrict__ misc, int count_slot,
                                                       int check_capacity, uint32_t *__restrict__ group_sum,
                                                       uint32_t *__restrict__ group_excl,
                                                       uint32_t *__restrict__ digit_base) {
    __shared__ uint32_t s_q[4][kRadix];
    __shared__ uint32_t s_wsum[kRadix / 32];
    const int d = threadIdx.x & (kRadix - 1), q = threadIdx.x >> 8;
    const uint32_t n = key_count(misc, count_slot, check_capacity);
    const uint32_t ngroups = (n + kSortTile * kGroupTiles - 1) / (kSortTile * kGroupTiles);
    const uint32_t per = (ngroups + 3) / 4;
    const uint32_t g0 = min(ngroups, q * per), g1 = min(ngroups, g0 + per);
    uint32_t sum = 0;
    for (uint32_t g = g0; g < g1; g += 8) {
        uint32_t v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = g + u < g1 ? group_sum[(uint64_t)(g + u) * kRadix + d] : 0u;
#pragma unroll
        for (int u = 0; u < 8; ++u) sum += v[u];
    }
    s_q[q][d] = sum;
    __syncthreads();
    uint32_t run = 0;
    for (int k = 0; k < q; ++k) run += s_q[k][d];
    for (uint32_t g = g0; g < g1; g += 8) {
        uint32_t v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = g + u < g1 ? group_sum[(uint64_t)(g + u) * kRadix + d] : 0u;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (g + u < g1) {
                group_excl[(uint64_t)(g + u) * kRadix + d] = run;
                group_sum[(uint64_t)(g + u) * kRadix + d] = 0u;
            }
            run += v[u];
        }
    }
    __syncthreads();
    if (q == 0) {
        const int lane = d & 31, warp = d >> 5;
        const uint32_t tot = s_q[0][d] + s_q[1][d] + s_q[2][d] + s_q[3][d];
        uint32_t v = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) s_wsum[warp] = v;
        asm volatile("bar.sync 1, 256;");
        uint32_t pre = 0;
#pragma unroll
        for (int w = 0; w < kRadix / 32; ++w) pre += w < warp ? s_wsum[w] : 0u;
        digit_base[d] = pre + v - tot;
    }
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, const uint32_t *__restrict__ misc, int count_slot, int check_capacity, int shift,
    const uint32_t *__restrict__ tile_hist, const uint32_t *__restrict__ group_excl,
    const uint32_t *__restrict__ digit_base) {
    constexpr int W = kSortThreads / 32;
    __shared__ uint32_t s_whist[W][kRadix];
    __shared__ uint32_t s_match[W][kRadix];  // lane masks per digit, zero between ranking steps
    __shared__ uint32_t s_lbase[kRadix];  // start of each digit inside the tile
    __shared__ uint32_t s_out[kRadix];    // global position of the tile's first key of each digit
    __shared__ uint32_t s_wsum[W];
    __shared__ uint32_t s_key[kSortTile];
    __shared__ uint32_t s_val[kSortTile];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n = key_count(misc, count_slot, check_capacity);
    const uint32_t tile = blockIdx.x;
    if ((uint64_t)tile * kSortTile >= n) return;
    const uint32_t base_d = digit_base[tid];
    for (int i = tid; i < W * kRadix; i += kSortThreads) (&s_match[0][0])[i] = 0u;
    {
        for (int i = tid; i < W * kRadix; i += kSortThreads) (&s_whist[0][0])[i] = 0u;
        // this tile's global offset for digit tid
        const uint32_t g0 = (tile / kGroupTiles) * kGroupTiles;
        uint32_t off = base_d + group_excl[(uint64_t)(tile / kGroupTiles) * kRadix + tid];
        uint32_t part[kGroupTiles - 1];
#pragma unroll
        for (int r = 0; r < kGroupTiles - 1; ++r)
            part[r] = g0 + r < tile ? tile_hist[(uint64_t)(g0 + r) * kRadix + tid] : 0u;
#pragma unroll
        for (int r = 0; r < kGroupTiles - 1; ++r) off += part[r];
        s_out[tid] = off;
        __syncthreads();

        uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
        const uint64_t base = (uint64_t)tile * kSortTile + (uint64_t)warp * 32 * kSortItems + lane;
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            const uint64_t i = base + (uint64_t)k * 32;
            const bool v = i < n;
            key[k] = v ? kin[i] : 0u;
            val[k] = v ? vin[i] : 0u;
        }
        // stable ranking: warp by warp, item k by item k, lane by lane. The lanes
        // sharing a digit find each other through a per-warp shared mask per
        // digit (atomicOr of the lane bits), cleared again by the group leader.
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            const bool v = base + (uint64_t)k * 32 < n;
            const uint32_t d = (key[k] >> shift) & 0xffu;
            if (v) atomicOr(&s_match[warp][d], 1u << lane);
            __syncwarp();
            const uint32_t peers = v ? s_match[warp][d] : 0u;
            __syncwarp();
            const int leader = __ffs(peers) - 1;
            uint32_t b = 0;
            if (v && lane == leader) {
                b = s_whist[warp][d];
                s_whist[warp][d] = b + __popc(peers);
                s_match[warp][d] = 0u;
            }
            b = __shfl_sync(0xffffffffu, b, leader < 0 ? 0 : leader);
            rank[k] = v ? b + __popc(peers & lanemask_lt()) : 0xffffffffu;
            __syncwarp();
        }
        __syncthreads();
        // warp offsets inside the tile per digit, tile count per digit
        uint32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t c = s_whist[w][tid];
            s_whist[w][tid] = cnt;
            cnt += c;
        }
        // exclusive scan of the counts over the digits: start of each digit in the tile
        uint32_t v = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) s_wsum[warp] = v;
        __syncthreads();
        uint32_t pre = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) pre += w < warp ? s_wsum[w] : 0u;
        s_lbase[tid] = pre + v - cnt;
        __syncthreads();
        // reorder the tile by digit in shared memory
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            if (rank[k] != 0xffffffffu) {
                const uint32_t d = (key[k] >> shift) & 0xffu;
                const uint32_t lp = s_lbase[d] + s_whist[warp][d] + rank[k];
                s_key[lp] = key[k];
                s_val[lp] = val[k];
            }
        }
        __syncthreads();
        // contiguous writes of each digit run
        const uint32_t nt = (uint32_t)min((uint64_t)kSortTile, (uint64_t)n - (uint64_t)tile * kSortTile);
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            const uint32_t lp = (uint32_t)(k * kSortThreads + tid);
            if (lp < nt) {
                const uint32_t kk = s_key[lp];
                const uint32_t d = (kk >> shift) & 0xffu;
                const uint32_t pos = s_out[d] + (lp - s_lbase[d]);
                if (pos < n) {
                    kout[pos] = kk;
                    vout[pos] = s_val[lp];
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace

int sort_blocks_per_sm() {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_radix_scatter, kSortThreads, 0) != cudaSuccess) b = 1;
    return b < 1 ? 1 : b;
}

// One stable pass over digit `pass` of the keys in buffer `cur` (count in misc[slot]).
static cudaError_t radix_pass(geer_workspace *ws, uint32_t *const kbuf[2], uint32_t *const vbuf[2], int cur, int slot,
                              int check, int pass, int64_t cap_keys, cudaStream_t s) {
    const int shift = kRadixBits * pass;
    const int64_t tiles = (cap_keys + kSortTile - 1) / kSortTile;
    k_radix_hist<<<(unsigned)std::max<int64_t>(1, tiles), kSortThreads, 0, s>>>(kbuf[cur], ws->d_misc, slot, check,
                                                                                shift, ws->d_tile_hist, ws->d_group_sum);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_radix_groups<<<1, 1024, 0, s>>>(ws->d_misc, slot, check, ws->d_group_sum, ws->d_group_excl, ws->d_digit_base);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_radix_scatter<<<(unsigned)std::max<int64_t>(1, tiles), kSortThreads, 0, s>>>(
        kbuf[cur], vbuf[cur], kbuf[cur ^ 1], vbuf[cur ^ 1], ws->d_misc, slot, check, shift, ws->d_tile_hist,
        ws->d_group_excl, ws->d_digit_base);
    return cudaGetLastError();
}

// Stable sort of the live items by depth key (4 digits of the FP32 bits).
cudaError_t launch_depth_sort(geer_workspace *ws, cudaStream_t s) {
    int cur = 0;
    const int64_t items = (int64_t)ws->n_cams * ws->n_gauss;
    if (items > 0) {
        for (int p = 0; p < 4; ++p) {
            cudaError_t e = radix_pass(ws, ws->d_ikey, ws->d_iid, cur, kMiscLive, 0, p, items, s);
            if (e != cudaSuccess) return e;
            cur ^= 1;
        }
    }
    ws->depth_buf = cur;
    return cudaSuccess;
}

// Stable sort of the (super-tile, item) pairs by super-tile id (one or two
// 8-bit digits).
cudaError_t launch_tile_sort(geer_workspace *ws, cudaStream_t s) {
    int cur = 0;
    for (int p = 0; p < ws->n_sort_passes; ++p) {
        cudaError_t e = radix_pass(ws, ws->d_keys, ws->d_vals, cur, kMiscPairs, 1, p, ws->cap_pairs, s);
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    ws->sorted_buf = cur;
    return launch_sorted_ranges(ws, s);
}

}  // namespace geer
