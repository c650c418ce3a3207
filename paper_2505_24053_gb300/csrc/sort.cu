// sort.cu -- SortByKeys (Algorithm 1): stable LSD radix sort of u32 keys with
// u32 values, 8-bit digits, two kernels per digit and no device-side waits:
//
//   k_radix_hist     per sort tile (ITEMS x 256 keys): the 256-bin digit
//                    histogram, stored per tile and summed into its group of
//                    32 tiles. The last block to finish (an atomic
//                    counter after a memory fence; nothing waits) scans the
//                    group sums down the tiles per digit and the digit totals
//                    (the digit bases);
//   k_radix_scatter  per sort tile: stable warp-level ranking (peer masks from a
//                    per-warp shared atomicOr of lane bits), the tile's offset per
//                    digit = digit base + group prefix + sum over the earlier
//                    tiles of its group, reordering by digit in shared memory and
//                    contiguous writes of each digit run.
//
// Tiles hold 3072 keys. The key count stays on the device: both kernels launch one block per tile of
// the workspace capacity and the blocks past the count exit at once.
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

// dev_buf: the pass's input buffer is chosen on the device (kin0 or kin1): the
// one the previous pass wrote, or read, if that pass was skipped (its digit the
// same for every key). Otherwise kin0 is the input.
template <int ITEMS>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t *__restrict__ kin0,
                                                             const uint32_t *__restrict__ kin1, int dev_buf,
                                                             uint32_t *__restrict__ misc, int count_slot,
                                                             int check_capacity, int shift,
                                                             uint32_t *__restrict__ tile_hist,
                                                             uint32_t *__restrict__ group_sum,
                                                             uint32_t *__restrict__ group_excl,
                                                             uint32_t *__restrict__ digit_base) {
    grid_dep_sync();
    constexpr int W = kSortThreads / 32, TILE = kSortThreads * ITEMS, GROUP = kGroupTiles;
    __shared__ uint32_t s_h[W][kRadix];
    __shared__ uint32_t s_wsum[W];
    __shared__ bool s_is_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n = key_count(misc, count_slot, check_capacity);
    const uint32_t tile = blockIdx.x;
    const uint32_t ntiles = (n + TILE - 1) / TILE;
    if (tile >= ntiles) return;
    // read before the last block of this pass updates them (it finishes after every block started)
    const int in = dev_buf ? depth_sorted_buf(misc) : 0;
    const uint32_t *__restrict__ kin = in ? kin1 : kin0;
    for (int i = tid; i < W * kRadix; i += kSortThreads) (&s_h[0][0])[i] = 0u;
    const uint64_t base = (uint64_t)tile * TILE + (uint64_t)warp * 32 * ITEMS + lane;
    uint32_t key[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const uint64_t i = base + (uint64_t)k * 32;
        key[k] = i < n ? kin[i] : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ITEMS; ++k)
        if (base + (uint64_t)k * 32 < n) atomicAdd(&s_h[warp][(key[k] >> shift) & 0xffu], 1u);
    __syncthreads();
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) c += s_h[w][tid];
    tile_hist[(uint64_t)tile * kRadix + tid] = c;
    if (c) atomicAdd(&group_sum[(uint64_t)(tile / GROUP) * kRadix + tid], c);

    // the last block to finish scans the group sums (threadFenceReduction pattern)
    __threadfence();
    __syncthreads();
    if (tid == 0) s_is_last = atomicAdd(&misc[kMiscSortDone], 1u) == ntiles - 1u;
    __syncthreads();
    if (!s_is_last) return;
    __threadfence();
    const int d = tid;  // one digit per thread
    const uint32_t ngroups = (ntiles + GROUP - 1) / GROUP;
    uint32_t run = 0;
    for (uint32_t g = 0; g < ngroups; g += 16) {
        uint32_t v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = g + u < ngroups ? __ldcg(&group_sum[(uint64_t)(g + u) * kRadix + d]) : 0u;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            if (g + u < ngroups) {
                group_excl[(uint64_t)(g + u) * kRadix + d] = run;
                group_sum[(uint64_t)(g + u) * kRadix + d] = 0u;  // zero for the next pass
            }
            run += v[u];
        }
    }
    // digit bases: exclusive scan of the digit totals over the 256 digits
    uint32_t v = run;
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
    digit_base[d] = pre + v - run;
    // one digit holds every key: the pass keeps the order (its scatter copies, or
    // with dev_buf is skipped, the data staying in its input buffer)
    const bool all = __syncthreads_or(run == n);
    if (tid == 0) {
        misc[kMiscSortSame] = all ? 1u : 0u;
        if (dev_buf) misc[kMiscSortCur] = (uint32_t)in;
        misc[kMiscSortDone] = 0u;
    }
}

// With rout: also rout[pos] = ranges[value] for every key written (the last pass
// of the super-tile sort gathers the association ranges into list order).
template <int ITEMS>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint32_t *__restrict__ kin_, const uint32_t *__restrict__ vin_, uint32_t *__restrict__ kout_,
    uint32_t *__restrict__ vout_, int dev_buf, const uint32_t *__restrict__ misc, int count_slot,
    int check_capacity, int shift, const uint32_t *__restrict__ tile_hist, const uint32_t *__restrict__ group_excl,
    const uint32_t *__restrict__ digit_base, const uint4 *__restrict__ ranges, uint4 *__restrict__ rout) {
    grid_dep_sync();
    // dev_buf: (kin_, vin_) is buffer 0 and (kout_, vout_) buffer 1; the input is
    // the one the histogram kernel recorded, and an identity pass is skipped
    if (dev_buf && misc[kMiscSortSame]) return;
    const bool swap = dev_buf && misc[kMiscSortCur];
    const uint32_t *__restrict__ kin = swap ? kout_ : kin_;
    const uint32_t *__restrict__ vin = swap ? vout_ : vin_;
    uint32_t *__restrict__ kout = swap ? const_cast<uint32_t *>(kin_) : kout_;
    uint32_t *__restrict__ vout = swap ? const_cast<uint32_t *>(vin_) : vout_;
    constexpr int W = kSortThreads / 32, TILE = kSortThreads * ITEMS, GROUP = kGroupTiles;
    __shared__ uint32_t s_whist[W][kRadix];
    __shared__ uint32_t s_match[W][kRadix];  // lane masks per digit, zero between ranking steps
    __shared__ uint32_t s_lbase[kRadix];  // start of each digit inside the tile
    __shared__ uint32_t s_out[kRadix];    // global position of the tile's first key of each digit
    __shared__ uint32_t s_wsum[W];
    __shared__ uint32_t s_key[TILE];
    __shared__ uint32_t s_val[TILE];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n = key_count(misc, count_slot, check_capacity);
    const uint32_t tile = blockIdx.x;
    if ((uint64_t)tile * TILE >= n) return;
    if (misc[kMiscSortSame]) {  // identity pass: coalesced copy of the tile
        const uint32_t nt = (uint32_t)min((uint64_t)TILE, (uint64_t)n - (uint64_t)tile * TILE);
        const uint64_t t0 = (uint64_t)tile * TILE;
        for (uint32_t i = tid; i < nt; i += kSortThreads) {
            const uint32_t v = vin[t0 + i];
            kout[t0 + i] = kin[t0 + i];
            vout[t0 + i] = v;
            if (rout) rout[t0 + i] = ranges[v];
        }
        return;
    }
    const uint32_t base_d = digit_base[tid];
    for (int i = tid; i < W * kRadix; i += kSortThreads) (&s_match[0][0])[i] = 0u;
    for (int i = tid; i < W * kRadix; i += kSortThreads) (&s_whist[0][0])[i] = 0u;
    // this tile's global offset for digit tid
    const uint32_t g0 = (tile / GROUP) * GROUP;
    uint32_t off = base_d + group_excl[(uint64_t)(tile / GROUP) * kRadix + tid];
    uint32_t part[GROUP - 1];
#pragma unroll
    for (int r = 0; r < GROUP - 1; ++r)
        part[r] = g0 + r < tile ? tile_hist[(uint64_t)(g0 + r) * kRadix + tid] : 0u;
#pragma unroll
    for (int r = 0; r < GROUP - 1; ++r) off += part[r];
    s_out[tid] = off;
    __syncthreads();

    uint32_t key[ITEMS], val[ITEMS], rank[ITEMS];
    const uint64_t base = (uint64_t)tile * TILE + (uint64_t)warp * 32 * ITEMS + lane;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const uint64_t i = base + (uint64_t)k * 32;
        const bool v = i < n;
        key[k] = v ? kin[i] : 0u;
        val[k] = v ? vin[i] : 0u;
    }
    // stable ranking: warp by warp, item k by item k, lane by lane. The lanes
    // sharing a digit find each other through a per-warp shared mask per digit
    // (atomicOr of the lane bits), cleared again by the group leader.
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
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
    for (int k = 0; k < ITEMS; ++k) {
        if (rank[k] != 0xffffffffu) {
            const uint32_t d = (key[k] >> shift) & 0xffu;
            const uint32_t lp = s_lbase[d] + s_whist[warp][d] + rank[k];
            s_key[lp] = key[k];
            s_val[lp] = val[k];
        }
    }
    __syncthreads();
    // contiguous writes of each digit run
    const uint32_t nt = (uint32_t)min((uint64_t)TILE, (uint64_t)n - (uint64_t)tile * TILE);
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const uint32_t lp = (uint32_t)(k * kSortThreads + tid);
        if (lp < nt) {
            const uint32_t kk = s_key[lp];
            const uint32_t d = (kk >> shift) & 0xffu;
            const uint32_t pos = s_out[d] + (lp - s_lbase[d]);
            if (pos < n) {
                const uint32_t v = s_val[lp];
                kout[pos] = kk;
                vout[pos] = v;
                if (rout) rout[pos] = ranges[v];
            }
        }
    }
}

}  // namespace

int sort_blocks_per_sm() {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_radix_scatter<kSortItems>, kSortThreads, 0) !=
        cudaSuccess)
        b = 1;
    return b < 1 ? 1 : b;
}

template <int ITEMS>
static cudaError_t radix_pass_t(geer_workspace *ws, uint32_t *const kbuf[2], uint32_t *const vbuf[2], int cur,
                                int dev_buf, int slot, int check, int shift, int64_t cap_keys, uint4 *rout,
                                cudaStream_t s) {
    constexpr int TILE = kSortThreads * ITEMS;
    const unsigned tiles = (unsigned)std::max<int64_t>(1, (cap_keys + TILE - 1) / TILE);
    launch_k(k_radix_hist<ITEMS>, dim3(tiles), dim3(kSortThreads), 0, s, kbuf[cur], kbuf[cur ^ 1], dev_buf,
             ws->d_misc, slot, check, shift, ws->d_tile_hist, ws->d_group_sum, ws->d_group_excl, ws->d_digit_base);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    launch_k(k_radix_scatter<ITEMS>, dim3(tiles), dim3(kSortThreads), 0, s, kbuf[cur], vbuf[cur], kbuf[cur ^ 1],
             vbuf[cur ^ 1], dev_buf, ws->d_misc, slot, check, shift, ws->d_tile_hist, ws->d_group_excl,
             ws->d_digit_base, ws->d_ranges, rout);
    return cudaGetLastError();
}

// One stable pass over digit `pass` of the keys in buffer `cur` (count in
// misc[slot]); with dev_buf the buffers are chosen on the device and a pass
// whose digit is the same for every key is skipped.
// (Tiles of 1024 keys for small sorts were measured slower: 0.106 against 0.079 ms
// for the four passes over 1M depth keys.)
static cudaError_t radix_pass(geer_workspace *ws, uint32_t *const kbuf[2], uint32_t *const vbuf[2], int cur, int slot,
                              int check, int pass, int64_t cap_keys, cudaStream_t s, uint4 *rout = nullptr,
                              int dev_buf = 0) {
    return radix_pass_t<kSortItems>(ws, kbuf, vbuf, cur, dev_buf, slot, check, kRadixBits * pass, cap_keys, rout, s);
}

// Stable sort of the live items by depth key (4 digits of the FP32 bits). The
// passes choose their buffers on the device (see depth_sorted_buf): a digit
// that is the same for every key (the exponent's high bits when the depths span
// less than a factor of two) costs its histogram only.
cudaError_t launch_depth_sort(geer_workspace *ws, cudaStream_t s) {
    const int64_t items = (int64_t)ws->n_cams * ws->n_gauss;
    if (items > 0) {
        for (int p = 0; p < 4; ++p) {
            cudaError_t e = radix_pass(ws, ws->d_ikey, ws->d_iid, 0, kMiscLive, 0, p, items, s, nullptr, 1);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

// Stable sort of the (super-tile, item) pairs by super-tile id (one or two
// 8-bit digits); the last pass also writes the items' association ranges in
// list order (the render kernels' filters read them coalesced).
cudaError_t launch_tile_sort(geer_workspace *ws, cudaStream_t s) {
    int cur = 0;
    for (int p = 0; p < ws->n_sort_passes; ++p) {
        cudaError_t e = radix_pass(ws, ws->d_keys, ws->d_vals, cur, kMiscPairs, 1, p, ws->cap_pairs, s,
                                   p + 1 == ws->n_sort_passes ? ws->d_sranges : nullptr);
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    ws->sorted_buf = cur;
    return cudaSuccess;
}

}  // namespace geer
