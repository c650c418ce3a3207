// sort.cu -- SortByKeys and IdentifyFrustumRanges (Algorithm 1).
//
// Stable LSD radix sort of the 64-bit (tile << 32 | depth) keys with their
// 32-bit values, 8-bit digits, one "onesweep" kernel per digit: every block
// ranks its tile of keys in shared memory, publishes its per-digit counts and
// finds its global offsets by decoupled look-back over earlier tiles, then
// scatters. Tiles are handed out by an atomic counter, so a block only ever
// waits on tiles owned by blocks that started before it; every wait is also
// bounded and records a timeout in the status word instead of hanging.
#include "geer_internal.cuh"

namespace geer {
namespace {

constexpr uint64_t kFlagAgg = 1ull;
constexpr uint64_t kFlagPrefix = 2ull;
constexpr int kSpinLimit = 1 << 20;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint64_t ld_volatile(const uint64_t *p) {
    return *reinterpret_cast<const volatile uint64_t *>(p);
}

__device__ __forceinline__ void st_status(uint64_t *p, uint64_t v) {
    atomicExch(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
}

// Digit histograms of every pass in one read of the keys.
__global__ void __launch_bounds__(256) k_histogram(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ misc,
                                                   uint32_t *__restrict__ hist, int npass) {
    __shared__ uint32_t sh[kMaxPasses * kRadix];
    for (int i = threadIdx.x; i < npass * kRadix; i += blockDim.x) sh[i] = 0u;
    __syncthreads();
    const uint32_t P = misc[kMiscPairs];
    const bool over = misc[kMiscStatus] & kStatusCapacity;
    if (!over) {
        const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
        for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x; i0 < P; i0 += stride) {
            const uint64_t i = i0 + threadIdx.x;
            const bool v = i < P;
            const uint64_t k = v ? keys[i] : 0ull;
            const uint32_t active = __ballot_sync(0xffffffffu, v);
            if (!v) continue;
            for (int p = 0; p < npass; ++p) {
                const uint32_t d = (uint32_t)(k >> (8 * p)) & 0xffu;
                const uint32_t peers = __match_any_sync(active, d);
                if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&sh[p * kRadix + d], __popc(peers));
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npass * kRadix; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

__global__ void __launch_bounds__(kSortThreads) k_onesweep(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                           uint64_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                           const uint32_t *__restrict__ hist, uint32_t *__restrict__ misc,
                                                           uint64_t *__restrict__ lookback, int pass) {
    constexpr int W = kSortThreads / 32;
    __shared__ uint32_t s_whist[W][kRadix];
    __shared__ uint32_t s_gbase[kRadix];
    __shared__ uint32_t s_base[kRadix];
    __shared__ uint32_t s_wsum[W];
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t P = misc[kMiscPairs];
    if (misc[kMiscStatus] & kStatusCapacity) return;
    const uint64_t epoch = (uint64_t)((misc[kMiscFrame] * kMaxPasses + (uint32_t)pass) & 0x3fffffffu);
    const int shift = kRadixBits * pass;

    // global exclusive offsets of the digits of this pass (scan of the histogram)
    {
        const uint32_t c = hist[pass * kRadix + tid];
        uint32_t v = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) s_wsum[warp] = v;
        __syncthreads();
        uint32_t pre = 0;
        for (int w = 0; w < warp; ++w) pre += s_wsum[w];
        s_gbase[tid] = pre + v - c;
    }

    for (;;) {
        if (tid == 0) s_tile = atomicAdd(&misc[kMiscTileCtr + pass], 1u);
        for (int i = tid; i < W * kRadix; i += kSortThreads) (&s_whist[0][0])[i] = 0u;
        __syncthreads();
        const uint32_t tile = s_tile;
        if ((uint64_t)tile * kSortTile >= P) break;

        // load: item k of (warp, lane) is key tile*T + warp*32*ITEMS + k*32 + lane
        uint64_t key[kSortItems];
        uint32_t val[kSortItems], dig[kSortItems], rank[kSortItems];
        const uint64_t base = (uint64_t)tile * kSortTile + (uint64_t)warp * 32 * kSortItems + lane;
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            const uint64_t i = base + (uint64_t)k * 32;
            const bool v = i < P;
            key[k] = v ? kin[i] : 0ull;
            val[k] = v ? vin[i] : 0u;
            dig[k] = v ? ((uint32_t)(key[k] >> shift) & 0xffu) : kRadix;
        }
        // stable warp-level ranking
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            const uint32_t d = dig[k];
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const int leader = __ffs(peers) - 1;
            uint32_t b = 0;
            if (lane == leader && d < kRadix) {
                b = s_whist[warp][d];
                s_whist[warp][d] = b + __popc(peers);
            }
            b = __shfl_sync(0xffffffffu, b, leader);
            rank[k] = b + __popc(peers & lanemask_lt());
            __syncwarp();
        }
        __syncthreads();
        // per digit: offsets of each warp inside the block and the block count
        uint32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t c = s_whist[w][tid];
            s_whist[w][tid] = cnt;
            cnt += c;
        }
        // decoupled look-back for digit tid
        uint64_t *my = lookback + (uint64_t)tile * kRadix + tid;
        uint32_t excl = 0;
        if (tile == 0) {
            st_status(my, (epoch << 34) | (kFlagPrefix << 32) | cnt);
        } else {
            st_status(my, (epoch << 34) | (kFlagAgg << 32) | cnt);
            int64_t j = (int64_t)tile - 1;
            int spins = 0;
            while (j >= 0) {
                const uint64_t s = ld_volatile(lookback + (uint64_t)j * kRadix + tid);
                const uint64_t flag = (s >> 32) & 3ull;
                if ((s >> 34) == epoch && flag != 0) {
                    excl += (uint32_t)s;
                    if (flag == kFlagPrefix) break;
                    --j;
                    continue;
                }
                if (++spins > kSpinLimit) {
                    atomicOr(&misc[kMiscStatus], kStatusTimeout);
                    break;
                }
                __nanosleep(64);
            }
            st_status(my, (epoch << 34) | (kFlagPrefix << 32) | (excl + cnt));
        }
        s_base[tid] = s_gbase[tid] + excl;
        __syncthreads();
        // scatter
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            const uint32_t d = dig[k];
            if (d < kRadix) {
                const uint32_t pos = s_base[d] + s_whist[warp][d] + rank[k];
                if (pos < P) {  // always true unless a look-back wait timed out
                    kout[pos] = key[k];
                    vout[pos] = val[k];
                }
            }
        }
        __syncthreads();
    }
}

// IdentifyFrustumRanges: [start, end) of every tile in the sorted keys.
__global__ void __launch_bounds__(256) k_ranges(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ misc,
                                                uint2 *__restrict__ tr, uint32_t ntiles) {
    const uint32_t P = misc[kMiscPairs];
    if (misc[kMiscStatus] & kStatusCapacity) return;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += stride) {
        const uint32_t t = (uint32_t)(keys[i] >> 32);
        if (t >= ntiles) continue;  // only after a timed-out sort
        if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != t) tr[t].x = (uint32_t)i;
        if (i + 1 == P || (uint32_t)(keys[i + 1] >> 32) != t) tr[t].y = (uint32_t)(i + 1);
    }
}

}  // namespace

int sort_blocks_per_sm() {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_onesweep, kSortThreads, 0) != cudaSuccess) b = 1;
    return b < 1 ? 1 : b;
}

cudaError_t launch_sort(geer_workspace *ws, cudaStream_t s) {
    const int grid = ws->num_sms * 4;
    k_histogram<<<grid, 256, 0, s>>>(ws->d_keys[0], ws->d_misc, ws->d_hist, ws->n_passes);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int cur = 0;
    for (int p = 0; p < ws->n_passes; ++p) {
        k_onesweep<<<ws->sort_grid, kSortThreads, 0, s>>>(ws->d_keys[cur], ws->d_vals[cur], ws->d_keys[cur ^ 1],
                                                          ws->d_vals[cur ^ 1], ws->d_hist, ws->d_misc, ws->d_lookback, p);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    ws->sorted_buf = cur;
    return cudaSuccess;
}

cudaError_t launch_ranges(const geer_workspace *ws, cudaStream_t s) {
    k_ranges<<<ws->num_sms * 4, 256, 0, s>>>(ws->d_keys[ws->sorted_buf], ws->d_misc, ws->d_tile_range,
                                              (uint32_t)ws->n_tiles);
    return cudaGetLastError();
}

}  // namespace geer
