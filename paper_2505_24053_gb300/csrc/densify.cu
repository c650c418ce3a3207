// densify.cu -- adaptive density control of the training loop (Algorithm 2,
// refinement iterations; the 3DGS rules driven by the gradient of the
// view-space mean3D, App. G):
//   statistics  accum += |dL/dmu_c| (= |dL/dmu|, the map is rigid), denom += 1
//               for the Gaussians associated with some tile in the step;
//   classify    prune (sigma < min_opacity, or the largest scale above
//               max_scale when max_scale > 0), else densify when
//               accum / denom >= grad_threshold: clone when the largest scale is
//               <= clone_max_scale, split otherwise; else keep;
//   apply       the outputs in the originals' order: kept / cloned Gaussians
//               with their Adam moments, a clone's copy and split children
//               with zero moments; child i at mu + R(q) (s * z_i), log-scale
//               minus ln 1.6;
//   reset       logit <- min(logit, logit(value)), the changed Gaussians'
//               opacity moments zeroed.
// The decisions are FP32 comparisons on FP32 values: accum / denom, the largest
// log-scale against ln of the scale thresholds, the logit against
// logit(min_opacity) (host: FP64 ln of the FP32 parameters, rounded to FP32).
// HBM-bound: the statistics, classification and split children take a thread
// per Gaussian; the copies of the parameters and moments an element-parallel
// pass per array (coalesced reads and writes).
#include <cmath>

#include "geer_internal.cuh"

namespace geer {
namespace {

constexpr int kDensThreads = 256;

enum : uint8_t { kActPrune = 0, kActKeep = 1, kActClone = 2, kActSplit = 3 };

__device__ __forceinline__ uint32_t outputs_of(uint8_t a) { return a == kActPrune ? 0u : (a == kActKeep ? 1u : 2u); }

struct DensConst {
    float grad_threshold, log_clone, logit_min, log_max;
    int big;  // max_scale > 0
};

__global__ void __launch_bounds__(kDensThreads) k_densify_accum(int64_t n, int ncams, const uint32_t *__restrict__ count,
                                                                const float *__restrict__ d_mean,
                                                                float *__restrict__ accum, float *__restrict__ denom) {
    grid_dep_sync();
    const int64_t g = (int64_t)blockIdx.x * kDensThreads + threadIdx.x;
    if (g >= n) return;
    bool vis = false;
    for (int c = 0; c < ncams; ++c) vis |= count[(int64_t)c * n + g] > 0u;
    if (!vis) return;
    const float x = d_mean[3 * g], y = d_mean[3 * g + 1], z = d_mean[3 * g + 2];
    accum[g] += sqrtf(x * x + y * y + z * z);
    denom[g] += 1.0f;
}

// Block-wide exclusive scan of one value per thread (kDensThreads threads).
__device__ __forceinline__ uint32_t block_excl(uint32_t x, uint32_t *wsum, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    uint32_t pre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kDensThreads / 32; ++w) {
        const uint32_t t = wsum[w];
        pre += w < warp ? t : 0u;
        tot += t;
    }
    __syncthreads();
    total = tot;
    return pre + v - x;
}

__global__ void __launch_bounds__(kDensThreads) k_densify_classify(DensConst c, int64_t n,
                                                                   const float *__restrict__ log_scale,
                                                                   const float *__restrict__ logit,
                                                                   const float *__restrict__ accum,
                                                                   const float *__restrict__ denom,
                                                                   uint8_t *__restrict__ action,
                                                                   uint32_t *__restrict__ blocksum) {
    grid_dep_sync();
    __shared__ uint32_t wsum[kDensThreads / 32];
    const int64_t g = (int64_t)blockIdx.x * kDensThreads + threadIdx.x;
    uint32_t outs = 0;
    if (g < n) {
        const float ls = fmaxf(fmaxf(log_scale[3 * g], log_scale[3 * g + 1]), log_scale[3 * g + 2]);
        const float d = denom[g];
        const float gr = d > 0.0f ? accum[g] / d : 0.0f;
        uint8_t a;
        if (logit[g] < c.logit_min || (c.big && ls > c.log_max)) a = kActPrune;
        else if (gr >= c.grad_threshold) a = ls <= c.log_clone ? kActClone : kActSplit;
        else a = kActKeep;
        action[g] = a;
        outs = outputs_of(a);
    }
    uint32_t tot;
    block_excl(outs, wsum, tot);
    if (threadIdx.x == 0) blocksum[blockIdx.x] = tot;
}

// Exclusive scan of the block sums in place (one block of 1024 threads, each
// scanning a contiguous chunk); the total goes to *total.
__global__ void __launch_bounds__(1024) k_densify_scan(uint32_t *__restrict__ blocksum, int64_t m,
                                                       unsigned long long *__restrict__ total) {
    grid_dep_sync();
    __shared__ unsigned long long wt[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t chunk = (m + 1023) / 1024;
    const int64_t b = t * chunk, e = min(m, b + chunk);
    unsigned long long s = 0;
    for (int64_t i = b; i < e; ++i) s += blocksum[i];
    unsigned long long v = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) wt[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = wt[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wt[lane] = w;
    }
    __syncthreads();
    unsigned long long ex = v - s + (warp > 0 ? wt[warp - 1] : 0ull);
    for (int64_t i = b; i < e; ++i) {
        const uint32_t c = blocksum[i];
        blocksum[i] = (uint32_t)ex;
        ex += c;
    }
    if (t == 1023) *total = ex;
}

// Each original's first output row (the block's offset from the scan plus the
// exclusive prefix of the outputs within the block).
__global__ void __launch_bounds__(kDensThreads) k_densify_offsets(int64_t n, const uint8_t *__restrict__ action,
                                                                  const uint32_t *__restrict__ blockoff,
                                                                  uint32_t *__restrict__ out_off) {
    grid_dep_sync();
    __shared__ uint32_t wsum[kDensThreads / 32];
    const int64_t g = (int64_t)blockIdx.x * kDensThreads + threadIdx.x;
    uint32_t tot;
    const uint32_t pre = block_excl(g < n ? outputs_of(action[g]) : 0u, wsum, tot);
    if (g < n) out_off[g] = blockoff[blockIdx.x] + pre;
}

// One array of `width` floats per Gaussian (a parameter or a moment group),
// element-parallel so that reads and writes are coalesced: a kept Gaussian's
// row to its output row, a clone's to both rows, a split Gaussian's to both
// children (mean and log-scale: skip_split, written by k_densify_split).
// zero_new: a moment group (the clone's copy and split children start at 0).
// act 1: also write exp of the values (activated scale), 2: their sigmoid
// (activated opacity) into aux.
__global__ void __launch_bounds__(kDensThreads) k_densify_copy(int64_t n, int64_t no, int width,
                                                               const float *__restrict__ src, float *__restrict__ dst,
                                                               int zero_new, int skip_split, int act,
                                                               float *__restrict__ aux,
                                                               const uint8_t *__restrict__ action,
                                                               const uint32_t *__restrict__ out_off) {
    grid_dep_sync();
    const int64_t idx = (int64_t)blockIdx.x * kDensThreads + threadIdx.x;
    if (idx >= n * width) return;
    const int64_t g = idx / width;
    const int a = (int)(idx - g * width);
    const uint8_t ac = action[g];
    if (ac == kActPrune || (skip_split && ac == kActSplit)) return;
    const int64_t o = out_off[g];
    if (o + (int64_t)outputs_of(ac) > no) return;  // a plan that does not match: nothing written out of bounds
    const float x = src[idx];
    const float x0 = (zero_new && ac == kActSplit) ? 0.0f : x, x1 = zero_new ? 0.0f : x;
    dst[o * width + a] = x0;
    if (ac != kActKeep) dst[(o + 1) * width + a] = x1;
    if (act && aux) {
        const float y = act == 1 ? expf(x) : 1.0f / (1.0f + expf(-x));
        aux[o * width + a] = y;
        if (ac != kActKeep) aux[(o + 1) * width + a] = y;
    }
}

// Split children's means and log-scales (and activated scales): child i at
// mu + R(q) (s * z_i), log-scale - ln 1.6.
__global__ void __launch_bounds__(kDensThreads) k_densify_split(int64_t n, int64_t no, const float *__restrict__ mean,
                                                                const float *__restrict__ log_scale,
                                                                const float *__restrict__ quat,
                                                                const float *__restrict__ z,
                                                                const uint8_t *__restrict__ action,
                                                                const uint32_t *__restrict__ out_off,
                                                                float *__restrict__ o_mean,
                                                                float *__restrict__ o_log_scale,
                                                                float *__restrict__ o_scale) {
    grid_dep_sync();
    const int64_t g = (int64_t)blockIdx.x * kDensThreads + threadIdx.x;
    if (g >= n || action[g] != kActSplit) return;
    const int64_t o = out_off[g];
    if (o + 2 > no) return;
    const float q0 = quat[4 * g], q1 = quat[4 * g + 1], q2 = quat[4 * g + 2], q3 = quat[4 * g + 3];
    const float qn = rsqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    const float w = q0 * qn, x = q1 * qn, y = q2 * qn, zq = q3 * qn;
    const float R[9] = {1.0f - 2.0f * (y * y + zq * zq), 2.0f * (x * y - w * zq), 2.0f * (x * zq + w * y),
                        2.0f * (x * y + w * zq), 1.0f - 2.0f * (x * x + zq * zq), 2.0f * (y * zq - w * x),
                        2.0f * (x * zq - w * y), 2.0f * (y * zq + w * x), 1.0f - 2.0f * (x * x + y * y)};
    float mu[3], ls[3], s[3];
    for (int k = 0; k < 3; ++k) {
        mu[k] = mean[3 * g + k];
        ls[k] = log_scale[3 * g + k];
        s[k] = expf(ls[k]);
    }
    constexpr float kLn16 = 0.470003629245735553f;  // ln 1.6
    for (int i = 0; i < 2; ++i) {
        const float *zi = z + 6 * g + 3 * i;
        const float t0 = s[0] * zi[0], t1 = s[1] * zi[1], t2 = s[2] * zi[2];
        for (int k = 0; k < 3; ++k) {
            o_mean[3 * (o + i) + k] = mu[k] + (R[3 * k] * t0 + R[3 * k + 1] * t1 + R[3 * k + 2] * t2);
            const float lc = ls[k] - kLn16;
            o_log_scale[3 * (o + i) + k] = lc;
            if (o_scale) o_scale[3 * (o + i) + k] = expf(lc);
        }
    }
}

__global__ void __launch_bounds__(kDensThreads) k_opacity_reset(int64_t n, float cap, float *__restrict__ logit,
                                                                float *__restrict__ m_op, float *__restrict__ v_op,
                                                                float *__restrict__ opacity) {
    grid_dep_sync();
    const int64_t g = (int64_t)blockIdx.x * kDensThreads + threadIdx.x;
    if (g >= n) return;
    float l = logit[g];
    if (l > cap) {
        l = cap;
        logit[g] = cap;
        m_op[g] = 0.0f;
        v_op[g] = 0.0f;
    }
    if (opacity) opacity[g] = 1.0f / (1.0f + expf(-l));
}

inline int64_t dens_blocks(int64_t n) { return (n + kDensThreads - 1) / kDensThreads; }

}  // namespace

// Scratch: action u8[n] | block sums / offsets u32[blocks] | first output row
// u32[n] | the total (u64), each part 16-byte aligned.
inline int64_t r16(int64_t b) { return (b + 15) / 16 * 16; }
size_t densify_scratch_bytes(int64_t n) { return (size_t)(r16(n) + r16(4 * dens_blocks(n)) + r16(4 * n) + 16); }

cudaError_t launch_densify_accum(const geer_workspace *ws, const float *d_mean, float *accum, float *denom,
                                 cudaStream_t s) {
    const int64_t n = ws->n_gauss;
    if (n == 0) return cudaSuccess;
    launch_k(k_densify_accum, dim3((unsigned)dens_blocks(n)), dim3(kDensThreads), 0, s, n, ws->n_cams,
             (const uint32_t *)ws->d_count, d_mean, accum, denom);
    return cudaGetLastError();
}

cudaError_t launch_densify_plan(const geer_densify_params *hp, int64_t n, const float *log_scale, const float *logit,
                                const float *accum, const float *denom, void *scratch, unsigned long long *total,
                                cudaStream_t s) {
    DensConst c;
    c.grad_threshold = hp->grad_threshold;
    c.log_clone = (float)std::log((double)hp->clone_max_scale);
    c.logit_min = (float)std::log((double)hp->min_opacity / (1.0 - (double)hp->min_opacity));
    c.big = hp->max_scale > 0.0f;
    c.log_max = c.big ? (float)std::log((double)hp->max_scale) : 0.0f;
    const int64_t nb = dens_blocks(n);
    uint8_t *action = static_cast<uint8_t *>(scratch);
    uint32_t *bsum = reinterpret_cast<uint32_t *>(action + r16(n));
    if (n > 0)
        launch_k(k_densify_classify, dim3((unsigned)nb), dim3(kDensThreads), 0, s, c, n, log_scale, logit, accum,
                 denom, action, bsum);
    launch_k(k_densify_scan, dim3(1), dim3(1024), 0, s, bsum, nb, total);
    return cudaGetLastError();
}

cudaError_t launch_densify_apply(int64_t n, int32_t sh_degree, const float *mean, const float *log_scale,
                                 const float *quat, const float *logit, const float *sh, const float *m,
                                 const float *v, const float *z, void *scratch, int64_t n_out, float *o_mean,
                                 float *o_log_scale, float *o_quat, float *o_logit, float *o_sh, float *o_m,
                                 float *o_v, float *o_scale, float *o_opacity, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint8_t *action = static_cast<const uint8_t *>(scratch);
    const uint32_t *boff = reinterpret_cast<const uint32_t *>(action + r16(n));
    uint32_t *off = reinterpret_cast<uint32_t *>(static_cast<char *>(scratch) + r16(n) + r16(4 * dens_blocks(n)));
    const int K3 = 3 * (sh_degree + 1) * (sh_degree + 1);
    launch_k(k_densify_offsets, dim3((unsigned)dens_blocks(n)), dim3(kDensThreads), 0, s, n, action, boff, off);
    const int64_t no = n_out;
    // the moments' flat groups: [mean 3 | log-scale 3 | quat 4 | logit 1 | sh K3] per Gaussian
    const int wd[5] = {3, 3, 4, 1, K3};
    int64_t gi = 0, go = 0;
    for (int grp = 0; grp < 5; ++grp) {
        const int w = wd[grp];
        const unsigned blocks = (unsigned)((n * w + kDensThreads - 1) / kDensThreads);
        launch_k(k_densify_copy, dim3(blocks), dim3(kDensThreads), 0, s, n, no, w, m + gi, o_m + go, 1, 0, 0,
                 (float *)nullptr, action, (const uint32_t *)off);
        launch_k(k_densify_copy, dim3(blocks), dim3(kDensThreads), 0, s, n, no, w, v + gi, o_v + go, 1, 0, 0,
                 (float *)nullptr, action, (const uint32_t *)off);
        gi += w * n;
        go += w * no;
    }
    const float *src[5] = {mean, log_scale, quat, logit, sh};
    float *dst[5] = {o_mean, o_log_scale, o_quat, o_logit, o_sh};
    float *aux[5] = {nullptr, o_scale, nullptr, o_opacity, nullptr};
    const int act[5] = {0, 1, 0, 2, 0};
    for (int grp = 0; grp < 5; ++grp) {
        const int w = wd[grp];
        const unsigned blocks = (unsigned)((n * w + kDensThreads - 1) / kDensThreads);
        launch_k(k_densify_copy, dim3(blocks), dim3(kDensThreads), 0, s, n, no, w, src[grp], dst[grp], 0,
                 grp < 2 ? 1 : 0, act[grp], aux[grp], action, (const uint32_t *)off);
    }
    launch_k(k_densify_split, dim3((unsigned)dens_blocks(n)), dim3(kDensThreads), 0, s, n, no, mean, log_scale, quat,
             z, action, (const uint32_t *)off, o_mean, o_log_scale, o_scale);
    return cudaGetLastError();
}

cudaError_t launch_opacity_reset(int64_t n, float value, float *logit, float *m_op, float *v_op, float *opacity,
                                 cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const float cap = (float)std::log((double)value / (1.0 - (double)value));
    launch_k(k_opacity_reset, dim3((unsigned)dens_blocks(n)), dim3(kDensThreads), 0, s, n, cap, logit, m_op, v_op,
             opacity);
    return cudaGetLastError();
}

}  // namespace geer
