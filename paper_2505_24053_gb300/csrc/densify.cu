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
// Elementwise and HBM-bound; a thread per Gaussian.
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

struct DensIn {
    const float *mean, *log_scale, *quat, *logit, *sh, *m, *v, *z;
};
struct DensOut {
    float *mean, *log_scale, *quat, *logit, *sh, *m, *v, *scale, *opacity;
};

// One output row: parameters of Gaussian g (mean and log-scale given), moments
// of g (with_moments) or zeros.
__device__ __forceinline__ void emit(const DensIn &in, const DensOut &out, int64_t n, int64_t no, int K3, int64_t g,
                                     int64_t o, const float mu[3], const float ls[3], bool with_moments) {
    // the flat group offsets of the moments: [mean 3n | log-scale 3n | quat 4n | logit n | sh K3 n]
    const int64_t gi[5] = {0, 3 * n, 6 * n, 10 * n, 11 * n};
    const int64_t go[5] = {0, 3 * no, 6 * no, 10 * no, 11 * no};
    const int width[5] = {3, 3, 4, 1, K3};
    for (int a = 0; a < 3; ++a) {
        out.mean[3 * o + a] = mu[a];
        out.log_scale[3 * o + a] = ls[a];
        if (out.scale) out.scale[3 * o + a] = expf(ls[a]);
    }
    for (int a = 0; a < 4; ++a) out.quat[4 * o + a] = in.quat[4 * g + a];
    const float lg = in.logit[g];
    out.logit[o] = lg;
    if (out.opacity) out.opacity[o] = 1.0f / (1.0f + expf(-lg));
    for (int a = 0; a < K3; ++a) out.sh[(int64_t)K3 * o + a] = in.sh[(int64_t)K3 * g + a];
    for (int grp = 0; grp < 5; ++grp) {
        const int wdt = width[grp];
        for (int a = 0; a < wdt; ++a) {
            const int64_t src = gi[grp] + (int64_t)wdt * g + a, dst = go[grp] + (int64_t)wdt * o + a;
            out.m[dst] = with_moments ? in.m[src] : 0.0f;
            out.v[dst] = with_moments ? in.v[src] : 0.0f;
        }
    }
}

__global__ void __launch_bounds__(kDensThreads) k_densify_apply(int64_t n, int64_t no, int K3, DensIn in, DensOut out,
                                                                const uint8_t *__restrict__ action,
                                                                const uint32_t *__restrict__ blockoff) {
    grid_dep_sync();
    __shared__ uint32_t wsum[kDensThreads / 32];
    const int64_t g = (int64_t)blockIdx.x * kDensThreads + threadIdx.x;
    const uint8_t a = g < n ? action[g] : kActPrune;
    uint32_t tot;
    const uint32_t pre = block_excl(outputs_of(a), wsum, tot);
    if (g >= n || a == kActPrune) return;
    const int64_t o = (int64_t)blockoff[blockIdx.x] + pre;
    if (o + (int64_t)outputs_of(a) > no) return;  // a plan that does not match: nothing written out of bounds
    float mu[3], ls[3];
    for (int k = 0; k < 3; ++k) {
        mu[k] = in.mean[3 * g + k];
        ls[k] = in.log_scale[3 * g + k];
    }
    if (a != kActSplit) {
        emit(in, out, n, no, K3, g, o, mu, ls, true);
        if (a == kActClone) emit(in, out, n, no, K3, g, o + 1, mu, ls, false);
        return;
    }
    // split: the rotation of the normalised quaternion, children at mu + R (s * z_i)
    float q0 = in.quat[4 * g], q1 = in.quat[4 * g + 1], q2 = in.quat[4 * g + 2], q3 = in.quat[4 * g + 3];
    const float qn = rsqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    const float w = q0 * qn, x = q1 * qn, y = q2 * qn, z = q3 * qn;
    const float R[9] = {1.0f - 2.0f * (y * y + z * z), 2.0f * (x * y - w * z), 2.0f * (x * z + w * y),
                        2.0f * (x * y + w * z), 1.0f - 2.0f * (x * x + z * z), 2.0f * (y * z - w * x),
                        2.0f * (x * z - w * y), 2.0f * (y * z + w * x), 1.0f - 2.0f * (x * x + y * y)};
    const float s[3] = {expf(ls[0]), expf(ls[1]), expf(ls[2])};
    constexpr float kLn16 = 0.470003629245735553f;  // ln 1.6
    const float lsc[3] = {ls[0] - kLn16, ls[1] - kLn16, ls[2] - kLn16};
    for (int i = 0; i < 2; ++i) {
        const float *zi = in.z + 6 * g + 3 * i;
        const float t0 = s[0] * zi[0], t1 = s[1] * zi[1], t2 = s[2] * zi[2];
        float c[3];
        for (int k = 0; k < 3; ++k) c[k] = mu[k] + (R[3 * k] * t0 + R[3 * k + 1] * t1 + R[3 * k + 2] * t2);
        emit(in, out, n, no, K3, g, o + i, c, lsc, false);
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

size_t densify_scratch_bytes(int64_t n) {
    const int64_t nb = dens_blocks(n);
    return (size_t)(((n + 15) / 16) * 16 + 4 * ((nb + 3) / 4) * 4 + 16);
}

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
    uint32_t *bsum = reinterpret_cast<uint32_t *>(action + ((n + 15) / 16) * 16);
    if (n > 0)
        launch_k(k_densify_classify, dim3((unsigned)nb), dim3(kDensThreads), 0, s, c, n, log_scale, logit, accum,
                 denom, action, bsum);
    launch_k(k_densify_scan, dim3(1), dim3(1024), 0, s, bsum, nb, total);
    return cudaGetLastError();
}

cudaError_t launch_densify_apply(int64_t n, int32_t sh_degree, const float *mean, const float *log_scale,
                                 const float *quat, const float *logit, const float *sh, const float *m,
                                 const float *v, const float *z, const void *scratch, int64_t n_out, float *o_mean,
                                 float *o_log_scale, float *o_quat, float *o_logit, float *o_sh, float *o_m,
                                 float *o_v, float *o_scale, float *o_opacity, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint8_t *action = static_cast<const uint8_t *>(scratch);
    const uint32_t *boff = reinterpret_cast<const uint32_t *>(action + ((n + 15) / 16) * 16);
    const int K3 = 3 * (sh_degree + 1) * (sh_degree + 1);
    DensIn in{mean, log_scale, quat, logit, sh, m, v, z};
    DensOut out{o_mean, o_log_scale, o_quat, o_logit, o_sh, o_m, o_v, o_scale, o_opacity};
    launch_k(k_densify_apply, dim3((unsigned)dens_blocks(n)), dim3(kDensThreads), 0, s, n, n_out, K3, in, out, action,
             boff);
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
