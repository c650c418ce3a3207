// train.cu -- the optimiser step of the training loop (Algorithm 2 with the
// 3DGS optimiser and parameterisation): one Adam step (Kingma and Ba) over the
// raw parameters mean, log-scale, quaternion, logit-opacity and SH, each group
// with its learning rate (SH degree 0 and the higher degrees apart). The
// renderer's gradients are with respect to the activated scale = exp(log-scale)
// and opacity = sigmoid(logit); the chain rule is applied here, and the
// activated values of the updated parameters are written for the next render.
//
// The raw parameters, the gradients and the moments m, v are addressed by one
// flat element index over the groups [mean 3n | log-scale 3n | quat 4n |
// logit n | sh 3Kn] (K = (deg + 1)^2); a thread updates four consecutive
// elements with 128-bit accesses when the layout allows it, else one (all
// elementwise, HBM-bound: 16 B read and 12-16 B written per element).
#include <cmath>

#include "geer_internal.cuh"

namespace geer {
namespace {

struct AdamConst {
    float lr[6];  // mean, log-scale, quat, logit-opacity, SH degree 0, SH higher degrees
    float b1, b2, eps, inv_bc1, inv_bc2;  // inv_bc: 1 / (1 - beta^t)
};

__global__ void __launch_bounds__(256) k_adam_gaussians(AdamConst hp, int64_t n, int K3, float *__restrict__ mean,
                                                        float *__restrict__ log_scale, float *__restrict__ quat,
                                                        float *__restrict__ logit, float *__restrict__ sh,
                                                        const float *__restrict__ d_mean,
                                                        const float *__restrict__ d_scale,
                                                        const float *__restrict__ d_quat,
                                                        const float *__restrict__ d_opacity,
                                                        const float *__restrict__ d_sh, float *__restrict__ m,
                                                        float *__restrict__ v, float *__restrict__ scale,
                                                        float *__restrict__ opacity) {
    grid_dep_sync();
    const int64_t total = n * (11 + (int64_t)K3);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        float *p;
        float g, lr;
        int group;  // 1: log-scale, 3: logit (activated outputs), else none
        int64_t off;
        if (e < 3 * n) {
            off = e; p = mean + off; g = d_mean[off]; lr = hp.lr[0]; group = 0;
        } else if (e < 6 * n) {
            off = e - 3 * n; p = log_scale + off; g = d_scale[off]; lr = hp.lr[1]; group = 1;
        } else if (e < 10 * n) {
            off = e - 6 * n; p = quat + off; g = d_quat[off]; lr = hp.lr[2]; group = 2;
        } else if (e < 11 * n) {
            off = e - 10 * n; p = logit + off; g = d_opacity[off]; lr = hp.lr[3]; group = 3;
        } else {
            off = e - 11 * n; p = sh + off; g = d_sh[off]; group = 4;
            lr = ((uint64_t)off % (uint32_t)K3) < 3 ? hp.lr[4] : hp.lr[5];  // first 3 SH values: degree 0
        }
        const float x = *p;
        if (group == 1) {
            g *= expf(x);  // d scale / d log-scale = scale
        } else if (group == 3) {
            const float s = 1.0f / (1.0f + expf(-x));
            g *= s * (1.0f - s);  // d sigmoid / d logit
        }
        const float mm = hp.b1 * m[e] + (1.0f - hp.b1) * g;
        const float vv = hp.b2 * v[e] + (1.0f - hp.b2) * g * g;
        m[e] = mm;
        v[e] = vv;
        const float xn = x - lr * (mm * hp.inv_bc1) / (sqrtf(vv * hp.inv_bc2) + hp.eps);
        *p = xn;
        if (group == 1 && scale) scale[off] = expf(xn);
        if (group == 3 && opacity) opacity[off] = 1.0f / (1.0f + expf(-xn));
    }
}

// Four consecutive elements per thread with 128-bit accesses, for n % 4 == 0
// (the group boundaries 3n, 6n, 10n, 11n are then multiples of 4, so a chunk
// never straddles two groups) and 16-byte aligned arrays.
__device__ __forceinline__ float adam_one(const AdamConst &hp, float x, float g, float &m, float &v, float lr) {
    m = hp.b1 * m + (1.0f - hp.b1) * g;
    v = hp.b2 * v + (1.0f - hp.b2) * g * g;
    return x - lr * (m * hp.inv_bc1) / (sqrtf(v * hp.inv_bc2) + hp.eps);
}

__global__ void __launch_bounds__(256) k_adam_gaussians4(AdamConst hp, int64_t n, int K3, float *__restrict__ mean,
                                                         float *__restrict__ log_scale, float *__restrict__ quat,
                                                         float *__restrict__ logit, float *__restrict__ sh,
                                                         const float *__restrict__ d_mean,
                                                         const float *__restrict__ d_scale,
                                                         const float *__restrict__ d_quat,
                                                         const float *__restrict__ d_opacity,
                                                         const float *__restrict__ d_sh, float *__restrict__ m,
                                                         float *__restrict__ v, float *__restrict__ scale,
                                                         float *__restrict__ opacity) {
    grid_dep_sync();
    const int64_t chunks = n * (11 + (int64_t)K3) / 4;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= chunks) return;
    const int64_t e = 4 * c;
    float *p;
    const float *gp;
    int group;
    int64_t off;
    if (e < 3 * n) { off = e; p = mean; gp = d_mean; group = 0; }
    else if (e < 6 * n) { off = e - 3 * n; p = log_scale; gp = d_scale; group = 1; }
    else if (e < 10 * n) { off = e - 6 * n; p = quat; gp = d_quat; group = 2; }
    else if (e < 11 * n) { off = e - 10 * n; p = logit; gp = d_opacity; group = 3; }
    else { off = e - 11 * n; p = sh; gp = d_sh; group = 4; }
    float4 x = *reinterpret_cast<const float4 *>(p + off);
    float4 g = *reinterpret_cast<const float4 *>(gp + off);
    float4 mm = *reinterpret_cast<const float4 *>(m + e);
    float4 vv = *reinterpret_cast<const float4 *>(v + e);
    float lr[4];
    if (group < 4) {
        lr[0] = lr[1] = lr[2] = lr[3] = hp.lr[group];
    } else {
        const int base = (int)((uint64_t)off % (uint32_t)K3);  // position in the Gaussian's SH row
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int pos = base + i >= K3 ? base + i - K3 : base + i;
            lr[i] = pos < 3 ? hp.lr[4] : hp.lr[5];
        }
    }
    float *xs = &x.x, *gs = &g.x, *ms = &mm.x, *vs = &vv.x;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float gi = gs[i];
        if (group == 1) {
            gi *= expf(xs[i]);
        } else if (group == 3) {
            const float sg = 1.0f / (1.0f + expf(-xs[i]));
            gi *= sg * (1.0f - sg);
        }
        xs[i] = adam_one(hp, xs[i], gi, ms[i], vs[i], lr[i]);
    }
    *reinterpret_cast<float4 *>(p + off) = x;
    *reinterpret_cast<float4 *>(m + e) = mm;
    *reinterpret_cast<float4 *>(v + e) = vv;
    if (group == 1 && scale)
        *reinterpret_cast<float4 *>(scale + off) = make_float4(expf(x.x), expf(x.y), expf(x.z), expf(x.w));
    if (group == 3 && opacity)
        *reinterpret_cast<float4 *>(opacity + off) =
            make_float4(1.0f / (1.0f + expf(-x.x)), 1.0f / (1.0f + expf(-x.y)), 1.0f / (1.0f + expf(-x.z)),
                        1.0f / (1.0f + expf(-x.w)));
}

}  // namespace

cudaError_t launch_adam_gaussians(const geer_adam *hp, int64_t n, int32_t sh_degree, float *mean, float *log_scale,
                                  float *quat, float *logit_opacity, float *sh, const float *d_mean,
                                  const float *d_scale, const float *d_quat, const float *d_opacity,
                                  const float *d_sh, float *m, float *v, float *scale, float *opacity,
                                  cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    AdamConst c;
    c.lr[0] = hp->lr_mean;
    c.lr[1] = hp->lr_scale;
    c.lr[2] = hp->lr_quat;
    c.lr[3] = hp->lr_opacity;
    c.lr[4] = hp->lr_sh_dc;
    c.lr[5] = hp->lr_sh_rest;
    c.b1 = hp->beta1;
    c.b2 = hp->beta2;
    c.eps = hp->eps;
    c.inv_bc1 = (float)(1.0 / (1.0 - std::pow((double)hp->beta1, (double)hp->step)));
    c.inv_bc2 = (float)(1.0 / (1.0 - std::pow((double)hp->beta2, (double)hp->step)));
    const int K3 = 3 * (sh_degree + 1) * (sh_degree + 1);
    const int64_t total = n * (11 + (int64_t)K3);
    auto a16 = [](const void *q) { return q == nullptr || (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
    const bool vec = n % 4 == 0 && a16(mean) && a16(log_scale) && a16(quat) && a16(logit_opacity) && a16(sh) &&
                     a16(d_mean) && a16(d_scale) && a16(d_quat) && a16(d_opacity) && a16(d_sh) && a16(m) &&
                     a16(v) && a16(scale) && a16(opacity);
    if (vec) {
        const int64_t blocks = (total / 4 + 255) / 256;
        launch_k(k_adam_gaussians4, dim3((unsigned)blocks), dim3(256), 0, s, c, n, K3, mean, log_scale, quat,
                 logit_opacity, sh, d_mean, d_scale, d_quat, d_opacity, d_sh, m, v, scale, opacity);
    } else {
        const int64_t blocks = std::min<int64_t>((total + 255) / 256, (int64_t)1 << 30);
        launch_k(k_adam_gaussians, dim3((unsigned)blocks), dim3(256), 0, s, c, n, K3, mean, log_scale, quat,
                 logit_opacity, sh, d_mean, d_scale, d_quat, d_opacity, d_sh, m, v, scale, opacity);
    }
    return cudaGetLastError();
}

}  // namespace geer
