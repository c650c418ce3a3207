// render.cu -- the per-ray render (Algorithm 1 per-CSF loop: Cano_Ray, Dist,
// BlendInOrder) and its backward (App. C, RenderCUDA stage).
//
// One block per BEAP tile (a camera sub-frustum) of 16 x 16 rays, one thread per
// ray. The tile's depth-sorted Gaussian records are staged through shared
// memory in batches of 256 and every ray walks them front to back with the
// closed-form ray integral (Sec. 3.1):
//   d_u = W d, m_u = o_u x d_u, kappa = |m_u|^2 / |d_u|^2,
//   alpha = min(alpha_max, sigma exp(-kappa / 2)),
// skipping alpha < alpha_min and Gaussians whose closest approach lies behind
// the camera (o_u . d_u >= 0), stopping before the contributor that would take
// the transmittance below T_min (App. B.1 colour equation, 3DGS thresholds).
#include "geer_internal.cuh"

namespace geer {
namespace {

constexpr int kBatch = kTilePix;
constexpr float kNegHalfLog2e = -0.72134752044448170f;  // -log2(e) / 2

__device__ __forceinline__ int find_cam(const DevCam *cams, int ncams, int t) {
    int c = 0;
    for (int i = 1; i < ncams; ++i)
        if (cams[i].tile_base <= t) c = i;
    return c;
}

// One ray-Gaussian evaluation in the camera frame (Sec. 3.1): d_u = W d,
// m_u = o_u x d_u, kappa = |m_u|^2 / |d_u|^2 and the exponent argument
// log2(sigma) - kappa log2(e) / 2. The forward and the backward share it so that
// both take the same FP32 decisions.
struct Eval {
    float du0, du1, du2, m0, m1, m2, dd, kappa, arg;
    bool hit;  // alpha >= alpha_min and the closest approach lies in front of the camera
};

__device__ __forceinline__ Eval evaluate(const float4 &a, const float4 &b, const float4 &c, const float4 &e, float dx,
                                         float dy, float dz, float log2_amin) {
    Eval v;
    v.du0 = a.x * dx + a.y * dy + a.z * dz;
    v.du1 = a.w * dx + b.x * dy + b.y * dz;
    v.du2 = b.z * dx + b.w * dy + c.x * dz;
    v.m0 = c.z * v.du2 - c.w * v.du1;
    v.m1 = c.w * v.du0 - c.y * v.du2;
    v.m2 = c.y * v.du1 - c.z * v.du0;
    const float mm = v.m0 * v.m0 + v.m1 * v.m1 + v.m2 * v.m2;
    v.dd = v.du0 * v.du0 + v.du1 * v.du1 + v.du2 * v.du2;
    const float od = c.y * v.du0 + c.z * v.du1 + c.w * v.du2;
    v.kappa = __fdividef(mm, v.dd);
    v.arg = fmaf(v.kappa, kNegHalfLog2e, e.x);
    v.hit = !(v.arg < log2_amin || od >= 0.0f);
    return v;
}

__global__ void __launch_bounds__(kTilePix) k_render_fwd(const DevCam *__restrict__ cams, int ncams,
                                                        const float2 *__restrict__ ptab,
                                                        const uint2 *__restrict__ tile_range,
                                                        const uint32_t *__restrict__ vals,
                                                        const Record *__restrict__ rec,
                                                        const uint32_t *__restrict__ misc, Params p,
                                                        float *__restrict__ rgb, float *__restrict__ Tout,
                                                        float *__restrict__ Tfin, uint32_t *__restrict__ last_out,
                                                        uint2 *__restrict__ evals) {
    __shared__ float4 s_rec[kBatch * 4];
    __shared__ int s_cam;
    if (misc[kMiscStatus] & kStatusCapacity) return;
    const int t = blockIdx.x;
    const int tid = threadIdx.x;
    if (tid == 0) s_cam = find_cam(cams, ncams, t);
    __syncthreads();
    const DevCam &cam = cams[s_cam];
    const int lt = t - cam.tile_base;
    if (lt >= cam.tiles_x * cam.tiles_y) return;  // padding tile of a camera slot
    const int cx = lt % cam.tiles_x, cy = lt / cam.tiles_x;
    const int x = cx * kTile + (tid & (kTile - 1));
    const int y = cy * kTile + (tid / kTile);
    const bool inside = x < cam.width && y < cam.height;

    float dx = 0.0f, dy = 0.0f, dz = 1.0f;
    if (inside) {
        const float2 th = ptab[cam.pcol_off + x];  // (sin theta, cos theta)
        const float2 ph = ptab[cam.prow_off + y];  // (sin phi, cos phi)
        dx = th.x * ph.y;
        dy = th.y * ph.x;
        dz = th.y * ph.y;
    }
    const uint2 range = tile_range[t];
    const float log2_amin = log2f(p.alpha_min);
    float T = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
    uint32_t last = 0, n_eval = 0, n_applied = 0;
    bool done = !inside;

    for (uint32_t b0 = range.x; b0 < range.y; b0 += kBatch) {
        if (__syncthreads_count(done) == kTilePix) break;
        const uint32_t i = b0 + tid;
        if (i < range.y) {
            const float4 *src = reinterpret_cast<const float4 *>(rec + vals[i]);
#pragma unroll
            for (int k = 0; k < 4; ++k) s_rec[tid * 4 + k] = src[k];
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)kBatch, range.y - b0);
        if (!done) {
            for (int j = 0; j < cnt; ++j) {
                ++n_eval;
                const float4 a = s_rec[j * 4 + 0];  // W00 W01 W02 W10
                const float4 b = s_rec[j * 4 + 1];  // W11 W12 W20 W21
                const float4 c = s_rec[j * 4 + 2];  // W22 ou0 ou1 ou2
                const float4 e = s_rec[j * 4 + 3];  // log2 sigma, r, g, b
                const Eval v = evaluate(a, b, c, e, dx, dy, dz, log2_amin);
                if (!v.hit) continue;
                const float arg = v.arg;
                const float alpha = fminf(exp2f(arg), p.alpha_max);
                const float Tn = T * (1.0f - alpha);
                if (Tn < p.T_min) {
                    done = true;
                    break;
                }
                const float wgt = alpha * T;
                cr = fmaf(wgt, e.y, cr);
                cg = fmaf(wgt, e.z, cg);
                cb = fmaf(wgt, e.w, cb);
                T = Tn;
                ++n_applied;
                last = b0 - range.x + (uint32_t)j + 1u;
            }
        }
        __syncthreads();
    }
    if (inside) {
        const int64_t pix = cam.pix_base + (int64_t)y * cam.width + x;
        rgb[3 * pix + 0] = fmaf(T, cam.bg[0], cr);
        rgb[3 * pix + 1] = fmaf(T, cam.bg[1], cg);
        rgb[3 * pix + 2] = fmaf(T, cam.bg[2], cb);
        if (Tout) Tout[pix] = T;
        Tfin[pix] = T;
        last_out[pix] = last;
        evals[pix] = make_uint2(n_eval, n_applied);
    }
}

// RenderCUDA backward (App. C): reverse traversal of each ray's contributors
// from the last one composited, transmittance recovered as T_i = T_{i+1}/(1-a_i),
// colour behind accumulated back to front. Per (camera, Gaussian) it accumulates
// dL/dsigma, dL/dc, dL/dW through d_u (outer product with the ray direction)
// and dL/do_u (the PreprocessCUDA part chains o_u = -W mu_c). The 16 values are
// reduced over the warp (reduce-scatter by shuffles), over the block in shared
// memory, then added to global memory with one set of float4 atomics per
// (tile, Gaussian).
__global__ void __launch_bounds__(kTilePix) k_render_bwd(const DevCam *__restrict__ cams, int ncams,
                                                        const float2 *__restrict__ ptab,
                                                        const uint2 *__restrict__ tile_range,
                                                        const uint32_t *__restrict__ vals,
                                                        const Record *__restrict__ rec,
                                                        const uint32_t *__restrict__ misc, Params p,
                                                        const float *__restrict__ dL_drgb,
                                                        const float *__restrict__ Tfin,
                                                        const uint32_t *__restrict__ last_in,
                                                        GradAcc *__restrict__ gacc) {
    __shared__ float4 s_rec[kBatch * 4];
    __shared__ float s_acc[kBatch][17];
    __shared__ uint32_t s_last;
    __shared__ int s_cam;
    if (misc[kMiscStatus] & kStatusCapacity) return;
    const int t = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        s_cam = find_cam(cams, ncams, t);
        s_last = 0u;
    }
    __syncthreads();
    const DevCam &cam = cams[s_cam];
    const int lt = t - cam.tile_base;
    if (lt >= cam.tiles_x * cam.tiles_y) return;  // padding tile of a camera slot
    const int cx = lt % cam.tiles_x, cy = lt / cam.tiles_x;
    const int x = cx * kTile + (tid & (kTile - 1));
    const int y = cy * kTile + (tid / kTile);
    const bool inside = x < cam.width && y < cam.height;
    float dx = 0.0f, dy = 0.0f, dz = 1.0f;
    float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f, T = 1.0f;
    uint32_t lastp = 0;
    if (inside) {
        const float2 th = ptab[cam.pcol_off + x];
        const float2 ph = ptab[cam.prow_off + y];
        dx = th.x * ph.y;
        dy = th.y * ph.x;
        dz = th.y * ph.y;
        const int64_t pix = cam.pix_base + (int64_t)y * cam.width + x;
        g0 = dL_drgb[3 * pix + 0];
        g1 = dL_drgb[3 * pix + 1];
        g2 = dL_drgb[3 * pix + 2];
        T = Tfin[pix];
        lastp = last_in[pix];
        atomicMax(&s_last, lastp);
    }
    // colour composited behind the current contributor (starts with the background)
    float S0 = T * cam.bg[0], S1 = T * cam.bg[1], S2 = T * cam.bg[2];
    const uint2 range = tile_range[t];
    const float log2_amin = log2f(p.alpha_min);
    __syncthreads();
    const uint32_t block_last = s_last;

    for (int32_t b_end = (int32_t)block_last; b_end > 0; b_end -= kBatch) {
        const int32_t b_start = max(0, b_end - kBatch);
        const int cnt = b_end - b_start;
        if (tid < cnt) {
            const float4 *src = reinterpret_cast<const float4 *>(rec + vals[range.x + b_start + tid]);
#pragma unroll
            for (int k = 0; k < 4; ++k) s_rec[tid * 4 + k] = src[k];
        }
        for (int i = tid; i < kBatch * 17; i += kTilePix) (&s_acc[0][0])[i] = 0.0f;
        __syncthreads();
        for (int jj = cnt - 1; jj >= 0; --jj) {
            const uint32_t j = (uint32_t)(b_start + jj);
            float gv[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) gv[k] = 0.0f;
            bool contrib = false;
            if (inside && j < lastp) {
                const float4 a = s_rec[jj * 4 + 0];
                const float4 b = s_rec[jj * 4 + 1];
                const float4 c = s_rec[jj * 4 + 2];
                const float4 e = s_rec[jj * 4 + 3];
                const Eval v = evaluate(a, b, c, e, dx, dy, dz, log2_amin);
                if (v.hit) {
                    contrib = true;
                    const float ae = exp2f(v.arg);
                    const float alpha = fminf(ae, p.alpha_max);
                    const float om = 1.0f - alpha;
                    const float Ti = T / om;  // transmittance in front of this Gaussian
                    const float wgt = Ti * alpha;
                    gv[1] = g0 * wgt;
                    gv[2] = g1 * wgt;
                    gv[3] = g2 * wgt;
                    const float dLda = g0 * (Ti * e.y - S0 / om) + g1 * (Ti * e.z - S1 / om) + g2 * (Ti * e.w - S2 / om);
                    S0 = fmaf(wgt, e.y, S0);
                    S1 = fmaf(wgt, e.z, S1);
                    S2 = fmaf(wgt, e.w, S2);
                    T = Ti;
                    if (ae < p.alpha_max) {
                        gv[0] = dLda * exp2f(v.kappa * kNegHalfLog2e);  // dL/dsigma = dL/da e^{-kappa/2}
                        const float dLdk = -0.5f * dLda * ae;
                        const float inv_dd = 1.0f / v.dd;
                        const float gm0 = 2.0f * v.m0 * inv_dd, gm1 = 2.0f * v.m1 * inv_dd, gm2 = 2.0f * v.m2 * inv_dd;
                        const float sk = -2.0f * v.kappa * inv_dd;
                        // dkappa/dd_u = -(2 kappa/|d_u|^2) d_u + g_m x o_u
                        const float q0 = sk * v.du0 + (gm1 * c.w - gm2 * c.z);
                        const float q1 = sk * v.du1 + (gm2 * c.y - gm0 * c.w);
                        const float q2 = sk * v.du2 + (gm0 * c.z - gm1 * c.y);
                        // dkappa/do_u = d_u x g_m
                        gv[13] = dLdk * (v.du1 * gm2 - v.du2 * gm1);
                        gv[14] = dLdk * (v.du2 * gm0 - v.du0 * gm2);
                        gv[15] = dLdk * (v.du0 * gm1 - v.du1 * gm0);
                        const float r0 = dLdk * q0, r1 = dLdk * q1, r2 = dLdk * q2;
                        gv[4] = r0 * dx; gv[5] = r0 * dy; gv[6] = r0 * dz;
                        gv[7] = r1 * dx; gv[8] = r1 * dy; gv[9] = r1 * dz;
                        gv[10] = r2 * dx; gv[11] = r2 * dy; gv[12] = r2 * dz;
                    }
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
                // warp reduce-scatter of the 16 values: lane l ends with the sum of value (l >> 1)
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const bool up = lane & 16;
                    const float send = up ? gv[k] : gv[k + 8];
                    const float keep = up ? gv[k + 8] : gv[k];
                    gv[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const bool up = lane & 8;
                    const float send = up ? gv[k] : gv[k + 4];
                    const float keep = up ? gv[k + 4] : gv[k];
                    gv[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
                }
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const bool up = lane & 4;
                    const float send = up ? gv[k] : gv[k + 2];
                    const float keep = up ? gv[k + 2] : gv[k];
                    gv[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
                }
                {
                    const bool up = lane & 2;
                    const float send = up ? gv[0] : gv[1];
                    const float keep = up ? gv[1] : gv[0];
                    gv[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
                }
                gv[0] += __shfl_xor_sync(0xffffffffu, gv[0], 1);
                if ((lane & 1) == 0) atomicAdd(&s_acc[jj][lane >> 1], gv[0]);
            }
        }
        __syncthreads();
        // flush: one Gaussian of the batch per thread, four float4 atomics
        if (tid < cnt) {
            const float *v = s_acc[tid];
            bool any = false;
#pragma unroll
            for (int k = 0; k < 16; ++k) any |= v[k] != 0.0f;
            if (any) {
                float4 *dst = reinterpret_cast<float4 *>(gacc + vals[range.x + b_start + tid]);
                atomicAdd(dst + 0, make_float4(v[0], v[1], v[2], v[3]));
                atomicAdd(dst + 1, make_float4(v[4], v[5], v[6], v[7]));
                atomicAdd(dst + 2, make_float4(v[8], v[9], v[10], v[11]));
                atomicAdd(dst + 3, make_float4(v[12], v[13], v[14], v[15]));
            }
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_render_fwd(const geer_workspace *ws, float *rgb, float *T_final, cudaStream_t s) {
    if (ws->n_tiles == 0) return cudaSuccess;
    k_render_fwd<<<(unsigned)ws->n_tiles, kTilePix, 0, s>>>(
        ws->d_cams, ws->n_cams, ws->d_pix_tab, ws->d_tile_range, ws->d_vals[ws->sorted_buf], ws->d_rec, ws->d_misc,
        Params{ws->params.alpha_min, ws->params.T_min, ws->params.alpha_max, ws->params.lambda_pad}, rgb, T_final,
        ws->d_Tfin, ws->d_last, ws->d_evals);
    return cudaGetLastError();
}

cudaError_t launch_render_bwd(const geer_workspace *ws, const float *dL_drgb, cudaStream_t s) {
    if (ws->n_tiles == 0) return cudaSuccess;
    k_render_bwd<<<(unsigned)ws->n_tiles, kTilePix, 0, s>>>(
        ws->d_cams, ws->n_cams, ws->d_pix_tab, ws->d_tile_range, ws->d_vals[ws->sorted_buf], ws->d_rec, ws->d_misc,
        Params{ws->params.alpha_min, ws->params.T_min, ws->params.alpha_max, ws->params.lambda_pad}, dL_drgb,
        ws->d_Tfin, ws->d_last, ws->d_gacc);
    return cudaGetLastError();
}

}  // namespace geer
