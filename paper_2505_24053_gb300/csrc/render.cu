// render.cu -- the per-ray render (Algorithm 1 per-CSF loop: Cano_Ray, Dist,
// BlendInOrder) and its backward (App. C, RenderCUDA stage).
//
// A BEAP tile (a camera sub-frustum) of 16 x 16 rays is processed by 16 / ROWS
// blocks of ROWS x 16 threads, one thread per ray, tiles taken in the order of
// descending pair count (the costliest first); each block stages the tile's
// depth-sorted Gaussian records through shared memory in batches of BATCH and
// every ray walks them front to back with the closed-form ray integral (Sec. 3.1):
//   d_u = W d, m_u = o_u x d_u, kappa = |m_u|^2 / |d_u|^2,
//   alpha = min(alpha_max, sigma exp(-kappa / 2)),
// skipping alpha < alpha_min and Gaussians whose closest approach lies behind
// the camera (o_u . d_u >= 0), stopping before the contributor that would take
// the transmittance below T_min (App. B.1 colour equation, 3DGS thresholds).
#include "geer_internal.cuh"

namespace geer {
namespace {

#ifndef GEER_FWD_ROWS
#define GEER_FWD_ROWS 16
#endif
#ifndef GEER_FWD_BATCH
#define GEER_FWD_BATCH 256
#endif
#ifndef GEER_BWD_ROWS
#define GEER_BWD_ROWS 8
#endif
#ifndef GEER_BWD_BATCH
#define GEER_BWD_BATCH 128
#endif
#ifndef GEER_BWD_MINB
#define GEER_BWD_MINB 8
#endif
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
    float du0, du1, du2, m0, m1, m2, dd, od, kappa, arg;
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
    v.od = c.y * v.du0 + c.z * v.du1 + c.w * v.du2;
    v.kappa = __fdividef(mm, v.dd);
    v.arg = fmaf(v.kappa, kNegHalfLog2e, e.x);
    v.hit = !(v.arg < log2_amin || v.od >= 0.0f);
    return v;
}

template <int ROWS, int BATCH>
__global__ void __launch_bounds__(ROWS * kTile) k_render_fwd(const DevCam *__restrict__ cams, int ncams,
                                                            const float2 *__restrict__ ptab,
                                                            const uint2 *__restrict__ tile_range,
                                                            const uint32_t *__restrict__ tile_order,
                                                            const uint32_t *__restrict__ vals,
                                                            const Record *__restrict__ rec,
                                                            const uint32_t *__restrict__ misc, Params p,
                                                            float *__restrict__ rgb, float *__restrict__ Tout,
                                                            float *__restrict__ Tfin, uint32_t *__restrict__ last_out,
                                                            uint2 *__restrict__ evals) {
    constexpr int kThreads = ROWS * kTile, kParts = kTile / ROWS;
    __shared__ float4 s_rec[BATCH * 4];
    __shared__ int s_cam;
    if (misc[kMiscStatus] & kStatusCapacity) return;
    const int t = (int)tile_order[blockIdx.x / kParts], part = blockIdx.x % kParts;
    const int tid = threadIdx.x;
    if (tid == 0) s_cam = find_cam(cams, ncams, t);
    __syncthreads();
    const DevCam &cam = cams[s_cam];
    const int lt = t - cam.tile_base;
    if (lt >= cam.tiles_x * cam.tiles_y) return;  // padding tile of a camera slot
    const int cx = lt % cam.tiles_x, cy = lt / cam.tiles_x;
    const int x = cx * kTile + (tid & (kTile - 1));
    const int y = cy * kTile + part * ROWS + (tid / kTile);
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

    for (uint32_t b0 = range.x; b0 < range.y; b0 += BATCH) {
        if (__syncthreads_count(done) == kThreads) break;
        const int cnt = (int)min((uint32_t)BATCH, range.y - b0);
        for (int r = tid; r < cnt; r += kThreads) {
            const float4 *src = reinterpret_cast<const float4 *>(rec + vals[b0 + r]);
#pragma unroll
            for (int k = 0; k < 4; ++k) s_rec[r * 4 + k] = src[k];
        }
        __syncthreads();
        if (!done) {
            for (int j = 0; j < cnt; ++j) {
                ++n_eval;
                const float4 a = s_rec[j * 4 + 0];  // W00 W01 W02 W10
                const float4 b = s_rec[j * 4 + 1];  // W11 W12 W20 W21
                const float4 c = s_rec[j * 4 + 2];  // W22 ou0 ou1 ou2
                const float4 e = s_rec[j * 4 + 3];  // log2 sigma, r, g, b
                const Eval v = evaluate(a, b, c, e, dx, dy, dz, log2_amin);
                if (!v.hit) continue;
                const float alpha = fminf(exp2f(v.arg), p.alpha_max);
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
// and dL/do_u (the PreprocessCUDA part chains o_u = -W mu_c).
//
// The 16 values are reduced over the warp (reduce-scatter by shuffles), over the
// block in shared memory, then added to global memory with one set of float4
// atomics per (block, Gaussian). A warp skips list entries beyond the last
// contributor of its rays.
struct BwdRay {
    float dx, dy, dz, g0, g1, g2, T, S0, S1, S2;
    uint32_t last;
};

// One ray's contribution to the 16 accumulators of the Gaussian in (a, b, c, e)
// (GradAcc order), and the step of the ray's reverse compositing state.
__device__ __forceinline__ void ray_gradient(BwdRay &r, const float4 &a, const float4 &b, const float4 &c,
                                             const float4 &e, float log2_amin, float alpha_max, float gv[16],
                                             bool &contrib) {
    const Eval v = evaluate(a, b, c, e, r.dx, r.dy, r.dz, log2_amin);
    if (!v.hit) return;
    contrib = true;
    const float ae = exp2f(v.arg);
    const float alpha = fminf(ae, alpha_max);
    const float inv_om = __frcp_rn(1.0f - alpha);
    const float Ti = r.T * inv_om;  // transmittance in front of this Gaussian
    const float wgt = Ti * alpha;
    gv[1] = fmaf(r.g0, wgt, gv[1]);
    gv[2] = fmaf(r.g1, wgt, gv[2]);
    gv[3] = fmaf(r.g2, wgt, gv[3]);
    const float dLda = r.g0 * (Ti * e.y - r.S0 * inv_om) + r.g1 * (Ti * e.z - r.S1 * inv_om) +
                       r.g2 * (Ti * e.w - r.S2 * inv_om);
    r.S0 = fmaf(wgt, e.y, r.S0);
    r.S1 = fmaf(wgt, e.z, r.S1);
    r.S2 = fmaf(wgt, e.w, r.S2);
    r.T = Ti;
    if (ae < alpha_max) {
        gv[0] = fmaf(dLda, exp2f(v.kappa * kNegHalfLog2e), gv[0]);  // dL/dsigma = dL/da e^{-kappa/2}
        const float dLdk = -0.5f * dLda * ae;
        // with g_m = 2 m_u / |d_u|^2 (dkappa/dm_u), scaled by dL/dkappa:
        //   dL/dd_u = dL/dkappa (-(2 kappa / |d_u|^2) d_u + g_m x o_u),  dL/do_u = dL/dkappa (d_u x g_m)
        const float h = 2.0f * dLdk * __fdividef(1.0f, v.dd);
        const float gm0 = h * v.m0, gm1 = h * v.m1, gm2 = h * v.m2;
        const float sk = -h * v.kappa;
        const float r0 = sk * v.du0 + (gm1 * c.w - gm2 * c.z);
        const float r1 = sk * v.du1 + (gm2 * c.y - gm0 * c.w);
        const float r2 = sk * v.du2 + (gm0 * c.z - gm1 * c.y);
        gv[13] += v.du1 * gm2 - v.du2 * gm1;
        gv[14] += v.du2 * gm0 - v.du0 * gm2;
        gv[15] += v.du0 * gm1 - v.du1 * gm0;
        gv[4] = fmaf(r0, r.dx, gv[4]); gv[5] = fmaf(r0, r.dy, gv[5]); gv[6] = fmaf(r0, r.dz, gv[6]);
        gv[7] = fmaf(r1, r.dx, gv[7]); gv[8] = fmaf(r1, r.dy, gv[8]); gv[9] = fmaf(r1, r.dz, gv[9]);
        gv[10] = fmaf(r2, r.dx, gv[10]); gv[11] = fmaf(r2, r.dy, gv[11]); gv[12] = fmaf(r2, r.dz, gv[12]);
    }
}

template <int ROWS, int BATCH>
__global__ void __launch_bounds__(ROWS * kTile, GEER_BWD_MINB) k_render_bwd(const DevCam *__restrict__ cams, int ncams,
                                                            const float2 *__restrict__ ptab,
                                                            const uint2 *__restrict__ tile_range,
                                                            const uint32_t *__restrict__ tile_order,
                                                            const uint32_t *__restrict__ vals,
                                                            const Record *__restrict__ rec,
                                                            const uint32_t *__restrict__ misc, Params p,
                                                            const float *__restrict__ dL_drgb,
                                                            const float *__restrict__ Tfin,
                                                            const uint32_t *__restrict__ last_in,
                                                            GradAcc *__restrict__ gacc) {
    constexpr int kThreads = ROWS * kTile, kParts = kTile / ROWS;
    __shared__ float4 s_rec[BATCH * 4];
    __shared__ float s_acc[BATCH][17];
    __shared__ uint32_t s_last;
    __shared__ int s_cam;
    if (misc[kMiscStatus] & kStatusCapacity) return;
    const int t = (int)tile_order[blockIdx.x / kParts], part = blockIdx.x % kParts;
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
    const int y = cy * kTile + part * ROWS + (tid / kTile);
    BwdRay ray;
    ray.dx = 0.0f; ray.dy = 0.0f; ray.dz = 1.0f;
    ray.g0 = ray.g1 = ray.g2 = 0.0f;
    ray.T = 1.0f;
    ray.last = 0;
    if (x < cam.width && y < cam.height) {
        const float2 th = ptab[cam.pcol_off + x];
        const float2 ph = ptab[cam.prow_off + y];
        ray.dx = th.x * ph.y;
        ray.dy = th.y * ph.x;
        ray.dz = th.y * ph.y;
        const int64_t pix = cam.pix_base + (int64_t)y * cam.width + x;
        ray.g0 = dL_drgb[3 * pix + 0];
        ray.g1 = dL_drgb[3 * pix + 1];
        ray.g2 = dL_drgb[3 * pix + 2];
        ray.T = Tfin[pix];
        ray.last = last_in[pix];
    }
    // colour composited behind the current contributor (starts with the background)
    ray.S0 = ray.T * cam.bg[0];
    ray.S1 = ray.T * cam.bg[1];
    ray.S2 = ray.T * cam.bg[2];
    const uint32_t warp_last = __reduce_max_sync(0xffffffffu, ray.last);
    if (lane == 0) atomicMax(&s_last, warp_last);
    const uint2 range = tile_range[t];
    const float log2_amin = log2f(p.alpha_min);
    __syncthreads();
    const uint32_t block_last = s_last;

    for (int32_t b_end = (int32_t)block_last; b_end > 0; b_end -= BATCH) {
        const int32_t b_start = max(0, b_end - BATCH);
        const int cnt = b_end - b_start;
        for (int r = tid; r < cnt; r += kThreads) {
            const float4 *src = reinterpret_cast<const float4 *>(rec + vals[range.x + b_start + r]);
#pragma unroll
            for (int k = 0; k < 4; ++k) s_rec[r * 4 + k] = src[k];
        }
        for (int i = tid; i < cnt * 17; i += kThreads) (&s_acc[0][0])[i] = 0.0f;
        __syncthreads();
        const int jj_top = min(cnt, (int)warp_last - b_start) - 1;  // warp-uniform
        for (int jj = jj_top; jj >= 0; --jj) {
            const uint32_t j = (uint32_t)(b_start + jj);
            float gv[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) gv[k] = 0.0f;
            bool contrib = false;
            if (j < ray.last) {
                const float4 a = s_rec[jj * 4 + 0];
                const float4 b = s_rec[jj * 4 + 1];
                const float4 c = s_rec[jj * 4 + 2];
                const float4 e = s_rec[jj * 4 + 3];
                ray_gradient(ray, a, b, c, e, log2_amin, p.alpha_max, gv, contrib);
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
        for (int r = tid; r < cnt; r += kThreads) {
            const float *v = s_acc[r];
            bool any = false;
#pragma unroll
            for (int k = 0; k < 16; ++k) any |= v[k] != 0.0f;
            if (any) {
                float4 *dst = reinterpret_cast<float4 *>(gacc + vals[range.x + b_start + r]);
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
    constexpr int R = GEER_FWD_ROWS, B = GEER_FWD_BATCH;
    k_render_fwd<R, B><<<(unsigned)(ws->n_tiles * (kTile / R)), R * kTile, 0, s>>>(
        ws->d_cams, ws->n_cams, ws->d_pix_tab, ws->d_tile_range, ws->d_tile_order, ws->d_vals[ws->sorted_buf], ws->d_rec, ws->d_misc,
        Params{ws->params.alpha_min, ws->params.T_min, ws->params.alpha_max, ws->params.lambda_pad}, rgb, T_final,
        ws->d_Tfin, ws->d_last, ws->d_evals);
    return cudaGetLastError();
}

cudaError_t launch_render_bwd(const geer_workspace *ws, const float *dL_drgb, cudaStream_t s) {
    if (ws->n_tiles == 0) return cudaSuccess;
    constexpr int R = GEER_BWD_ROWS, B = GEER_BWD_BATCH;
    k_render_bwd<R, B><<<(unsigned)(ws->n_tiles * (kTile / R)), R * kTile, 0, s>>>(
        ws->d_cams, ws->n_cams, ws->d_pix_tab, ws->d_tile_range, ws->d_tile_order, ws->d_vals[ws->sorted_buf], ws->d_rec, ws->d_misc,
        Params{ws->params.alpha_min, ws->params.T_min, ws->params.alpha_max, ws->params.lambda_pad}, dL_drgb,
        ws->d_Tfin, ws->d_last, ws->d_gacc);
    return cudaGetLastError();
}

}  // namespace geer
