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
                const float du0 = a.x * dx + a.y * dy + a.z * dz;
                const float du1 = a.w * dx + b.x * dy + b.y * dz;
                const float du2 = b.z * dx + b.w * dy + c.x * dz;
                const float m0 = c.z * du2 - c.w * du1;
                const float m1 = c.w * du0 - c.y * du2;
                const float m2 = c.y * du1 - c.z * du0;
                const float mm = m0 * m0 + m1 * m1 + m2 * m2;
                const float dd = du0 * du0 + du1 * du1 + du2 * du2;
                const float od = c.y * du0 + c.z * du1 + c.w * du2;
                const float kappa = __fdividef(mm, dd);
                const float arg = fmaf(kappa, kNegHalfLog2e, e.x);
                if (arg < log2_amin || od >= 0.0f) continue;
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

}  // namespace

cudaError_t launch_render_fwd(const geer_workspace *ws, float *rgb, float *T_final, cudaStream_t s) {
    if (ws->n_tiles == 0) return cudaSuccess;
    k_render_fwd<<<(unsigned)ws->n_tiles, kTilePix, 0, s>>>(
        ws->d_cams, ws->n_cams, ws->d_pix_tab, ws->d_tile_range, ws->d_vals[ws->sorted_buf], ws->d_rec, ws->d_misc,
        Params{ws->params.alpha_min, ws->params.T_min, ws->params.alpha_max, ws->params.lambda_pad}, rgb, T_final,
        ws->d_Tfin, ws->d_last, ws->d_evals);
    return cudaGetLastError();
}

}  // namespace geer
