// backward.cu -- PreprocessCUDA backward (App. C): per Gaussian, sum over the
// cameras of the chain from the render-stage accumulators to the parameters
// (for the splat alpha, from its centre and conic: splat_chain).
//
//   o_u = -W mu_c, mu_c = R_cw mu + t:  dL/dW += dL/do_u (-mu_c)^T,
//                                       dL/dmu += -R_cw^T W^T dL/do_u;
//   W = S^-1 M^T, M = R_cw R(q/|q|):    dL/ds_k = -sum_i dL/dW_ki M_ik / s_k^2,
//                                       dL/dM_ik = dL/dW_ki / s_k, dL/dR = R_cw^T dL/dM,
//                                       then the unit-quaternion polynomial and
//                                       the normalisation (I - q q^T)/|q|;
//   colour = max(0, SH(dir) + 1/2), dir = (mu - o)/|mu - o|:
//                                       dL/dsh_k = dL/dc Y_k(dir), and the
//                                       direction term into mu.
// Also a small L1-loss gradient kernel for training-style steps.
#include <algorithm>

#include "geer_internal.cuh"

namespace geer {
namespace {

// Real SH basis (3DGS convention, as in the forward): term k and its gradient
// with respect to the (unit) direction components. Called with k a compile-time
// constant inside unrolled loops, so each call folds to its own polynomial and no
// table of all terms is held in registers.
struct ShDir {
    float x, y, z, xx, yy, zz;
};

__device__ __forceinline__ float sh_value(int k, const ShDir &d) {
    const float k1 = 0.4886025119029199f;
    const float a = 1.0925484305920792f, b = 0.31539156525252005f, c = 0.5462742152960396f;
    const float e = 0.5900435899266435f, f = 2.890611442640554f, h = 0.4570457994644658f;
    const float pp = 0.3731763325901154f, r = 1.445305721320277f;
    const float x = d.x, y = d.y, z = d.z, xx = d.xx, yy = d.yy, zz = d.zz;
    switch (k) {
        case 0: return 0.28209479177387814f;
        case 1: return -k1 * y;
        case 2: return k1 * z;
        case 3: return -k1 * x;
        case 4: return a * x * y;
        case 5: return -a * y * z;
        case 6: return b * (2.0f * zz - xx - yy);
        case 7: return -a * x * z;
        case 8: return c * (xx - yy);
        case 9: return -e * y * (3.0f * xx - yy);
        case 10: return f * x * y * z;
        case 11: return -h * y * (4.0f * zz - xx - yy);
        case 12: return pp * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
        case 13: return -h * x * (4.0f * zz - xx - yy);
        case 14: return r * z * (xx - yy);
        default: return -e * x * (xx - 3.0f * yy);
    }
}

__device__ __forceinline__ void sh_grad(int k, const ShDir &d, float g[3]) {
    const float k1 = 0.4886025119029199f;
    const float a = 1.0925484305920792f, b = 0.31539156525252005f, c = 0.5462742152960396f;
    const float e = 0.5900435899266435f, f = 2.890611442640554f, h = 0.4570457994644658f;
    const float pp = 0.3731763325901154f, r = 1.445305721320277f;
    const float x = d.x, y = d.y, z = d.z, xx = d.xx, yy = d.yy, zz = d.zz;
    g[0] = g[1] = g[2] = 0.0f;
    switch (k) {
        case 0: break;
        case 1: g[1] = -k1; break;
        case 2: g[2] = k1; break;
        case 3: g[0] = -k1; break;
        case 4: g[0] = a * y; g[1] = a * x; break;
        case 5: g[1] = -a * z; g[2] = -a * y; break;
        case 6: g[0] = -2.0f * b * x; g[1] = -2.0f * b * y; g[2] = 4.0f * b * z; break;
        case 7: g[0] = -a * z; g[2] = -a * x; break;
        case 8: g[0] = 2.0f * c * x; g[1] = -2.0f * c * y; break;
        case 9: g[0] = -6.0f * e * x * y; g[1] = -e * (3.0f * xx - 3.0f * yy); break;
        case 10: g[0] = f * y * z; g[1] = f * x * z; g[2] = f * x * y; break;
        case 11: g[0] = 2.0f * h * x * y; g[1] = -h * (4.0f * zz - xx - 3.0f * yy); g[2] = -8.0f * h * y * z; break;
        case 12: g[0] = -6.0f * pp * x * z; g[1] = -6.0f * pp * y * z; g[2] = pp * (6.0f * zz - 3.0f * xx - 3.0f * yy);
            break;
        case 13: g[0] = -h * (4.0f * zz - 3.0f * xx - yy); g[1] = 2.0f * h * x * y; g[2] = -8.0f * h * x * z; break;
        case 14: g[0] = 2.0f * r * x * z; g[1] = -2.0f * r * y * z; g[2] = r * (xx - yy); break;
        default: g[0] = -e * (3.0f * xx - 3.0f * yy); g[1] = 6.0f * e * x * y; break;
    }
}

// One block per 64 Gaussians. The block's SH coefficients are staged into shared
// memory with coalesced asynchronous copies (row stride made odd so that
// per-thread rows do not share banks) while each thread loads its own
// parameters; each thread then runs the chain for its Gaussian over the cameras
// and collects its dL/dsh in shared memory, and the block adds that to dL/dsh in
// global memory coalesced. With one camera the SH row itself is overwritten by
// its gradient term by term (each coefficient is read before its slot is
// written), which halves the block's shared memory; with several cameras the
// gradient has a row of its own.
constexpr int kPBThreads = 64;
#ifndef GEER_PB_MINB
#define GEER_PB_MINB 14  // resident blocks of the one-camera variant: caps registers at 72
#endif

// The splat alpha's chain (GEER_ALPHA_SPLAT) from dL/d(theta_c, phi_c) and
// dL/d(A, B, C) (the conic K = Sigma_2^-1, B its off-diagonal) to the camera-frame
// mean, the axes M and the scales: dL/dSigma_2 = -K G K with G the symmetric
// gradient [[gA, gB/2], [gB/2, gC]]; Sigma_2 = sum_k f_k f_k^T with
// f_k = s_k J M_k, J the gradients of the screen angles at the mean (the EWA
// covariance of the forward); then J and the centre (atan2(x, z), atan2(y, z))
// differentiated with respect to the mean.
__device__ __forceinline__ void splat_chain(const float mc[3], const float M[9], const float s[3], float gt, float gp,
                                            float gA, float gB, float gC, float dmc[3], float dM[9], float ds[3]) {
    const float x = mc[0], y = mc[1], z = mc[2];
    const float qx = x * x + z * z, qy = y * y + z * z, rx = 1.0f / qx, ry = 1.0f / qy;
    const float ja0 = z * rx, ja2 = -x * rx, jb1 = z * ry, jb2 = -y * ry;
    float fx[3], fy[3], c00 = 0.0f, c01 = 0.0f, c11 = 0.0f, det = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        fx[k] = s[k] * (ja0 * M[k] + ja2 * M[6 + k]);
        fy[k] = s[k] * (jb1 * M[3 + k] + jb2 * M[6 + k]);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        c00 += fx[k] * fx[k];
        c01 += fx[k] * fy[k];
        c11 += fy[k] * fy[k];
        const int l = (k + 1) % 3;
        const float mk = fx[k] * fy[l] - fy[k] * fx[l];
        det += mk * mk;
    }
    const float id = 1.0f / det;
    const float K00 = c11 * id, K01 = -c01 * id, K11 = c00 * id;
    // H = -K G K (symmetric): dL = tr(H dSigma_2)
    const float G01 = 0.5f * gB;
    const float t00 = gA * K00 + G01 * K01, t01 = gA * K01 + G01 * K11;  // (G K) rows
    const float t10 = G01 * K00 + gC * K01, t11 = G01 * K01 + gC * K11;
    const float h00 = -(K00 * t00 + K01 * t10), h01 = -(K00 * t01 + K01 * t11), h11 = -(K01 * t01 + K11 * t11);
    // dL/df_k from c00 = sum fx^2, c01 = sum fx fy (both off-diagonal slots), c11 = sum fy^2
    float dja0 = 0.0f, dja2 = 0.0f, djb1 = 0.0f, djb2 = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float dfx = 2.0f * (h00 * fx[k] + h01 * fy[k]);
        const float dfy = 2.0f * (h11 * fy[k] + h01 * fx[k]);
        ds[k] += dfx * (ja0 * M[k] + ja2 * M[6 + k]) + dfy * (jb1 * M[3 + k] + jb2 * M[6 + k]);
        dM[k] = dfx * s[k] * ja0;
        dM[3 + k] = dfy * s[k] * jb1;
        dM[6 + k] = s[k] * (dfx * ja2 + dfy * jb2);
        dja0 += dfx * s[k] * M[k];
        dja2 += dfx * s[k] * M[6 + k];
        djb1 += dfy * s[k] * M[3 + k];
        djb2 += dfy * s[k] * M[6 + k];
    }
    const float rx2 = rx * rx, ry2 = ry * ry;
    // J = (z, 0, -x) / (x^2 + z^2), (0, z, -y) / (y^2 + z^2); centre angles atan2(x, z), atan2(y, z)
    dmc[0] = dja0 * (-2.0f * x * z * rx2) + dja2 * ((x * x - z * z) * rx2) + gt * z * rx;
    dmc[1] = djb1 * (-2.0f * y * z * ry2) + djb2 * ((y * y - z * z) * ry2) + gp * z * ry;
    dmc[2] = dja0 * ((x * x - z * z) * rx2) + dja2 * (2.0f * x * z * rx2) + djb1 * ((y * y - z * z) * ry2) +
             djb2 * (2.0f * y * z * ry2) - gt * x * rx - gp * y * ry;
}

template <int DEG, bool ONE_CAM, bool SPLAT>
__global__ void __launch_bounds__(kPBThreads, ONE_CAM ? GEER_PB_MINB : 1) k_preprocess_bwd(
    const DevCam *__restrict__ cams, int ncams, const float *__restrict__ mean, const float *__restrict__ scale,
    const float *__restrict__ quat, const float *__restrict__ sh, int64_t n, const uint32_t *__restrict__ count,
    const GradAcc *__restrict__ gacc, float *__restrict__ d_mean, float *__restrict__ d_scale,
    float *__restrict__ d_quat, float *__restrict__ d_opacity, float *__restrict__ d_sh, int accumulate) {
    grid_dep_sync();
    constexpr int NB = (DEG + 1) * (DEG + 1), NC = 3 * NB, ST = NC | 1;
    __shared__ float s_sh[kPBThreads * ST];
    __shared__ float s_dsh[ONE_CAM ? 1 : kPBThreads * ST];
    __shared__ uint8_t s_live[kPBThreads];
    const int tid = threadIdx.x;
    const int64_t g0 = (int64_t)blockIdx.x * kPBThreads;
    const int nloc = (int)min((int64_t)kPBThreads, n - g0);
    {
        // asynchronous 4-byte copies into the padded rows: no registers held while
        // the block's rows are in flight
        const float *src = sh + g0 * NC;
        for (int i = tid; i < nloc * NC; i += kPBThreads) {
            const int gl = i / NC, k = i - gl * NC;
            cp_async4(&s_sh[gl * ST + k], src + i);
        }
        if (!ONE_CAM)
            for (int i = tid; i < kPBThreads * ST; i += kPBThreads) s_dsh[i] = 0.0f;
    }
    const int64_t g = g0 + tid;
    bool any = false;
    if (tid < nloc)
        for (int ci = 0; ci < ncams; ++ci) any |= count[(int64_t)ci * n + g] > 0;
    float mu[3], s[3], q[4];
    float4 pa[4];  // the one camera's accumulators, loaded with the parameters
    if (any) {  // a Gaussian not associated with any tile has no gradient
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mu[a] = mean[3 * g + a];
            s[a] = scale[3 * g + a];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) q[a] = quat[4 * g + a];
        if (ONE_CAM) {
            const float4 *ap = reinterpret_cast<const float4 *>(gacc + g);
#pragma unroll
            for (int k = 0; k < 4; ++k) pa[k] = ap[k];
        }
    }
    s_live[tid] = any ? 1 : 0;
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    const bool block_any = __syncthreads_or(any);
    if (!block_any && accumulate) return;
    if (any) {
        float *shc = s_sh + tid * ST;
        float *dsh = ONE_CAM ? shc : s_dsh + tid * ST;
        float is[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) is[a] = 1.0f / s[a];
        const float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        const float w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
        float R[9];
        R[0] = 1.0f - 2.0f * (y * y + z * z); R[1] = 2.0f * (x * y - w * z);        R[2] = 2.0f * (x * z + w * y);
        R[3] = 2.0f * (x * y + w * z);        R[4] = 1.0f - 2.0f * (x * x + z * z); R[5] = 2.0f * (y * z - w * x);
        R[6] = 2.0f * (x * z - w * y);        R[7] = 2.0f * (y * z + w * x);        R[8] = 1.0f - 2.0f * (x * x + y * y);
        float dmu[3] = {0, 0, 0}, ds[3] = {0, 0, 0}, dR[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, dsig = 0.0f;

        for (int ci = 0; ci < (ONE_CAM ? 1 : ncams); ++ci) {
            const int64_t idx = (int64_t)ci * n + g;
            if (!ONE_CAM && count[idx] == 0) continue;
            const DevCam &cam = cams[ci];
            float4 a0, a1, a2, a3;
            if (ONE_CAM) {
                a0 = pa[0]; a1 = pa[1]; a2 = pa[2]; a3 = pa[3];
            } else {
                const float4 *ap = reinterpret_cast<const float4 *>(gacc + idx);
                a0 = ap[0]; a1 = ap[1]; a2 = ap[2]; a3 = ap[3];
            }
            dsig += a0.x;
            const float *Rc = cam.R;
            // camera-frame mean and Gaussian axes M = R_cw R (W = S^-1 M^T)
            float mc[3], M[9];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                mc[i] = Rc[3 * i] * mu[0] + Rc[3 * i + 1] * mu[1] + Rc[3 * i + 2] * mu[2] + cam.t[i];
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    M[3 * i + j] = Rc[3 * i] * R[j] + Rc[3 * i + 1] * R[3 + j] + Rc[3 * i + 2] * R[6 + j];
            }
            float dmc[3], dM[9];
            if (SPLAT) {
                splat_chain(mc, M, s, a1.x, a1.y, a1.z, a1.w, a2.x, dmc, dM, ds);
            } else {
                const float dou[3] = {a3.y, a3.z, a3.w};
                const float dWr[9] = {a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w, a3.x};
                // o_u = -W mu_c: dL/dW = dW|RC - dL/do_u mu_c^T, dL/dmu_c = -W^T dL/do_u
                float dW[9];
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int i = 0; i < 3; ++i) dW[3 * k + i] = dWr[3 * k + i] - dou[k] * mc[i];
#pragma unroll
                for (int i = 0; i < 3; ++i)
                    dmc[i] = -(M[3 * i] * is[0] * dou[0] + M[3 * i + 1] * is[1] * dou[1] + M[3 * i + 2] * is[2] * dou[2]);
                // W_ki = M_ik / s_k: scales and the rotation
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    float acc_s = 0.0f;
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        acc_s += dW[3 * k + i] * M[3 * i + k];
                        dM[3 * i + k] = dW[3 * k + i] * is[k];
                    }
                    ds[k] -= acc_s * is[k] * is[k];
                }
            }
            // dL/dmu += R_cw^T dL/dmu_c
#pragma unroll
            for (int j = 0; j < 3; ++j) dmu[j] += Rc[j] * dmc[0] + Rc[3 + j] * dmc[1] + Rc[6 + j] * dmc[2];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    dR[3 * j + k] += Rc[j] * dM[k] + Rc[3 + j] * dM[3 + k] + Rc[6 + j] * dM[6 + k];
            // colour: SH at the world direction from the camera centre
            const float vx = mu[0] - cam.o[0], vy = mu[1] - cam.o[1], vz = mu[2] - cam.o[2];
            const float vn = sqrtf(vx * vx + vy * vy + vz * vz);
            ShDir u;
            u.x = vx / vn; u.y = vy / vn; u.z = vz / vn;
            u.xx = u.x * u.x; u.yy = u.y * u.y; u.zz = u.z * u.z;
            const float drgb[3] = {a0.y, a0.z, a0.w};
            float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const float Yk = sh_value(k, u);
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) raw[ch] += Yk * shc[3 * k + ch];
            }
            float dLdc[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) dLdc[ch] = raw[ch] > 0.0f ? drgb[ch] : 0.0f;
            float ddir[3] = {0, 0, 0};
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const float Yk = sh_value(k, u);
                float gk[3];
                sh_grad(k, u, gk);
                float wk = 0.0f;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    wk += dLdc[ch] * shc[3 * k + ch];
                    if (ONE_CAM) dsh[3 * k + ch] = dLdc[ch] * Yk;  // slot read just above
                    else dsh[3 * k + ch] += dLdc[ch] * Yk;
                }
                ddir[0] += wk * gk[0];
                ddir[1] += wk * gk[1];
                ddir[2] += wk * gk[2];
            }
            const float dp = ddir[0] * u.x + ddir[1] * u.y + ddir[2] * u.z;
            dmu[0] += (ddir[0] - u.x * dp) / vn;
            dmu[1] += (ddir[1] - u.y * dp) / vn;
            dmu[2] += (ddir[2] - u.z * dp) / vn;
        }
        // unit-quaternion polynomial R(w, x, y, z) (App. C.4) then the normalisation
        const float gw = 2.0f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
        const float gx = 2.0f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.0f * x * dR[4] - w * dR[5] + z * dR[6] +
                                 w * dR[7] - 2.0f * x * dR[8]);
        const float gy = 2.0f * (-2.0f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] +
                                 z * dR[7] - 2.0f * y * dR[8]);
        const float gz = 2.0f * (-2.0f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.0f * z * dR[4] +
                                 y * dR[5] + x * dR[6] + y * dR[7]);
        const float proj = gw * w + gx * x + gy * y + gz * z;
        // accumulating: the previous gradients are all read before any is written,
        // so that their loads are in flight together
        float om[3] = {0, 0, 0}, os[3] = {0, 0, 0}, oq[4] = {0, 0, 0, 0}, oo = 0.0f;
        if (accumulate) {
            if (d_mean)
#pragma unroll
                for (int a = 0; a < 3; ++a) om[a] = d_mean[3 * g + a];
            if (d_scale)
#pragma unroll
                for (int a = 0; a < 3; ++a) os[a] = d_scale[3 * g + a];
            if (d_quat)
#pragma unroll
                for (int a = 0; a < 4; ++a) oq[a] = d_quat[4 * g + a];
            if (d_opacity) oo = d_opacity[g];
        }
        if (d_quat) {
            d_quat[4 * g + 0] = oq[0] + (gw - w * proj) / qn;
            d_quat[4 * g + 1] = oq[1] + (gx - x * proj) / qn;
            d_quat[4 * g + 2] = oq[2] + (gy - y * proj) / qn;
            d_quat[4 * g + 3] = oq[3] + (gz - z * proj) / qn;
        }
        if (d_mean)
#pragma unroll
            for (int a = 0; a < 3; ++a) d_mean[3 * g + a] = om[a] + dmu[a];
        if (d_scale)
#pragma unroll
            for (int a = 0; a < 3; ++a) d_scale[3 * g + a] = os[a] + ds[a];
        if (d_opacity) d_opacity[g] = oo + dsig;
    } else if (!accumulate && tid < nloc) {  // overwriting: no gradient is a zero gradient
        if (d_mean)
#pragma unroll
            for (int a = 0; a < 3; ++a) d_mean[3 * g + a] = 0.0f;
        if (d_scale)
#pragma unroll
            for (int a = 0; a < 3; ++a) d_scale[3 * g + a] = 0.0f;
        if (d_quat)
#pragma unroll
            for (int a = 0; a < 4; ++a) d_quat[4 * g + a] = 0.0f;
        if (d_opacity) d_opacity[g] = 0.0f;
    }
    __syncthreads();
    if (d_sh) {
        // accumulating, rows of Gaussians without a gradient are left untouched;
        // overwriting, they are zeroed
        const float *acc = ONE_CAM ? s_sh : s_dsh;
        float *dst = d_sh + g0 * NC;
#ifndef GEER_PB_BATCH
#define GEER_PB_BATCH 24
#endif
        constexpr int kBatch = GEER_PB_BATCH;  // values in flight per thread
        if (!accumulate) {
            for (int i = tid; i < nloc * NC; i += kPBThreads) {
                const int gl = i / NC;
                dst[i] = s_live[gl] ? acc[gl * ST + (i - gl * NC)] : 0.0f;
            }
            return;
        }
        for (int i0 = tid; i0 < nloc * NC; i0 += kBatch * kPBThreads) {
            float v[kBatch];
#pragma unroll
            for (int b = 0; b < kBatch; ++b) {
                const int i = i0 + b * kPBThreads, gl = i / NC;
                v[b] = (i < nloc * NC && s_live[gl]) ? dst[i] : 0.0f;
            }
#pragma unroll
            for (int b = 0; b < kBatch; ++b) {
                const int i = i0 + b * kPBThreads, gl = i / NC;
                if (i < nloc * NC && s_live[gl]) dst[i] = v[b] + acc[gl * ST + (i - gl * NC)];
            }
        }
    }
}

// L1 loss mean |C - target| over all values and its gradient sign(C - target)/m.
__global__ void __launch_bounds__(256) k_l1_grad(const float *__restrict__ pred, const float *__restrict__ target,
                                                 int64_t m, float *__restrict__ grad, float *__restrict__ loss) {
    grid_dep_sync();
    __shared__ float red[8];
    const float inv = 1.0f / (float)m;
    float acc = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = pred[i] - target[i];
        grad[i] = d > 0.0f ? inv : (d < 0.0f ? -inv : 0.0f);
        acc += fabsf(d);
    }
    if (loss) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.0f;
            for (int w = 0; w < 8; ++w) t += red[w];
            atomicAdd(loss, t * inv);
        }
    }
}

}  // namespace

cudaError_t launch_preprocess_bwd(const geer_workspace *ws, const geer_gaussians *g, float *d_mean, float *d_scale,
                                  float *d_quat, float *d_opacity, float *d_sh, int accumulate, cudaStream_t s) {
    if (g->n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((g->n + kPBThreads - 1) / kPBThreads);
    const bool splat = ws->params.alpha_model != GEER_ALPHA_EXACT;
#define GEER_PB_LAUNCH(D)                                                                                      \
    if (ws->n_cams == 1)                                                                                       \
        launch_k(splat ? k_preprocess_bwd<D, true, true> : k_preprocess_bwd<D, true, false>, dim3(blocks),     \
                 dim3(kPBThreads), 0, s, ws->d_cams, 1, g->mean, g->scale, g->quat, g->sh, g->n, ws->d_count,   \
                 ws->d_gacc, d_mean, d_scale, d_quat, d_opacity, d_sh, accumulate);                             \
    else                                                                                                       \
        launch_k(splat ? k_preprocess_bwd<D, false, true> : k_preprocess_bwd<D, false, false>, dim3(blocks),   \
                 dim3(kPBThreads), 0, s, ws->d_cams, ws->n_cams, g->mean, g->scale, g->quat, g->sh, g->n,       \
                 ws->d_count, ws->d_gacc, d_mean, d_scale, d_quat, d_opacity, d_sh, accumulate)
    switch (g->sh_degree) {
        case 0: GEER_PB_LAUNCH(0); break;
        case 1: GEER_PB_LAUNCH(1); break;
        case 2: GEER_PB_LAUNCH(2); break;
        default: GEER_PB_LAUNCH(3); break;
    }
#undef GEER_PB_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_l1_grad(const float *pred, const float *target, int64_t m, float *grad, float *loss,
                           int num_sms, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    if (loss) {
        cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), s);
        if (e != cudaSuccess) return e;
    }
    const int64_t blocks = std::min<int64_t>((m + 255) / 256, (int64_t)num_sms * 8);
    launch_k(k_l1_grad, dim3((unsigned)blocks), dim3(256), 0, s, pred, target, m, grad, loss);
    return cudaGetLastError();
}

}  // namespace geer
