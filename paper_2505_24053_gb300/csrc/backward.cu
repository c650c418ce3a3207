// backward.cu -- PreprocessCUDA backward (App. C): per Gaussian, sum over the
// cameras of the chain from the render-stage accumulators to the parameters.
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

// Real SH basis (3DGS convention, as in the forward) and its gradient with
// respect to the (unit) direction components.
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, float Y[16], float dY[16][3]) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        Y[k] = 0.0f;
        dY[k][0] = dY[k][1] = dY[k][2] = 0.0f;
    }
    Y[0] = 0.28209479177387814f;
    if (deg >= 1) {
        const float k1 = 0.4886025119029199f;
        Y[1] = -k1 * y; dY[1][1] = -k1;
        Y[2] = k1 * z;  dY[2][2] = k1;
        Y[3] = -k1 * x; dY[3][0] = -k1;
    }
    if (deg >= 2) {
        const float a = 1.0925484305920792f, b = 0.31539156525252005f, c = 0.5462742152960396f;
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = a * x * y;                  dY[4][0] = a * y;  dY[4][1] = a * x;
        Y[5] = -a * y * z;                 dY[5][1] = -a * z; dY[5][2] = -a * y;
        Y[6] = b * (2.0f * zz - xx - yy);  dY[6][0] = -2.0f * b * x; dY[6][1] = -2.0f * b * y; dY[6][2] = 4.0f * b * z;
        Y[7] = -a * x * z;                 dY[7][0] = -a * z; dY[7][2] = -a * x;
        Y[8] = c * (xx - yy);              dY[8][0] = 2.0f * c * x; dY[8][1] = -2.0f * c * y;
        if (deg >= 3) {
            const float e = 0.5900435899266435f, f = 2.890611442640554f, h = 0.4570457994644658f;
            const float pp = 0.3731763325901154f, r = 1.445305721320277f;
            Y[9] = -e * y * (3.0f * xx - yy);
            dY[9][0] = -6.0f * e * x * y; dY[9][1] = -e * (3.0f * xx - 3.0f * yy);
            Y[10] = f * x * y * z;
            dY[10][0] = f * y * z; dY[10][1] = f * x * z; dY[10][2] = f * x * y;
            Y[11] = -h * y * (4.0f * zz - xx - yy);
            dY[11][0] = 2.0f * h * x * y; dY[11][1] = -h * (4.0f * zz - xx - 3.0f * yy); dY[11][2] = -8.0f * h * y * z;
            Y[12] = pp * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
            dY[12][0] = -6.0f * pp * x * z; dY[12][1] = -6.0f * pp * y * z;
            dY[12][2] = pp * (6.0f * zz - 3.0f * xx - 3.0f * yy);
            Y[13] = -h * x * (4.0f * zz - xx - yy);
            dY[13][0] = -h * (4.0f * zz - 3.0f * xx - yy); dY[13][1] = 2.0f * h * x * y; dY[13][2] = -8.0f * h * x * z;
            Y[14] = r * z * (xx - yy);
            dY[14][0] = 2.0f * r * x * z; dY[14][1] = -2.0f * r * y * z; dY[14][2] = r * (xx - yy);
            Y[15] = -e * x * (xx - 3.0f * yy);
            dY[15][0] = -e * (3.0f * xx - 3.0f * yy); dY[15][1] = 6.0f * e * x * y;
        }
    }
}

// One block per 64 Gaussians. The block's SH coefficients and its slice of
// dL/dsh are staged through shared memory with coalesced loads (row stride made
// odd so that per-thread rows do not share banks); each thread then runs the
// chain for its Gaussian over the cameras, adds its SH gradient in shared
// memory, and the block writes dL/dsh back coalesced.
constexpr int kPBThreads = 64;

template <int DEG>
__global__ void __launch_bounds__(kPBThreads) k_preprocess_bwd(
    const DevCam *__restrict__ cams, int ncams, const float *__restrict__ mean, const float *__restrict__ scale,
    const float *__restrict__ quat, const float *__restrict__ sh, int64_t n, const uint32_t *__restrict__ count,
    const GradAcc *__restrict__ gacc, float *__restrict__ d_mean, float *__restrict__ d_scale,
    float *__restrict__ d_quat, float *__restrict__ d_opacity, float *__restrict__ d_sh) {
    constexpr int NB = (DEG + 1) * (DEG + 1), NC = 3 * NB, ST = NC | 1;
    __shared__ float s_sh[kPBThreads * ST];
    __shared__ float s_dsh[kPBThreads * ST];
    const int tid = threadIdx.x;
    const int64_t g0 = (int64_t)blockIdx.x * kPBThreads;
    const int nloc = (int)min((int64_t)kPBThreads, n - g0);
    {
        const float *src = sh + g0 * NC;
        const float *dsrc = d_sh ? d_sh + g0 * NC : nullptr;
        if (nloc == kPBThreads) {
            // a full block's rows are kPBThreads * NC * 4 bytes (a multiple of 16) from a
            // 16-byte aligned base: all its 16-byte loads are issued before any is used
            constexpr int kF = kPBThreads * NC / 4;                // float4 in the block's rows
            constexpr int kV = (kF + kPBThreads - 1) / kPBThreads;  // per thread
            float4 a[kV], b[kV];
#pragma unroll
            for (int u = 0; u < kV; ++u) {
                if (u * kPBThreads + tid < kF) {
                    a[u] = reinterpret_cast<const float4 *>(src)[u * kPBThreads + tid];
                    if (dsrc) b[u] = reinterpret_cast<const float4 *>(dsrc)[u * kPBThreads + tid];
                }
            }
#pragma unroll
            for (int u = 0; u < kV; ++u) {
                if (u * kPBThreads + tid >= kF) continue;
                const int i = 4 * (u * kPBThreads + tid);
                const float va[4] = {a[u].x, a[u].y, a[u].z, a[u].w};
                const float vb[4] = {b[u].x, b[u].y, b[u].z, b[u].w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int gl = (i + q) / NC, k = i + q - gl * NC;
                    s_sh[gl * ST + k] = va[q];
                    if (dsrc) s_dsh[gl * ST + k] = vb[q];
                }
            }
        } else {
            for (int i = tid; i < nloc * NC; i += kPBThreads) {
                const int gl = i / NC, k = i - gl * NC;
                s_sh[gl * ST + k] = src[i];
                if (dsrc) s_dsh[gl * ST + k] = dsrc[i];
            }
        }
    }
    __syncthreads();
    const int64_t g = g0 + tid;
    bool any = false;
    if (tid < nloc)
        for (int ci = 0; ci < ncams; ++ci) any |= count[(int64_t)ci * n + g] > 0;
    if (any) {  // a Gaussian not associated with any tile has no gradient
        const float *shc = s_sh + tid * ST;
        float *dsh = s_dsh + tid * ST;
        float mu[3], s[3], is[3], q[4];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mu[a] = mean[3 * g + a];
            s[a] = scale[3 * g + a];
            is[a] = 1.0f / s[a];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) q[a] = quat[4 * g + a];
        const float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        const float w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
        float R[9];
        R[0] = 1.0f - 2.0f * (y * y + z * z); R[1] = 2.0f * (x * y - w * z);        R[2] = 2.0f * (x * z + w * y);
        R[3] = 2.0f * (x * y + w * z);        R[4] = 1.0f - 2.0f * (x * x + z * z); R[5] = 2.0f * (y * z - w * x);
        R[6] = 2.0f * (x * z - w * y);        R[7] = 2.0f * (y * z + w * x);        R[8] = 1.0f - 2.0f * (x * x + y * y);
        float dmu[3] = {0, 0, 0}, ds[3] = {0, 0, 0}, dR[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, dsig = 0.0f;

        for (int ci = 0; ci < ncams; ++ci) {
            const int64_t idx = (int64_t)ci * n + g;
            if (count[idx] == 0) continue;
            const DevCam &cam = cams[ci];
            const float4 *ap = reinterpret_cast<const float4 *>(gacc + idx);
            const float4 a0 = ap[0], a1 = ap[1], a2 = ap[2], a3 = ap[3];
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
            const float dou[3] = {a3.y, a3.z, a3.w};
            const float dWr[9] = {a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w, a3.x};
            // o_u = -W mu_c: dL/dW = dW|RC - dL/do_u mu_c^T, dL/dmu_c = -W^T dL/do_u, dL/dmu += R_cw^T dL/dmu_c
            float dW[9], dmc[3];
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int i = 0; i < 3; ++i) dW[3 * k + i] = dWr[3 * k + i] - dou[k] * mc[i];
#pragma unroll
            for (int i = 0; i < 3; ++i)
                dmc[i] = -(M[3 * i] * is[0] * dou[0] + M[3 * i + 1] * is[1] * dou[1] + M[3 * i + 2] * is[2] * dou[2]);
#pragma unroll
            for (int j = 0; j < 3; ++j) dmu[j] += Rc[j] * dmc[0] + Rc[3 + j] * dmc[1] + Rc[6 + j] * dmc[2];
            // W_ki = M_ik / s_k: scales and the rotation
            float dM[9];
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
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    dR[3 * j + k] += Rc[j] * dM[k] + Rc[3 + j] * dM[3 + k] + Rc[6 + j] * dM[6 + k];
            // colour: SH at the world direction from the camera centre
            const float vx = mu[0] - cam.o[0], vy = mu[1] - cam.o[1], vz = mu[2] - cam.o[2];
            const float vn = sqrtf(vx * vx + vy * vy + vz * vz);
            const float ux = vx / vn, uy = vy / vn, uz = vz / vn;
            float Y[16], dY[16][3];
            sh_basis_grad(DEG, ux, uy, uz, Y, dY);
            const float drgb[3] = {a0.y, a0.z, a0.w};
            float dLdc[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float raw = 0.5f;
#pragma unroll
                for (int k = 0; k < NB; ++k) raw += Y[k] * shc[3 * k + ch];
                dLdc[ch] = raw > 0.0f ? drgb[ch] : 0.0f;
            }
            float ddir[3] = {0, 0, 0};
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                float wk = 0.0f;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    dsh[3 * k + ch] += dLdc[ch] * Y[k];
                    wk += dLdc[ch] * shc[3 * k + ch];
                }
                ddir[0] += wk * dY[k][0];
                ddir[1] += wk * dY[k][1];
                ddir[2] += wk * dY[k][2];
            }
            const float dp = ddir[0] * ux + ddir[1] * uy + ddir[2] * uz;
            dmu[0] += (ddir[0] - ux * dp) / vn;
            dmu[1] += (ddir[1] - uy * dp) / vn;
            dmu[2] += (ddir[2] - uz * dp) / vn;
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
        if (d_quat) {
            d_quat[4 * g + 0] += (gw - w * proj) / qn;
            d_quat[4 * g + 1] += (gx - x * proj) / qn;
            d_quat[4 * g + 2] += (gy - y * proj) / qn;
            d_quat[4 * g + 3] += (gz - z * proj) / qn;
        }
        if (d_mean)
#pragma unroll
            for (int a = 0; a < 3; ++a) d_mean[3 * g + a] += dmu[a];
        if (d_scale)
#pragma unroll
            for (int a = 0; a < 3; ++a) d_scale[3 * g + a] += ds[a];
        if (d_opacity) d_opacity[g] += dsig;
    }
    __syncthreads();
    if (d_sh) {
        float *dst = d_sh + g0 * NC;
        for (int i = tid; i < nloc * NC; i += kPBThreads) {
            const int gl = i / NC, k = i - gl * NC;
            dst[i] = s_dsh[gl * ST + k];
        }
    }
}

// L1 loss mean |C - target| over all values and its gradient sign(C - target)/m.
__global__ void __launch_bounds__(256) k_l1_grad(const float *__restrict__ pred, const float *__restrict__ target,
                                                 int64_t m, float *__restrict__ grad, float *__restrict__ loss) {
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
                                  float *d_quat, float *d_opacity, float *d_sh, cudaStream_t s) {
    if (g->n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((g->n + kPBThreads - 1) / kPBThreads);
#define GEER_PB_LAUNCH(D)                                                                                      \
    k_preprocess_bwd<D><<<blocks, kPBThreads, 0, s>>>(ws->d_cams, ws->n_cams, g->mean, g->scale, g->quat, g->sh, \
                                                      g->n, ws->d_count, ws->d_gacc, d_mean, d_scale, d_quat,   \
                                                      d_opacity, d_sh)
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
    k_l1_grad<<<(unsigned)blocks, 256, 0, s>>>(pred, target, m, grad, loss);
    return cudaGetLastError();
}

}  // namespace geer
