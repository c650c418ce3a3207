// metrics.cu -- evaluation of a native-camera image against a reference image
// (the paper's evaluation of renders reprojected to the native fisheye image):
// per region, the sum of squared errors over pixels and channels, the sum of
// the per-pixel SSIM (mean over the three channels) and the pixel count.
//
// SSIM (Wang et al. 2004, as 3DGS-style evaluations compute it): local means,
// variances and covariance under an 11 x 11 Gaussian window (sigma 1.5,
// normalised), zero padding at the image border, C1 = 0.01^2, C2 = 0.03^2 for
// values in [0, 1]. A block takes a 16 x 16 tile: the tile and a 5-pixel halo of
// both images are staged in shared memory, the window is applied as a
// horizontal then a vertical 11-tap pass to the five quantities x, y, x^2, y^2,
// xy of each channel, and the block's sums per region are added to FP64
// accumulators with one atomic each.
#include "geer_internal.cuh"

namespace geer {
namespace {

constexpr int kMT = 16;                // output tile edge
constexpr int kHalo = 5;               // window radius
constexpr int kIn = kMT + 2 * kHalo;   // staged tile edge
constexpr int kQ = 15;                 // 5 quantities x 3 channels
constexpr int kMaxRegions = 8;

__global__ void __launch_bounds__(kMT * kMT) k_image_metrics(const float *__restrict__ pred,
                                                             const float *__restrict__ gt, int w, int h,
                                                             const uint8_t *__restrict__ regions, int nreg,
                                                             double *__restrict__ acc) {
    grid_dep_sync();
    __shared__ float sx[3][kIn][kIn], sy[3][kIn][kIn];
    __shared__ float hs[kQ][kIn][kMT];
    __shared__ float gw[2 * kHalo + 1];
    __shared__ float red[kMT * kMT / 32][kMaxRegions][3];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = (int)blockIdx.x * kMT - kHalo, y0 = (int)blockIdx.y * kMT - kHalo;
    if (tid < 2 * kHalo + 1) {
        const float k = (float)(tid - kHalo);
        gw[tid] = expf(-k * k / (2.0f * 1.5f * 1.5f));
    }
    for (int i = tid; i < kIn * kIn; i += kMT * kMT) {
        const int iy = i / kIn, ix = i - iy * kIn, gx = x0 + ix, gy = y0 + iy;
        const bool in = gx >= 0 && gx < w && gy >= 0 && gy < h;
        const int64_t p = (int64_t)gy * w + gx;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            sx[ch][iy][ix] = in ? pred[3 * p + ch] : 0.0f;
            sy[ch][iy][ix] = in ? gt[3 * p + ch] : 0.0f;
        }
    }
    __syncthreads();
    if (tid == 0) {
        float s = 0.0f;
        for (int k = 0; k < 2 * kHalo + 1; ++k) s += gw[k];
        for (int k = 0; k < 2 * kHalo + 1; ++k) gw[k] /= s;
    }
    __syncthreads();
    // horizontal pass: rows of the staged tile, the block's 16 output columns
    for (int o = tid; o < kIn * kMT; o += kMT * kMT) {
        const int r = o / kMT, c = o - r * kMT;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float m0 = 0, m1 = 0, m2 = 0, m3 = 0, m4 = 0;
#pragma unroll
            for (int k = 0; k < 2 * kHalo + 1; ++k) {
                const float a = sx[ch][r][c + k], b = sy[ch][r][c + k], g = gw[k];
                m0 = fmaf(g, a, m0);
                m1 = fmaf(g, b, m1);
                m2 = fmaf(g, a * a, m2);
                m3 = fmaf(g, b * b, m3);
                m4 = fmaf(g, a * b, m4);
            }
            hs[5 * ch + 0][r][c] = m0;
            hs[5 * ch + 1][r][c] = m1;
            hs[5 * ch + 2][r][c] = m2;
            hs[5 * ch + 3][r][c] = m3;
            hs[5 * ch + 4][r][c] = m4;
        }
    }
    __syncthreads();
    // vertical pass and SSIM for this thread's pixel
    const int py = tid / kMT, px = tid - py * kMT;
    const int gx = (int)blockIdx.x * kMT + px, gy = (int)blockIdx.y * kMT + py;
    int reg = -1;
    float se = 0.0f, ss = 0.0f;
    if (gx < w && gy < h) {
        const int64_t p = (int64_t)gy * w + gx;
        reg = regions ? (int)regions[p] : 0;
        if (reg >= nreg) reg = -1;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float m[5] = {0, 0, 0, 0, 0};
#pragma unroll
            for (int k = 0; k < 2 * kHalo + 1; ++k) {
                const float g = gw[k];
#pragma unroll
                for (int q = 0; q < 5; ++q) m[q] = fmaf(g, hs[5 * ch + q][py + k][px], m[q]);
            }
            const float mx = m[0], my = m[1];
            const float vx = m[2] - mx * mx, vy = m[3] - my * my, cxy = m[4] - mx * my;
            const float c1 = 0.01f * 0.01f, c2 = 0.03f * 0.03f;
            ss += ((2.0f * mx * my + c1) * (2.0f * cxy + c2)) / ((mx * mx + my * my + c1) * (vx + vy + c2));
            const float d = sx[ch][py + kHalo][px + kHalo] - sy[ch][py + kHalo][px + kHalo];
            se = fmaf(d, d, se);
        }
        ss *= 1.0f / 3.0f;
    }
    // block sums per region
    for (int r = 0; r < nreg; ++r) {
        float a = reg == r ? se : 0.0f, b = reg == r ? ss : 0.0f, c = reg == r ? 1.0f : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        if (lane == 0) {
            red[warp][r][0] = a;
            red[warp][r][1] = b;
            red[warp][r][2] = c;
        }
    }
    __syncthreads();
    if (tid < 3 * nreg) {
        const int r = tid / 3, q = tid - 3 * r;
        double t = 0.0;
        for (int v = 0; v < kMT * kMT / 32; ++v) t += (double)red[v][r][q];
        if (t != 0.0) atomicAdd(&acc[3 * r + q], t);
    }
}

}  // namespace

cudaError_t launch_image_metrics(const float *pred, const float *gt, int width, int height, const uint8_t *regions,
                                 int n_regions, double *acc, cudaStream_t s) {
    if (n_regions < 1 || n_regions > kMaxRegions) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * 3 * n_regions, s);
    if (e != cudaSuccess || width == 0 || height == 0) return e;
    launch_k(k_image_metrics, dim3((unsigned)((width + kMT - 1) / kMT), (unsigned)((height + kMT - 1) / kMT)),
             dim3(kMT * kMT), 0, s, pred, gt, width, height, regions, n_regions, acc);
    return cudaGetLastError();
}

}  // namespace geer
