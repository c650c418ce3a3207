// remap.cu -- resampling a BEAP render into the camera's native image (App. E,
// inverse interpolation, read in reverse: native pixel -> ray -> BEAP angles).
//
// Native intrinsics: square pixels, principal point at the image centre, and the
// focal length that maps the horizontal half field of view to w/2 (the same
// reading that fixes the BEAP grid's vertical field of view):
//   pinhole       x_p = f tan(theta) + c_x                (App. E)
//   fisheye (KB)  x_p = f phi_d / r tan(theta) + c_x,
//                 r = sqrt(tan^2 theta + tan^2 phi), phi = atan r,
//                 phi_d = phi (1 + k1 phi^2 + k2 phi^4 + k3 phi^6 + k4 phi^8)
//                 (equidistant: k = 0).
// A native pixel's ray inverts these (Newton on phi_d(phi) = r_d); its BEAP
// angles are theta = atan2(x, z), phi = atan(y / z), its BEAP coordinate
// u = theta / FoV_x w + w/2 - 1/2 (likewise v), and its colour the bilinear
// interpolation of the BEAP image there. Rays outside the BEAP grid (beyond half
// a pixel) or where the distortion cannot be inverted get the fill colour.
//
// The same pass can label each native pixel with its evaluation region: central
// when its ray's BEAP angles satisfy |theta| <= w / (2f), |phi| <= h / (2f) (f the
// native focal length), peripheral otherwise, none without a ray in the grid.
#include <cstring>

#include "geer_internal.cuh"

namespace geer {
namespace {

struct RemapCam {
    int32_t model, width, height, pad_;
    float f, fov_x, fov_y, phi_max;
    float k[4];
    float fill[3];
    float cen_th, cen_ph;  // central-region half angles w / (2f), h / (2f)
};

__device__ __forceinline__ float kb_poly(const float k[4], float p, float &dp) {
    const float p2 = p * p;
    const float s = 1.0f + p2 * (k[0] + p2 * (k[1] + p2 * (k[2] + p2 * k[3])));
    // d/dp of p s(p^2) = s + p * 2p s'(p^2)
    const float ds = k[0] + p2 * (2.0f * k[1] + p2 * (3.0f * k[2] + p2 * 4.0f * k[3]));
    dp = s + 2.0f * p2 * ds;
    return p * s;
}

// beap / out NULL: regions only; regions NULL: image only.
__global__ void __launch_bounds__(256) k_remap_to_native(const float *__restrict__ beap, RemapCam c,
                                                         float *__restrict__ out, uint8_t *__restrict__ regions) {
    grid_dep_sync();
    const int64_t n = (int64_t)c.width * c.height;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int i = (int)(idx % c.width), j = (int)(idx / c.width);
    const float u = ((float)i + 0.5f - 0.5f * (float)c.width) / c.f;
    const float v = ((float)j + 0.5f - 0.5f * (float)c.height) / c.f;
    float dx, dy, dz;
    bool ok = true;
    if (c.model == GEER_PINHOLE) {
        dx = u; dy = v; dz = 1.0f;
    } else {
        const float rd = sqrtf(u * u + v * v);
        float p = rd;  // Newton on phi_d(phi) = rd from phi = rd
        for (int it = 0; it < 12; ++it) {
            float dp;
            const float val = kb_poly(c.k, p, dp);
            if (!(dp > 0.0f)) { ok = false; break; }
            p = fminf(fmaxf(p - (val - rd) / dp, 0.0f), c.phi_max);
        }
        float dp;
        if (ok && fabsf(kb_poly(c.k, p, dp) - rd) > 1e-5f * (1.0f + rd)) ok = false;
        const float sp = sinf(p), cp = cosf(p);
        if (rd > 0.0f) { dx = sp * u / rd; dy = sp * v / rd; } else { dx = 0.0f; dy = 0.0f; }
        dz = cp;
    }
    float r = c.fill[0], g = c.fill[1], b = c.fill[2];
    uint8_t region = kRegionNone;
    if (ok && dz != 0.0f) {
        const float th = atan2f(dx, dz);
        const float ph = atanf(dy / dz);
        const float ub = th / c.fov_x * (float)c.width + 0.5f * (float)c.width - 0.5f;
        const float vb = ph / c.fov_y * (float)c.height + 0.5f * (float)c.height - 0.5f;
        if (ub >= -0.5f && ub <= (float)c.width - 0.5f && vb >= -0.5f && vb <= (float)c.height - 0.5f && beap) {
            const float uc = fminf(fmaxf(ub, 0.0f), (float)(c.width - 1));
            const float vc = fminf(fmaxf(vb, 0.0f), (float)(c.height - 1));
            const int x0 = min((int)uc, c.width - 2 < 0 ? 0 : c.width - 2);
            const int y0 = min((int)vc, c.height - 2 < 0 ? 0 : c.height - 2);
            const int x1 = min(x0 + 1, c.width - 1), y1 = min(y0 + 1, c.height - 1);
            const float ax = uc - (float)x0, ay = vc - (float)y0;
            const float *p00 = beap + 3 * ((int64_t)y0 * c.width + x0);
            const float *p01 = beap + 3 * ((int64_t)y0 * c.width + x1);
            const float *p10 = beap + 3 * ((int64_t)y1 * c.width + x0);
            const float *p11 = beap + 3 * ((int64_t)y1 * c.width + x1);
            float o[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float top = p00[ch] + ax * (p01[ch] - p00[ch]);
                const float bot = p10[ch] + ax * (p11[ch] - p10[ch]);
                o[ch] = top + ay * (bot - top);
            }
            r = o[0]; g = o[1]; b = o[2];
        }
        if (ub >= -0.5f && ub <= (float)c.width - 0.5f && vb >= -0.5f && vb <= (float)c.height - 0.5f)
            region = (fabsf(th) <= c.cen_th && fabsf(ph) <= c.cen_ph) ? kRegionCentral : kRegionPeripheral;
    }
    if (out) {
        out[3 * idx + 0] = r;
        out[3 * idx + 1] = g;
        out[3 * idx + 2] = b;
    }
    if (regions) regions[idx] = region;
}

// The supervision of a BEAP render from a native image (BEAP ray sampling with
// ground-truth interpolation): each BEAP pixel's ray (Sec. 3.3) projected into
// the native image (App. E with the intrinsics above: pinhole f (x, y) / z;
// fisheye f phi_d(p) (x, y) / sqrt(x^2 + y^2) with the polar angle
// p = atan2(sqrt(x^2 + y^2), z) on the invertible branch) and the native image
// interpolated bilinearly at pixel-centre coordinates; valid 0 where the point
// is not within half a pixel of the image or the ray has no projection.
__global__ void __launch_bounds__(256) k_native_to_beap(const float *__restrict__ native, RemapCam c,
                                                        float *__restrict__ beap, uint8_t *__restrict__ valid) {
    grid_dep_sync();
    const int64_t n = (int64_t)c.width * c.height;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int i = (int)(idx % c.width), j = (int)(idx / c.width);
    const float th = (((float)i + 0.5f) / (float)c.width - 0.5f) * c.fov_x;
    const float ph = (((float)j + 0.5f) / (float)c.height - 0.5f) * c.fov_y;
    float st, ct, sp, cp;
    sincosf(th, &st, &ct);
    sincosf(ph, &sp, &cp);
    const float dx = st * cp, dy = ct * sp, dz = ct * cp;
    bool ok;
    float x = 0.0f, y = 0.0f;
    if (c.model == GEER_PINHOLE) {
        ok = dz > 0.0f;
        if (ok) { x = c.f * dx / dz; y = c.f * dy / dz; }
    } else {
        const float rho = sqrtf(dx * dx + dy * dy);
        const float p = atan2f(rho, dz);
        ok = p <= c.phi_max;
        if (ok && rho > 0.0f) {
            float dp;
            const float s = c.f * kb_poly(c.k, p, dp) / rho;
            x = s * dx;
            y = s * dy;
        }
    }
    const float u = x + 0.5f * (float)c.width - 0.5f, v = y + 0.5f * (float)c.height - 0.5f;
    ok = ok && u >= -0.5f && u <= (float)c.width - 0.5f && v >= -0.5f && v <= (float)c.height - 0.5f;
    float o[3] = {0.0f, 0.0f, 0.0f};
    if (ok) {
        const float uc = fminf(fmaxf(u, 0.0f), (float)(c.width - 1));
        const float vc = fminf(fmaxf(v, 0.0f), (float)(c.height - 1));
        const int x0 = min((int)uc, c.width - 2 < 0 ? 0 : c.width - 2);
        const int y0 = min((int)vc, c.height - 2 < 0 ? 0 : c.height - 2);
        const int x1 = min(x0 + 1, c.width - 1), y1 = min(y0 + 1, c.height - 1);
        const float ax = uc - (float)x0, ay = vc - (float)y0;
        const float *p00 = native + 3 * ((int64_t)y0 * c.width + x0);
        const float *p01 = native + 3 * ((int64_t)y0 * c.width + x1);
        const float *p10 = native + 3 * ((int64_t)y1 * c.width + x0);
        const float *p11 = native + 3 * ((int64_t)y1 * c.width + x1);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float top = p00[ch] + ax * (p01[ch] - p00[ch]);
            const float bot = p10[ch] + ax * (p11[ch] - p10[ch]);
            o[ch] = top + ay * (bot - top);
        }
    }
    beap[3 * idx + 0] = o[0];
    beap[3 * idx + 1] = o[1];
    beap[3 * idx + 2] = o[2];
    if (valid) valid[idx] = ok ? 1 : 0;
}

}  // namespace

cudaError_t launch_native_to_beap(const float *native, const geer_camera *cam, double fov_y, double focal,
                                  double phi_max, float *beap, uint8_t *valid, cudaStream_t s) {
    RemapCam c;
    memset(&c, 0, sizeof(c));
    c.model = cam->model;
    c.width = cam->width;
    c.height = cam->height;
    c.f = (float)focal;
    c.fov_x = cam->fov_x;
    c.fov_y = (float)fov_y;
    c.phi_max = (float)phi_max;
    for (int i = 0; i < 4; ++i) c.k[i] = cam->model == GEER_KANNALA_BRANDT ? cam->k[i] : 0.0f;
    const int64_t n = (int64_t)cam->width * cam->height;
    if (n == 0) return cudaSuccess;
    launch_k(k_native_to_beap, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, s, native, c, beap, valid);
    return cudaGetLastError();
}

cudaError_t launch_remap_to_native(const float *beap, const geer_camera *cam, double fov_y, double focal,
                                   double phi_max, const float *fill, float *out, uint8_t *regions, cudaStream_t s) {
    RemapCam c;
    c.model = cam->model;
    c.width = cam->width;
    c.height = cam->height;
    c.pad_ = 0;
    c.f = (float)focal;
    c.fov_x = cam->fov_x;
    c.fov_y = (float)fov_y;
    c.phi_max = (float)phi_max;
    for (int i = 0; i < 4; ++i) c.k[i] = cam->model == GEER_KANNALA_BRANDT ? cam->k[i] : 0.0f;
    for (int i = 0; i < 3; ++i) c.fill[i] = fill ? fill[i] : 0.0f;
    c.cen_th = (float)(0.5 * cam->width / focal);
    c.cen_ph = (float)(0.5 * cam->height / focal);
    const int64_t n = (int64_t)cam->width * cam->height;
    if (n == 0) return cudaSuccess;
    launch_k(k_remap_to_native, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, s, beap, c, out, regions);
    return cudaGetLastError();
}

}  // namespace geer
