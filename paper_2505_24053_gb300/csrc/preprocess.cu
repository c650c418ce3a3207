// preprocess.cu -- per-Gaussian preprocessing (Algorithm 1: CullGaussian,
// ViewspaceGaussians, PBF_Intersect, PCA_Whitening), the pair-count scan and
// DuplicateWithKeys.
//
// The PBF part runs in exactly rounded FP32 operations in a fixed order
// (__fmul_rn / __fadd_rn / __fsub_rn / __fdiv_rn / __fsqrt_rn, which the
// compiler never contracts), so the tile ranges and depth keys are bit-for-bit
// reproducible by an independent FP32 implementation of the same sequence.
#include <algorithm>

#include "geer_internal.cuh"

namespace geer {
namespace {

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fsq(float a) { return __fsqrt_rn(a); }

// An arc of dihedral angle in half-angle-tangent space tau = tan(angle / 2)
// (the mirror transform with xi = 1, App. D.2). kind 0 empty, 1 [lo, hi],
// 2 wrapping [lo, +inf) u (-inf, hi], 3 full circle.
struct Arc {
    int kind;
    float lo, hi;
};

// tan(angle/2) of the planar direction (x, z), angle measured from +z towards +x.
__device__ float half_tan(float x, float z) {
    float r = fsq(fa(fm(x, x), fm(z, z)));
    return (z >= 0.0f) ? fdv(x, fa(r, z)) : fdv(fs(r, z), x);
}

// PBF bounds about one camera axis (Sec. 3.2, App. D.1): the bounding planes
// through the axis have tangent c solving T22 c^2 - 2 T02 c + T00 = 0 with
// T = lambda^2 Sigma_c - mu_c mu_c^T. The discriminant T02^2 - T00 T22 equals
// lambda^2 (P - lambda^2 D) with P = mu^T adj(Sigma_pp) mu and D = det(Sigma_pp),
// evaluated without cancellation. No real root: the axis pierces the ellipsoid
// and the arc is the full circle (clamp to the full FoV, App. D.1). The four
// mirrored candidates are reduced to the two nearest the centre's mirrored
// angle (App. D.2) and widened by a 2^-18 (1 + tau^2) margin.
__device__ Arc pbf_arc(float mx, float mz, float T00, float T02, float T22, float P, float D, float lam2) {
    Arc a{3, 0.0f, 0.0f};
    float disc = fm(lam2, fs(P, fm(lam2, D)));
    if (!(disc > 0.0f)) return a;
    float sq = fsq(disc);
    float qq = fa(T02, (T02 >= 0.0f) ? sq : -sq);
    if (qq == 0.0f) return a;
    float cand[4];
    cand[0] = half_tan(qq, T22);
    cand[1] = half_tan(-qq, -T22);
    cand[2] = half_tan(T00, qq);
    cand[3] = half_tan(-T00, -qq);
    float tm = half_tan(mx, mz);
    if (!isfinite(tm)) return a;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (!isfinite(cand[i])) return a;
    bool have_lo = false, have_hi = false;
    float lo = 0.0f, hi = 0.0f, mn = cand[0], mxv = cand[0];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float v = cand[i];
        if (v < mn) mn = v;
        if (v > mxv) mxv = v;
        if (v < tm && (!have_lo || v > lo)) { lo = v; have_lo = true; }
        if (v > tm && (!have_hi || v < hi)) { hi = v; have_hi = true; }
    }
    a.kind = 1;
    if (!have_hi) { hi = mn; a.kind = 2; }
    if (!have_lo) { lo = mxv; a.kind = 2; }
    const float margin = 3.814697265625e-06f;  // 2^-18
    a.lo = fs(lo, fm(margin, fa(1.0f, fm(lo, lo))));
    a.hi = fa(hi, fm(margin, fa(1.0f, fm(hi, hi))));
    return a;
}

// The arc rotated by pi (tau -> -1/tau), for rays whose other BEAP angle is
// beyond 90 degrees.
__device__ Arc shift_arc(Arc a) {
    Arc r = a;
    if (a.kind == 0 || a.kind == 3) return r;
    if (a.lo == 0.0f || a.hi == 0.0f) { r.kind = 3; return r; }
    r.lo = fdv(-1.0f, a.lo);
    r.hi = fdv(-1.0f, a.hi);
    if (a.kind == 2) r.kind = 1;
    else r.kind = (a.lo < 0.0f && a.hi > 0.0f) ? 2 : 1;
    return r;
}

// The first tile index k in [0, n] with pred(k) (false before, true from k on:
// pred is monotone in k), searched from a guess: the guess only sets where the
// probes start, so the result is exactly the first true index whatever the guess.
template <typename Pred>
__device__ __forceinline__ int first_true_from(int guess, int n, Pred pred) {
    int k = min(max(guess, 0), n);
    while (k > 0 && pred(k - 1)) --k;
    while (k < n && !pred(k)) ++k;
    return k;
}

// Tile range [lo, hi) whose half-angle span [ta, tb] (tab[i].x, tab[i].y, both
// increasing in i) meets the arc; prefix u suffix becomes the whole range. BEAP
// angles are linear in the pixel index (Sec. 3.3), so the pixel of a bound tau
// is about (2 atan(tau)) * ppr + (w - 1) / 2: that tile is the first probe
// (ppr: pixels per radian, half: (w - 1) / 2), and a probe or two more find the
// first index of each condition exactly.
__device__ void arc_range(Arc a, const float4 *tab, int n, float ppr, float half, int &olo, int &ohi) {
    olo = 0;
    ohi = 0;
    if (a.kind == 0) return;
    if (a.kind == 3) { ohi = n; return; }
    const float plo = fmaf(2.0f * atanf(a.lo), ppr, half), phi = fmaf(2.0f * atanf(a.hi), ppr, half);
    // first index with tb >= a.lo (tb: the tile's last ray), then first with ta > a.hi
    const int first = first_true_from((int)floorf((plo - (kTile - 1)) / kTile), n,
                                      [&](int k) { return tab[k].y >= a.lo; });
    const int last = first_true_from((int)floorf(phi / kTile) + 1, n,
                                     [&](int k) { return tab[k].x > a.hi; }) - 1;
    if (a.kind == 1) {
        if (first <= last) { olo = first; ohi = last + 1; }
        return;
    }
    bool suf = first < n, pre = last >= 0;
    if (suf && pre) { olo = 0; ohi = n; }
    else if (suf) { olo = first; ohi = n; }
    else if (pre) { olo = 0; ohi = last + 1; }
}

// lambda^2 >= 2 ln(sigma / alpha_min) with basic operations only, times (1 + pad):
// ln m <= 2 (z + z^3 / (3 (1 - z^2))), z = (m - 1)/(m + 1), m in [1, 2).
__device__ float lambda2(float sigma, float alpha_min, float pad) {
    float x = fdv(sigma, alpha_min);
    int e;
    float m = frexpf(x, &e);
    m = fm(m, 2.0f);
    e = e - 1;
    float z = fdv(fs(m, 1.0f), fa(m, 1.0f));
    float z2 = fm(z, z);
    float t = fdv(fm(z, z2), fm(3.0f, fs(1.0f, z2)));
    float lnm = fm(2.0f, fa(z, t));
    float lnx = fa(fm((float)e, 0.693147182464599609375f), lnm);
    return fm(fm(2.0f, lnx), fa(1.0f, pad));
}

// ---- Splatting bounds (the association ablation, Sec. 4) -------------------
// The EWA and UT alternatives to PBF bound the Gaussian's projection onto the
// BEAP screen (theta, phi) = (atan2(x, z), atan2(y, z)) by a box; the box's
// angle intervals become arcs of the same half-angle-tangent form as PBF's,
// so the tile ranges and everything after them are shared. Plain FP32
// arithmetic (no reproducibility contract: the bounds are compared with an
// FP64 definition within a tolerance).
constexpr float kPiF = 3.14159265358979f, kTwoPiF = 6.28318530717959f;
constexpr float kSplatNear = 0.2f;  // near plane of the splatting pipelines
constexpr float kSqrt3 = 1.7320508075688772f;

// tan(a / 2) for a in [-pi, pi]; the half angle is kept below pi / 2 so that the
// FP32 rounding of pi cannot turn the tangent's sign at the ends.
__device__ __forceinline__ float tan_half(float a) {
    return tanf(fminf(fmaxf(0.5f * a, -1.5707962f), 1.5707962f));
}

// The arc of the angles [lo, hi] taken modulo 2 pi.
__device__ Arc angle_arc(float lo, float hi) {
    Arc a{3, 0.0f, 0.0f};
    if (!(hi - lo < kTwoPiF) || !isfinite(lo) || !isfinite(hi)) return a;
    const float k = floorf((lo + kPiF) / kTwoPiF);  // lo into [-pi, pi)
    lo -= k * kTwoPiF;
    hi -= k * kTwoPiF;
    if (hi <= kPiF) {
        a.kind = 1;
        a.lo = tan_half(lo);
        a.hi = tan_half(hi);
    } else {  // through pi: [lo, pi] u (-pi, hi - 2 pi]
        a.kind = 2;
        a.lo = tan_half(lo);
        a.hi = tan_half(hi - kTwoPiF);
    }
    return a;
}

// The splatting box of a live item as four arcs: theta (a), theta turned by pi
// (a1: rows whose rays have cos(phi) < 0 see atan2(x, z) = theta + pi), phi (b)
// and phi turned (b1). (x, y, z): camera-frame mean; column k of M: axis k;
// s: scales. EWA: Sigma_2 = J Sigma_c J^T with the rows of J the gradients of
// the two angles, summed over the axes as s_k^2 (J M_k)(J M_k)^T. UT: the six
// off-centre sigma points mu +- sqrt(3) s_k M_k, their angles taken relative to
// the mean's (atan2 of the cross and dot products with the offset split out,
// so small Gaussians lose no digits); weights 1/6 each, the centre point 0 for
// the mean and 2 for the covariance.
// The EWA factor of Sigma_2 = sum_k f_k f_k^T: f_k = s_k J M_k, J the gradients
// of the two screen angles at the mean (x, y, z).
__device__ __forceinline__ void ewa_factor(float x, float y, float z, const float M[9], const float s[3], float fx[3],
                                           float fy[3]) {
    const float rx = 1.0f / (x * x + z * z), ry = 1.0f / (y * y + z * z);
    const float ja0 = z * rx, ja2 = -x * rx, jb1 = z * ry, jb2 = -y * ry;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        fx[k] = s[k] * (ja0 * M[k] + ja2 * M[6 + k]);
        fy[k] = s[k] * (jb1 * M[3 + k] + jb2 * M[6 + k]);
    }
}

// The EWA splat of a live item for GEER_ALPHA_SPLAT: the mean's screen angles
// and the conic Sigma_2^-1 = (A, B; B, C), out = {theta, phi, A, B, C}. The
// determinant is the sum of the squared 2 x 2 minors of the factor
// (Cauchy-Binet), free of the cancellation of c00 c11 - c01^2. False when
// Sigma_2 is singular (the item is culled).
__device__ __forceinline__ bool splat_conic(float x, float y, float z, const float M[9], const float s[3],
                                            float out[5]) {
    float fx[3], fy[3];
    ewa_factor(x, y, z, M, s, fx, fy);
    float c00 = 0.0f, c01 = 0.0f, c11 = 0.0f, det = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        c00 += fx[k] * fx[k];
        c01 += fx[k] * fy[k];
        c11 += fy[k] * fy[k];
        const int l = (k + 1) % 3;
        const float mk = fx[k] * fy[l] - fy[k] * fx[l];
        det += mk * mk;
    }
    if (!(det > 0.0f) || !isfinite(det)) return false;
    const float inv = 1.0f / det;
    out[0] = atan2f(x, z);
    out[1] = atan2f(y, z);
    out[2] = c11 * inv;
    out[3] = -c01 * inv;
    out[4] = c00 * inv;
    return isfinite(out[2]) && isfinite(out[4]);
}

__device__ __forceinline__ void splat_arcs(int mode, int snug, float amin, float sigma, float x, float y, float z,
                                           const float M[9], const float s[3], Arc &a, Arc &a1, Arc &b, Arc &b1) {
    float tc = atan2f(x, z), pc = atan2f(y, z);
    float c00 = 0.0f, c01 = 0.0f, c11 = 0.0f;
    if (mode == GEER_ASSOC_EWA) {
        float fx[3], fy[3];
        ewa_factor(x, y, z, M, s, fx, fy);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            c00 += fx[k] * fx[k];
            c01 += fx[k] * fy[k];
            c11 += fy[k] * fy[k];
        }
    } else {
        float dt[6], dp[6], mt = 0.0f, mp = 0.0f;
        const float rxz = x * x + z * z, ryz = y * y + z * z;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float f = (h == 0 ? kSqrt3 : -kSqrt3) * s[k];
                const float ox = f * M[k], oy = f * M[3 + k], oz = f * M[6 + k];
                dt[2 * k + h] = atan2f(ox * z - oz * x, rxz + ox * x + oz * z);
                dp[2 * k + h] = atan2f(oy * z - oz * y, ryz + oy * y + oz * z);
                mt += dt[2 * k + h];
                mp += dp[2 * k + h];
            }
        }
        mt *= (1.0f / 6.0f);
        mp *= (1.0f / 6.0f);
        c00 = 2.0f * mt * mt;
        c01 = 2.0f * mt * mp;
        c11 = 2.0f * mp * mp;
        float q00 = 0.0f, q01 = 0.0f, q11 = 0.0f;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const float et = dt[i] - mt, ep = dp[i] - mp;
            q00 += et * et;
            q01 += et * ep;
            q11 += ep * ep;
        }
        c00 += q00 * (1.0f / 6.0f);
        c01 += q01 * (1.0f / 6.0f);
        c11 += q11 * (1.0f / 6.0f);
        tc += mt;
        pc += mp;
    }
    float et, ep;
    if (snug) {  // bounding box of the alpha_min ellipse
        const float t = 2.0f * logf(sigma / amin);
        et = sqrtf(fmaxf(t * c00, 0.0f));
        ep = sqrtf(fmaxf(t * c11, 0.0f));
    } else {  // 3 sqrt of the larger eigenvalue, both axes
        const float h = 0.5f * (c00 + c11), d = 0.5f * (c00 - c11);
        et = ep = 3.0f * sqrtf(fmaxf(h + sqrtf(d * d + c01 * c01), 0.0f));
    }
    a = angle_arc(tc - et, tc + et);
    a1 = angle_arc(tc - et + kPiF, tc + et + kPiF);
    b = angle_arc(pc - ep, pc + ep);
    b1 = angle_arc(pc - ep + kPiF, pc + ep + kPiF);
}


// Real SH of degree <= 3 in the 3DGS convention (Condon-Shortley phase, index
// l^2 + l + m), written out as polynomials of the unit direction. The constants
// are K_lm sqrt(2)^(m != 0) = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (* sqrt 2).
__device__ __forceinline__ void sh_colour(int deg, const float *c, float x, float y, float z, float rgb[3]) {
    float Y[16];
    Y[0] = 0.28209479177387814f;  // 1/(2 sqrt(pi))
    int nb = 1;
    if (deg >= 1) {
        const float k1 = 0.4886025119029199f;  // sqrt(3/(4 pi))
        Y[1] = -k1 * y; Y[2] = k1 * z; Y[3] = -k1 * x;
        nb = 4;
    }
    if (deg >= 2) {
        float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = 1.0925484305920792f * x * y;               // sqrt(15/pi)/2
        Y[5] = -1.0925484305920792f * y * z;
        Y[6] = 0.31539156525252005f * (2.0f * zz - xx - yy);  // sqrt(5/pi)/4
        Y[7] = -1.0925484305920792f * x * z;
        Y[8] = 0.5462742152960396f * (xx - yy);           // sqrt(15/pi)/4
        nb = 9;
        if (deg >= 3) {
            Y[9] = -0.5900435899266435f * y * (3.0f * xx - yy);        // sqrt(35/(2 pi))/4
            Y[10] = 2.890611442640554f * x * y * z;                    // sqrt(105/pi)/2
            Y[11] = -0.4570457994644658f * y * (4.0f * zz - xx - yy);  // sqrt(21/(2 pi))/4
            Y[12] = 0.3731763325901154f * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);  // sqrt(7/pi)/4
            Y[13] = -0.4570457994644658f * x * (4.0f * zz - xx - yy);
            Y[14] = 1.445305721320277f * z * (xx - yy);                // sqrt(105/pi)/4
            Y[15] = -0.5900435899266435f * x * (xx - 3.0f * yy);
            nb = 16;
        }
    }
    float r = 0.5f, g = 0.5f, b = 0.5f;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        if (k < nb) {
            r += Y[k] * c[3 * k];
            g += Y[k] * c[3 * k + 1];
            b += Y[k] * c[3 * k + 2];
        }
    }
    rgb[0] = fmaxf(r, 0.0f);
    rgb[1] = fmaxf(g, 0.0f);
    rgb[2] = fmaxf(b, 0.0f);
}

// True when the association predicate reduces to the rectangle X0 x Y0: no
// flipped-angle ranges and X0, Y0 inside the tiles whose rays all have
// cos(theta) >= 0 (columns) and cos(phi) >= 0 (rows).
__device__ __forceinline__ bool is_rect(const DevCam &cam, const int rg[8]) {
    if (rg[2] < rg[3] || rg[6] < rg[7]) return false;
    if (rg[0] >= rg[1] || rg[4] >= rg[5]) return true;  // empty
    return rg[0] >= cam.c0lo && rg[1] <= cam.c0hi && rg[4] >= cam.r0lo && rg[5] <= cam.r0hi;
}


// The association predicate tile_assoc(x, y) = (z_row(y) & x in X0 | w_row(y) & x in X1)
// & (z_col(x) & y in Y0 | w_col(x) & y in Y1), with the z / w flag sets of the
// camera's rows and columns (one interval / two runs, DevCam), is a union of
// products of row and column sets. Its count over a region follows in constant
// time by inclusion-exclusion, and the set itself is the union of at most nine
// rectangles.
__device__ __forceinline__ int ilen(int lo, int hi) { return hi > lo ? hi - lo : 0; }

// Members of [lo, hi) in a flag set: kind 0 the z interval, 1 the w runs, 2 both.
__device__ __forceinline__ int flag_count(int lo, int hi, const int32_t z[2], const int32_t w[2], int kind) {
    if (kind == 0) return ilen(max(lo, z[0]), min(hi, z[1]));
    int alo = lo, ahi = min(hi, w[0]), blo = max(lo, w[1]), bhi = hi;
    if (kind == 2) {
        alo = max(alo, z[0]);
        ahi = min(ahi, z[1]);
        blo = max(blo, z[0]);
        bhi = min(bhi, z[1]);
    }
    return ilen(alo, ahi) + ilen(blo, bhi);
}

// Associated tiles of the item with ranges rg in [x0, x1) x [y0, y1).
__device__ __forceinline__ uint32_t assoc_count(const DevCam &cam, const int rg[8], int x0, int x1, int y0, int y1) {
    // column sets of the terms a0 (X0), a1 (X1), a0 a1; row sets of b0 (Y0), b1 (Y1), b0 b1
    const int alo[3] = {rg[0], rg[2], max(rg[0], rg[2])}, ahi[3] = {rg[1], rg[3], min(rg[1], rg[3])};
    const int blo[3] = {rg[4], rg[6], max(rg[4], rg[6])}, bhi[3] = {rg[5], rg[7], min(rg[5], rg[7])};
    int64_t total = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            // rows with the flag of term i inside Y_j, columns with the flag of term j inside X_i
            const int rows = flag_count(max(y0, blo[j]), min(y1, bhi[j]), cam.zr, cam.wr, i);
            if (rows == 0) continue;
            const int cols = flag_count(max(x0, alo[i]), min(x1, ahi[i]), cam.zc, cam.wc, j);
            const int sg = (i == 2) != (j == 2) ? -1 : 1;
            total += (int64_t)sg * rows * cols;
        }
    }
    return (uint32_t)total;
}

// The associated set as rectangles {x0, x1, y0, y1} (at most nine, overlapping
// only on rows / columns that carry both flags); returns their number.
__device__ __forceinline__ int assoc_rects(const DevCam &cam, const int rg[8], int4 rc[9]) {
    int n = 0;
#pragma unroll
    for (int i = 0; i < 2; ++i) {      // rows of the z interval (i = 0) or the w runs (i = 1) ...
#pragma unroll
        for (int j = 0; j < 2; ++j) {  // ... crossed with columns of the z interval or the w runs
            const int xlo = rg[2 * i], xhi = rg[2 * i + 1];      // X_i
            const int ylo = rg[4 + 2 * j], yhi = rg[5 + 2 * j];  // Y_j
            if (xlo >= xhi || ylo >= yhi) continue;
#pragma unroll
            for (int ri = 0; ri < 2; ++ri) {
                if (i == 0 && ri == 1) break;
                const int r0 = i == 0 ? cam.zr[0] : (ri == 0 ? 0 : cam.wr[1]);
                const int r1 = i == 0 ? cam.zr[1] : (ri == 0 ? cam.wr[0] : cam.tiles_y);
                const int y0 = max(ylo, r0), y1 = min(yhi, r1);
                if (y0 >= y1) continue;
#pragma unroll
                for (int ci = 0; ci < 2; ++ci) {
                    if (j == 0 && ci == 1) break;
                    const int c0 = j == 0 ? cam.zc[0] : (ci == 0 ? 0 : cam.wc[1]);
                    const int c1 = j == 0 ? cam.zc[1] : (ci == 0 ? cam.wc[0] : cam.tiles_x);
                    const int x0 = max(xlo, c0), x1 = min(xhi, c1);
                    if (x0 < x1) rc[n++] = make_int4(x0, x1, y0, y1);
                }
            }
        }
    }
    return n;
}

// The super-tiles (S x S tiles) holding an associated tile: the union of the
// rectangles' super-tile boxes, each super-tile visited once.
template <typename F>
__device__ __forceinline__ void for_each_super_general(const DevCam &cam, int S, const int rg[8], F f) {
    int4 rc[9];
    const int n = assoc_rects(cam, rg, rc);
    for (int k = 0; k < n; ++k) {
        const int sx0 = rc[k].x / S, sx1 = (rc[k].y - 1) / S + 1, sy0 = rc[k].z / S, sy1 = (rc[k].w - 1) / S + 1;
        for (int sy = sy0; sy < sy1; ++sy)
            for (int sx = sx0; sx < sx1; ++sx) {
                bool seen = false;
                for (int q = 0; q < k && !seen; ++q)
                    seen = sx >= rc[q].x / S && sx <= (rc[q].y - 1) / S && sy >= rc[q].z / S && sy <= (rc[q].w - 1) / S;
                if (!seen) f(sx, sy);
            }
    }
}

// Block-wide exclusive scan (256 threads); returns the exclusive prefix and the block total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t *wsum, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    uint32_t pre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kPrepThreads / 32; ++w) {
        const uint32_t t = wsum[w];
        pre += w < warp ? t : 0u;
        tot += t;
    }
    __syncthreads();
    total = tot;
    return pre + v - x;
}

__device__ __forceinline__ uint32_t block_sum_u32(uint32_t v, uint32_t *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    uint32_t t = 0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;  // valid in warp 0
}

// Thread per Gaussian, loop over cameras (the Gaussian's parameters are read once).
// Two blocks per SM (128 registers): measured faster than one block without
// spills and than three with more.
// SH rows of the block staged in shared memory: row stride NC | 1 floats (odd, so
// that the threads' rows do not share banks).
template <int DEG>
struct PrepSh {
    static constexpr int kStride = (3 * (DEG + 1) * (DEG + 1)) | 1;
};

#ifndef GEER_PREP_MINB
#define GEER_PREP_MINB 3  // resident blocks per SM: caps registers at 80
#endif
// SPLAT: the instance for the association ablation and the splat alpha (any
// GEER_ASSOC_* / GEER_ALPHA_*); the PBF / exact-integral instance (SPLAT false)
// holds none of that code.
template <int DEG, bool SPLAT>
__global__ void __launch_bounds__(kPrepThreads, GEER_PREP_MINB) k_preprocess(
    const DevCam *__restrict__ cams, int ncams, const float4 *__restrict__ ttab, Params p,
    const float *__restrict__ mean, const float *__restrict__ scale, const float *__restrict__ quat,
    const float *__restrict__ opacity, const float *__restrict__ sh, int64_t n, Record *__restrict__ rec,
    uint4 *__restrict__ ranges, GradAcc *__restrict__ gacc, uint32_t *__restrict__ count, uint32_t *__restrict__ key,
    uint32_t *__restrict__ blocksum, int64_t nblk) {
    grid_dep_sync();
    constexpr int NC = 3 * (DEG + 1) * (DEG + 1), ST = PrepSh<DEG>::kStride;
    extern __shared__ float s_sh[];  // [kPrepThreads][ST]
    __shared__ uint32_t red[kPrepThreads / 32];
    const int64_t g0 = (int64_t)blockIdx.x * kPrepThreads;
    const int64_t g = g0 + threadIdx.x;
    {
        // the block's SH coefficients, copied asynchronously while the bounds are
        // computed; read only for the colour
        const int nloc = (int)min((int64_t)kPrepThreads, n - g0);
        const float *src = sh + g0 * NC;
        for (int i = threadIdx.x; i < nloc * NC; i += kPrepThreads) {
            const int gl = i / NC;
            cp_async4(&s_sh[gl * ST + (i - gl * NC)], src + i);
        }
    }
    bool ok = g < n;
    float mu[3] = {0, 0, 0}, sc[3] = {1, 1, 1}, qt[4] = {1, 0, 0, 0}, sigma = 0.0f;
    if (ok) {
#pragma unroll
        for (int a = 0; a < 3; ++a) { mu[a] = mean[3 * g + a]; sc[a] = scale[3 * g + a]; }
#pragma unroll
        for (int a = 0; a < 4; ++a) qt[a] = quat[4 * g + a];
        sigma = opacity[g];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (!isfinite(mu[a]) || !isfinite(sc[a]) || !(sc[a] > 0.0f)) ok = false;
#pragma unroll
        for (int a = 0; a < 4; ++a)
            if (!isfinite(qt[a])) ok = false;
        if (!isfinite(sigma) || !(sigma >= p.alpha_min)) ok = false;
    }
    // normalised quaternion and rotation, exactly rounded
    float R[9];
    float lam2 = 0.0f;
    if (ok) {
        float qn = fsq(fa(fa(fa(fm(qt[0], qt[0]), fm(qt[1], qt[1])), fm(qt[2], qt[2])), fm(qt[3], qt[3])));
        if (!(qn > 0.0f)) ok = false;
        float w = fdv(qt[0], qn), x = fdv(qt[1], qn), y = fdv(qt[2], qn), z = fdv(qt[3], qn);
        R[0] = fs(1.0f, fm(2.0f, fa(fm(y, y), fm(z, z))));
        R[1] = fm(2.0f, fs(fm(x, y), fm(w, z)));
        R[2] = fm(2.0f, fa(fm(x, z), fm(w, y)));
        R[3] = fm(2.0f, fa(fm(x, y), fm(w, z)));
        R[4] = fs(1.0f, fm(2.0f, fa(fm(x, x), fm(z, z))));
        R[5] = fm(2.0f, fs(fm(y, z), fm(w, x)));
        R[6] = fm(2.0f, fs(fm(x, z), fm(w, y)));
        R[7] = fm(2.0f, fa(fm(y, z), fm(w, x)));
        R[8] = fs(1.0f, fm(2.0f, fa(fm(x, x), fm(y, y))));
        lam2 = lambda2(sigma, p.alpha_min, p.lambda_pad);
        if (!(lam2 > 0.0f)) ok = false;
    }
    const float s2[3] = {fm(sc[0], sc[0]), fm(sc[1], sc[1]), fm(sc[2], sc[2])};
    const float ss[3] = {fm(sc[1], sc[2]), fm(sc[0], sc[2]), fm(sc[0], sc[1])};

    for (int ci = 0; ci < ncams; ++ci) {
        const DevCam &cam = cams[ci];
        const int64_t idx = (int64_t)ci * n + g;
        uint32_t cnt = 0;
        bool live = ok;
        float m0 = 0, m1 = 0, m2 = 0, M[9], u[3];
        Record r;
        if (live) {
            const float *Rc = cam.R;
            m0 = fa(fa(fa(fm(Rc[0], mu[0]), fm(Rc[1], mu[1])), fm(Rc[2], mu[2])), cam.t[0]);
            m1 = fa(fa(fa(fm(Rc[3], mu[0]), fm(Rc[4], mu[1])), fm(Rc[5], mu[2])), cam.t[1]);
            m2 = fa(fa(fa(fm(Rc[6], mu[0]), fm(Rc[7], mu[1])), fm(Rc[8], mu[2])), cam.t[2]);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    M[3 * i + j] = fa(fa(fm(Rc[3 * i], R[j]), fm(Rc[3 * i + 1], R[3 + j])), fm(Rc[3 * i + 2], R[6 + j]));
            // camera inside the lambda-ellipsoid: cull (App. B.2: t < 0 matters only
            // when the optical centre is inside the contour)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                u[k] = fdv(fa(fa(fm(M[k], m0), fm(M[3 + k], m1)), fm(M[6 + k], m2)), sc[k]);
            float ou2 = fa(fa(fm(u[0], u[0]), fm(u[1], u[1])), fm(u[2], u[2]));
            if (!(ou2 > lam2)) live = false;
            // the splatting bounds and the splat alpha project through z: their near plane as well
            if (SPLAT && (p.assoc != GEER_ASSOC_PBF || p.alpha_model != GEER_ALPHA_EXACT) && !(m2 > kSplatNear))
                live = false;
        }
        float sp[5];  // GEER_ALPHA_SPLAT: the splat's centre and conic
        if (SPLAT && live && p.alpha_model != GEER_ALPHA_EXACT && !splat_conic(m0, m1, m2, M, sc, sp)) live = false;
        if (live) {
            Arc A, B, A1, B1;
            if (!SPLAT || p.assoc == GEER_ASSOC_PBF) {
                auto SIG = [&](int a, int b) {
                    return fa(fa(fm(s2[0], fm(M[3 * a], M[3 * b])), fm(s2[1], fm(M[3 * a + 1], M[3 * b + 1]))),
                              fm(s2[2], fm(M[3 * a + 2], M[3 * b + 2])));
                };
                float Sxx = SIG(0, 0), Syy = SIG(1, 1), Szz = SIG(2, 2), Sxz = SIG(0, 2), Syz = SIG(1, 2);
                float T00 = fs(fm(lam2, Sxx), fm(m0, m0));
                float T11 = fs(fm(lam2, Syy), fm(m1, m1));
                float T22 = fs(fm(lam2, Szz), fm(m2, m2));
                float T02 = fs(fm(lam2, Sxz), fm(m0, m2));
                float T12 = fs(fm(lam2, Syz), fm(m1, m2));
                float pxz[3], pyz[3], dxz[3], dyz[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    float cx = fs(fm(m0, M[6 + k]), fm(m2, M[k]));
                    float cy = fs(fm(m1, M[6 + k]), fm(m2, M[3 + k]));
                    pxz[k] = fm(s2[k], fm(cx, cx));
                    pyz[k] = fm(s2[k], fm(cy, cy));
                    float ax = fm(ss[k], M[3 + k]);
                    float ay = fm(ss[k], M[k]);
                    dxz[k] = fm(ax, ax);
                    dyz[k] = fm(ay, ay);
                }
                float Pxz = fa(fa(pxz[0], pxz[1]), pxz[2]), Pyz = fa(fa(pyz[0], pyz[1]), pyz[2]);
                float Dxz = fa(fa(dxz[0], dxz[1]), dxz[2]), Dyz = fa(fa(dyz[0], dyz[1]), dyz[2]);
                A = pbf_arc(m0, m2, T00, T02, T22, Pxz, Dxz, lam2);
                B = pbf_arc(m1, m2, T11, T12, T22, Pyz, Dyz, lam2);
                A1 = shift_arc(A);
                B1 = shift_arc(B);
            } else {
                splat_arcs(p.assoc, p.snug, p.alpha_min, sigma, m0, m1, m2, M, sc, A, A1, B, B1);
            }
            const float4 *ctab = ttab + cam.tcol_off;
            const float4 *rtab = ttab + cam.trow_off;
            int rg[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            const float chalf = 0.5f * (float)(cam.width - 1), rhalf = 0.5f * (float)(cam.height - 1);
            arc_range(A, ctab, cam.tiles_x, cam.col_ppr, chalf, rg[0], rg[1]);
            arc_range(B, rtab, cam.tiles_y, cam.row_ppr, rhalf, rg[4], rg[5]);
            if (cam.any_row_flip) arc_range(A1, ctab, cam.tiles_x, cam.col_ppr, chalf, rg[2], rg[3]);
            if (cam.any_col_flip) arc_range(B1, rtab, cam.tiles_y, cam.row_ppr, rhalf, rg[6], rg[7]);
            if (is_rect(cam, rg))
                cnt = (uint32_t)(rg[1] - rg[0]) * (uint32_t)(rg[5] - rg[4]);
            else
                cnt = assoc_count(cam, rg, 0, cam.tiles_x, 0, cam.tiles_y);
            float dist = fsq(fa(fa(fm(m0, m0), fm(m1, m1)), fm(m2, m2)));
            key[idx] = __float_as_uint(dist);
            ranges[idx] = make_uint4((uint32_t)rg[0] | ((uint32_t)rg[1] << 16), (uint32_t)rg[2] | ((uint32_t)rg[3] << 16),
                                     (uint32_t)rg[4] | ((uint32_t)rg[5] << 16), (uint32_t)rg[6] | ((uint32_t)rg[7] << 16));
            // render record: W = S^-1 M^T (camera frame), o_u = -W mu_c = -u; for the
            // splat alpha, W[0..4] = the splat's centre and conic instead
            if (!SPLAT || p.alpha_model == GEER_ALPHA_EXACT) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    float inv = 1.0f / sc[k];
                    r.W[3 * k + 0] = M[k] * inv;
                    r.W[3 * k + 1] = M[3 + k] * inv;
                    r.W[3 * k + 2] = M[6 + k] * inv;
                    r.ou[k] = -u[k];
                }
            } else {
#pragma unroll
                for (int k = 0; k < 9; ++k) r.W[k] = k < 5 ? sp[k] : 0.0f;
#pragma unroll
                for (int k = 0; k < 3; ++k) r.ou[k] = 0.0f;
            }
            r.log2_sigma = log2f(sigma);
        } else if (g < n) {
            key[idx] = 0u;
            ranges[idx] = make_uint4(0, 0, 0, 0);
        }
        if (ci == 0) {  // the SH rows have arrived (block-uniform)
            asm volatile("cp.async.wait_all;\n" ::: "memory");
            __syncthreads();
        }
        if (live) {
            float dx = mu[0] - cam.o[0], dy = mu[1] - cam.o[1], dz = mu[2] - cam.o[2];
            float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
            sh_colour(DEG, s_sh + threadIdx.x * ST, dx * inv, dy * inv, dz * inv, r.rgb);
            float4 *dst = reinterpret_cast<float4 *>(rec + idx);
            const float4 *src = reinterpret_cast<const float4 *>(&r);
#pragma unroll
            for (int i = 0; i < 4; ++i) dst[i] = src[i];
        }
        if (g < n) count[idx] = cnt;
        if (g < n && gacc) {  // every item's backward accumulators start from zero
            float4 *acc = reinterpret_cast<float4 *>(gacc + idx);
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
        uint32_t tot = block_sum_u32(cnt > 0 ? 1u : 0u, red);
        if (threadIdx.x == 0) blocksum[(int64_t)ci * nblk + blockIdx.x] = tot;
    }
}

// Exclusive scan of per-block counts (one block; each thread scans a contiguous
// chunk serially). mode 0 (live items): total -> misc[kMiscLive]; also clears the
// per-super-tile pair counts. mode 1 ((super-tile, item) pairs): total ->
// misc[kMiscPairs] (clamped to cap) with the capacity check. mode 2 ((tile, item)
// associations P): total -> misc[kMiscTileLo / Hi]. With two blocks, block 1
// scans blocksum_b in mode_b at the same time (one launch for two arrays).
__global__ void __launch_bounds__(1024) k_scan_blocks(uint32_t *__restrict__ blocksum, int64_t m,
                                                      uint32_t *__restrict__ misc, uint2 *__restrict__ srange,
                                                      int64_t nst, int64_t cap, int mode,
                                                      uint32_t *__restrict__ blocksum_b = nullptr, int mode_b = 0) {
    grid_dep_sync();
    __shared__ unsigned long long warp_tot[32];
    if (blockIdx.x == 1) {
        blocksum = blocksum_b;
        mode = mode_b;
    }
    const int t = threadIdx.x;
    const int64_t chunk = (m + 1023) / 1024;
    const int64_t b = t * chunk, e = min(m, b + chunk);
    unsigned long long s = 0;
    for (int64_t i = b; i < e; ++i) s += blocksum[i];
    unsigned long long v = s;
    const int lane = t & 31, warp = t >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    unsigned long long excl = v - s + (warp > 0 ? warp_tot[warp - 1] : 0ull);
    for (int64_t i = b; i < e; ++i) {
        uint32_t c = blocksum[i];
        blocksum[i] = (uint32_t)min(excl, 0xffffffffull);
        excl += c;
    }
    if (t == 1023) {
        const unsigned long long total = excl;
        if (mode == 0) {
            misc[kMiscLive] = (uint32_t)total;
            // the depth sort's first pass reads buffer 0 (see depth_sorted_buf)
            misc[kMiscSortCur] = 1u;
            misc[kMiscSortSame] = 0u;
        } else if (mode == 2) {
            misc[kMiscTileLo] = (uint32_t)total;
            misc[kMiscTileHi] = (uint32_t)(total >> 32);
        } else {
            misc[kMiscPairs] = (uint32_t)min(total, (unsigned long long)cap);
            misc[kMiscPairsHi] = (uint32_t)(total >> 32);
            misc[kMiscTotalLo] = (uint32_t)total;
            if (total > (unsigned long long)cap) atomicOr(&misc[kMiscStatus], kStatusCapacity);
        }
    }
    if (mode == 0) {
        uint32_t *scount = reinterpret_cast<uint32_t *>(srange + nst);
        for (int64_t i = t; i < nst; i += 1024) scount[i] = 0u;
    }
}

// Compaction of the live (camera, Gaussian) items, in index order, into
// (depth key, item) arrays.
__global__ void __launch_bounds__(kPrepThreads) k_compact(int ncams, int64_t n, const uint32_t *__restrict__ count,
                                                          const uint32_t *__restrict__ key,
                                                          const uint32_t *__restrict__ blocksum, int64_t nblk,
                                                          uint32_t *__restrict__ okey, uint32_t *__restrict__ oid) {
    grid_dep_sync();
    __shared__ uint32_t wsum[kPrepThreads / 32];
    const int64_t g = (int64_t)blockIdx.x * kPrepThreads + threadIdx.x;
    for (int ci = 0; ci < ncams; ++ci) {
        const int64_t idx = (int64_t)ci * n + g;
        const bool live = g < n && count[idx] > 0;
        uint32_t tot;
        const uint32_t pre = block_excl_scan(live ? 1u : 0u, wsum, tot);
        if (live) {
            const uint32_t k = key[idx];
            const uint32_t pos = blocksum[(int64_t)ci * nblk + blockIdx.x] + pre;
            okey[pos] = k;
            oid[pos] = (uint32_t)idx;
        }
    }
}

// Number of (super-tile, item) pairs of an item with c associated tiles.
__device__ __forceinline__ uint32_t super_count(const DevCam &cam, int S, const int rg[8], uint32_t c, bool rect) {
    if (c == 0) return 0u;
    if (rect) {
        const int sx0 = rg[0] / S, sx1 = (rg[1] - 1) / S + 1, sy0 = rg[4] / S, sy1 = (rg[5] - 1) / S + 1;
        return (uint32_t)((sx1 - sx0) * (sy1 - sy0));
    }
    uint32_t k = 0;
    for_each_super_general(cam, S, rg, [&](int, int) { ++k; });
    return k;
}

// Per block of depth-sorted live items: their super-tile pairs (emission
// offsets) and their tile pairs (the total, for the capacity check).
__global__ void __launch_bounds__(kPrepThreads) k_gather_counts(const DevCam *__restrict__ cams,
                                                                const float4 *__restrict__ ttab, int64_t n, int S,
                                                                const uint32_t *__restrict__ sorted0,
                                                                const uint32_t *__restrict__ sorted1,
                                                                const uint32_t *__restrict__ count,
                                                                const uint4 *__restrict__ ranges,
                                                                const uint32_t *__restrict__ misc,
                                                                uint32_t *__restrict__ bs_super,
                                                                uint32_t *__restrict__ bs_tile) {
    grid_dep_sync();
    __shared__ uint32_t red[kPrepThreads / 32];
    const uint32_t L = misc[kMiscLive];
    const uint32_t *__restrict__ sorted_id = depth_sorted_buf(misc) ? sorted1 : sorted0;
    const int64_t i = (int64_t)blockIdx.x * kPrepThreads + threadIdx.x;
    uint32_t c = 0, sc = 0;
    if (i < L) {
        const uint32_t item = sorted_id[i];
        c = count[item];
        int rg[8];
        unpack_ranges(ranges[item], rg);
        const DevCam &cam = cams[item / (uint32_t)n];
        sc = super_count(cam, S, rg, c, is_rect(cam, rg));
    }
    const uint32_t tot = block_sum_u32(c, red);
    if (threadIdx.x == 0) bs_tile[blockIdx.x] = tot;
    __syncthreads();
    const uint32_t stot = block_sum_u32(sc, red);
    if (threadIdx.x == 0) bs_super[blockIdx.x] = stot;
}

// DuplicateWithKeys in depth order, at super-tile granularity: item i of the
// depth-sorted list emits one (global super-tile, item) pair per super-tile
// holding an associated tile, in row-major order, and counts the pairs per
// super-tile. Items whose association is a rectangle are emitted by the whole
// warp together (lane j writes output j: coalesced); others loop per thread.
__global__ void __launch_bounds__(kPrepThreads) k_duplicate(
    const DevCam *__restrict__ cams, const float4 *__restrict__ ttab, int64_t n, int S,
    const uint32_t *__restrict__ sorted0, const uint32_t *__restrict__ sorted1, const uint4 *__restrict__ ranges,
    const uint32_t *__restrict__ count, uint32_t *__restrict__ misc, const uint32_t *__restrict__ blocksum,
    uint32_t *__restrict__ okeys,
    uint32_t *__restrict__ ovals, uint32_t *__restrict__ scount, int nst, int64_t cap) {
    grid_dep_sync();
    __shared__ uint32_t wsum[kPrepThreads / 32];
    extern __shared__ uint32_t sh[];  // per-super-tile pair counts when they fit (nst <= kSmemTiles)
    const bool smem = nst <= kSmemTiles;
    if (smem)
        for (int k = threadIdx.x; k < nst; k += kPrepThreads) sh[k] = 0u;
    const uint32_t L = misc[kMiscLive];
    const uint32_t *__restrict__ sorted_id = depth_sorted_buf(misc) ? sorted1 : sorted0;
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * kPrepThreads + threadIdx.x;
    uint32_t item = 0, cnt = 0;
    int rg[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int ci = 0;
    bool rect = true;
    if (i < L) {
        item = sorted_id[i];
        ci = (int)(item / (uint32_t)n);
        unpack_ranges(ranges[item], rg);
        rect = is_rect(cams[ci], rg);
        cnt = super_count(cams[ci], S, rg, count[item], rect);
    }
    uint32_t tot;
    const uint32_t pre = block_excl_scan(cnt, wsum, tot);
    const int64_t off = (int64_t)blocksum[blockIdx.x] + pre;
    const bool fits = off + cnt <= cap;
    const DevCam &cam = cams[ci];
    __syncthreads();  // the per-super-tile counters are cleared
    int sx0 = 0, sy0 = 0, rw = 1;
    if (rect && fits && cnt > 0) {
        sx0 = rg[0] / S;
        sy0 = rg[4] / S;
        rw = (rg[1] - 1) / S + 1 - sx0;
    }
    // cooperative emission of the rectangle items of this warp
    const uint32_t rc = (rect && fits) ? cnt : 0u;
    uint32_t incl = rc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t wtot = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t sb = (uint32_t)(cam.stile_base + sy0 * cam.stiles_x + sx0);
    for (uint32_t j0 = 0; j0 < wtot; j0 += 32) {
        const uint32_t j = j0 + lane;
        // owner: first lane whose inclusive count exceeds j
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t v = __shfl_sync(0xffffffffu, incl, lo + step - 1);
            if (v <= j) lo += step;
        }
        const uint32_t o_incl = __shfl_sync(0xffffffffu, incl, lo);
        const uint32_t o_cnt = __shfl_sync(0xffffffffu, rc, lo);
        const int o_rw = __shfl_sync(0xffffffffu, rw, lo);
        const uint32_t o_sb = __shfl_sync(0xffffffffu, sb, lo);
        const int o_sx = __shfl_sync(0xffffffffu, cam.stiles_x, lo);
        const uint32_t o_item = __shfl_sync(0xffffffffu, item, lo);
        const int64_t o_off = __shfl_sync(0xffffffffu, off, lo);
        if (j < wtot) {
            const uint32_t k = j - (o_incl - o_cnt);
            const uint32_t ky = k / (uint32_t)o_rw, kx = k - ky * (uint32_t)o_rw;
            const uint32_t st = o_sb + ky * (uint32_t)o_sx + kx;
            okeys[o_off + k] = st;
            ovals[o_off + k] = o_item;
            if (in_bounds(st, (uint64_t)nst, kSiteDupSuper, misc)) atomicAdd(smem ? &sh[st] : &scount[st], 1u);
        }
    }
    // per-thread emission of the other items (flipped angular ranges)
    if (!rect && fits && cnt > 0) {
        int64_t o = off;
        const int64_t end = off + cnt;
        for_each_super_general(cam, S, rg, [&](int sx, int sy) {
            if (o < end) {
                const uint32_t st = (uint32_t)(cam.stile_base + sy * cam.stiles_x + sx);
                okeys[o] = st;
                ovals[o] = item;
                if (in_bounds(st, (uint64_t)nst, kSiteDupSuper, misc)) atomicAdd(smem ? &sh[st] : &scount[st], 1u);
                ++o;
            }
        });
    }
    __syncthreads();
    if (smem)
        for (int k = threadIdx.x; k < nst; k += kPrepThreads)
            if (sh[k]) atomicAdd(&scount[k], sh[k]);
}

// Warp-aggregated bucket atomic: the lanes with ok hold bucket bk; one atomic
// per distinct bucket of the warp adds the lanes' count to hist[bk]. Returns the
// lane's slot (old value + its rank among the lanes of its bucket). All lanes of
// the warp must call it.
__device__ __forceinline__ uint32_t bucket_add(uint32_t *hist, bool ok, int bk) {
    const unsigned peers = __match_any_sync(0xffffffffu, ok ? bk : -1);
    const int leader = __ffs(peers) - 1, lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (ok && lane == leader) base = atomicAdd(&hist[bk], (uint32_t)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
}

// Exclusive scan of the kOrderBuckets bucket sizes in place (warp 0; the block
// synchronises before and after).
__device__ __forceinline__ void bucket_scan(uint32_t *hist) {
    if (threadIdx.x >= 32) return;
    constexpr int kPer = (kOrderBuckets + 31) / 32;
    const int lane = threadIdx.x, b0 = lane * kPer;
    uint32_t v[kPer], sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        v[k] = b0 + k < kOrderBuckets ? hist[b0 + k] : 0u;
        sum += v[k];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    uint32_t run = incl - sum;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        if (b0 + k < kOrderBuckets) hist[b0 + k] = run;
        run += v[k];
    }
}

// Exclusive scan over [0, m) of counts held as contiguous per-thread chunks by a
// 1024-thread block: returns the prefix of the thread's chunk (s = the chunk's sum).
__device__ __forceinline__ uint32_t block_chunk_prefix(uint32_t s, uint32_t *warp_tot) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    uint32_t v = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    const uint32_t pre = v - s + (warp > 0 ? warp_tot[warp - 1] : 0u);
    __syncthreads();
    return pre;
}

// One block, IdentifyFrustumRanges at super-tile granularity: each super-tile's
// [start, end) in the sorted super-tile pairs (exclusive scan of its pair
// count), and the order in which the render blocks take the tiles: by
// descending length of their super-tile's list (bucketed), so that the costliest
// tiles start first and the grid does not end on a tail of heavy tiles. (Measured
// on the 1M-Gaussian fisheye workload: 0.344 ms forward against 0.358 - 0.409 ms
// with the length capped at 16K - 1K entries and 0.424 ms in tile order.)
__global__ void __launch_bounds__(1024) k_tile_offsets(const DevCam *__restrict__ cams, int ncams, int S,
                                                       int ntiles, uint2 *__restrict__ srange, int nst,
                                                       uint32_t *__restrict__ misc,
                                                       uint32_t *__restrict__ tile_order,
                                                       uint32_t *__restrict__ queue, uint32_t queue_n) {
    grid_dep_sync();
    // the fused render's unit queue and its counters start afresh with every binning
    if (queue) {
        for (uint32_t i = threadIdx.x; i < queue_n; i += 1024) queue[i] = 0xffffffffu;
        if (threadIdx.x < 4) misc[kMiscFwdNext + threadIdx.x] = 0u;
    }
    constexpr int kOrderSmem = 16384;  // super-tiles / tiles whose buckets the block keeps in shared memory
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t hist[kOrderBuckets];
    __shared__ uint8_t s_sbk[kOrderSmem], s_tbk[kOrderSmem];
    if (misc[kMiscStatus] & kStatusCapacity) return;
    const int t = threadIdx.x;
    const bool keep_s = nst <= kOrderSmem, keep_t = ntiles <= kOrderSmem;
    for (int i = t; i < kOrderBuckets; i += 1024) hist[i] = 0u;
    // super-tile ranges
    const uint32_t *scount = reinterpret_cast<const uint32_t *>(srange + nst);
    const int schunk = (nst + 1023) / 1024;
    const int sb = t * schunk, se = min(nst, sb + schunk);
    uint32_t ss = 0;
    for (int i = sb; i < se; ++i) ss += scount[i];
    uint32_t srun = block_chunk_prefix(ss, warp_tot);
    for (int i = sb; i < se; ++i) {
        const uint32_t cnt = scount[i];
        srange[i] = make_uint2(srun, srun + cnt);
        if (keep_s) s_sbk[i] = (uint8_t)order_bucket(cnt);
        srun += cnt;
    }
    __syncthreads();
    // each tile's cost estimate: its super-tile's list length (0 for padding tiles),
    // bucketed in the first pass and kept for the second
    const int chunk = (ntiles + 1023) / 1024;
    const int b = t * chunk, e = min(ntiles, b + chunk);
    int c = 0;
    for (int k = 1; k < ncams; ++k)
        if (cams[k].tile_base <= b) c = k;
    for (int pass = 0; pass < 2; ++pass) {
        int cc = c;
        for (int k = 0; k < chunk; ++k) {  // the same trip count in every lane (warp-wide atomics)
            const int i = b + k;
            int bk = kOrderBuckets - 1;
            if (i < e && pass == 1 && keep_t) {
                bk = s_tbk[i];
            } else if (i < e) {
                while (cc + 1 < ncams && cams[cc + 1].tile_base <= i) ++cc;
                const DevCam &cm = cams[cc];
                const int lt = i - cm.tile_base;
                if (lt >= 0 && lt < cm.tiles_x * cm.tiles_y) {
                    const int cy = lt / cm.tiles_x, cx = lt - cy * cm.tiles_x;
                    const int si = cm.stile_base + (cy / S) * cm.stiles_x + cx / S;
                    if (keep_s) {
                        bk = s_sbk[si];
                    } else {
                        const uint2 r = srange[si];
                        bk = order_bucket(r.y - r.x);
                    }
                }
                if (keep_t) s_tbk[i] = (uint8_t)bk;
            }
            const uint32_t slot = bucket_add(hist, i < e, bk);
            if (pass == 1 && i < e) tile_order[slot] = (uint32_t)i;
        }
        __syncthreads();
        if (pass == 0) bucket_scan(hist);
        __syncthreads();
    }
}

// One block: the backward's units and their schedule. A tile whose forward walk
// covered W > 0 list entries and passed the checkpoints B_1 < ... < B_m < W
// has the units k = 0..m, entries [B_k, B_{k+1}) with B_0 = 0 and B_{m+1} = W.
// The forward leaves per tile their number and schedule buckets (unit_rec: the
// bucket of each unit's cost, the (entry, warp) pairs whose hit byte it set in
// the unit: a backward warp walks those steps, so a dense tile's unit costs
// more than a sparse one's of the same length). The units are ordered by
// descending cost, units[slot] = tile << 4 | k. Also sets the unit count and
// resets the counter the persistent backward blocks take units from.
__global__ void __launch_bounds__(1024) k_bwd_order(const uint4 *__restrict__ unit_rec, int ntiles,
                                                    uint32_t *__restrict__ misc, uint32_t *__restrict__ order) {
    grid_dep_sync();
    __shared__ uint32_t hist[kOrderBuckets];
    __shared__ uint32_t s_total;
    if (misc[kMiscStatus] & kStatusCapacity) return;
    const int t = threadIdx.x;
    for (int i = t; i < kOrderBuckets; i += 1024) hist[i] = 0u;
    if (t == 0) s_total = 0u;
    __syncthreads();
    const int chunk = (ntiles + 1023) / 1024;
    const int b = t * chunk, e = min(ntiles, b + chunk);
    constexpr int G = 4;  // tiles whose records are loaded together
    for (int pass = 0; pass < 2; ++pass) {
        uint32_t mine = 0;
        for (int c0 = 0; c0 < chunk; c0 += G) {  // the same trip counts in every lane (warp-wide atomics)
            uint4 r[G];
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const int i = b + c0 + u;
                r[u] = c0 + u < chunk && i < e ? unit_rec[i] : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const int i = b + c0 + u;
                const uint32_t units = min((r[u].w >> (8 * (kUnitCountByte & 3))) & 0xffu, (uint32_t)kCkptMax + 1u);
#pragma unroll
                for (int k = 0; k <= kCkptMax; ++k) {
                    if (!__any_sync(0xffffffffu, (uint32_t)k < units)) break;
                    const bool ok = (uint32_t)k < units;
                    const uint32_t word = k < 4 ? r[u].x : (k < 8 ? r[u].y : r[u].z);
                    const int bk = min((int)((word >> (8 * (k & 3))) & 0xffu), kOrderBuckets - 1);
                    const uint32_t slot = bucket_add(hist, ok, bk);
                    if (pass == 1 && ok) order[slot] = ((uint32_t)i << 4) | (uint32_t)k;
                }
                mine += units;
            }
        }
        if (pass == 0) {
            atomicAdd(&s_total, mine);
            __syncthreads();
            bucket_scan(hist);
        }
        __syncthreads();
    }
    if (t == 0) {
        misc[kMiscUnits] = s_total;
        misc[kMiscUnitNext] = 0u;
    }
}

}  // namespace

cudaError_t launch_preprocess(const geer_workspace *ws, const geer_gaussians *g, cudaStream_t s) {
    const int64_t nblk = prep_blocks(g->n);
    if (nblk == 0) return cudaSuccess;
    const Params prm = ws->params;
    const bool splat = prm.assoc != GEER_ASSOC_PBF || prm.alpha_model != GEER_ALPHA_EXACT;
#define GEER_PREP_LAUNCH(D)                                                                                      \
    {                                                                                                            \
        const int smem = kPrepThreads * PrepSh<D>::kStride * (int)sizeof(float);                               \
        auto *kern = splat ? k_preprocess<D, true> : k_preprocess<D, false>;                                     \
        if (smem > 48 * 1024) {                                                                                  \
            const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);  \
            if (e != cudaSuccess) return e;                                                                      \
        }                                                                                                        \
        launch_k(kern, dim3((unsigned)nblk), dim3(kPrepThreads), smem, s, ws->d_cams, ws->n_cams,                 \
                 ws->d_tile_tab, prm, g->mean, g->scale, g->quat, g->opacity, g->sh, g->n, ws->d_rec,            \
                 ws->d_ranges, ws->trains ? ws->d_gacc : nullptr, ws->d_count, ws->d_key,                    \
                 ws->d_blocksum, nblk);                                                                   \
    }
    switch (g->sh_degree) {
        case 0: GEER_PREP_LAUNCH(0); break;
        case 1: GEER_PREP_LAUNCH(1); break;
        case 2: GEER_PREP_LAUNCH(2); break;
        default: GEER_PREP_LAUNCH(3); break;
    }
#undef GEER_PREP_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_bin_front(const geer_workspace *ws, cudaStream_t s) {
    const int64_t nblk = prep_blocks(ws->n_gauss);
    launch_k(k_scan_blocks, dim3(1), dim3(1024), 0, s, ws->d_blocksum, nblk * ws->n_cams, ws->d_misc, ws->d_srange,
             ws->n_stiles, ws->cap_pairs, 0, nullptr, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || nblk == 0) return e;
    launch_k(k_compact, dim3((unsigned)nblk), dim3(kPrepThreads), 0, s, ws->n_cams, ws->n_gauss, ws->d_count,
             ws->d_key, ws->d_blocksum, nblk, ws->d_ikey[0], ws->d_iid[0]);
    return cudaGetLastError();
}

cudaError_t launch_count_pairs(const geer_workspace *ws, cudaStream_t s) {
    const int64_t m = prep_blocks((int64_t)ws->n_cams * ws->n_gauss);
    if (m > 0) {
        launch_k(k_gather_counts, dim3((unsigned)m), dim3(kPrepThreads), 0, s, ws->d_cams, ws->d_tile_tab,
                 ws->n_gauss, ws->super_size, ws->d_iid[0], ws->d_iid[1], ws->d_count, ws->d_ranges, ws->d_misc,
                 ws->d_blocksum2, ws->d_blocksum3);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // super-tile pairs: emission offsets and the capacity check; tile associations: the count P
    launch_k(k_scan_blocks, dim3(2), dim3(1024), 0, s, ws->d_blocksum2, m, ws->d_misc, nullptr, 0, ws->cap_pairs, 1,
             ws->d_blocksum3, 2);
    return cudaGetLastError();
}

cudaError_t launch_duplicate(const geer_workspace *ws, cudaStream_t s) {
    const int64_t m = prep_blocks((int64_t)ws->n_cams * ws->n_gauss);
    uint32_t *scount = reinterpret_cast<uint32_t *>(ws->d_srange + ws->n_stiles);
    if (m > 0) {
        const size_t smem = ws->n_stiles <= kSmemTiles ? sizeof(uint32_t) * ws->n_stiles : 0;
        launch_k(k_duplicate, dim3((unsigned)m), dim3(kPrepThreads), smem, s, ws->d_cams, ws->d_tile_tab,
                 ws->n_gauss, ws->super_size, ws->d_iid[0], ws->d_iid[1], ws->d_ranges, ws->d_count, ws->d_misc,
                 ws->d_blocksum2, ws->d_keys[0], ws->d_vals[0], scount, (int)ws->n_stiles, ws->cap_pairs);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    launch_k(k_tile_offsets, dim3(1), dim3(1024), 0, s, ws->d_cams, ws->n_cams, ws->super_size, (int)ws->n_tiles,
             ws->d_srange, (int)ws->n_stiles, ws->d_misc, ws->d_tile_order,
             ws->trains ? ws->d_bwd_order : nullptr, (uint32_t)(ws->n_tiles * (kCkptMax + 1)));
    return cudaGetLastError();
}

cudaError_t launch_bwd_order(const geer_workspace *ws, cudaStream_t s) {
    if (ws->n_tiles == 0) return cudaSuccess;
    launch_k(k_bwd_order, dim3(1), dim3(1024), 0, s, ws->d_unit_rec, (int)ws->n_tiles, ws->d_misc,
             ws->d_bwd_order);
    return cudaGetLastError();
}

}  // namespace geer
