/*
 * geer_oracle.c -- slow, plain CPU oracle for the exact ray-Gaussian renderer of
 * 3DGEER (arXiv 2505.24053).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load this library. The product path (the CUDA library)
 * never calls it, and the two share no code, header or table generator.
 *
 * Part 1 -- FP64 definition of the rendered image (no PBF culling):
 *   - BEAP ray of pixel (i, j): equiangular grid (Sec. 3.3 "BEAP" equation;
 *     pixel centres, 0-based) and the direction of App. E.
 *   - Gaussian: Sigma = R S S^T R^T, R from the normalised quaternion
 *     (App. B.1); whitening W = S^-1 R^T (App. C.1).
 *   - Closed-form ray integral: o_u = W(o - mu), d_u = W d, m_u = o_u x d_u,
 *     kappa = |m_u|^2 / |d_u|^2, alpha = sigma exp(-kappa/2)
 *     (Sec. 3.1 closed-form transmittance; App. B.2, Mahalanobis distance eq.).
 *   - Colour: real spherical harmonics of the 3DGS convention evaluated at the
 *     world direction (mu - o)/|mu - o| (App. B.1 colour equation), +0.5,
 *     clamped at 0. The basis is built from associated Legendre functions.
 *   - Compositing: contributors in depth-key order, C += T a c, T *= (1 - a)
 *     (App. B.1 colour equation) with the 3DGS thresholds alpha_min, alpha_max,
 *     T_min and a background term.
 * Part 2 -- FP32 replica of the per-Gaussian decisions that are integers
 *   decided by floating point, in the exact operation order the GPU uses:
 *   cull flag, depth key (FP32 |mu_c|), and the Particle Bounding Frustum tile
 *   ranges (Sec. 3.2 tangency quadratic; App. D.1 T-matrix form; App. D.2
 *   half-angle mirror transform with xi = 1). This file must be compiled with
 *   -ffp-contract=off and without fast-math.
 * Part 3 -- FP64 analytic gradients of an L1-type loss (App. C cookbook, with
 *   the cross-product signs written for m_u = o_u x d_u).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TILE 16

typedef struct {
    int32_t model; /* 0 pinhole, 1 equidistant fisheye, 2 Kannala-Brandt */
    int32_t width, height;
    float fov_x, fov_y; /* radians; fov_y <= 0 means derived from the model */
    float k[4];         /* Kannala-Brandt k1..k4 */
    float R_cw[9];      /* world -> camera rotation, row-major */
    float t_cw[3];      /* world -> camera translation */
    float bg[3];        /* background colour */
} orc_camera;

typedef struct {
    int64_t n;
    int32_t sh_degree;
    int32_t pad_;
    const float *mean;    /* [n][3] */
    const float *scale;   /* [n][3], linear */
    const float *quat;    /* [n][4], (w, x, y, z), any norm */
    const float *opacity; /* [n], activated */
    const float *sh;      /* [n][(deg+1)^2][3] */
} orc_gaussians;

typedef struct {
    float alpha_min, T_min, alpha_max, lambda_pad;
} orc_params;

/* ------------------------------------------------------------------------- */
/* Part 1: FP64 definition                                                    */
/* ------------------------------------------------------------------------- */

static double kb_distort(const double k[4], double phi)
{
    /* Kannala-Brandt distorted angle (App. E): phi (1 + k1 phi^2 + ... + k4 phi^8) */
    double p2 = phi * phi;
    return phi * (1.0 + k[0] * p2 + k[1] * p2 * p2 + k[2] * p2 * p2 * p2 + k[3] * p2 * p2 * p2 * p2);
}

/* Vertical field of view of the BEAP grid. The paper gives the grid in terms of
 * FoV_x and FoV_y (Sec. 3.3) without saying how FoV_y follows from a camera;
 * reading: the vertical angular half-extent along the image's vertical centre
 * line at the same focal length that maps FoV_x/2 to w/2. */
double orc_fov_y(const orc_camera *c)
{
    if (c->fov_y > 0.0f) return (double)c->fov_y;
    double fx = c->fov_x, w = c->width, h = c->height;
    if (c->model == 0) return 2.0 * atan(tan(0.5 * fx) * h / w);
    if (c->model == 1) return fx * h / w;
    double k[4];
    for (int i = 0; i < 4; ++i) k[i] = c->k[i];
    double edge = kb_distort(k, 0.5 * fx);
    if (!(edge > 0.0)) return NAN;
    double target = edge * h / w; /* (h/2) / f with f = (w/2) / edge */
    /* smallest phi in (0, fx/2] with kb_distort(phi) = target */
    const int steps = 8192;
    double lo = 0.0, hi = 0.5 * fx;
    for (int s = 1; s <= steps; ++s) {
        double p = 0.5 * fx * s / steps;
        if (kb_distort(k, p) >= target) { hi = p; lo = 0.5 * fx * (s - 1) / steps; break; }
    }
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (kb_distort(k, mid) >= target) hi = mid; else lo = mid;
    }
    return 2.0 * hi;
}

/* BEAP pixel-centre angles (Sec. 3.3): pixel i (0-based) sits at
 * theta_i = ((i + 1/2)/w - 1/2) FoV_x, likewise phi_j with FoV_y. */
static double beap_theta(int i, int w, double fov) { return ((i + 0.5) / w - 0.5) * fov; }

/* Camera-frame BEAP direction (App. E), normalised. */
static void beap_dir(double th, double ph, double d[3])
{
    double x = sin(th) * cos(ph), y = cos(th) * sin(ph), z = cos(th) * cos(ph);
    double n = sqrt(x * x + y * y + z * z);
    d[0] = x / n; d[1] = y / n; d[2] = z / n;
}

/* World-space ray (o, d) of BEAP pixel (i, j): o = -R_cw^T t_cw, d = R_cw^T d_cam. */
void orc_pixel_ray(const orc_camera *c, int i, int j, double o[3], double d[3])
{
    double fy = orc_fov_y(c);
    double th = beap_theta(i, c->width, c->fov_x), ph = beap_theta(j, c->height, fy);
    double dc[3];
    beap_dir(th, ph, dc);
    for (int a = 0; a < 3; ++a) {
        o[a] = 0.0; d[a] = 0.0;
        for (int b = 0; b < 3; ++b) {
            o[a] -= (double)c->R_cw[3 * b + a] * c->t_cw[b];
            d[a] += (double)c->R_cw[3 * b + a] * dc[b];
        }
    }
}

/* Rotation of the normalised quaternion (w, x, y, z). */
static void quat_rot(const float *q, double R[9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double n = sqrt(w * w + x * x + y * y + z * z);
    w /= n; x /= n; y /= n; z /= n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Whitening W = S^-1 R^T (App. C.1), row-major. */
static void whitening(const float *q, const float *s, double W[9])
{
    double R[9];
    quat_rot(q, R);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) W[3 * i + j] = R[3 * j + i] / (double)s[i];
}

static void matvec(const double M[9], const double v[3], double r[3])
{
    for (int i = 0; i < 3; ++i) r[i] = M[3 * i] * v[0] + M[3 * i + 1] * v[1] + M[3 * i + 2] * v[2];
}

static void cross(const double a[3], const double b[3], double r[3])
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Squared canonical distance kappa between ray (o, d) and Gaussian (mu, s, q)
 * (App. B.2): cross-product form, never the expanded |o_u|^2|d_u|^2 - (o_u.d_u)^2
 * (App. C, numerical stability). Also returns t* = -(o_u.d_u)/|d_u|^2, the ray
 * parameter of closest approach, and |o_u|. */
double orc_kappa(const float *mu, const float *s, const float *q, const double o[3], const double d[3],
                 double *tstar, double *ou_norm)
{
    double W[9], v[3], ou[3], du[3], m[3];
    whitening(q, s, W);
    for (int a = 0; a < 3; ++a) v[a] = o[a] - (double)mu[a];
    matvec(W, v, ou);
    matvec(W, d, du);
    cross(ou, du, m);
    double dd = dot(du, du);
    if (tstar) *tstar = -dot(ou, du) / dd;
    if (ou_norm) *ou_norm = sqrt(dot(ou, ou));
    return dot(m, m) / dd;
}

/* Real spherical harmonics, 3DGS convention (Condon-Shortley phase kept, index
 * l^2 + l + m, m = -l..l), built from associated Legendre functions:
 *   m = 0: K_l0 P_l^0(z);  m > 0: sqrt2 K_lm P_l^m(z) cos(m phi);
 *   m < 0: sqrt2 K_l|m| P_l^|m|(z) sin(|m| phi),
 *   K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!). */
void orc_sh_basis(int deg, const double dir[3], double *Y)
{
    double x = dir[0], y = dir[1], z = dir[2];
    double az = atan2(y, x);
    double st = sqrt(fmax(0.0, 1.0 - z * z));
    double P[4][4]; /* P[l][m] */
    memset(P, 0, sizeof(P));
    for (int m = 0; m <= deg; ++m) {
        double pmm = 1.0;
        for (int i = 1; i <= m; ++i) pmm *= -(2.0 * i - 1.0) * st; /* (-1)^m (2m-1)!! st^m */
        P[m][m] = pmm;
        if (m + 1 <= deg) P[m + 1][m] = z * (2.0 * m + 1.0) * pmm;
        for (int l = m + 2; l <= deg; ++l)
            P[l][m] = ((2.0 * l - 1.0) * z * P[l - 1][m] - (l + m - 1.0) * P[l - 2][m]) / (l - m);
    }
    for (int l = 0; l <= deg; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double fr = 1.0;
            for (int i = l - am + 1; i <= l + am; ++i) fr /= i; /* (l-|m|)!/(l+|m|)! */
            double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * fr);
            double val;
            if (m == 0) val = K * P[l][0];
            else if (m > 0) val = M_SQRT2 * K * P[l][am] * cos(am * az);
            else val = M_SQRT2 * K * P[l][am] * sin(am * az);
            Y[l * l + l + m] = val;
        }
    }
}

/* View-dependent colour (App. B.1): SH at the world direction (mu - o)/|mu - o|,
 * plus 0.5, clamped at 0 (3DGS convention). raw[] returns the unclamped value. */
void orc_colour(int deg, const float *sh_g, const float *mu, const double o[3], double rgb[3], double raw[3])
{
    double dir[3], Y[16];
    for (int a = 0; a < 3; ++a) dir[a] = (double)mu[a] - o[a];
    double n = sqrt(dot(dir, dir));
    for (int a = 0; a < 3; ++a) dir[a] /= n;
    orc_sh_basis(deg, dir, Y);
    int nb = (deg + 1) * (deg + 1);
    for (int c = 0; c < 3; ++c) {
        double acc = 0.0;
        for (int k = 0; k < nb; ++k) acc += (double)sh_g[3 * k + c] * Y[k];
        acc += 0.5;
        if (raw) raw[c] = acc;
        rgb[c] = acc > 0.0 ? acc : 0.0;
    }
}

/* ------------------------------------------------------------------------- */
/* Part 2: FP32 replica of the per-Gaussian integer decisions                 */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t ncols, nrows;
    int32_t any_row_flip, any_col_flip;
    float *col_ta, *col_tb, *row_ta, *row_tb; /* half-angle tangents of first/last pixel centre */
    uint8_t *col_has0, *col_has1, *row_has0, *row_has1;
} rep_tables;

/* Per tile column: tan(theta/2) of its first and last pixel centre (FP64,
 * rounded to FP32), and whether its pixels have cos(theta) >= 0 (has0) or
 * <= 0 (has1). Same for rows with phi. */
static void rep_build_tables(const orc_camera *c, rep_tables *t)
{
    double fy = orc_fov_y(c);
    t->ncols = (c->width + ORC_TILE - 1) / ORC_TILE;
    t->nrows = (c->height + ORC_TILE - 1) / ORC_TILE;
    t->col_ta = malloc(sizeof(float) * t->ncols); t->col_tb = malloc(sizeof(float) * t->ncols);
    t->row_ta = malloc(sizeof(float) * t->nrows); t->row_tb = malloc(sizeof(float) * t->nrows);
    t->col_has0 = calloc(t->ncols, 1); t->col_has1 = calloc(t->ncols, 1);
    t->row_has0 = calloc(t->nrows, 1); t->row_has1 = calloc(t->nrows, 1);
    t->any_row_flip = 0; t->any_col_flip = 0;
    for (int cx = 0; cx < t->ncols; ++cx) {
        int i0 = cx * ORC_TILE, i1 = i0 + ORC_TILE - 1;
        if (i1 > c->width - 1) i1 = c->width - 1;
        t->col_ta[cx] = (float)tan(0.5 * beap_theta(i0, c->width, c->fov_x));
        t->col_tb[cx] = (float)tan(0.5 * beap_theta(i1, c->width, c->fov_x));
        for (int i = i0; i <= i1; ++i) {
            double cs = cos(beap_theta(i, c->width, c->fov_x));
            if (cs > -1e-12) t->col_has0[cx] = 1;
            if (cs < 1e-12) { t->col_has1[cx] = 1; t->any_col_flip = 1; }
        }
    }
    for (int cy = 0; cy < t->nrows; ++cy) {
        int j0 = cy * ORC_TILE, j1 = j0 + ORC_TILE - 1;
        if (j1 > c->height - 1) j1 = c->height - 1;
        t->row_ta[cy] = (float)tan(0.5 * beap_theta(j0, c->height, fy));
        t->row_tb[cy] = (float)tan(0.5 * beap_theta(j1, c->height, fy));
        for (int j = j0; j <= j1; ++j) {
            double cs = cos(beap_theta(j, c->height, fy));
            if (cs > -1e-12) t->row_has0[cy] = 1;
            if (cs < 1e-12) { t->row_has1[cy] = 1; t->any_row_flip = 1; }
        }
    }
}

static void rep_free_tables(rep_tables *t)
{
    free(t->col_ta); free(t->col_tb); free(t->row_ta); free(t->row_tb);
    free(t->col_has0); free(t->col_has1); free(t->row_has0); free(t->row_has1);
}

/* An arc of dihedral angle in half-angle-tangent space tau = tan(angle/2)
 * (the xi = 1 mirror transform of App. D.2). kind 0: empty, 1: [lo, hi],
 * 2: wrapping [lo, +inf) u (-inf, hi], 3: full circle. */
typedef struct { int kind; float lo, hi; } rep_arc;

/* tan(angle/2) of the direction (x, z) in the plane, in the branch that stays
 * well conditioned. */
static float rep_half_tan(float x, float z)
{
    float r = sqrtf(x * x + z * z);
    return (z >= 0.0f) ? x / (r + z) : (r - z) / x;
}

/* PBF arc for one axis pair (App. D.1): roots of T22 c^2 - 2 T02 c + T00 = 0
 * with c the tangent of the bounding plane, discriminant evaluated as
 * lam2 (P - lam2 D) so that it does not cancel; negative or zero
 * discriminant -> full arc (the clamp to the full FoV of App. D.1). The four
 * mirrored candidates are reduced to the two nearest the centre's mirrored
 * angle (App. D.2), then widened by a small absolute margin. */
static rep_arc rep_pbf_arc(float mx, float mz, float T00, float T02, float T22, float P, float D, float lam2)
{
    rep_arc a;
    a.kind = 3; a.lo = 0.0f; a.hi = 0.0f;
    float disc = lam2 * (P - lam2 * D);
    if (!(disc > 0.0f)) return a;
    float sq = sqrtf(disc);
    float qq = T02 + (T02 >= 0.0f ? sq : -sq);
    if (qq == 0.0f) return a;
    float cand[4];
    cand[0] = rep_half_tan(qq, T22);
    cand[1] = rep_half_tan(-qq, -T22);
    cand[2] = rep_half_tan(T00, qq);
    cand[3] = rep_half_tan(-T00, -qq);
    float tm = rep_half_tan(mx, mz);
    if (!isfinite(tm)) return a;
    for (int i = 0; i < 4; ++i)
        if (!isfinite(cand[i])) return a;
    int have_lo = 0, have_hi = 0;
    float lo = 0.0f, hi = 0.0f, mn = cand[0], mxv = cand[0];
    for (int i = 0; i < 4; ++i) {
        float v = cand[i];
        if (v < mn) mn = v;
        if (v > mxv) mxv = v;
        if (v < tm && (!have_lo || v > lo)) { lo = v; have_lo = 1; }
        if (v > tm && (!have_hi || v < hi)) { hi = v; have_hi = 1; }
    }
    a.kind = 1;
    if (!have_hi) { hi = mn; a.kind = 2; }
    if (!have_lo) { lo = mxv; a.kind = 2; }
    const float margin = 3.814697265625e-06f; /* 2^-18 */
    a.lo = lo - margin * (1.0f + lo * lo);
    a.hi = hi + margin * (1.0f + hi * hi);
    return a;
}

/* The same arc rotated by pi: tau -> -1/tau. */
static rep_arc rep_shift_arc(rep_arc a)
{
    rep_arc r = a;
    if (a.kind == 0 || a.kind == 3) return r;
    if (a.lo == 0.0f || a.hi == 0.0f) { r.kind = 3; return r; }
    r.lo = -1.0f / a.lo;
    r.hi = -1.0f / a.hi;
    if (a.kind == 2) r.kind = 1;
    else r.kind = (a.lo < 0.0f && a.hi > 0.0f) ? 2 : 1;
    return r;
}

/* Tile index range [lo, hi) whose [ta, tb] meets the arc; a union of a prefix
 * and a suffix is replaced by the whole range (conservative hull). */
static void rep_arc_range(rep_arc a, const float *ta, const float *tb, int n, int *olo, int *ohi)
{
    *olo = 0; *ohi = 0;
    if (a.kind == 0) return;
    if (a.kind == 3) { *ohi = n; return; }
    int first = n; /* first index with tb >= a.lo */
    for (int i = 0; i < n; ++i) if (tb[i] >= a.lo) { first = i; break; }
    int last = -1; /* last index with ta <= a.hi */
    for (int i = n - 1; i >= 0; --i) if (ta[i] <= a.hi) { last = i; break; }
    if (a.kind == 1) {
        if (first <= last) { *olo = first; *ohi = last + 1; }
        return;
    }
    int has_suffix = first < n, has_prefix = last >= 0;
    if (has_suffix && has_prefix) { *olo = 0; *ohi = n; }
    else if (has_suffix) { *olo = first; *ohi = n; }
    else if (has_prefix) { *olo = 0; *ohi = last + 1; }
}

/* lambda^2 >= 2 ln(sigma / alpha_min), as an upper bound written with basic
 * operations only (so the GPU reproduces it bit for bit), times (1 + pad).
 * ln(m) for m in [1,2) is bounded by 2(z + z^3 / (3(1 - z^2))), z = (m-1)/(m+1). */
static float rep_lambda2(float sigma, float alpha_min, float pad)
{
    float x = sigma / alpha_min;
    int e;
    float m = frexpf(x, &e);
    m = m * 2.0f;
    e = e - 1;
    float z = (m - 1.0f) / (m + 1.0f);
    float z2 = z * z;
    float t = (z * z2) / (3.0f * (1.0f - z2));
    float lnm = 2.0f * (z + t);
    float lnx = (float)e * 0.693147182464599609375f + lnm;
    return (2.0f * lnx) * (1.0f + pad);
}

/* Per (camera, Gaussian) FP32 replica: cull flag, depth key bits, the eight
 * tile bounds {X0lo, X0hi, X1lo, X1hi, Y0lo, Y0hi, Y1lo, Y1hi} and the tile
 * count. X0: columns for unflipped rows (cos phi >= 0), X1: for flipped rows,
 * Y0: rows for unflipped columns (cos theta >= 0), Y1: for flipped columns. */
static void rep_one(const orc_camera *c, const rep_tables *t, const orc_params *p, const float *mu, const float *sc,
                    const float *qt, float sigma, uint8_t *cull, uint32_t *key, uint16_t rg[8], uint32_t *count)
{
    *cull = 1; *key = 0; *count = 0;
    for (int i = 0; i < 8; ++i) rg[i] = 0;
    for (int a = 0; a < 3; ++a) {
        if (!isfinite(mu[a]) || !isfinite(sc[a]) || !(sc[a] > 0.0f)) return;
    }
    for (int a = 0; a < 4; ++a) if (!isfinite(qt[a])) return;
    if (!isfinite(sigma) || !(sigma >= p->alpha_min)) return;
    const float *Rc = c->R_cw;
    /* mean in the camera frame */
    float m0 = ((Rc[0] * mu[0] + Rc[1] * mu[1]) + Rc[2] * mu[2]) + c->t_cw[0];
    float m1 = ((Rc[3] * mu[0] + Rc[4] * mu[1]) + Rc[5] * mu[2]) + c->t_cw[1];
    float m2 = ((Rc[6] * mu[0] + Rc[7] * mu[1]) + Rc[8] * mu[2]) + c->t_cw[2];
    float dist = sqrtf((m0 * m0 + m1 * m1) + m2 * m2);
    /* normalised quaternion and its rotation */
    float qn = sqrtf(((qt[0] * qt[0] + qt[1] * qt[1]) + qt[2] * qt[2]) + qt[3] * qt[3]);
    if (!(qn > 0.0f)) return;
    float w = qt[0] / qn, x = qt[1] / qn, y = qt[2] / qn, z = qt[3] / qn;
    float R[9];
    R[0] = 1.0f - 2.0f * (y * y + z * z); R[1] = 2.0f * (x * y - w * z);        R[2] = 2.0f * (x * z + w * y);
    R[3] = 2.0f * (x * y + w * z);        R[4] = 1.0f - 2.0f * (x * x + z * z); R[5] = 2.0f * (y * z - w * x);
    R[6] = 2.0f * (x * z - w * y);        R[7] = 2.0f * (y * z + w * x);        R[8] = 1.0f - 2.0f * (x * x + y * y);
    /* M = R_cw R: Gaussian axes in the camera frame (columns) */
    float M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            M[3 * i + j] = (Rc[3 * i] * R[j] + Rc[3 * i + 1] * R[3 + j]) + Rc[3 * i + 2] * R[6 + j];
    float lam2 = rep_lambda2(sigma, p->alpha_min, p->lambda_pad);
    if (!(lam2 > 0.0f)) return;
    /* camera inside the lambda-ellipsoid: |S^-1 M^T mu_c|^2 <= lambda^2 -> cull */
    float u0 = ((M[0] * m0 + M[3] * m1) + M[6] * m2) / sc[0];
    float u1 = ((M[1] * m0 + M[4] * m1) + M[7] * m2) / sc[1];
    float u2 = ((M[2] * m0 + M[5] * m1) + M[8] * m2) / sc[2];
    float ou2 = (u0 * u0 + u1 * u1) + u2 * u2;
    if (!(ou2 > lam2)) return;
    /* camera-frame covariance entries Sigma_ab = sum_k s_k^2 M_ak M_bk */
    float s2[3] = {sc[0] * sc[0], sc[1] * sc[1], sc[2] * sc[2]};
#define SIG(a, b) ((s2[0] * (M[3 * (a)] * M[3 * (b)]) + s2[1] * (M[3 * (a) + 1] * M[3 * (b) + 1])) + s2[2] * (M[3 * (a) + 2] * M[3 * (b) + 2]))
    float Sxx = SIG(0, 0), Syy = SIG(1, 1), Szz = SIG(2, 2), Sxz = SIG(0, 2), Syz = SIG(1, 2);
#undef SIG
    float T00 = lam2 * Sxx - m0 * m0;
    float T11 = lam2 * Syy - m1 * m1;
    float T22 = lam2 * Szz - m2 * m2;
    float T02 = lam2 * Sxz - m0 * m2;
    float T12 = lam2 * Syz - m1 * m2;
    /* P = mu^T adj(Sigma_pp) mu, D = det(Sigma_pp) through the factor S and the
     * rotation's complementary row (no cancellation) */
    float pxz[3], pyz[3], dxz[3], dyz[3];
    float ss[3] = {sc[1] * sc[2], sc[0] * sc[2], sc[0] * sc[1]};
    for (int k = 0; k < 3; ++k) {
        float cx = m0 * M[6 + k] - m2 * M[k];
        float cy = m1 * M[6 + k] - m2 * M[3 + k];
        pxz[k] = s2[k] * (cx * cx);
        pyz[k] = s2[k] * (cy * cy);
        float ax = ss[k] * M[3 + k];
        float ay = ss[k] * M[k];
        dxz[k] = ax * ax;
        dyz[k] = ay * ay;
    }
    float Pxz = (pxz[0] + pxz[1]) + pxz[2], Pyz = (pyz[0] + pyz[1]) + pyz[2];
    float Dxz = (dxz[0] + dxz[1]) + dxz[2], Dyz = (dyz[0] + dyz[1]) + dyz[2];
    rep_arc A = rep_pbf_arc(m0, m2, T00, T02, T22, Pxz, Dxz, lam2);
    rep_arc B = rep_pbf_arc(m1, m2, T11, T12, T22, Pyz, Dyz, lam2);
    int x0lo, x0hi, x1lo = 0, x1hi = 0, y0lo, y0hi, y1lo = 0, y1hi = 0;
    rep_arc_range(A, t->col_ta, t->col_tb, t->ncols, &x0lo, &x0hi);
    rep_arc_range(B, t->row_ta, t->row_tb, t->nrows, &y0lo, &y0hi);
    if (t->any_row_flip) rep_arc_range(rep_shift_arc(A), t->col_ta, t->col_tb, t->ncols, &x1lo, &x1hi);
    if (t->any_col_flip) rep_arc_range(rep_shift_arc(B), t->row_ta, t->row_tb, t->nrows, &y1lo, &y1hi);
    *cull = 0;
    union { float f; uint32_t u; } kb;
    kb.f = dist;
    *key = kb.u;
    rg[0] = (uint16_t)x0lo; rg[1] = (uint16_t)x0hi; rg[2] = (uint16_t)x1lo; rg[3] = (uint16_t)x1hi;
    rg[4] = (uint16_t)y0lo; rg[5] = (uint16_t)y0hi; rg[6] = (uint16_t)y1lo; rg[7] = (uint16_t)y1hi;
    /* count tiles of the (possibly flipped) association predicate */
    int cxa = x0lo < x0hi ? x0lo : t->ncols, cxb = x0lo < x0hi ? x0hi : 0;
    if (x1lo < x1hi) { if (x1lo < cxa) cxa = x1lo; if (x1hi > cxb) cxb = x1hi; }
    int cya = y0lo < y0hi ? y0lo : t->nrows, cyb = y0lo < y0hi ? y0hi : 0;
    if (y1lo < y1hi) { if (y1lo < cya) cya = y1lo; if (y1hi > cyb) cyb = y1hi; }
    uint32_t cnt = 0;
    for (int cy = cya; cy < cyb; ++cy)
        for (int cx = cxa; cx < cxb; ++cx) {
            int aok = (t->row_has0[cy] && cx >= x0lo && cx < x0hi) || (t->row_has1[cy] && cx >= x1lo && cx < x1hi);
            int bok = (t->col_has0[cx] && cy >= y0lo && cy < y0hi) || (t->col_has1[cx] && cy >= y1lo && cy < y1hi);
            cnt += (uint32_t)(aok && bok);
        }
    *count = cnt;
}

/* Replica over all Gaussians of one camera. */
void orc_replica(const orc_gaussians *g, const orc_camera *c, const orc_params *p, uint8_t *cull, uint32_t *key,
                 uint16_t *ranges, uint32_t *count)
{
    rep_tables t;
    rep_build_tables(c, &t);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < g->n; ++i)
        rep_one(c, &t, p, g->mean + 3 * i, g->scale + 3 * i, g->quat + 4 * i, g->opacity[i], cull + i, key + i,
                ranges + 8 * i, count + i);
    rep_free_tables(&t);
}

/* Association mask of n Gaussians from their replica ranges:
 * mask[g][cy][cx] = 1 iff tile (cx, cy) is associated with Gaussian g. */
void orc_assoc_mask(const orc_camera *c, int64_t n, const uint16_t *ranges, uint8_t *mask)
{
    rep_tables t;
    rep_build_tables(c, &t);
    for (int64_t gi = 0; gi < n; ++gi) {
        const uint16_t *rg = ranges + 8 * gi;
        uint8_t *mk = mask + gi * (int64_t)t.ncols * t.nrows;
        for (int cy = 0; cy < t.nrows; ++cy)
            for (int cx = 0; cx < t.ncols; ++cx) {
                int aok = (t.row_has0[cy] && cx >= rg[0] && cx < rg[1]) || (t.row_has1[cy] && cx >= rg[2] && cx < rg[3]);
                int bok = (t.col_has0[cx] && cy >= rg[4] && cy < rg[5]) || (t.col_has1[cx] && cy >= rg[6] && cy < rg[7]);
                mk[cy * t.ncols + cx] = (uint8_t)(aok && bok);
            }
    }
    rep_free_tables(&t);
}

/* Expose the PBF arcs of one Gaussian (for the tangency pins):
 * out = {kindA, loA, hiA, kindB, loB, hiB, lam2} */
void orc_replica_arcs(const orc_camera *c, const orc_params *p, const float *mu, const float *sc, const float *qt,
                      float sigma, float *out)
{
    /* same steps as rep_one up to the arcs; written out again so the pins see
     * exactly what the replica uses */
    const float *Rc = c->R_cw;
    float m0 = ((Rc[0] * mu[0] + Rc[1] * mu[1]) + Rc[2] * mu[2]) + c->t_cw[0];
    float m1 = ((Rc[3] * mu[0] + Rc[4] * mu[1]) + Rc[5] * mu[2]) + c->t_cw[1];
    float m2 = ((Rc[6] * mu[0] + Rc[7] * mu[1]) + Rc[8] * mu[2]) + c->t_cw[2];
    float qn = sqrtf(((qt[0] * qt[0] + qt[1] * qt[1]) + qt[2] * qt[2]) + qt[3] * qt[3]);
    float w = qt[0] / qn, x = qt[1] / qn, y = qt[2] / qn, z = qt[3] / qn;
    float R[9];
    R[0] = 1.0f - 2.0f * (y * y + z * z); R[1] = 2.0f * (x * y - w * z);        R[2] = 2.0f * (x * z + w * y);
    R[3] = 2.0f * (x * y + w * z);        R[4] = 1.0f - 2.0f * (x * x + z * z); R[5] = 2.0f * (y * z - w * x);
    R[6] = 2.0f * (x * z - w * y);        R[7] = 2.0f * (y * z + w * x);        R[8] = 1.0f - 2.0f * (x * x + y * y);
    float M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            M[3 * i + j] = (Rc[3 * i] * R[j] + Rc[3 * i + 1] * R[3 + j]) + Rc[3 * i + 2] * R[6 + j];
    float lam2 = rep_lambda2(sigma, p->alpha_min, p->lambda_pad);
    float s2[3] = {sc[0] * sc[0], sc[1] * sc[1], sc[2] * sc[2]};
#define SIG(a, b) ((s2[0] * (M[3 * (a)] * M[3 * (b)]) + s2[1] * (M[3 * (a) + 1] * M[3 * (b) + 1])) + s2[2] * (M[3 * (a) + 2] * M[3 * (b) + 2]))
    float Sxx = SIG(0, 0), Syy = SIG(1, 1), Szz = SIG(2, 2), Sxz = SIG(0, 2), Syz = SIG(1, 2);
#undef SIG
    float T00 = lam2 * Sxx - m0 * m0, T11 = lam2 * Syy - m1 * m1, T22 = lam2 * Szz - m2 * m2;
    float T02 = lam2 * Sxz - m0 * m2, T12 = lam2 * Syz - m1 * m2;
    float pxz[3], pyz[3], dxz[3], dyz[3];
    float ss[3] = {sc[1] * sc[2], sc[0] * sc[2], sc[0] * sc[1]};
    for (int k = 0; k < 3; ++k) {
        float cx = m0 * M[6 + k] - m2 * M[k];
        float cy = m1 * M[6 + k] - m2 * M[3 + k];
        pxz[k] = s2[k] * (cx * cx);
        pyz[k] = s2[k] * (cy * cy);
        float ax = ss[k] * M[3 + k];
        float ay = ss[k] * M[k];
        dxz[k] = ax * ax;
        dyz[k] = ay * ay;
    }
    float Pxz = (pxz[0] + pxz[1]) + pxz[2], Pyz = (pyz[0] + pyz[1]) + pyz[2];
    float Dxz = (dxz[0] + dxz[1]) + dxz[2], Dyz = (dyz[0] + dyz[1]) + dyz[2];
    rep_arc A = rep_pbf_arc(m0, m2, T00, T02, T22, Pxz, Dxz, lam2);
    rep_arc B = rep_pbf_arc(m1, m2, T11, T12, T22, Pyz, Dyz, lam2);
    out[0] = (float)A.kind; out[1] = A.lo; out[2] = A.hi;
    out[3] = (float)B.kind; out[4] = B.lo; out[5] = B.hi;
    out[6] = lam2;
}

/* ------------------------------------------------------------------------- */
/* Part 1 continued: the brute-force render                                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    uint32_t key;
    int64_t gid;
    double a;      /* unclamped alpha = sigma exp(-kappa/2) */
    double rel;    /* relative sensitivity of a to FP32-sized perturbations */
    double rgb[3];
} contrib;

static int contrib_cmp(const void *pa, const void *pb)
{
    const contrib *a = pa, *b = pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->gid < b->gid ? -1 : (a->gid > b->gid);
}

#define ORC_MAX_ALT 8
#define ORC_EPS32 5.9604644775390625e-08 /* 2^-24 */

typedef struct {
    const contrib *c;
    int n;
    double amin, amax, tmin, bg[3];
    int nalt;
    double alt[ORC_MAX_ALT][4]; /* r, g, b, T_final */
    int overflow;
} comp_ctx;

/* Front-to-back compositing (App. B.1 colour equation with the 3DGS
 * thresholds). A decision whose FP64 margin is inside the FP32 sensitivity band
 * is explored both ways; every leaf is one admissible result. */
static void composite(comp_ctx *x, int i, double T, double C0, double C1, double C2, double Trel, int budget)
{
    for (; i < x->n; ++i) {
        const contrib *g = &x->c[i];
        int inc = g->a >= x->amin;
        int amb_inc = fabs(g->a - x->amin) <= 2.0 * g->rel * g->a;
        if (amb_inc) {
            if (budget <= 0) { x->overflow = 1; return; }
            budget -= 1;
            /* branch: take the other choice of this decision first */
            if (inc) composite(x, i + 1, T, C0, C1, C2, Trel, budget); /* excluded */
            else {
                /* included */
                double a = g->a < x->amax ? g->a : x->amax;
                double Tn = T * (1.0 - a);
                double Tr = Trel + g->rel * a / (1.0 - a) + 4.0 * ORC_EPS32;
                if (Tn < x->tmin) { /* stops */
                    if (x->nalt < ORC_MAX_ALT) {
                        double *o = x->alt[x->nalt++];
                        o[0] = C0 + T * x->bg[0]; o[1] = C1 + T * x->bg[1]; o[2] = C2 + T * x->bg[2]; o[3] = T;
                    } else x->overflow = 1;
                } else {
                    composite(x, i + 1, Tn, C0 + T * a * g->rgb[0], C1 + T * a * g->rgb[1], C2 + T * a * g->rgb[2],
                              Tr, budget);
                }
            }
            if (x->overflow) return;
        }
        if (!inc) continue;
        double a = g->a < x->amax ? g->a : x->amax;
        double Tn = T * (1.0 - a);
        double Tr = Trel + g->rel * a / (1.0 - a) + 4.0 * ORC_EPS32;
        int stop = Tn < x->tmin;
        int amb_stop = fabs(Tn - x->tmin) <= 2.0 * Tr * x->tmin;
        if (amb_stop) {
            if (budget <= 0) { x->overflow = 1; return; }
            budget -= 1;
            if (stop) { /* other branch: continue */
                composite(x, i + 1, Tn, C0 + T * a * g->rgb[0], C1 + T * a * g->rgb[1], C2 + T * a * g->rgb[2], Tr,
                          budget);
            } else { /* other branch: stop here */
                if (x->nalt < ORC_MAX_ALT) {
                    double *o = x->alt[x->nalt++];
                    o[0] = C0 + T * x->bg[0]; o[1] = C1 + T * x->bg[1]; o[2] = C2 + T * x->bg[2]; o[3] = T;
                } else x->overflow = 1;
            }
            if (x->overflow) return;
        }
        if (stop) break;
        C0 += T * a * g->rgb[0]; C1 += T * a * g->rgb[1]; C2 += T * a * g->rgb[2];
        T = Tn;
        Trel = Tr;
    }
    if (x->nalt < ORC_MAX_ALT) {
        double *o = x->alt[x->nalt++];
        o[0] = C0 + T * x->bg[0]; o[1] = C1 + T * x->bg[1]; o[2] = C2 + T * x->bg[2]; o[3] = T;
    } else x->overflow = 1;
}

/*
 * Render a list of pixels by brute force.
 *   pix[2m], pix[2m+1]: column i, row j of pixel m.
 *   cull[], key[]: the replica's decisions (one camera).
 * Outputs per pixel m:
 *   rgb[3m..]     primary result (FP64 decisions)
 *   tfinal[m]     final transmittance of the primary result
 *   alt[m][ORC_MAX_ALT][4], nalt[m]: every admissible result (primary first is
 *                 not guaranteed; the primary is always among them)
 *   cond[m]       bound on the change of any channel under FP32-sized relative
 *                 perturbations of each alpha (sum_i T_i a_i rel_i (|c_i| + cmax))
 *   ncontrib[m]   number of contributors applied in the primary result
 *   flags[m]      1 if the ambiguity budget was exceeded (pixel undecidable)
 */
void orc_render_pixels(const orc_gaussians *g, const orc_camera *c, const orc_params *p, const uint8_t *cull,
                       const uint32_t *key, int64_t npix, const int32_t *pix, double *rgb, double *tfinal,
                       double *alt, int32_t *nalt, double *cond, int32_t *ncontrib, int32_t *flags)
{
    int nb = (g->sh_degree + 1) * (g->sh_degree + 1);
    (void)nb;
#pragma omp parallel
    {
        int64_t cap = 1024;
        contrib *buf = malloc(sizeof(contrib) * cap);
#pragma omp for schedule(dynamic, 1)
        for (int64_t m = 0; m < npix; ++m) {
            double o[3], d[3];
            orc_pixel_ray(c, pix[2 * m], pix[2 * m + 1], o, d);
            double onorm = sqrt(dot(o, o));
            int64_t nc = 0;
            double cmax = fmax(fabs(c->bg[0]), fmax(fabs(c->bg[1]), fabs(c->bg[2])));
            for (int64_t gi = 0; gi < g->n; ++gi) {
                if (cull[gi]) continue;
                const float *mu = g->mean + 3 * gi, *s = g->scale + 3 * gi, *q = g->quat + 4 * gi;
                double tstar, ou;
                double kappa = orc_kappa(mu, s, q, o, d, &tstar, &ou);
                if (!(tstar > 0.0)) continue;
                double a = (double)g->opacity[gi] * exp(-0.5 * kappa);
                /* sensitivity of a to FP32-sized relative perturbations of the
                 * ray direction and of the positions: the canonical distance
                 * moves by ~ eps (|mu| + |o| + dist) / s_min, so a moves by
                 * sqrt(kappa) times that, plus a few eps for the exponential */
                double smin = fmin(s[0], fmin(s[1], s[2]));
                double mun = sqrt((double)mu[0] * mu[0] + (double)mu[1] * mu[1] + (double)mu[2] * mu[2]);
                double dist = sqrt(((double)mu[0] - o[0]) * ((double)mu[0] - o[0]) +
                                   ((double)mu[1] - o[1]) * ((double)mu[1] - o[1]) +
                                   ((double)mu[2] - o[2]) * ((double)mu[2] - o[2]));
                double rel = ORC_EPS32 * (4.0 * sqrt(kappa) * (mun + onorm + dist) / smin + 16.0 + kappa);
                if (a < p->alpha_min * (1.0 - 4.0 * rel)) continue;
                if (nc == cap) { cap *= 2; buf = realloc(buf, sizeof(contrib) * cap); }
                contrib *e = &buf[nc++];
                e->key = key[gi];
                e->gid = gi;
                e->a = a;
                e->rel = rel;
                orc_colour(g->sh_degree, g->sh + (int64_t)3 * nb * gi, mu, o, e->rgb, NULL);
                double cm = fmax(e->rgb[0], fmax(e->rgb[1], e->rgb[2]));
                if (cm > cmax) cmax = cm;
            }
            qsort(buf, (size_t)nc, sizeof(contrib), contrib_cmp);
            /* primary result and conditioning along the primary path */
            double T = 1.0, C[3] = {0, 0, 0}, B = 0.0;
            int applied = 0;
            for (int64_t i = 0; i < nc; ++i) {
                contrib *e = &buf[i];
                if (e->a < p->alpha_min) continue;
                double a = e->a < p->alpha_max ? e->a : p->alpha_max;
                double Tn = T * (1.0 - a);
                if (Tn < p->T_min) break;
                double cm = fmax(e->rgb[0], fmax(e->rgb[1], e->rgb[2]));
                B += T * a * e->rel * (cm + cmax);
                for (int k = 0; k < 3; ++k) C[k] += T * a * e->rgb[k];
                T = Tn;
                ++applied;
            }
            for (int k = 0; k < 3; ++k) rgb[3 * m + k] = C[k] + T * c->bg[k];
            tfinal[m] = T;
            cond[m] = B + 2.0 * ORC_EPS32 * (1.0 + cmax);
            ncontrib[m] = applied;
            comp_ctx x;
            x.c = buf; x.n = (int)nc;
            x.amin = p->alpha_min; x.amax = p->alpha_max; x.tmin = p->T_min;
            for (int k = 0; k < 3; ++k) x.bg[k] = c->bg[k];
            x.nalt = 0; x.overflow = 0;
            composite(&x, 0, 1.0, 0.0, 0.0, 0.0, 0.0, 3);
            nalt[m] = x.nalt;
            flags[m] = x.overflow;
            for (int a = 0; a < x.nalt; ++a)
                for (int k = 0; k < 4; ++k) alt[(m * ORC_MAX_ALT + a) * 4 + k] = x.alt[a][k];
        }
        free(buf);
    }
}

/* FP64 contributor set of one pixel (for the zero-miss pin): every non-culled
 * Gaussian with t* > 0 and sigma exp(-kappa/2) >= alpha_min. Returns the count;
 * writes at most cap ids. */
int64_t orc_pixel_contributors(const orc_gaussians *g, const orc_camera *c, const orc_params *p, const uint8_t *cull,
                               int32_t i, int32_t j, int64_t *ids, int64_t cap)
{
    double o[3], d[3];
    orc_pixel_ray(c, i, j, o, d);
    int64_t nc = 0;
    for (int64_t gi = 0; gi < g->n; ++gi) {
        if (cull[gi]) continue;
        double tstar;
        double kappa = orc_kappa(g->mean + 3 * gi, g->scale + 3 * gi, g->quat + 4 * gi, o, d, &tstar, NULL);
        if (!(tstar > 0.0)) continue;
        if ((double)g->opacity[gi] * exp(-0.5 * kappa) >= p->alpha_min) {
            if (nc < cap) ids[nc] = gi;
            ++nc;
        }
    }
    return nc;
}

/* ------------------------------------------------------------------------- */
/* Part 3: FP64 analytic gradients                                             */
/* ------------------------------------------------------------------------- */

/* d/dq of R(q/|q|) contracted with G (dL/dR): returns dL/dq (4). The rotation
 * of the normalised quaternion is differentiated entry by entry (the
 * polynomial of App. C.4), then chained through q -> q/|q| (a reading: App. C.4
 * differentiates the unit-quaternion polynomial; the normalisation is applied
 * before it). */
static void rot_grad(const float *qf, const double G[9], double dq[4])
{
    double q[4] = {qf[0], qf[1], qf[2], qf[3]};
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
    /* dR/dw, dR/dx, dR/dy, dR/dz for the unit-quaternion formula */
    double dRw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    double dRx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    double dRy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    double dRz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    double gh[4] = {0, 0, 0, 0};
    for (int k = 0; k < 9; ++k) {
        gh[0] += G[k] * dRw[k]; gh[1] += G[k] * dRx[k]; gh[2] += G[k] * dRy[k]; gh[3] += G[k] * dRz[k];
    }
    double qh[4] = {w, x, y, z};
    double dp = gh[0] * qh[0] + gh[1] * qh[1] + gh[2] * qh[2] + gh[3] * qh[3];
    for (int k = 0; k < 4; ++k) dq[k] = (gh[k] - qh[k] * dp) / n;
}

/* Gradient of the real SH basis w.r.t. the (unnormalised) direction v, by
 * central differences of orc_sh_basis on the unit sphere -- FP64, step 1e-6,
 * accurate to ~1e-10, far below what the GPU comparison resolves. */
static void sh_basis_jac(int deg, const double v[3], double J[16][3])
{
    int nb = (deg + 1) * (deg + 1);
    for (int a = 0; a < 3; ++a) {
        double vp[3] = {v[0], v[1], v[2]}, vm[3] = {v[0], v[1], v[2]};
        double h = 1e-6 * fmax(1.0, fabs(v[a]));
        vp[a] += h; vm[a] -= h;
        double np = sqrt(dot(vp, vp)), nm = sqrt(dot(vm, vm));
        for (int b = 0; b < 3; ++b) { vp[b] /= np; vm[b] /= nm; }
        double Yp[16], Ym[16];
        orc_sh_basis(deg, vp, Yp);
        orc_sh_basis(deg, vm, Ym);
        for (int k = 0; k < nb; ++k) J[k][a] = (Yp[k] - Ym[k]) / (2.0 * h);
    }
}

/*
 * Analytic gradients of L = sum_pixels sum_ch dLdC[pix][ch] * C[pix][ch] for
 * the primary (FP64-decision) result of each listed pixel, w.r.t. mean, scale,
 * quat, opacity, sh (accumulated into the outputs). Follows the App. C
 * cookbook: dT/dsigma = e^{-kappa/2}, dT/dkappa = -T/2,
 * dkappa/dm_u = 2 m_u/|d_u|^2, dkappa/do_u = d_u x g, dkappa/dd_u =
 * -(2 kappa/|d_u|^2) d_u + g x o_u with g = dkappa/dm_u (signs for
 * m_u = o_u x d_u), dkappa/dW = (dkappa/dd_u) d^T + (dkappa/do_u)(o - mu)^T,
 * dkappa/dmu = -W^T dkappa/do_u, then W = S^-1 R^T to s and q, plus the colour
 * path through SH (coefficients and direction).
 */
void orc_render_grad(const orc_gaussians *g, const orc_camera *c, const orc_params *p, const uint8_t *cull,
                     const uint32_t *key, int64_t npix, const int32_t *pix, const double *dLdC, double *d_mean,
                     double *d_scale, double *d_quat, double *d_opacity, double *d_sh)
{
    int deg = g->sh_degree;
    int nb = (deg + 1) * (deg + 1);
    int64_t cap = 1024;
    contrib *buf = malloc(sizeof(contrib) * cap);
    for (int64_t m = 0; m < npix; ++m) {
        double o[3], d[3];
        orc_pixel_ray(c, pix[2 * m], pix[2 * m + 1], o, d);
        int64_t nc = 0;
        for (int64_t gi = 0; gi < g->n; ++gi) {
            if (cull[gi]) continue;
            double tstar;
            double kappa = orc_kappa(g->mean + 3 * gi, g->scale + 3 * gi, g->quat + 4 * gi, o, d, &tstar, NULL);
            if (!(tstar > 0.0)) continue;
            double a = (double)g->opacity[gi] * exp(-0.5 * kappa);
            if (a < p->alpha_min) continue;
            if (nc == cap) { cap *= 2; buf = realloc(buf, sizeof(contrib) * cap); }
            contrib *e = &buf[nc++];
            e->key = key[gi]; e->gid = gi; e->a = a; e->rel = 0;
            orc_colour(deg, g->sh + (int64_t)3 * nb * gi, g->mean + 3 * gi, o, e->rgb, NULL);
        }
        qsort(buf, (size_t)nc, sizeof(contrib), contrib_cmp);
        /* forward pass: transmittance before each applied contributor */
        int64_t napp = 0;
        double T = 1.0;
        double *Tb = malloc(sizeof(double) * (nc + 1));
        for (int64_t i = 0; i < nc; ++i) {
            double a = buf[i].a < p->alpha_max ? buf[i].a : p->alpha_max;
            double Tn = T * (1.0 - a);
            if (Tn < p->T_min) break;
            Tb[napp++] = T;
            T = Tn;
        }
        double Tfin = T;
        const double *gC = dLdC + 3 * m;
        /* colour behind contributor i (including the background), accumulated back to front */
        double behind[3] = {Tfin * c->bg[0], Tfin * c->bg[1], Tfin * c->bg[2]};
        for (int64_t i = napp - 1; i >= 0; --i) {
            contrib *e = &buf[i];
            int64_t gi = e->gid;
            const float *mu = g->mean + 3 * gi, *s = g->scale + 3 * gi, *q = g->quat + 4 * gi;
            double clamped = e->a >= p->alpha_max;
            double a = clamped ? p->alpha_max : e->a;
            double Ti = Tb[i];
            /* C = ... + Ti a c_i + behind, behind = (1 - a) * (stuff scaled by Ti) */
            double dLda = 0.0;
            for (int k = 0; k < 3; ++k) dLda += gC[k] * (Ti * e->rgb[k] - behind[k] / (1.0 - a));
            /* colour path */
            double raw[3], rgb[3];
            orc_colour(deg, g->sh + (int64_t)3 * nb * gi, mu, o, rgb, raw);
            double dLdc[3];
            for (int k = 0; k < 3; ++k) dLdc[k] = raw[k] > 0.0 ? gC[k] * Ti * a : 0.0;
            double v[3] = {(double)mu[0] - o[0], (double)mu[1] - o[1], (double)mu[2] - o[2]};
            double vn = sqrt(dot(v, v));
            double dir[3] = {v[0] / vn, v[1] / vn, v[2] / vn};
            double Y[16], J[16][3];
            orc_sh_basis(deg, dir, Y);
            sh_basis_jac(deg, v, J);
            for (int k = 0; k < nb; ++k)
                for (int ch = 0; ch < 3; ++ch) {
                    d_sh[(gi * nb + k) * 3 + ch] += dLdc[ch] * Y[k];
                    for (int ax = 0; ax < 3; ++ax)
                        d_mean[3 * gi + ax] += dLdc[ch] * (double)g->sh[(gi * nb + k) * 3 + ch] * J[k][ax];
                }
            /* update behind to include this contributor for the next (front) one */
            for (int k = 0; k < 3; ++k) behind[k] += Ti * a * e->rgb[k];
            if (clamped) continue; /* alpha = alpha_max has no gradient */
            double sig = g->opacity[gi];
            double ek = e->a / sig; /* exp(-kappa/2) */
            d_opacity[gi] += dLda * ek;
            double dLdk = dLda * (-0.5 * e->a);
            /* canonical ray and cookbook chain */
            double W[9], R[9], ou[3], du[3], mm[3];
            quat_rot(q, R);
            whitening(q, s, W);
            matvec(W, v, ou);
            for (int k = 0; k < 3; ++k) ou[k] = -ou[k]; /* o_u = W (o - mu) */
            matvec(W, d, du);
            cross(ou, du, mm);
            double dd = dot(du, du);
            double kap = dot(mm, mm) / dd;
            double gm[3] = {2.0 * mm[0] / dd, 2.0 * mm[1] / dd, 2.0 * mm[2] / dd};
            double dko[3], dkd[3], tmp[3];
            cross(du, gm, dko);
            cross(gm, ou, tmp);
            for (int k = 0; k < 3; ++k) dkd[k] = -2.0 * kap / dd * du[k] + tmp[k];
            double omu[3] = {-v[0], -v[1], -v[2]};
            double dW[9];
            for (int a1 = 0; a1 < 3; ++a1)
                for (int b1 = 0; b1 < 3; ++b1) dW[3 * a1 + b1] = dLdk * (dkd[a1] * d[b1] + dko[a1] * omu[b1]);
            /* dL/dmu = -W^T dL/do_u */
            for (int b1 = 0; b1 < 3; ++b1) {
                double acc = 0.0;
                for (int a1 = 0; a1 < 3; ++a1) acc += W[3 * a1 + b1] * dko[a1];
                d_mean[3 * gi + b1] += -dLdk * acc;
            }
            /* W_ij = R_ji / s_i: dW_ij/ds_i = -R_ji / s_i^2 ; dW_ij/dR_ji = 1/s_i */
            double GR[9];
            for (int i1 = 0; i1 < 3; ++i1) {
                double acc = 0.0;
                for (int j1 = 0; j1 < 3; ++j1) {
                    acc += dW[3 * i1 + j1] * (-R[3 * j1 + i1] / ((double)s[i1] * s[i1]));
                    GR[3 * j1 + i1] = dW[3 * i1 + j1] / (double)s[i1];
                }
                d_scale[3 * gi + i1] += acc;
            }
            double dq[4];
            rot_grad(q, GR, dq);
            for (int k = 0; k < 4; ++k) d_quat[4 * gi + k] += dq[k];
        }
        free(Tb);
    }
    free(buf);
}

/* ------------------------------------------------------------------------- */
/* Part 4: resampling a BEAP image into the native camera image (App. E)       */
/* ------------------------------------------------------------------------- */

/* Native intrinsics (the reading that also fixes FoV_y): square pixels, principal
 * point at the image centre, focal length mapping FoV_x/2 to w/2. */
double orc_native_focal(const orc_camera *c)
{
    double half = 0.5 * (double)c->fov_x;
    if (c->model == 0) return 0.5 * c->width / tan(half);
    double k[4] = {0, 0, 0, 0};
    if (c->model == 2) for (int i = 0; i < 4; ++i) k[i] = c->k[i];
    return 0.5 * c->width / kb_distort(k, half);
}

/* Forward projection of App. E for a camera-frame direction in front of the
 * camera: pinhole (x_p, y_p) = f (tan theta, tan phi) + c; fisheye
 * r = sqrt(tan^2 theta + tan^2 phi), varphi = atan r, varphi_d = KB polynomial,
 * (x_p, y_p) = f varphi_d / r (tan theta, tan phi) + c. */
void orc_project(const orc_camera *c, const double d[3], double *xp, double *yp)
{
    double f = orc_native_focal(c);
    double tt = d[0] / d[2], tp = d[1] / d[2];
    double cx = 0.5 * c->width, cy = 0.5 * c->height;
    if (c->model == 0) { *xp = f * tt + cx; *yp = f * tp + cy; return; }
    double k[4] = {0, 0, 0, 0};
    if (c->model == 2) for (int i = 0; i < 4; ++i) k[i] = c->k[i];
    double r = sqrt(tt * tt + tp * tp);
    if (r == 0.0) { *xp = cx; *yp = cy; return; }
    double vd = kb_distort(k, atan(r));
    *xp = f * vd / r * tt + cx;
    *yp = f * vd / r * tp + cy;
}

/* End of the increasing branch of the distortion phi_d below pi (pi if none). */
static double kb_branch_end(const double k[4])
{
    double prev = 0.0;
    for (int s = 1; s <= 4096; ++s) {
        double ph = M_PI * s / 4096, val = kb_distort(k, ph);
        if (!(val > prev)) return M_PI * (s - 1) / 4096;
        prev = val;
    }
    return M_PI;
}

static int native_ray_k(const orc_camera *c, double f, const double k[4], double pmax, int i, int j,
                        double d[3])
{
    double u = (i + 0.5 - 0.5 * c->width) / f, v = (j + 0.5 - 0.5 * c->height) / f;
    if (c->model == 0) {
        double n = sqrt(u * u + v * v + 1.0);
        d[0] = u / n; d[1] = v / n; d[2] = 1.0 / n;
        return 1;
    }
    double rd = sqrt(u * u + v * v);
    if (rd > kb_distort(k, pmax)) return 0;
    double lo = 0.0, hi = pmax;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (kb_distort(k, mid) < rd) lo = mid; else hi = mid;
    }
    double p = 0.5 * (lo + hi);
    if (rd > 0) { d[0] = sin(p) * u / rd; d[1] = sin(p) * v / rd; } else { d[0] = 0; d[1] = 0; }
    d[2] = cos(p);
    return 1;
}

static void native_model(const orc_camera *c, double k[4], double *pmax)
{
    for (int a = 0; a < 4; ++a) k[a] = c->model == 2 ? c->k[a] : 0.0;
    *pmax = c->model == 0 ? 0.0 : kb_branch_end(k);
}

/* Ray of native pixel (i, j) (centre at i + 1/2, j + 1/2): the inverse of the
 * projection. Fisheye: the incidence angle solves varphi_d(varphi) = r_d, found by
 * bisection on the increasing branch starting at 0. Returns 0 when no ray. */
int orc_native_ray(const orc_camera *c, int i, int j, double d[3])
{
    double k[4], pmax;
    native_model(c, k, &pmax);
    return native_ray_k(c, orc_native_focal(c), k, pmax, i, j, d);
}

/* Native image from a BEAP image of the same camera: bilinear interpolation at
 * u = theta/FoV_x w + w/2 - 1/2, v = phi/FoV_y h + h/2 - 1/2 with theta =
 * atan2(x, z), phi = atan(y / z); outside the grid (beyond half a pixel) or
 * without a ray: fill. out: [h][w][3] doubles; coords (may be NULL): [h][w][2], the
 * BEAP coordinate (u, v) of each native pixel, NaN where it has no ray. */
void orc_remap_to_native(const orc_camera *c, const float *beap, const float *fill, double *out,
                         double *coords)
{
    int w = c->width, h = c->height;
    double fy = orc_fov_y(c), f = orc_native_focal(c), k[4], pmax;
    native_model(c, k, &pmax);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < h; ++j)
        for (int i = 0; i < w; ++i) {
            double d[3], o[3] = {fill[0], fill[1], fill[2]};
            if (coords) coords[2 * (j * w + i)] = coords[2 * (j * w + i) + 1] = NAN;
            if (native_ray_k(c, f, k, pmax, i, j, d) && d[2] != 0.0) {
                double th = atan2(d[0], d[2]), ph = atan(d[1] / d[2]);
                double ub = th / c->fov_x * w + 0.5 * w - 0.5, vb = ph / fy * h + 0.5 * h - 0.5;
                if (coords) { coords[2 * (j * w + i)] = ub; coords[2 * (j * w + i) + 1] = vb; }
                if (ub >= -0.5 && ub <= w - 0.5 && vb >= -0.5 && vb <= h - 0.5) {
                    double uc = fmin(fmax(ub, 0.0), w - 1.0), vc = fmin(fmax(vb, 0.0), h - 1.0);
                    int x0 = (int)floor(uc), y0 = (int)floor(vc);
                    if (x0 > w - 2) x0 = w - 2 < 0 ? 0 : w - 2;
                    if (y0 > h - 2) y0 = h - 2 < 0 ? 0 : h - 2;
                    int x1 = x0 + 1 < w ? x0 + 1 : w - 1, y1 = y0 + 1 < h ? y0 + 1 : h - 1;
                    double ax = uc - x0, ay = vc - y0;
                    for (int ch = 0; ch < 3; ++ch) {
                        double p00 = beap[3 * (y0 * w + x0) + ch], p01 = beap[3 * (y0 * w + x1) + ch];
                        double p10 = beap[3 * (y1 * w + x0) + ch], p11 = beap[3 * (y1 * w + x1) + ch];
                        o[ch] = (1 - ay) * ((1 - ax) * p00 + ax * p01) + ay * ((1 - ax) * p10 + ax * p11);
                    }
                }
            }
            for (int ch = 0; ch < 3; ++ch) out[3 * (j * w + i) + ch] = o[ch];
        }
}
