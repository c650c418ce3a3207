// geer_host.cu -- the C ABI (include/geer.h): argument checks, camera and BEAP
// table setup, workspace layout and the launch sequence of each stage.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "geer_internal.cuh"

using namespace geer;

namespace {

struct Layout {
    size_t off = 0;
    size_t take(size_t bytes) {
        size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return o;
    }
};

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Kannala-Brandt distorted angle phi (1 + k1 phi^2 + k2 phi^4 + k3 phi^6 + k4 phi^8) (App. E).
double kb_theta_d(const float k[4], double phi) {
    const double p2 = phi * phi;
    return phi * (1.0 + p2 * (k[0] + p2 * (k[1] + p2 * (k[2] + p2 * k[3]))));
}

// Vertical BEAP field of view: the vertical half-angle that the focal length
// mapping fov_x/2 to w/2 maps to h/2 (pinhole: tan; equidistant: linear;
// Kannala-Brandt: smallest root of the distortion polynomial).
double derived_fov_y(const geer_camera &c) {
    if (c.fov_y > 0.0f) return (double)c.fov_y;
    const double fx = c.fov_x, w = c.width, h = c.height;
    if (c.model == GEER_PINHOLE) return 2.0 * atan(tan(0.5 * fx) * h / w);
    if (c.model == GEER_EQUIDISTANT) return fx * h / w;
    const double edge = kb_theta_d(c.k, 0.5 * fx);
    if (!(edge > 0.0)) return NAN;
    const double target = edge * h / w;
    // bracket the first crossing on a fine grid, then bisect
    double lo = 0.0, hi = 0.5 * fx;
    const int n = 8192;
    for (int s = 1; s <= n; ++s) {
        const double ph = 0.5 * fx * s / n;
        if (kb_theta_d(c.k, ph) >= target) {
            hi = ph;
            lo = 0.5 * fx * (s - 1) / n;
            break;
        }
    }
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (kb_theta_d(c.k, mid) >= target) hi = mid; else lo = mid;
    }
    return 2.0 * hi;
}

// BEAP pixel-centre angle (Sec. 3.3): ((i + 1/2)/w - 1/2) FoV.
inline double beap_angle(int i, int w, double fov) { return ((i + 0.5) / w - 0.5) * fov; }

bool camera_ok(const geer_camera &c) {
    if (c.width <= 0 || c.height <= 0 || c.width > 65535 * kTile || c.height > 65535 * kTile) return false;
    if (!(c.fov_x > 0.0f) || !(c.fov_x < 6.2831f)) return false;
    if (c.model < GEER_PINHOLE || c.model > GEER_KANNALA_BRANDT) return false;
    if (c.model == GEER_PINHOLE && !(c.fov_x < 3.1415f)) return false;
    const double fy = derived_fov_y(c);
    if (!(fy > 0.0) || !(fy < 6.2831)) return false;
    if (c.model == GEER_PINHOLE && !(fy < 3.1415)) return false;
    for (float v : c.R_cw) if (!isfinite(v)) return false;
    for (float v : c.t_cw) if (!isfinite(v)) return false;
    return true;
}

struct CamTables {
    std::vector<DevCam> cams;
    std::vector<float4> ttab;
    std::vector<float2> ptab;
    int64_t pixels = 0, tiles = 0;
    int32_t super_size = 4;
    int64_t stiles = 0;
    bool ok = true;  // every camera's flag sets have the interval shape the kernels assume
};

// The tile columns (or rows) of a camera whose rays have cos >= 0 form one
// interval, those with cos <= 0 a leading and a trailing run (the BEAP angles
// grow monotonically): records them for the association counts and checks the
// shape.
bool flag_intervals(const float4 *tab, int n, int32_t z[2], int32_t w[2]) {
    z[0] = n;
    z[1] = 0;
    for (int i = 0; i < n; ++i)
        if (tab[i].z != 0.0f) {
            z[0] = std::min(z[0], i);
            z[1] = i + 1;
        }
    int a = 0, b = n;
    while (a < n && tab[a].w != 0.0f) ++a;
    while (b > a && tab[b - 1].w != 0.0f) --b;
    w[0] = a;
    w[1] = b;
    for (int i = 0; i < n; ++i) {
        if ((tab[i].z != 0.0f) != (i >= z[0] && i < z[1])) return false;
        if ((tab[i].w != 0.0f) != (i < a || i >= b)) return false;
    }
    return true;
}

// Super-tile grid of each camera (binning is by super-tiles of S x S tiles; the
// render filters a super-tile's list down to its tile). Free layouts take the
// smallest S in 4..8 that keeps every super-tile id below 256 (one radix pass),
// else 4. Slot layouts take S = 4 and the slot's own tile ids, so that every
// launch shape depends on the slot count only.
void assign_super(DevCam *cams, int n, int64_t slot_tiles, int32_t &S, int64_t &n_stiles) {
    if (slot_tiles > 0) {
        S = 4;
        for (int ci = 0; ci < n; ++ci) {
            DevCam &d = cams[ci];
            d.stiles_x = (int32_t)ceil_div(d.tiles_x, S);
            d.stile_base = (int32_t)(ci * slot_tiles);
        }
        n_stiles = n * slot_tiles;
        return;
    }
    S = 4;
    for (int e = 4; e <= 8; ++e) {
        int64_t tot = 0;
        for (int ci = 0; ci < n; ++ci) tot += ceil_div(cams[ci].tiles_x, e) * ceil_div(cams[ci].tiles_y, e);
        if (tot <= kRadix) {
            S = e;
            break;
        }
    }
    int64_t sb = 0;
    for (int ci = 0; ci < n; ++ci) {
        DevCam &d = cams[ci];
        d.stiles_x = (int32_t)ceil_div(d.tiles_x, S);
        d.stile_base = (int32_t)sb;
        sb += (int64_t)d.stiles_x * ceil_div(d.tiles_y, S);
    }
    n_stiles = sb;
}

int32_t sort_passes(int64_t ids) {
    int bits = 1;
    while ((int64_t(1) << bits) < ids) ++bits;
    return (bits + kRadixBits - 1) / kRadixBits;
}

// Per camera: tile-column/-row half-angle spans tan(angle/2) of the first and
// last ray of the tile with flags for cos(angle) >= 0 / <= 0 (rays beyond 90 deg
// flip the other dihedral angle by pi), per-pixel sin/cos of theta and phi.
void build_tables(const geer_camera *cams, int n, CamTables &out, const uint8_t *active = nullptr,
                  int64_t slot_tiles = 0, int64_t slot_pixels = 0) {
    out = CamTables();
    for (int ci = 0; ci < n; ++ci) {
        const geer_camera &c = cams[ci];
        DevCam d;
        memset(&d, 0, sizeof(d));
        if (slot_tiles > 0) {
            // fixed slot placement: camera ci owns tiles [ci * slot_tiles, ...) and
            // pixels [ci * slot_pixels, ...); an inactive slot has no tiles at all
            out.tiles = (int64_t)ci * slot_tiles;
            out.pixels = (int64_t)ci * slot_pixels;
            if (active && !active[ci]) {
                d.tile_base = (int32_t)out.tiles;
                d.pix_base = out.pixels;
                d.tcol_off = d.trow_off = (int32_t)out.ttab.size();
                d.pcol_off = d.prow_off = (int32_t)out.ptab.size();
                out.cams.push_back(d);
                out.tiles = (int64_t)(ci + 1) * slot_tiles;
                out.pixels = (int64_t)(ci + 1) * slot_pixels;
                continue;
            }
        }
        d.width = c.width;
        d.height = c.height;
        d.tiles_x = (int)ceil_div(c.width, kTile);
        d.tiles_y = (int)ceil_div(c.height, kTile);
        d.tile_base = (int32_t)out.tiles;
        d.pix_base = out.pixels;
        const double fx = c.fov_x, fy = derived_fov_y(c);
        d.col_ppr = (float)(c.width / fx);
        d.row_ppr = (float)(c.height / fy);
        d.tcol_off = (int32_t)out.ttab.size();
        for (int tx = 0; tx < d.tiles_x; ++tx) {
            const int i0 = tx * kTile, i1 = std::min(i0 + kTile - 1, c.width - 1);
            float4 v;
            v.x = (float)tan(0.5 * beap_angle(i0, c.width, fx));
            v.y = (float)tan(0.5 * beap_angle(i1, c.width, fx));
            v.z = 0.0f;
            v.w = 0.0f;
            for (int i = i0; i <= i1; ++i) {
                const double cs = cos(beap_angle(i, c.width, fx));
                if (cs > -1e-12) v.z = 1.0f;
                if (cs < 1e-12) { v.w = 1.0f; d.any_col_flip = 1; }
            }
            out.ttab.push_back(v);
        }
        d.trow_off = (int32_t)out.ttab.size();
        for (int ty = 0; ty < d.tiles_y; ++ty) {
            const int j0 = ty * kTile, j1 = std::min(j0 + kTile - 1, c.height - 1);
            float4 v;
            v.x = (float)tan(0.5 * beap_angle(j0, c.height, fy));
            v.y = (float)tan(0.5 * beap_angle(j1, c.height, fy));
            v.z = 0.0f;
            v.w = 0.0f;
            for (int j = j0; j <= j1; ++j) {
                const double cs = cos(beap_angle(j, c.height, fy));
                if (cs > -1e-12) v.z = 1.0f;
                if (cs < 1e-12) { v.w = 1.0f; d.any_row_flip = 1; }
            }
            out.ttab.push_back(v);
        }
        d.pcol_off = (int32_t)out.ptab.size();
        for (int i = 0; i < c.width; ++i) {
            const double a = beap_angle(i, c.width, fx);
            out.ptab.push_back(make_float2((float)sin(a), (float)cos(a)));
        }
        d.prow_off = (int32_t)out.ptab.size();
        for (int j = 0; j < c.height; ++j) {
            const double a = beap_angle(j, c.height, fy);
            out.ptab.push_back(make_float2((float)sin(a), (float)cos(a)));
        }
        out.ok &= flag_intervals(out.ttab.data() + d.tcol_off, d.tiles_x, d.zc, d.wc);
        out.ok &= flag_intervals(out.ttab.data() + d.trow_off, d.tiles_y, d.zr, d.wr);
        // tiles whose rays all have cos >= 0 (a contiguous middle range)
        d.c0lo = d.tiles_x; d.c0hi = 0;
        for (int tx = 0; tx < d.tiles_x; ++tx) {
            const float4 v = out.ttab[d.tcol_off + tx];
            if (v.z != 0.0f && v.w == 0.0f) { d.c0lo = std::min(d.c0lo, tx); d.c0hi = tx + 1; }
        }
        d.r0lo = d.tiles_y; d.r0hi = 0;
        for (int ty = 0; ty < d.tiles_y; ++ty) {
            const float4 v = out.ttab[d.trow_off + ty];
            if (v.z != 0.0f && v.w == 0.0f) { d.r0lo = std::min(d.r0lo, ty); d.r0hi = ty + 1; }
        }
        for (int k = 0; k < 9; ++k) d.R[k] = c.R_cw[k];
        for (int k = 0; k < 3; ++k) {
            d.t[k] = c.t_cw[k];
            d.bg[k] = c.bg[k];
            double o = 0.0;
            for (int b = 0; b < 3; ++b) o -= (double)c.R_cw[3 * b + k] * (double)c.t_cw[b];
            d.o[k] = (float)o;
        }
        out.cams.push_back(d);
        out.tiles += (int64_t)d.tiles_x * d.tiles_y;
        out.pixels += (int64_t)c.width * c.height;
        if (slot_tiles > 0) {
            out.tiles = (int64_t)(ci + 1) * slot_tiles;
            out.pixels = (int64_t)(ci + 1) * slot_pixels;
        }
    }
    assign_super(out.cams.data(), (int)out.cams.size(), slot_tiles, out.super_size, out.stiles);
}

struct Caps {
    int32_t cams;
    int64_t pixels, tiles, tile_tab, pix_tab, gauss, pairs, sort_tiles, prep_blocks;
    int64_t hit_entries;  // per tile: the forward's hit record for the backward (0: none)
};

Caps caps_of(const CamTables &t, int32_t n_cams, int64_t n_gauss, int64_t pair_capacity) {
    Caps c;
    c.cams = n_cams;
    c.pixels = std::max<int64_t>(t.pixels, 1);
    c.tiles = std::max<int64_t>(t.tiles, 1);
    c.tile_tab = std::max<int64_t>((int64_t)t.ttab.size(), 1);
    c.pix_tab = std::max<int64_t>((int64_t)t.ptab.size(), 1);
    c.gauss = std::max<int64_t>(n_gauss, 1);
    c.pairs = std::max<int64_t>(pair_capacity, 1);
    c.sort_tiles = ceil_div(std::max<int64_t>(c.pairs, (int64_t)n_cams * c.gauss), kSortTile) + 1;
    c.prep_blocks = prep_blocks(c.gauss);
    c.hit_entries = kHitEntries;
    return c;
}

// Lays the arrays out; with base == nullptr only measures.
size_t layout(const Caps &c, char *base, geer_workspace *ws) {
    Layout L;
    const int64_t cg = (int64_t)c.cams * c.gauss;
    size_t o_cams = L.take(sizeof(DevCam) * c.cams);
    size_t o_ttab = L.take(sizeof(float4) * c.tile_tab);
    size_t o_ptab = L.take(sizeof(float2) * c.pix_tab);
    size_t o_rec = L.take(sizeof(Record) * cg);
    size_t o_rng = L.take(sizeof(uint4) * cg);
    size_t o_cnt = L.take(sizeof(uint32_t) * cg);
    size_t o_key = L.take(sizeof(uint32_t) * cg);
    size_t o_bs = L.take(sizeof(uint32_t) * c.cams * c.prep_blocks);
    size_t o_bs2 = L.take(sizeof(uint32_t) * prep_blocks(cg));
    size_t o_bs3 = L.take(sizeof(uint32_t) * prep_blocks(cg));
    size_t o_ik0 = L.take(sizeof(uint32_t) * cg);
    size_t o_ik1 = L.take(sizeof(uint32_t) * cg);
    size_t o_ii0 = L.take(sizeof(uint32_t) * cg);
    size_t o_ii1 = L.take(sizeof(uint32_t) * cg);
    size_t o_k0 = L.take(sizeof(uint32_t) * c.pairs);
    size_t o_k1 = L.take(sizeof(uint32_t) * c.pairs);
    size_t o_v0 = L.take(sizeof(uint32_t) * c.pairs);
    size_t o_v1 = L.take(sizeof(uint32_t) * c.pairs);
    size_t o_srg = L.take(sizeof(uint4) * c.pairs);
    const int64_t groups = ceil_div(c.sort_tiles, kGroupTiles) + 1;
    size_t o_th = L.take(sizeof(uint32_t) * kRadix * c.sort_tiles);
    size_t o_gs = L.take(sizeof(uint32_t) * kRadix * groups);
    size_t o_ge = L.take(sizeof(uint32_t) * kRadix * groups);
    size_t o_db = L.take(sizeof(uint32_t) * kRadix);
    size_t o_misc = L.take(sizeof(uint32_t) * kMiscCount);
    size_t o_tr = L.take((sizeof(uint2) + sizeof(uint32_t)) * c.tiles);
    size_t o_to = L.take(sizeof(uint32_t) * c.tiles);
    const bool bwd = c.hit_entries > 0;  // the forward-only layout has no backward state
    size_t o_bo = L.take(sizeof(uint32_t) * c.tiles * (bwd ? kCkptMax + 1 : 1));
    size_t o_sr = L.take((sizeof(uint2) + sizeof(uint32_t)) * c.tiles);
    size_t o_last = L.take(sizeof(uint32_t) * c.pixels);
    size_t o_tfin = L.take(sizeof(float) * c.pixels);
    size_t o_ev = L.take(sizeof(uint2) * c.pixels);
    size_t o_gacc = L.take(sizeof(GradAcc) * cg);
    size_t o_hit = L.take(sizeof(uint2) * c.tiles * c.hit_entries);
    size_t o_idr = L.take(sizeof(uint32_t) * c.tiles * c.hit_entries);
    size_t o_mask = L.take(bwd ? sizeof(uint8_t) * c.tiles : 0);  // not in the forward-only layout
    size_t o_ck = L.take(bwd ? sizeof(float4) * c.tiles * kCkptMax * kTilePix : 0);
    size_t o_cka = L.take(bwd ? sizeof(uint2) * c.tiles * kCkptMax : 0);
    size_t o_ckn = L.take(bwd ? sizeof(uint32_t) * c.tiles : 0);
    size_t o_ckw = L.take(bwd ? sizeof(uint4) * c.tiles : 0);
    size_t o_cf = L.take(bwd ? sizeof(float4) * c.pixels : 0);
    if (base && ws) {
        ws->d_cams = reinterpret_cast<DevCam *>(base + o_cams);
        ws->d_tile_tab = reinterpret_cast<float4 *>(base + o_ttab);
        ws->d_pix_tab = reinterpret_cast<float2 *>(base + o_ptab);
        ws->d_rec = reinterpret_cast<Record *>(base + o_rec);
        ws->d_ranges = reinterpret_cast<uint4 *>(base + o_rng);
        ws->d_count = reinterpret_cast<uint32_t *>(base + o_cnt);
        ws->d_key = reinterpret_cast<uint32_t *>(base + o_key);
        ws->d_blocksum = reinterpret_cast<uint32_t *>(base + o_bs);
        ws->d_blocksum2 = reinterpret_cast<uint32_t *>(base + o_bs2);
        ws->d_blocksum3 = reinterpret_cast<uint32_t *>(base + o_bs3);
        ws->d_ikey[0] = reinterpret_cast<uint32_t *>(base + o_ik0);
        ws->d_ikey[1] = reinterpret_cast<uint32_t *>(base + o_ik1);
        ws->d_iid[0] = reinterpret_cast<uint32_t *>(base + o_ii0);
        ws->d_iid[1] = reinterpret_cast<uint32_t *>(base + o_ii1);
        ws->d_keys[0] = reinterpret_cast<uint32_t *>(base + o_k0);
        ws->d_keys[1] = reinterpret_cast<uint32_t *>(base + o_k1);
        ws->d_vals[0] = reinterpret_cast<uint32_t *>(base + o_v0);
        ws->d_vals[1] = reinterpret_cast<uint32_t *>(base + o_v1);
        ws->d_sranges = reinterpret_cast<uint4 *>(base + o_srg);
        ws->d_tile_hist = reinterpret_cast<uint32_t *>(base + o_th);
        ws->d_group_sum = reinterpret_cast<uint32_t *>(base + o_gs);
        ws->d_group_excl = reinterpret_cast<uint32_t *>(base + o_ge);
        ws->d_digit_base = reinterpret_cast<uint32_t *>(base + o_db);
        ws->d_misc = reinterpret_cast<uint32_t *>(base + o_misc);
        ws->d_tile_walk = reinterpret_cast<uint2 *>(base + o_tr);
        ws->d_tile_order = reinterpret_cast<uint32_t *>(base + o_to);
        ws->d_bwd_order = reinterpret_cast<uint32_t *>(base + o_bo);
        ws->d_srange = reinterpret_cast<uint2 *>(base + o_sr);
        ws->d_last = reinterpret_cast<uint32_t *>(base + o_last);
        ws->d_Tfin = reinterpret_cast<float *>(base + o_tfin);
        ws->d_evals = reinterpret_cast<uint2 *>(base + o_ev);
        ws->d_gacc = reinterpret_cast<GradAcc *>(base + o_gacc);
        ws->d_hit = c.hit_entries > 0 ? reinterpret_cast<uint2 *>(base + o_hit) : nullptr;
        ws->d_idrec = c.hit_entries > 0 ? reinterpret_cast<uint32_t *>(base + o_idr) : nullptr;
        ws->hit_entries = c.hit_entries;
        ws->d_tile_mask = bwd ? reinterpret_cast<uint8_t *>(base + o_mask) : nullptr;
        ws->d_ckpt = bwd ? reinterpret_cast<float4 *>(base + o_ck) : nullptr;
        ws->d_ckpt_at = bwd ? reinterpret_cast<uint2 *>(base + o_cka) : nullptr;
        ws->d_ckpt_cnt = bwd ? reinterpret_cast<uint32_t *>(base + o_ckn) : nullptr;
        ws->d_unit_rec = bwd ? reinterpret_cast<uint4 *>(base + o_ckw) : nullptr;
        ws->d_Cfin = bwd ? reinterpret_cast<float4 *>(base + o_cf) : nullptr;
    }
    return L.off;
}

geer_status cuda_status(cudaError_t e) { return e == cudaSuccess ? GEER_OK : GEER_ERR_CUDA; }

// Records the begin/end events of one stage when timing is enabled.
struct StageTimer {
    geer_workspace *ws;
    int stage, slot;
    cudaStream_t s;
    StageTimer(geer_workspace *w, int st, cudaStream_t str) : ws(w), stage(st), slot(-1), s(str) {
        if (ws->timing && ((ws->timing_mask >> stage) & 1u)) {
            slot = ws->ev_count[stage] % kTimingRing;
            cudaEventRecord(ws->ev[stage][slot][0], s);
        }
    }
    ~StageTimer() {
        if (slot >= 0) {
            cudaEventRecord(ws->ev[stage][slot][1], s);
            ws->ev_count[stage] += 1;
        }
    }
};

geer_status check_cams(const geer_camera *cams, int32_t n) {
    if (!cams || n <= 0 || n > kMaxCams) return GEER_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (!camera_ok(cams[i])) return GEER_ERR_ARG;
    return GEER_OK;
}

geer_status check_params(const geer_params *p) {
    if (!p) return GEER_ERR_ARG;
    if (p->tile_w != kTile || p->tile_h != kTile) return GEER_ERR_UNSUPPORTED;
    if (!(p->alpha_min > 0.0f) || !(p->alpha_min < 1.0f)) return GEER_ERR_ARG;
    if (!(p->alpha_max > 0.0f) || !(p->alpha_max < 1.0f) || p->alpha_max < p->alpha_min) return GEER_ERR_ARG;
    if (!(p->T_min >= 0.0f) || !(p->T_min < 1.0f)) return GEER_ERR_ARG;
    if (!(p->lambda_pad >= 0.0f) || !(p->lambda_pad < 1.0f)) return GEER_ERR_ARG;
    if (p->assoc != GEER_ASSOC_PBF && p->assoc != GEER_ASSOC_EWA && p->assoc != GEER_ASSOC_UT) return GEER_ERR_ARG;
    if (p->snugbox != 0 && p->snugbox != 1) return GEER_ERR_ARG;
    if (p->alpha_model != GEER_ALPHA_EXACT && p->alpha_model != GEER_ALPHA_SPLAT) return GEER_ERR_ARG;
    return GEER_OK;
}

geer_status check_gaussians(const geer_workspace *ws, const geer_gaussians *g) {
    if (!g || g->n < 0 || g->n > ws->cap_gauss) return GEER_ERR_ARG;
    if (g->sh_degree < 0 || g->sh_degree > 3 || g->sh_degree > ws->cap_sh_degree) return GEER_ERR_ARG;
    if ((int64_t)ws->n_cams * g->n > 0xffffffffll) return GEER_ERR_ARG;
    if (g->n > 0 && (!g->mean || !g->scale || !g->quat || !g->opacity || !g->sh)) return GEER_ERR_ARG;
    if (g->n > 0 && (reinterpret_cast<uintptr_t>(g->sh) & 15)) return GEER_ERR_ARG;
    return GEER_OK;
}

// Upload the camera set: stage in pinned memory, then one async copy per array.
geer_status upload_cams(geer_workspace *ws, const CamTables &t, cudaStream_t s) {
    const size_t b0 = sizeof(DevCam) * t.cams.size();
    const size_t b1 = sizeof(float4) * t.ttab.size();
    const size_t b2 = sizeof(float2) * t.ptab.size();
    if (b0 + b1 + b2 > ws->stage_bytes) return GEER_ERR_ARG;
    if (t.stiles > ws->cap_tiles) return GEER_ERR_ARG;
    // the staging buffer may still be read by a previous copy on this stream
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return GEER_ERR_CUDA;
    char *h = static_cast<char *>(ws->h_stage);
    memcpy(h, t.cams.data(), b0);
    memcpy(h + b0, t.ttab.data(), b1);
    memcpy(h + b0 + b1, t.ptab.data(), b2);
    if ((e = cudaMemcpyAsync(ws->d_cams, h, b0, cudaMemcpyHostToDevice, s)) != cudaSuccess) return GEER_ERR_CUDA;
    if (b1 && (e = cudaMemcpyAsync(ws->d_tile_tab, h + b0, b1, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return GEER_ERR_CUDA;
    if (b2 && (e = cudaMemcpyAsync(ws->d_pix_tab, h + b0 + b1, b2, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return GEER_ERR_CUDA;
    ws->n_cams = (int32_t)t.cams.size();
    ws->n_pixels = t.pixels;
    ws->n_tiles = t.tiles;
    std::copy(t.cams.begin(), t.cams.end(), ws->cams);
    ws->super_size = t.super_size;
    ws->n_stiles = t.stiles;
    ws->n_sort_passes = sort_passes(t.stiles);
    ws->stage = 0;
    ws->tile_mask_on = 0;  // tile indices refer to the new camera set
    return GEER_OK;
}

}  // namespace

extern "C" {

const char *geer_status_string(geer_status s) {
    switch (s) {
        case GEER_OK: return "ok";
        case GEER_ERR_ARG: return "invalid argument";
        case GEER_ERR_CAPACITY: return "pair capacity exceeded";
        case GEER_ERR_CUDA: return "CUDA error";
        case GEER_ERR_TIMEOUT: return "bounded device wait timed out";
        case GEER_ERR_UNSUPPORTED: return "unsupported";
        case GEER_ERR_STATE: return "call out of order";
        case GEER_ERR_BOUNDS: return "a device bounds guard skipped an access";
    }
    return "unknown status";
}

geer_status geer_default_params(geer_params *p) {
    if (!p) return GEER_ERR_ARG;
    p->tile_w = kTile;
    p->tile_h = kTile;
    p->alpha_min = 1.0f / 255.0f;
    p->T_min = 1e-4f;
    p->alpha_max = 0.99f;
    p->lambda_pad = 1e-3f;
    p->assoc = GEER_ASSOC_PBF;
    p->snugbox = 0;
    p->alpha_model = GEER_ALPHA_EXACT;
    return GEER_OK;
}

geer_status geer_workspace_size(const geer_camera *cams, int32_t n_cams, int64_t n_gauss, int32_t sh_degree,
                                int64_t pair_capacity, size_t *bytes) {
    if (!bytes || n_gauss < 0 || pair_capacity < 0 || sh_degree < 0 || sh_degree > 3) return GEER_ERR_ARG;
    geer_status st = check_cams(cams, n_cams);
    if (st != GEER_OK) return st;
    if ((int64_t)n_cams * n_gauss > 0xffffffffll || pair_capacity > 0xffffffffll) return GEER_ERR_ARG;
    CamTables t;
    build_tables(cams, n_cams, t);
    if (!t.ok) return GEER_ERR_UNSUPPORTED;
    *bytes = layout(caps_of(t, n_cams, n_gauss, pair_capacity), nullptr, nullptr);
    return GEER_OK;
}

geer_status geer_workspace_init(void *dev_mem, size_t bytes, const geer_camera *cams, int32_t n_cams,
                                int64_t n_gauss, int32_t sh_degree, int64_t pair_capacity,
                                const geer_params *params, geer_workspace **out) {
    if (!out) return GEER_ERR_ARG;
    *out = nullptr;
    if (!dev_mem || (reinterpret_cast<uintptr_t>(dev_mem) & 255)) return GEER_ERR_ARG;
    size_t need = 0;
    geer_status st = geer_workspace_size(cams, n_cams, n_gauss, sh_degree, pair_capacity, &need);
    if (st != GEER_OK) return st;
    if (bytes < need) return GEER_ERR_ARG;
    geer_params pd;
    geer_default_params(&pd);
    if (!params) params = &pd;
    if ((st = check_params(params)) != GEER_OK) return st;

    geer_workspace *ws = static_cast<geer_workspace *>(calloc(1, sizeof(geer_workspace)));
    if (!ws) return GEER_ERR_ARG;
    CamTables t;
    build_tables(cams, n_cams, t);
    const Caps c = caps_of(t, n_cams, n_gauss, pair_capacity);
    layout(c, static_cast<char *>(dev_mem), ws);
    ws->cap_cams = c.cams;
    ws->cap_pixels = c.pixels;
    ws->cap_tiles = c.tiles;
    ws->cap_tile_tab = c.tile_tab;
    ws->cap_pix_tab = c.pix_tab;
    ws->cap_gauss = n_gauss;
    ws->cap_pairs = pair_capacity;
    ws->cap_sh_degree = sh_degree;
    ws->cap_sort_tiles = c.sort_tiles;
    ws->params = Params{params->alpha_min, params->T_min, params->alpha_max, params->lambda_pad, params->assoc,
                        params->snugbox, params->alpha_model};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ws->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) { free(ws); return GEER_ERR_CUDA; }
    ws->sort_grid = ws->num_sms * sort_blocks_per_sm();
    ws->bwd_grid = ws->num_sms * render_bwd_blocks_per_sm(ws->params.alpha_model);
    ws->train_grid = ws->num_sms * render_train_blocks_per_sm(ws->params.alpha_model);
    ws->stage_bytes = sizeof(DevCam) * c.cams + sizeof(float4) * c.tile_tab + sizeof(float2) * c.pix_tab;
    if (cudaMallocHost(&ws->h_stage, ws->stage_bytes) != cudaSuccess) { free(ws); return GEER_ERR_CUDA; }
    // status words and radix group sums start from zero
    e = cudaMemset(ws->d_misc, 0, sizeof(uint32_t) * kMiscCount);
    if (e == cudaSuccess)
        e = cudaMemset(ws->d_group_sum, 0, sizeof(uint32_t) * kRadix * (ceil_div(c.sort_tiles, kGroupTiles) + 1));
    if (e != cudaSuccess) { cudaFreeHost(ws->h_stage); free(ws); return GEER_ERR_CUDA; }
    st = upload_cams(ws, t, 0);
    if (st == GEER_OK && cudaStreamSynchronize(0) != cudaSuccess) st = GEER_ERR_CUDA;
    if (st != GEER_OK) { cudaFreeHost(ws->h_stage); free(ws); return st; }
    *out = ws;
    return GEER_OK;
}

geer_status geer_workspace_destroy(geer_workspace *ws) {
    if (!ws) return GEER_ERR_ARG;
    if (ws->timing)
        for (int a = 0; a < kStageCount; ++a)
            for (int b = 0; b < kTimingRing; ++b) {
                cudaEventDestroy(ws->ev[a][b][0]);
                cudaEventDestroy(ws->ev[a][b][1]);
            }
    if (ws->h_stage) cudaFreeHost(ws->h_stage);
    free(ws);
    return GEER_OK;
}

geer_status geer_set_cameras(geer_workspace *ws, const geer_camera *cams, int32_t n_cams, void *stream) {
    if (!ws) return GEER_ERR_ARG;
    geer_status st = check_cams(cams, n_cams);
    if (st != GEER_OK) return st;
    if (n_cams > ws->cap_cams) return GEER_ERR_ARG;
    CamTables t;
    build_tables(cams, n_cams, t);
    if (!t.ok) return GEER_ERR_UNSUPPORTED;
    if (t.pixels > ws->cap_pixels || t.tiles > ws->cap_tiles || (int64_t)t.ttab.size() > ws->cap_tile_tab ||
        (int64_t)t.ptab.size() > ws->cap_pix_tab)
        return GEER_ERR_ARG;
    return upload_cams(ws, t, static_cast<cudaStream_t>(stream));
}

geer_status geer_set_camera_slots(geer_workspace *ws, const geer_camera *cams, int32_t n_slots, const uint8_t *active,
                                  int64_t slot_tiles, int64_t slot_pixels, void *stream) {
    if (!ws || !cams || n_slots <= 0 || n_slots > ws->cap_cams || slot_tiles <= 0 || slot_pixels <= 0)
        return GEER_ERR_ARG;
    for (int i = 0; i < n_slots; ++i) {
        if (active && !active[i]) continue;
        if (!camera_ok(cams[i])) return GEER_ERR_ARG;
        const int64_t tiles = ceil_div(cams[i].width, kTile) * ceil_div(cams[i].height, kTile);
        if (tiles > slot_tiles || (int64_t)cams[i].width * cams[i].height > slot_pixels) return GEER_ERR_ARG;
    }
    CamTables t;
    build_tables(cams, n_slots, t, active, slot_tiles, slot_pixels);
    if (!t.ok) return GEER_ERR_UNSUPPORTED;
    if (t.pixels > ws->cap_pixels || t.tiles > ws->cap_tiles || (int64_t)t.ttab.size() > ws->cap_tile_tab ||
        (int64_t)t.ptab.size() > ws->cap_pix_tab)
        return GEER_ERR_ARG;
    return upload_cams(ws, t, static_cast<cudaStream_t>(stream));
}

geer_status geer_preprocess(geer_workspace *ws, const geer_gaussians *g, void *stream) {
    if (!ws) return GEER_ERR_ARG;
    geer_status st = check_gaussians(ws, g);
    if (st != GEER_OK) return st;
    ws->n_gauss = g->n;
    ws->sh_degree = g->sh_degree;
    ws->stage = 1;
    StageTimer tm(ws, kStagePreprocess, static_cast<cudaStream_t>(stream));
    st = cuda_status(launch_preprocess(ws, g, static_cast<cudaStream_t>(stream)));
    ws->acc_zero = st == GEER_OK && ws->trains;  // the kernel zeroed the items' accumulators
    return st;
}

geer_status geer_bin_sort(geer_workspace *ws, int64_t *pairs_needed, void *stream) {
    if (!ws) return GEER_ERR_ARG;
    if (ws->stage < 1) return GEER_ERR_STATE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ws->queue_ready = false;
    // live items in index order -> stable depth sort -> pair counts in depth order
    {
        StageTimer tm(ws, kStageBinFront, s);
        if (launch_bin_front(ws, s) != cudaSuccess) return GEER_ERR_CUDA;
    }
    {
        StageTimer tm(ws, kStageDepthSort, s);
        if (launch_depth_sort(ws, s) != cudaSuccess) return GEER_ERR_CUDA;
    }
    {
        StageTimer tm(ws, kStageCountPairs, s);
        if (launch_count_pairs(ws, s) != cudaSuccess) return GEER_ERR_CUDA;
    }
    if (pairs_needed) {
        uint32_t m[kMiscCount];
        if (cudaMemcpyAsync(m, ws->d_misc, sizeof(m), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return GEER_ERR_CUDA;
        const int64_t total = ((int64_t)m[kMiscPairsHi] << 32) | (int64_t)m[kMiscTotalLo];
        *pairs_needed = total;
        if (total > ws->cap_pairs) {
            // clear the capacity bit: the caller resizes and retries
            uint32_t zero = 0;
            cudaMemcpyAsync(ws->d_misc + kMiscStatus, &zero, sizeof(zero), cudaMemcpyHostToDevice, s);
            cudaStreamSynchronize(s);
            ws->stage = 1;
            return GEER_ERR_CAPACITY;
        }
    }
    // emit (tile, item) pairs in depth order, stable sort by tile, ranges
    {
        StageTimer tm(ws, kStageDuplicate, s);
        if (launch_duplicate(ws, s) != cudaSuccess) return GEER_ERR_CUDA;
    }
    {
        StageTimer tm(ws, kStageTileSort, s);
        if (launch_tile_sort(ws, s) != cudaSuccess) return GEER_ERR_CUDA;
    }
    ws->queue_ready = ws->trains;  // the render order's kernel reset the unit queue
    ws->stage = 2;
    return GEER_OK;
}

geer_status geer_render_fwd(geer_workspace *ws, float *rgb, float *T_final, void *stream) {
    if (!ws || !rgb) return GEER_ERR_ARG;
    if (ws->stage < 2) return GEER_ERR_STATE;
    ws->trains = false;  // forward-only steps: the next preprocess leaves the accumulators (a backward turns it back on)
    geer_status st;
    {
        StageTimer tm(ws, kStageRenderFwd, static_cast<cudaStream_t>(stream));
        st = cuda_status(launch_render_fwd(ws, rgb, T_final, static_cast<cudaStream_t>(stream)));
    }
    if (st == GEER_OK) ws->stage = 3;
    return st;
}

geer_status geer_render_bwd(geer_workspace *ws, const geer_gaussians *g, const float *dL_drgb, float *d_mean,
                            float *d_scale, float *d_quat, float *d_opacity, float *d_sh, int32_t accumulate,
                            void *stream) {
    if (!ws || !dL_drgb) return GEER_ERR_ARG;
    if (ws->stage < 3) return GEER_ERR_STATE;
    geer_status st = check_gaussians(ws, g);
    if (st != GEER_OK) return st;
    if (g->n != ws->n_gauss || g->sh_degree != ws->sh_degree) return GEER_ERR_ARG;
    if (d_sh && (reinterpret_cast<uintptr_t>(d_sh) & 15)) return GEER_ERR_ARG;
    if ((st = geer_render_bwd_tiles(ws, dL_drgb, stream)) != GEER_OK) return st;
    return geer_preprocess_bwd(ws, g, d_mean, d_scale, d_quat, d_opacity, d_sh, accumulate, stream);
}

geer_status geer_render_bwd_tiles(geer_workspace *ws, const float *dL_drgb, void *stream) {
    if (!ws || !dL_drgb) return GEER_ERR_ARG;
    if (ws->stage < 3) return GEER_ERR_STATE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t items = (int64_t)ws->n_cams * ws->n_gauss;
    if (!ws->acc_zero && items > 0 && cudaMemsetAsync(ws->d_gacc, 0, sizeof(GradAcc) * items, s) != cudaSuccess)
        return GEER_ERR_CUDA;
    ws->acc_zero = false;
    ws->queue_ready = false;  // the unit order overwrites the queue
    ws->trains = true;        // from now on the preprocess zeroes the accumulators
    {
        StageTimer tm(ws, kStageRenderBwd, s);
        if (launch_bwd_order(ws, s) != cudaSuccess || launch_render_bwd(ws, dL_drgb, s) != cudaSuccess)
            return GEER_ERR_CUDA;
    }
    ws->stage = 4;
    return GEER_OK;
}

geer_status geer_render_train_l1(geer_workspace *ws, const float *target, float *rgb, float *T_final,
                                 float *dL_drgb, float *loss, void *stream) {
    if (!ws || !target || !rgb || !dL_drgb) return GEER_ERR_ARG;
    if (ws->stage < 2) return GEER_ERR_STATE;
    if (ws->hit_entries == 0) return GEER_ERR_UNSUPPORTED;  // a forward-only workspace has no backward state
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t items = (int64_t)ws->n_cams * ws->n_gauss;
    // the accumulators and the unit queue: zeroed / reset by the preprocess and the
    // binning of this step unless a backward has used them since
    if ((!ws->acc_zero && items > 0 && cudaMemsetAsync(ws->d_gacc, 0, sizeof(GradAcc) * items, s) != cudaSuccess) ||
        (loss && cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) ||
        (!ws->queue_ready &&
         (cudaMemsetAsync(ws->d_bwd_order, 0xff, sizeof(uint32_t) * ws->n_tiles * (kCkptMax + 1), s) != cudaSuccess ||
          cudaMemsetAsync(ws->d_misc + kMiscFwdNext, 0, sizeof(uint32_t) * (kMiscTrainNext - kMiscFwdNext + 1), s) !=
              cudaSuccess)))
        return GEER_ERR_CUDA;
    ws->acc_zero = false;
    ws->queue_ready = false;
    ws->trains = true;  // from now on the preprocess and the binning prepare the accumulators and the queue
    {
        StageTimer tm(ws, kStageRenderTrain, s);
        if (launch_render_train(ws, target, rgb, T_final, dL_drgb, loss, s) != cudaSuccess) return GEER_ERR_CUDA;
    }
    ws->stage = 4;
    return GEER_OK;
}

geer_status geer_grad_accumulators(geer_workspace *ws, float **acc, int64_t *n_floats) {
    if (!ws || !acc || !n_floats) return GEER_ERR_ARG;
    *acc = reinterpret_cast<float *>(ws->d_gacc);
    *n_floats = (int64_t)ws->n_cams * ws->n_gauss * (int64_t)(sizeof(GradAcc) / sizeof(float));
    return GEER_OK;
}

geer_status geer_preprocess_bwd(geer_workspace *ws, const geer_gaussians *g, float *d_mean, float *d_scale,
                                float *d_quat, float *d_opacity, float *d_sh, int32_t accumulate, void *stream) {
    if (!ws) return GEER_ERR_ARG;
    if (ws->stage != 4) return GEER_ERR_STATE;
    geer_status st = check_gaussians(ws, g);
    if (st != GEER_OK) return st;
    if (g->n != ws->n_gauss || g->sh_degree != ws->sh_degree) return GEER_ERR_ARG;
    if (d_sh && (reinterpret_cast<uintptr_t>(d_sh) & 15)) return GEER_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StageTimer tm(ws, kStagePreprocessBwd, s);
    return cuda_status(launch_preprocess_bwd(ws, g, d_mean, d_scale, d_quat, d_opacity, d_sh, accumulate ? 1 : 0, s));
}

geer_status geer_tile_owners(const geer_camera *cams, int32_t n_cams, int32_t n_parts, int32_t *owner) {
    if (!owner || n_parts < 1) return GEER_ERR_ARG;
    geer_status st = check_cams(cams, n_cams);
    if (st != GEER_OK) return st;
    int64_t t = 0;
    for (int c = 0; c < n_cams; ++c) {
        const int64_t tx = ceil_div(cams[c].width, kTile), ty = ceil_div(cams[c].height, kTile);
        for (int64_t cy = 0; cy < ty; ++cy)
            for (int64_t cx = 0; cx < tx; ++cx) owner[t++] = (int32_t)((cx + cy + c) % n_parts);
    }
    return GEER_OK;
}

geer_status geer_set_tile_mask(geer_workspace *ws, const uint8_t *mask, int64_t n_tiles, void *stream) {
    if (!ws) return GEER_ERR_ARG;
    if (!mask) {
        ws->tile_mask_on = 0;
        return GEER_OK;
    }
    if (n_tiles != ws->n_tiles || !ws->d_tile_mask) return GEER_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n_tiles > 0 && (cudaMemcpyAsync(ws->d_tile_mask, mask, (size_t)n_tiles, cudaMemcpyHostToDevice, s) !=
                            cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
        return GEER_ERR_CUDA;
    ws->tile_mask_on = 1;
    return GEER_OK;
}

geer_status geer_last_device_status(geer_workspace *ws, int64_t *pairs, void *stream) {
    if (!ws) return GEER_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t m[kMiscCount];
    if (cudaMemcpyAsync(m, ws->d_misc, sizeof(m), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GEER_ERR_CUDA;
    if (pairs) *pairs = ((int64_t)m[kMiscPairsHi] << 32) | (int64_t)m[kMiscTotalLo];
    if (m[kMiscStatus] != 0) {
        uint32_t zero = 0;
        if (cudaMemcpyAsync(ws->d_misc + kMiscStatus, &zero, sizeof(zero), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return GEER_ERR_CUDA;
    }
    if (m[kMiscStatus] & kStatusCapacity) return GEER_ERR_CAPACITY;
    if (m[kMiscStatus] & kStatusBounds) return GEER_ERR_BOUNDS;
    if (m[kMiscStatus] & kStatusTimeout) return GEER_ERR_TIMEOUT;
    return GEER_OK;
}

int32_t geer_checked_build(void) { return GEER_CHECKED; }

geer_status geer_bounds_violation(geer_workspace *ws, uint32_t *site, int64_t *index, void *stream) {
    if (!ws || !site || !index) return GEER_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t m[kMiscCount];
    if (cudaMemcpyAsync(m, ws->d_misc, sizeof(m), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GEER_ERR_CUDA;
    *site = m[kMiscCheckSite];
    *index = (int64_t)(((uint64_t)m[kMiscCheckHi] << 32) | (uint64_t)m[kMiscCheckLo]);
    if (*site != 0) {
        const uint32_t zero[3] = {0u, 0u, 0u};
        const uint32_t status = m[kMiscStatus] & ~kStatusBounds;
        if (cudaMemcpyAsync(ws->d_misc + kMiscCheckSite, zero, sizeof(zero), cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(ws->d_misc + kMiscStatus, &status, sizeof(status), cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return GEER_ERR_CUDA;
    }
    return GEER_OK;
}

geer_status geer_debug_set_render_order(geer_workspace *ws, const uint32_t *order, int64_t n, void *stream) {
    if (!ws || (!order && n > 0)) return GEER_ERR_ARG;
    if (ws->stage < 2) return GEER_ERR_STATE;
    if (n != ws->n_tiles) return GEER_ERR_ARG;
    // tile indices must lie within the current camera set; a checked build lets
    // through indices within the workspace's tile capacity, for its device guards
    const int64_t limit = GEER_CHECKED ? ws->cap_tiles : ws->n_tiles;
    for (int64_t i = 0; i < n; ++i)
        if ((int64_t)order[i] >= limit) return GEER_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n > 0 && (cudaMemcpyAsync(ws->d_tile_order, order, sizeof(uint32_t) * n, cudaMemcpyHostToDevice, s) !=
                      cudaSuccess ||
                  cudaStreamSynchronize(s) != cudaSuccess))
        return GEER_ERR_CUDA;
    return GEER_OK;
}

geer_status geer_debug_preprocess(geer_workspace *ws, uint16_t *ranges, uint32_t *counts, uint32_t *keys,
                                  uint8_t *cull, void *stream) {
    if (!ws) return GEER_ERR_ARG;
    if (ws->stage < 1) return GEER_ERR_STATE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t m = (int64_t)ws->n_cams * ws->n_gauss;
    if (m == 0) return GEER_OK;
    std::vector<uint4> r(m);
    std::vector<uint32_t> cnt(m), k(m);
    if (cudaMemcpyAsync(r.data(), ws->d_ranges, sizeof(uint4) * m, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(cnt.data(), ws->d_count, sizeof(uint32_t) * m, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(k.data(), ws->d_key, sizeof(uint32_t) * m, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GEER_ERR_CUDA;
    for (int64_t i = 0; i < m; ++i) {
        const uint32_t w[4] = {r[i].x, r[i].y, r[i].z, r[i].w};
        if (ranges)
            for (int j = 0; j < 4; ++j) {
                ranges[8 * i + 2 * j] = (uint16_t)(w[j] & 0xffff);
                ranges[8 * i + 2 * j + 1] = (uint16_t)(w[j] >> 16);
            }
        if (counts) counts[i] = cnt[i];
        if (keys) keys[i] = k[i];
        if (cull) cull[i] = k[i] == 0u ? 1 : 0;  // a live Gaussian has a positive depth key
    }
    return GEER_OK;
}

geer_status geer_debug_pairs(geer_workspace *ws, uint64_t *keys, uint32_t *values, int64_t cap, int64_t *count,
                             void *stream) {
    if (!ws || !count || cap < 0) return GEER_ERR_ARG;
    if (ws->stage < 2) return GEER_ERR_STATE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t m[kMiscCount];
    if (cudaMemcpyAsync(m, ws->d_misc, sizeof(m), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GEER_ERR_CUDA;
    if (m[kMiscStatus] & kStatusCapacity) return GEER_ERR_CAPACITY;
    const int64_t P = ((int64_t)m[kMiscTileHi] << 32) | (int64_t)m[kMiscTileLo];
    *count = P;
    const int64_t n = std::min(P, cap);
    if (n == 0) return GEER_OK;
    // every tile's full list, filtered from its super-tile's list as the renders
    // do: count, offsets on the host, then the lists (into the free sort buffer)
    if (P > ws->cap_pairs) return GEER_ERR_CAPACITY;
    uint32_t *scratch = reinterpret_cast<uint32_t *>(ws->d_tile_walk + ws->n_tiles);
    uint32_t *lists = ws->d_keys[ws->sorted_buf ^ 1];
    std::vector<uint32_t> cnt(ws->n_tiles), off(ws->n_tiles);
    if (launch_expand_tiles(ws, scratch, nullptr, s) != cudaSuccess ||
        cudaMemcpyAsync(cnt.data(), scratch, sizeof(uint32_t) * ws->n_tiles, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GEER_ERR_CUDA;
    int64_t run = 0;
    for (int64_t t = 0; t < ws->n_tiles; ++t) {
        off[t] = (uint32_t)run;
        run += cnt[t];
    }
    if (run != P) return GEER_ERR_CUDA;  // the filtered lists must hold exactly the counted associations
    const int64_t items = (int64_t)ws->n_cams * ws->n_gauss;
    std::vector<uint32_t> v(P), depth(items);
    if (cudaMemcpyAsync(scratch, off.data(), sizeof(uint32_t) * ws->n_tiles, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        launch_expand_tiles(ws, scratch, lists, s) != cudaSuccess ||
        cudaMemcpyAsync(v.data(), lists, sizeof(uint32_t) * P, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(depth.data(), ws->d_key, sizeof(uint32_t) * items, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GEER_ERR_CUDA;
    for (int64_t t = 0; t < ws->n_tiles; ++t)
        for (int64_t i = off[t]; i < (int64_t)off[t] + cnt[t] && i < n; ++i) {
            if (keys) keys[i] = ((uint64_t)t << 32) | (v[i] < items ? depth[v[i]] : 0u);
            if (values) values[i] = v[i];
        }
    return GEER_OK;
}

geer_status geer_tile_counts(geer_workspace *ws, uint32_t *counts, void *stream) {
    if (!ws || !counts) return GEER_ERR_ARG;
    if (ws->stage < 2) return GEER_ERR_STATE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t m[kMiscCount];
    if (cudaMemcpyAsync(m, ws->d_misc, sizeof(m), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GEER_ERR_CUDA;
    if (m[kMiscStatus] & kStatusCapacity) return GEER_ERR_CAPACITY;
    if (ws->n_tiles == 0) return GEER_OK;
    uint32_t *scratch = reinterpret_cast<uint32_t *>(ws->d_tile_walk + ws->n_tiles);
    if (launch_expand_tiles(ws, scratch, nullptr, s) != cudaSuccess ||
        cudaMemcpyAsync(counts, scratch, sizeof(uint32_t) * ws->n_tiles, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GEER_ERR_CUDA;
    return GEER_OK;
}

geer_status geer_debug_render_state(geer_workspace *ws, uint32_t *evals, uint32_t *last, uint32_t *walk,
                                    void *stream) {
    if (!ws) return GEER_ERR_ARG;
    if (ws->stage < 3) return GEER_ERR_STATE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((evals && cudaMemcpyAsync(evals, ws->d_evals, sizeof(uint2) * ws->n_pixels, cudaMemcpyDeviceToHost, s) !=
                      cudaSuccess) ||
        (last && cudaMemcpyAsync(last, ws->d_last, sizeof(uint32_t) * ws->n_pixels, cudaMemcpyDeviceToHost, s) !=
                     cudaSuccess) ||
        (walk && cudaMemcpyAsync(walk, ws->d_tile_walk, sizeof(uint2) * ws->n_tiles, cudaMemcpyDeviceToHost, s) !=
                     cudaSuccess) ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GEER_ERR_CUDA;
    return GEER_OK;
}

geer_status geer_pair_counts(geer_workspace *ws, int64_t *tile_pairs, int64_t *super_pairs, int32_t *sort_passes,
                             int64_t *live_items, void *stream) {
    if (!ws) return GEER_ERR_ARG;
    if (ws->stage < 2) return GEER_ERR_STATE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t m[kMiscCount];
    if (cudaMemcpyAsync(m, ws->d_misc, sizeof(m), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GEER_ERR_CUDA;
    if (tile_pairs) *tile_pairs = ((int64_t)m[kMiscTileHi] << 32) | (int64_t)m[kMiscTileLo];
    if (super_pairs) *super_pairs = ((int64_t)m[kMiscPairsHi] << 32) | (int64_t)m[kMiscTotalLo];
    if (sort_passes) *sort_passes = ws->n_sort_passes;
    if (live_items) *live_items = m[kMiscLive];
    return GEER_OK;
}

geer_status geer_l1_loss_grad(const float *rgb, const float *target, int64_t n_values, float *dL_drgb, float *loss,
                              void *stream) {
    if (n_values < 0 || (n_values > 0 && (!rgb || !target || !dL_drgb))) return GEER_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GEER_ERR_CUDA;
    return cuda_status(launch_l1_grad(rgb, target, n_values, dL_drgb, loss, sms, static_cast<cudaStream_t>(stream)));
}

geer_status geer_render_counts(geer_workspace *ws, uint64_t *evaluated, uint64_t *applied, uint64_t *walked_back,
                               void *stream) {
    if (!ws || !evaluated || !applied) return GEER_ERR_ARG;
    if (ws->stage < 3) return GEER_ERR_STATE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<uint2> v(ws->n_pixels);
    std::vector<uint32_t> last(ws->n_pixels);
    if (cudaMemcpyAsync(v.data(), ws->d_evals, sizeof(uint2) * ws->n_pixels, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(last.data(), ws->d_last, sizeof(uint32_t) * ws->n_pixels, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GEER_ERR_CUDA;
    uint64_t e = 0, a = 0, w = 0;
    for (int64_t i = 0; i < ws->n_pixels; ++i) {
        e += v[i].x;
        a += v[i].y;
        w += last[i];
    }
    *evaluated = e;
    *applied = a;
    if (walked_back) *walked_back = w;
    return GEER_OK;
}

// The native camera's vertical BEAP field of view, focal length and largest
// invertible angle of its distortion (App. E), for the remap kernel.
static void native_params(const geer_camera *cam, double &fy, double &focal, double &phi_max) {
    fy = derived_fov_y(*cam);
    const double half = 0.5 * (double)cam->fov_x;
    if (cam->model == GEER_PINHOLE) {
        focal = 0.5 * cam->width / tan(half);
        phi_max = 0.0;
    } else {
        float k0[4] = {0, 0, 0, 0};
        const float *k = cam->model == GEER_KANNALA_BRANDT ? cam->k : k0;
        focal = 0.5 * cam->width / kb_theta_d(k, half);
        // the distortion must stay invertible (increasing) up to phi_max: the first
        // turning point of phi_d(phi) below pi, or pi
        phi_max = M_PI;
        const int steps = 4096;
        double prev = 0.0;
        for (int s2 = 1; s2 <= steps; ++s2) {
            const double ph = M_PI * s2 / steps, val = kb_theta_d(k, ph);
            if (!(val > prev)) { phi_max = M_PI * (s2 - 1) / steps; break; }
            prev = val;
        }
    }
}

geer_status geer_remap_to_native(const float *beap_rgb, const geer_camera *cam, const float *fill_rgb,
                                 float *native_rgb, void *stream) {
    if (!beap_rgb || !cam || !native_rgb || !camera_ok(*cam)) return GEER_ERR_ARG;
    double fy, focal, phi_max;
    native_params(cam, fy, focal, phi_max);
    return cuda_status(launch_remap_to_native(beap_rgb, cam, fy, focal, phi_max, fill_rgb, native_rgb, nullptr,
                                              static_cast<cudaStream_t>(stream)));
}

geer_status geer_native_to_beap(const float *native_rgb, const geer_camera *cam, float *beap_rgb, uint8_t *valid,
                                void *stream) {
    if (!native_rgb || !cam || !beap_rgb || !camera_ok(*cam)) return GEER_ERR_ARG;
    double fy, focal, phi_max;
    native_params(cam, fy, focal, phi_max);
    return cuda_status(launch_native_to_beap(native_rgb, cam, fy, focal, phi_max, beap_rgb, valid,
                                             static_cast<cudaStream_t>(stream)));
}

geer_status geer_adam_step(const geer_adam *hp, int64_t n, int32_t sh_degree, float *mean, float *log_scale,
                           float *quat, float *logit_opacity, float *sh, const float *d_mean, const float *d_scale,
                           const float *d_quat, const float *d_opacity, const float *d_sh, float *m, float *v,
                           float *scale, float *opacity, void *stream) {
    if (!hp || n < 0 || sh_degree < 0 || sh_degree > 3 || hp->step < 1 || !(hp->beta1 >= 0.0f && hp->beta1 < 1.0f) ||
        !(hp->beta2 >= 0.0f && hp->beta2 < 1.0f) || !(hp->eps >= 0.0f))
        return GEER_ERR_ARG;
    if (n > 0 && (!mean || !log_scale || !quat || !logit_opacity || !sh || !d_mean || !d_scale || !d_quat ||
                  !d_opacity || !d_sh || !m || !v))
        return GEER_ERR_ARG;
    return cuda_status(launch_adam_gaussians(hp, n, sh_degree, mean, log_scale, quat, logit_opacity, sh, d_mean,
                                             d_scale, d_quat, d_opacity, d_sh, m, v, scale, opacity,
                                             static_cast<cudaStream_t>(stream)));
}

geer_status geer_densify_accumulate(geer_workspace *ws, const float *d_mean, float *accum, float *denom,
                                    void *stream) {
    if (!ws || (ws->n_gauss > 0 && (!d_mean || !accum || !denom))) return GEER_ERR_ARG;
    if (ws->stage < 1) return GEER_ERR_STATE;  // needs a preprocess
    return cuda_status(launch_densify_accum(ws, d_mean, accum, denom, static_cast<cudaStream_t>(stream)));
}

size_t geer_densify_scratch_bytes(int64_t n) { return n < 0 ? 0 : densify_scratch_bytes(n); }

namespace {
bool densify_params_ok(const geer_densify_params *hp) {
    return hp && hp->grad_threshold >= 0.0f && std::isfinite(hp->grad_threshold) && hp->clone_max_scale > 0.0f &&
           std::isfinite(hp->clone_max_scale) && hp->min_opacity > 0.0f && hp->min_opacity < 1.0f &&
           hp->max_scale >= 0.0f && std::isfinite(hp->max_scale);
}
bool scratch_ok(const void *scratch, size_t bytes, int64_t n) {
    return scratch && (reinterpret_cast<uintptr_t>(scratch) & 15) == 0 && bytes >= densify_scratch_bytes(n);
}
}  // namespace

geer_status geer_densify_plan(const geer_densify_params *hp, int64_t n, const float *log_scale,
                              const float *logit_opacity, const float *accum, const float *denom, void *scratch,
                              size_t scratch_bytes, int64_t *n_out, void *stream) {
    // n <= 2^30: the outputs (at most 2 n) are indexed in 32 bits
    if (!densify_params_ok(hp) || n < 0 || n > ((int64_t)1 << 30) || !n_out || !scratch_ok(scratch, scratch_bytes, n))
        return GEER_ERR_ARG;
    if (n > 0 && (!log_scale || !logit_opacity || !accum || !denom)) return GEER_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto *total = reinterpret_cast<unsigned long long *>(static_cast<char *>(scratch) + densify_scratch_bytes(n) - 16);
    unsigned long long h = 0;
    if (launch_densify_plan(hp, n, log_scale, logit_opacity, accum, denom, scratch, total, s) != cudaSuccess ||
        cudaMemcpyAsync(&h, total, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GEER_ERR_CUDA;
    *n_out = (int64_t)h;
    return GEER_OK;
}

geer_status geer_densify_apply(int64_t n, int32_t sh_degree, const float *mean, const float *log_scale,
                               const float *quat, const float *logit_opacity, const float *sh, const float *m,
                               const float *v, const float *z, void *scratch, size_t scratch_bytes,
                               int64_t n_out, float *o_mean, float *o_log_scale, float *o_quat, float *o_logit,
                               float *o_sh, float *o_m, float *o_v, float *o_scale, float *o_opacity, void *stream) {
    if (n < 0 || n > ((int64_t)1 << 30) || n_out < 0 || n_out > 2 * n || sh_degree < 0 || sh_degree > 3 ||
        !scratch_ok(scratch, scratch_bytes, n))
        return GEER_ERR_ARG;
    if (n > 0 && (!mean || !log_scale || !quat || !logit_opacity || !sh || !m || !v || !z))
        return GEER_ERR_ARG;
    if (n_out > 0 && (!o_mean || !o_log_scale || !o_quat || !o_logit || !o_sh || !o_m || !o_v)) return GEER_ERR_ARG;
    return cuda_status(launch_densify_apply(n, sh_degree, mean, log_scale, quat, logit_opacity, sh, m, v, z, scratch,
                                            n_out, o_mean, o_log_scale, o_quat, o_logit, o_sh, o_m, o_v, o_scale,
                                            o_opacity, static_cast<cudaStream_t>(stream)));
}

geer_status geer_opacity_reset(int64_t n, int32_t sh_degree, float value, float *logit_opacity, float *m, float *v,
                               float *opacity, void *stream) {
    if (n < 0 || sh_degree < 0 || sh_degree > 3 || !(value > 0.0f && value < 1.0f)) return GEER_ERR_ARG;
    if (n > 0 && (!logit_opacity || !m || !v)) return GEER_ERR_ARG;
    // the opacity block of the moments starts at 10 n (after mean, log-scale and quaternion)
    return cuda_status(launch_opacity_reset(n, value, logit_opacity, m + 10 * n, v + 10 * n, opacity,
                                            static_cast<cudaStream_t>(stream)));
}

geer_status geer_native_regions(const geer_camera *cam, uint8_t *regions, void *stream) {
    if (!cam || !regions || !camera_ok(*cam)) return GEER_ERR_ARG;
    double fy, focal, phi_max;
    native_params(cam, fy, focal, phi_max);
    return cuda_status(launch_remap_to_native(nullptr, cam, fy, focal, phi_max, nullptr, nullptr, regions,
                                              static_cast<cudaStream_t>(stream)));
}

geer_status geer_image_metrics(const float *pred, const float *gt, int32_t width, int32_t height,
                               const uint8_t *regions, int32_t n_regions, double *acc, double *out, void *stream) {
    if (!pred || !gt || !acc || !out || width < 0 || height < 0 || n_regions < 1 || n_regions > 8)
        return GEER_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double sums[3 * 8];
    if (launch_image_metrics(pred, gt, width, height, regions, n_regions, acc, s) != cudaSuccess ||
        cudaMemcpyAsync(sums, acc, sizeof(double) * 3 * n_regions, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GEER_ERR_CUDA;
    for (int r = 0; r < n_regions; ++r) {
        const double sse = sums[3 * r], ssim = sums[3 * r + 1], cnt = sums[3 * r + 2];
        double *o = out + 5 * r;
        o[0] = sse;
        o[1] = ssim;
        o[2] = cnt;
        // PSNR of values in [0, 1]: 10 log10(1 / MSE), MSE over the region's pixels and 3 channels
        o[3] = cnt > 0.0 ? (sse > 0.0 ? 10.0 * log10(3.0 * cnt / sse) : INFINITY) : NAN;
        o[4] = cnt > 0.0 ? ssim / cnt : NAN;
    }
    return GEER_OK;
}

static const char *kStageNames[kStageCount] = {"preprocess", "bin_front", "depth_sort", "count_pairs", "duplicate",
                                               "tile_sort", "render_fwd", "render_bwd", "preprocess_bwd",
                                               "render_train"};

const char *geer_stage_name(int32_t stage) {
    return (stage >= 0 && stage < kStageCount) ? kStageNames[stage] : "unknown";
}

geer_status geer_enable_stage_timing(geer_workspace *ws, uint32_t mask) {
    if (!ws) return GEER_ERR_ARG;
    mask &= (1u << kStageCount) - 1u;
    geer_status st = geer_enable_timing(ws, mask ? 1 : 0);
    if (st == GEER_OK) ws->timing_mask = mask;
    return st;
}

geer_status geer_enable_timing(geer_workspace *ws, int32_t enable) {
    if (!ws) return GEER_ERR_ARG;
    ws->timing_mask = (1u << kStageCount) - 1u;
    if (enable && !ws->timing) {
        for (int a = 0; a < kStageCount; ++a) {
            ws->ev_count[a] = 0;
            for (int b = 0; b < kTimingRing; ++b)
                if (cudaEventCreate(&ws->ev[a][b][0]) != cudaSuccess || cudaEventCreate(&ws->ev[a][b][1]) != cudaSuccess)
                    return GEER_ERR_CUDA;
        }
        ws->timing = 1;
    } else if (!enable && ws->timing) {
        for (int a = 0; a < kStageCount; ++a)
            for (int b = 0; b < kTimingRing; ++b) {
                cudaEventDestroy(ws->ev[a][b][0]);
                cudaEventDestroy(ws->ev[a][b][1]);
            }
        ws->timing = 0;
    }
    return GEER_OK;
}

geer_status geer_stage_times(geer_workspace *ws, float *ms, int32_t n, int32_t *counts, void *stream) {
    if (!ws || !ms || n < kStageCount) return GEER_ERR_ARG;
    if (!ws->timing) return GEER_ERR_STATE;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return GEER_ERR_CUDA;
    for (int a = 0; a < kStageCount; ++a) {
        const int k = std::min(ws->ev_count[a], kTimingRing);
        double tot = 0.0;
        for (int b = 0; b < k; ++b) {
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, ws->ev[a][b][0], ws->ev[a][b][1]) != cudaSuccess) return GEER_ERR_CUDA;
            tot += t;
        }
        ms[a] = k ? (float)(tot / k) : 0.0f;
        if (counts) counts[a] = k;
    }
    return GEER_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free render of one small camera (geer_render_noalloc).
//
// All device scratch lives in the file-scope array g_noalloc_scratch below;
// every GPU that loads the library holds it until the process exits. Host code
// sees only a host-side stand-in for the symbol, so the device address is
// taken once per device with cudaGetSymbolAddress (with that device current)
// and handed to the kernels. Host-side state is static as well: no heap,
// no cudaMalloc/cudaMallocHost/cudaFree.
namespace {

constexpr int64_t kNoAllocMaxGauss = 32768;
constexpr int64_t kNoAllocMaxPixels = 512 * 512;
constexpr int64_t kNoAllocMaxPairs = int64_t(1) << 19;  // (super-tile, Gaussian) pairs
constexpr int64_t kNoAllocMaxTileTab = 2 * 1024;   // tile columns + rows
constexpr int64_t kNoAllocMaxPixTab = 8 * 1024;    // pixel columns + rows
constexpr int64_t kNoAllocMaxTiles = 2 * 1024;
constexpr size_t kNoAllocBytes = size_t(28) << 20;  // 28 MiB, checked against the layout at set-up
constexpr int kNoAllocMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocState {
    bool ready;
    char *base;  // device address of g_noalloc_scratch on this device
    int num_sms;
    geer_workspace ws;
    DevCam cam;
    float4 ttab[kNoAllocMaxTileTab];
    float2 ptab[kNoAllocMaxPixTab];
};
NoAllocState g_noalloc[kNoAllocMaxDevices];

// The per-camera tables of build_tables, for one camera, into fixed arrays.
bool noalloc_tables(const geer_camera &c, NoAllocState &st, int64_t &ntt, int64_t &npt) {
    DevCam &d = st.cam;
    memset(&d, 0, sizeof(d));
    d.width = c.width;
    d.height = c.height;
    d.tiles_x = (int)ceil_div(c.width, kTile);
    d.tiles_y = (int)ceil_div(c.height, kTile);
    ntt = (int64_t)d.tiles_x + d.tiles_y;
    npt = (int64_t)c.width + c.height;
    if (ntt > kNoAllocMaxTileTab || npt > kNoAllocMaxPixTab || (int64_t)d.tiles_x * d.tiles_y > kNoAllocMaxTiles)
        return false;
    const double fx = c.fov_x, fy = derived_fov_y(c);
    d.col_ppr = (float)(c.width / fx);
    d.row_ppr = (float)(c.height / fy);
    d.tcol_off = 0;
    for (int tx = 0; tx < d.tiles_x; ++tx) {
        const int i0 = tx * kTile, i1 = std::min(i0 + kTile - 1, c.width - 1);
        float4 v = make_float4((float)tan(0.5 * beap_angle(i0, c.width, fx)),
                               (float)tan(0.5 * beap_angle(i1, c.width, fx)), 0.0f, 0.0f);
        for (int i = i0; i <= i1; ++i) {
            const double cs = cos(beap_angle(i, c.width, fx));
            if (cs > -1e-12) v.z = 1.0f;
            if (cs < 1e-12) { v.w = 1.0f; d.any_col_flip = 1; }
        }
        st.ttab[tx] = v;
    }
    d.trow_off = d.tiles_x;
    for (int ty = 0; ty < d.tiles_y; ++ty) {
        const int j0 = ty * kTile, j1 = std::min(j0 + kTile - 1, c.height - 1);
        float4 v = make_float4((float)tan(0.5 * beap_angle(j0, c.height, fy)),
                               (float)tan(0.5 * beap_angle(j1, c.height, fy)), 0.0f, 0.0f);
        for (int j = j0; j <= j1; ++j) {
            const double cs = cos(beap_angle(j, c.height, fy));
            if (cs > -1e-12) v.z = 1.0f;
            if (cs < 1e-12) { v.w = 1.0f; d.any_row_flip = 1; }
        }
        st.ttab[d.tiles_x + ty] = v;
    }
    d.pcol_off = 0;
    for (int i = 0; i < c.width; ++i) {
        const double a = beap_angle(i, c.width, fx);
        st.ptab[i] = make_float2((float)sin(a), (float)cos(a));
    }
    d.prow_off = c.width;
    for (int j = 0; j < c.height; ++j) {
        const double a = beap_angle(j, c.height, fy);
        st.ptab[c.width + j] = make_float2((float)sin(a), (float)cos(a));
    }
    if (!flag_intervals(st.ttab, d.tiles_x, d.zc, d.wc) || !flag_intervals(st.ttab + d.tiles_x, d.tiles_y, d.zr, d.wr))
        return false;
    d.c0lo = d.tiles_x; d.c0hi = 0;
    for (int tx = 0; tx < d.tiles_x; ++tx) {
        const float4 v = st.ttab[tx];
        if (v.z != 0.0f && v.w == 0.0f) { d.c0lo = std::min(d.c0lo, tx); d.c0hi = tx + 1; }
    }
    d.r0lo = d.tiles_y; d.r0hi = 0;
    for (int ty = 0; ty < d.tiles_y; ++ty) {
        const float4 v = st.ttab[d.tiles_x + ty];
        if (v.z != 0.0f && v.w == 0.0f) { d.r0lo = std::min(d.r0lo, ty); d.r0hi = ty + 1; }
    }
    for (int k = 0; k < 9; ++k) d.R[k] = c.R_cw[k];
    for (int k = 0; k < 3; ++k) {
        d.t[k] = c.t_cw[k];
        d.bg[k] = c.bg[k];
        double o = 0.0;
        for (int b = 0; b < 3; ++b) o -= (double)c.R_cw[3 * b + k] * (double)c.t_cw[b];
        d.o[k] = (float)o;
    }
    return true;
}

}  // namespace

extern "C" geer_status geer_render_noalloc(const geer_gaussians *g, const geer_camera *cam, const geer_params *params,
                                           float *rgb, float *T_final, void *stream) {
    if (!g || !cam || !rgb) return GEER_ERR_ARG;
    geer_params pd;
    geer_default_params(&pd);
    if (!params) params = &pd;
    geer_status st = check_params(params);
    if (st != GEER_OK) return st;
    if (!camera_ok(*cam)) return GEER_ERR_ARG;
    if (g->n < 0 || g->sh_degree < 0 || g->sh_degree > 3) return GEER_ERR_ARG;
    if (g->n > 0 && (!g->mean || !g->scale || !g->quat || !g->opacity || !g->sh)) return GEER_ERR_ARG;
    if (g->n > 0 && (reinterpret_cast<uintptr_t>(g->sh) & 15)) return GEER_ERR_ARG;
    if (g->n > kNoAllocMaxGauss || (int64_t)cam->width * cam->height > kNoAllocMaxPixels) return GEER_ERR_CAPACITY;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GEER_ERR_CUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return GEER_ERR_UNSUPPORTED;
    NoAllocState &S = g_noalloc[dev];
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!S.ready) {
        // once per device, with the device current: the device address of the scratch array
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return GEER_ERR_CUDA;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GEER_ERR_CUDA;
        S.base = static_cast<char *>(ptr);
        S.num_sms = sms;
        S.ready = true;
    }
    int64_t ntt = 0, npt = 0;
    if (!noalloc_tables(*cam, S, ntt, npt)) return GEER_ERR_CAPACITY;
    // lay the workspace out in the scratch array for the fixed maxima
    Caps c;
    c.cams = 1;
    c.pixels = kNoAllocMaxPixels;
    c.tiles = kNoAllocMaxTiles;
    c.tile_tab = kNoAllocMaxTileTab;
    c.pix_tab = kNoAllocMaxPixTab;
    c.gauss = kNoAllocMaxGauss;
    c.pairs = kNoAllocMaxPairs;
    c.sort_tiles = ceil_div(std::max<int64_t>(c.pairs, c.gauss), kSortTile) + 1;
    c.prep_blocks = prep_blocks(c.gauss);
    c.hit_entries = 0;  // forward only: no hit record
    if (layout(c, nullptr, nullptr) > kNoAllocBytes) return GEER_ERR_UNSUPPORTED;
    geer_workspace &ws = S.ws;
    memset(&ws, 0, sizeof(ws));
    layout(c, S.base, &ws);
    ws.cap_cams = 1;
    ws.cap_pixels = c.pixels;
    ws.cap_tiles = c.tiles;
    ws.cap_tile_tab = c.tile_tab;
    ws.cap_pix_tab = c.pix_tab;
    ws.cap_gauss = kNoAllocMaxGauss;
    ws.cap_pairs = kNoAllocMaxPairs;
    ws.cap_sh_degree = 3;
    ws.cap_sort_tiles = c.sort_tiles;
    ws.params = Params{params->alpha_min, params->T_min, params->alpha_max, params->lambda_pad, params->assoc,
                       params->snugbox, params->alpha_model};
    ws.num_sms = S.num_sms;
    ws.sort_grid = S.num_sms * sort_blocks_per_sm();
    ws.n_cams = 1;
    ws.n_pixels = (int64_t)cam->width * cam->height;
    ws.n_tiles = (int64_t)S.cam.tiles_x * S.cam.tiles_y;
    assign_super(&S.cam, 1, 0, ws.super_size, ws.n_stiles);
    ws.n_sort_passes = sort_passes(ws.n_stiles);
    ws.cams[0] = S.cam;
    ws.n_gauss = g->n;
    ws.sh_degree = g->sh_degree;
    // the array keeps the previous call's contents: clear what must start at zero
    // and upload this camera's tables (from static host buffers)
    if (cudaMemsetAsync(ws.d_misc, 0, sizeof(uint32_t) * kMiscCount, s) != cudaSuccess ||
        cudaMemsetAsync(ws.d_group_sum, 0, sizeof(uint32_t) * kRadix * (ceil_div(c.sort_tiles, kGroupTiles) + 1),
                        s) != cudaSuccess ||
        cudaMemcpyAsync(ws.d_cams, &S.cam, sizeof(DevCam), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(ws.d_tile_tab, S.ttab, sizeof(float4) * ntt, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(ws.d_pix_tab, S.ptab, sizeof(float2) * npt, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return GEER_ERR_CUDA;
    if (launch_preprocess(&ws, g, s) != cudaSuccess || launch_bin_front(&ws, s) != cudaSuccess ||
        launch_depth_sort(&ws, s) != cudaSuccess || launch_count_pairs(&ws, s) != cudaSuccess)
        return GEER_ERR_CUDA;
    static uint32_t h_misc[kNoAllocMaxDevices][kMiscCount];
    if (cudaMemcpyAsync(h_misc[dev], ws.d_misc, sizeof(uint32_t) * kMiscCount, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GEER_ERR_CUDA;
    if (h_misc[dev][kMiscPairsHi] != 0 || (int64_t)h_misc[dev][kMiscTotalLo] > kNoAllocMaxPairs)
        return GEER_ERR_CAPACITY;
    if (launch_duplicate(&ws, s) != cudaSuccess || launch_tile_sort(&ws, s) != cudaSuccess ||
        launch_render_fwd(&ws, rgb, T_final, s) != cudaSuccess)
        return GEER_ERR_CUDA;
    return GEER_OK;
}
