// geer_internal.cuh -- shared declarations of the CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/geer.h"

namespace geer {

constexpr int kTile = 16;                   // BEAP tile edge in rays (a camera sub-frustum)
constexpr int kTilePix = kTile * kTile;
constexpr int kTileWarps = kTilePix / 32;    // warps of a tile's rays (one byte each in the hit record)
constexpr uint8_t kRegionCentral = 0, kRegionPeripheral = 1, kRegionNone = 255;  // native evaluation regions
constexpr int64_t kHitEntries = 2048;      // tile-list entries per tile whose hit bytes are recorded
// Forward checkpoints: the rays' (T, C) at the end of the first forward batch
// reaching tile-list index kCkptFirst, then every kCkptStride entries, at most
// kCkptMax per tile. The backward splits a tile's walk there into units that
// run in parallel.
constexpr int kCkptMax = 8;
constexpr uint32_t kCkptFirst = 192, kCkptStride = 256;
constexpr int kPrepThreads = 256;           // preprocess / duplicate block size
constexpr int kSortThreads = 256;           // onesweep block size (8 warps)
constexpr int kSortItems = 12;              // keys per thread per sort tile
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kMaxCams = 256;
constexpr int kGroupTiles = 32;            // sort tiles per group (radix offsets are scanned per group)
constexpr int kSmemTiles = 12288;          // per-block tile histogram in shared memory up to this many tiles

// Device status word bits.
constexpr uint32_t kStatusCapacity = 1u;
constexpr uint32_t kStatusListOverflow = 2u;  // inspection: a tile list differs from its counted length
constexpr uint32_t kStatusBounds = 4u;        // GEER_CHECKED build: a bounds guard skipped an access
constexpr uint32_t kStatusTimeout = 8u;       // a bounded wait (a shared-memory barrier, the fused render's unit queue) gave up

// Indices into the misc u32 array of the workspace.
enum Misc : int {
    kMiscStatus = 0,      // device status bits
    kMiscPairs = 1,       // (super-tile, item) pairs to sort (clamped to the capacity)
    kMiscPairsHi = 2,     // unclamped pair count / 2^32
    kMiscTotalLo = 4,     // unclamped pair count mod 2^32
    kMiscLive = 5,        // live (camera, Gaussian) items (tile count > 0)
    kMiscTileLo = 6,      // (tile, item) associations P mod 2^32
    kMiscTileHi = 7,      // P / 2^32
    kMiscSortDone = 8,    // radix histogram blocks finished in the current pass
    kMiscSortSame = 9,    // the current pass's digit is the same for every key (an identity pass, skipped)
    kMiscCheckSite = 10,  // GEER_CHECKED build: site of the first bounds violation (0: none)
    kMiscCheckLo = 11,    // its index mod 2^32
    kMiscCheckHi = 12,    // its index / 2^32
    kMiscUnits = 13,      // backward units of the last geer_render_bwd_tiles (tile walks split at checkpoints)
    kMiscUnitNext = 14,   // the next backward unit to take (persistent blocks)
    kMiscSortCur = 15,    // depth sort: the buffer the current pass reads (set by its histogram kernel)
    kMiscFwdNext = 16,    // fused render: the next forward tile (of the render order) to take
    kMiscFwdDone = 17,    // fused render: forward tiles finished, their units published
    kMiscUnitsPub = 18,   // fused render: backward units published (slots reserved in the unit queue)
    kMiscTrainNext = 19,  // fused render: the next queue slot a block takes
    kMiscCount = 32
};

#ifndef GEER_CHECKED
#define GEER_CHECKED 0  // 1: bounds guards record their first violation (libgeer_checked.so)
#endif

// Sites of the bounds guards (reported by geer_bounds_violation).
enum CheckSite : uint32_t {
    kSiteFwdTile = 1,     // render forward: tile index from the render order
    kSiteFwdList = 2,     // render forward: super-tile list range [start, end) against the pair capacity
    kSiteFwdItem = 3,     // render forward: item id from the sorted pairs
    kSiteBwdTile = 4,     // render backward: tile index from the backward order
    kSiteBwdList = 5,     // render backward: super-tile list range
    kSiteBwdItem = 6,     // render backward: item id (record gather, accumulator scatter)
    kSiteDupSuper = 7,    // duplicate: super-tile id of an emitted pair
};

// Guard of an index that comes from an earlier kernel (or from the caller's
// data): true when i < n; otherwise the caller skips the access. In a
// GEER_CHECKED build a failing guard also records the first violation (site,
// index) next to the device status word, where geer_bounds_violation reads it.
__device__ __forceinline__ bool in_bounds(uint64_t i, uint64_t n, uint32_t site, uint32_t *misc) {
    if (i < n) return true;
#if GEER_CHECKED
    if (atomicCAS(misc + kMiscCheckSite, 0u, site) == 0u) {
        misc[kMiscCheckLo] = (uint32_t)i;
        misc[kMiscCheckHi] = (uint32_t)(i >> 32);
    }
    atomicOr(misc + kMiscStatus, kStatusBounds);
#else
    (void)site;
    (void)misc;
#endif
    return false;
}

// One camera as the kernels see it. Angles and tables are precomputed on the
// host in FP64 and rounded to FP32.
struct DevCam {
    int32_t width, height, tiles_x, tiles_y;
    int32_t tile_base;   // global index of tile (0, 0)
    int32_t any_row_flip, any_col_flip;
    int32_t tcol_off, trow_off;  // offsets (in float4) of the per-tile tables
    int32_t pcol_off, prow_off;  // offsets (in float2) of the per-pixel tables
    int32_t c0lo, c0hi, r0lo, r0hi;  // tile columns / rows whose rays all have cos >= 0
    int32_t stiles_x;    // super-tiles per row (ceil(tiles_x / super-tile size))
    int32_t stile_base;  // global index of super-tile (0, 0)
    // tile columns / rows holding rays with cos >= 0 (the z flag): one interval [lo, hi);
    // with cos <= 0 (the w flag): the runs [0, a) and [b, n)
    int32_t zc[2], wc[2], zr[2], wr[2];
    int32_t pad_;
    float col_ppr, row_ppr;  // BEAP pixels per radian (width / fov_x, height / fov_y)
    int64_t pix_base;    // offset of pixel (0, 0) in the batched image (in pixels)
    float R[9], t[3];    // world -> camera
    float o[3];          // camera centre in world coordinates
    float bg[3];
};

// Per (camera, Gaussian) render record, 64 bytes: the whitening W = S^-1 (R_cw R)^T
// (camera frame, row-major), o_u = W (0 - mu_c), log2(sigma) and the colour.
struct __align__(16) Record {
    float W[9];
    float ou[3];
    float log2_sigma;
    float rgb[3];
};
static_assert(sizeof(Record) == 64, "record must be 64 bytes");

// Per (camera, Gaussian) render-stage gradient accumulators (App. C, RenderCUDA
// part): dL/dsigma, dL/drgb, dL/dW|RC = sum dL/dd_u d^T and dL/do_u. 16 floats.
// (Summing instead the ray moments of t = o_u.d_u/|d_u|^2 and forming dL/dW from
// them afterwards needs fewer operations per ray but loses two to three decimal
// digits in FP32 to the cancellation between its two terms.)
struct __align__(16) GradAcc {
    float d_sigma;   // dL/dsigma
    float d_rgb[3];  // dL/dc
    float d_W[9];    // dL/dW through d_u (RenderCUDA part)
    float d_ou[3];   // dL/do_u
};
static_assert(sizeof(GradAcc) == 64, "grad accumulator must be 64 bytes");

struct Params {
    float alpha_min, T_min, alpha_max, lambda_pad;
    int32_t assoc, snug;  // GEER_ASSOC_*, SnugBox flag
    int32_t alpha_model;  // GEER_ALPHA_*
};

// PBF association ranges of a (camera, Gaussian) item, packed as u16 pairs:
// [0,1) columns and [4,5) rows of the direct arcs, [2,3) and [6,7) of the arcs
// shifted by pi (rays beyond 90 degrees).
#ifndef GEER_PDL
#define GEER_PDL 1  // programmatic dependent launch of the library's kernels
#endif

// Programmatic dependent launch: every kernel first lets the next kernel on its
// stream begin launching (its blocks may become resident while this grid's last
// blocks run), then waits until its own predecessor grid has completed and its
// writes are visible (griddepcontrol). The next grid launches only once every
// block of this one has started, so a waiting block never keeps a predecessor's
// block from starting. For an ordinary stream-ordered launch both are no-ops.
__device__ __forceinline__ void grid_dep_sync() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Launches a kernel on stream s with programmatic stream serialization (GEER_PDL).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = GEER_PDL;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Asynchronous 4-byte global -> shared copy (completed by cp.async.wait_all).
__device__ __forceinline__ void cp_async4(float *smem, const float *gmem) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem) : "memory");
}

// Bulk (TMA engine) copies into shared memory that complete on an mbarrier.
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Arrive once on the barrier, announcing `bytes` more to be written by bulk copies.
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// bytes (a multiple of 16, both addresses 16-byte aligned) from global to this
// CTA's shared memory; completion is counted on bar.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Orders this thread's earlier generic accesses of shared memory before later
// bulk copies into it.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Waits for the barrier's phase `parity` to complete, at most `limit` polls;
// false if it did not (the caller records a timeout and goes on).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void unpack_ranges(const uint4 r4, int rg[8]) {
    rg[0] = (int)(r4.x & 0xffff); rg[1] = (int)(r4.x >> 16); rg[2] = (int)(r4.y & 0xffff); rg[3] = (int)(r4.y >> 16);
    rg[4] = (int)(r4.z & 0xffff); rg[5] = (int)(r4.z >> 16); rg[6] = (int)(r4.w & 0xffff); rg[7] = (int)(r4.w >> 16);
}

// Association of tile (cx, cy) with an item: the column test takes the arc kind
// of the tile's rows (cos(phi) >= 0: direct, < 0: shifted) and the row test that
// of its columns; col / row are the tile's table entries (z, w: the tile has rays
// with cos >= 0 / cos <= 0).
__device__ __forceinline__ bool tile_assoc(const float4 &col, const float4 &row, int cx, int cy, const int rg[8]) {
    bool aok = (row.z != 0.0f && cx >= rg[0] && cx < rg[1]) || (row.w != 0.0f && cx >= rg[2] && cx < rg[3]);
    bool bok = (col.z != 0.0f && cy >= rg[4] && cy < rg[5]) || (col.w != 0.0f && cy >= rg[6] && cy < rg[7]);
    return aok && bok;
}

// Schedule bucket of a cost c (a tile's pair count, a backward unit's steps):
// larger costs first, four buckets per octave, zero cost last.
constexpr int kOrderBuckets = 129;
__device__ __forceinline__ int order_bucket(uint32_t c) {
    if (c == 0) return kOrderBuckets - 1;
    const int lg = 31 - __clz(c);
    const int sub = (int)((c >> (lg >= 2 ? lg - 2 : 0)) & 3u);
    return 127 - (lg * 4 + (lg >= 2 ? sub : 0));
}

// A tile's backward units as the forward leaves them (one uint4 per tile):
// byte k (k <= kCkptMax) the schedule bucket of unit k, byte 15 the number of
// units (0: nothing to walk back).
constexpr int kUnitCountByte = 15;
static_assert(kMiscTrainNext == kMiscFwdNext + 3, "the fused render's four counters are contiguous");
static_assert(kCkptMax + 1 <= kUnitCountByte, "the unit buckets and their count share one uint4");

// Stages timed by geer_enable_timing (CUDA events around each stage's kernels).
enum Stage : int {
    kStagePreprocess = 0,
    kStageBinFront,      // live-item scan + compaction
    kStageDepthSort,
    kStageCountPairs,
    kStageDuplicate,     // super-tile pairs, super-tile ranges, render order
    kStageTileSort,      // sort of the super-tile pairs
    kStageRenderFwd,
    kStageRenderBwd,
    kStagePreprocessBwd,
    kStageRenderTrain,   // the fused forward + L1 + render-stage backward
    kStageCount
};
constexpr int kTimingRing = 64;

}  // namespace geer

// Host-side workspace handle.
struct geer_workspace {
    // capacities fixed at init
    int32_t cap_cams;
    int64_t cap_pixels, cap_tiles, cap_tile_tab, cap_pix_tab;
    int64_t cap_gauss, cap_pairs;
    int32_t cap_sh_degree;
    int64_t cap_sort_tiles;
    geer::Params params;

    // current camera set
    int32_t n_cams;
    int64_t n_pixels, n_tiles;
    int32_t super_size;      // super-tile edge in tiles
    int64_t n_stiles;        // super-tile id range
    int32_t n_sort_passes;   // radix passes over the super-tile ids
    geer::DevCam cams[geer::kMaxCams];

    // device arrays (inside the caller's memory)
    geer::DevCam *d_cams;
    float4 *d_tile_tab;
    float2 *d_pix_tab;
    geer::Record *d_rec;
    uint4 *d_ranges;
    uint32_t *d_count, *d_key;
    uint32_t *d_blocksum;   // live items per preprocess block
    uint32_t *d_blocksum2;  // super-tile pairs per block of depth-sorted items (scanned: emission offsets)
    uint32_t *d_blocksum3;  // (tile, item) associations per block of depth-sorted items
    uint32_t *d_ikey[2];    // depth keys of the live items (ping-pong)
    uint32_t *d_iid[2];     // item ids (camera * n + gaussian) of the live items
    uint32_t *d_keys[2];    // super-tile ids of the (super-tile, item) pairs (ping-pong)
    uint32_t *d_vals[2];    // item ids of the pairs
    uint32_t *d_tile_hist;  // [cap_sort_tiles][kRadix] digit histogram per sort tile
    uint32_t *d_group_sum;  // [cap_sort_groups][kRadix] (zero between passes)
    uint32_t *d_group_excl; // [cap_sort_groups][kRadix]
    uint32_t *d_digit_base; // [kRadix]
    uint32_t *d_misc;       // [kMiscCount]
    uint2 *d_tile_walk;     // [cap_tiles] per tile, where the forward's scan of its super-tile list ended:
                            // (position, tile-list entries found before it); followed by [cap_tiles] u32 scratch
    uint32_t *d_tile_order; // [cap_tiles] tiles by descending super-tile list length: the forward's schedule
    uint32_t *d_bwd_order;  // [cap_tiles * (kCkptMax + 1)] backward units (tile << 4 | piece) by descending length
    float4 *d_ckpt;         // [cap_tiles][kCkptMax][kTilePix] rays' (T, C) at the forward's checkpoints (or null)
    uint2 *d_ckpt_at;       // [cap_tiles][kCkptMax] checkpoint (tile-list index, super-list position)
    uint32_t *d_ckpt_cnt;   // [cap_tiles] checkpoints recorded by the last forward
    uint4 *d_unit_rec;      // [cap_tiles] the tile's backward units: their schedule buckets and count
    float4 *d_Cfin;         // [cap_pixels] composited colour before the background (tiles with checkpoints)
    int bwd_grid;           // persistent backward blocks
    int train_grid;         // persistent blocks of the fused forward + L1 + backward render
    uint4 *d_sranges;       // [cap_pairs] association ranges of the sorted pairs' items (in list order)
    uint2 *d_srange;        // [cap_tiles] super-tile [start, end) in the sorted pairs, followed by [cap_tiles] u32 counts
    uint32_t *d_last;       // [cap_pixels] list entries walked per ray
    float *d_Tfin;          // [cap_pixels] final transmittance (for the backward)
    uint2 *d_evals;         // [cap_pixels] ray-Gaussian evaluations executed / contributors applied
    geer::GradAcc *d_gacc;  // [cap_cams * cap_gauss]
    uint2 *d_hit;           // [cap_tiles][hit_entries] per tile-list entry, one byte per warp of the tile:
                            // nonzero when one of the warp's rays hit the entry in the forward (or null)
    uint32_t *d_idrec;      // [cap_tiles][hit_entries] the item id of each of those tile-list entries
    int64_t hit_entries;    // list entries recorded per tile (0: none)
    uint8_t *d_tile_mask;   // [cap_tiles] tiles the forward renders (geer_set_tile_mask; null: no mask room)
    int tile_mask_on;       // the mask is in effect for the current camera set

    // state of the last calls
    int64_t n_gauss;
    int32_t sh_degree;
    int stage;               // 0 none, 1 preprocessed, 2 sorted, 3 rendered, 4 render-stage gradients
    bool trains;             // the last render stage was a backward: the preprocess and the binning prepare the next
    bool acc_zero;           // the last preprocess zeroed the items' accumulators; no backward since
    bool queue_ready;        // the last bin_sort reset the fused render's unit queue; not used since
    int sorted_buf;          // which ping-pong buffer holds the sorted super-tile pairs
    int sort_grid;           // grid of the radix kernels (grid-stride over sort tiles)
    int num_sms;

    // pinned staging for asynchronous camera uploads
    void *h_stage;
    size_t stage_bytes;

    // optional stage timing: a ring of (begin, end) events per stage
    int timing;
    uint32_t timing_mask;    // the stages that record events (bit s = stage s)
    cudaEvent_t ev[geer::kStageCount][geer::kTimingRing][2];
    int ev_count[geer::kStageCount];
};

namespace geer {

// Launchers (defined in the .cu files).
cudaError_t launch_preprocess(const geer_workspace *ws, const geer_gaussians *g, cudaStream_t s);
cudaError_t launch_bin_front(const geer_workspace *ws, cudaStream_t s);
cudaError_t launch_depth_sort(geer_workspace *ws, cudaStream_t s);
cudaError_t launch_count_pairs(const geer_workspace *ws, cudaStream_t s);
cudaError_t launch_duplicate(const geer_workspace *ws, cudaStream_t s);
cudaError_t launch_bwd_order(const geer_workspace *ws, cudaStream_t s);
cudaError_t launch_expand_tiles(const geer_workspace *ws, uint32_t *counts_or_offsets, uint32_t *lists, cudaStream_t s);
cudaError_t launch_tile_sort(geer_workspace *ws, cudaStream_t s);
cudaError_t launch_render_fwd(const geer_workspace *ws, float *rgb, float *T_final, cudaStream_t s);
cudaError_t launch_render_bwd(const geer_workspace *ws, const float *dL_drgb, cudaStream_t s);
cudaError_t launch_render_train(const geer_workspace *ws, const float *target, float *rgb, float *T_final,
                                float *dL_drgb, float *loss, cudaStream_t s);
cudaError_t launch_preprocess_bwd(const geer_workspace *ws, const geer_gaussians *g, float *d_mean, float *d_scale,
                                  float *d_quat, float *d_opacity, float *d_sh, int accumulate, cudaStream_t s);
cudaError_t launch_l1_grad(const float *pred, const float *target, int64_t m, float *grad, float *loss, int num_sms,
                           cudaStream_t s);
cudaError_t launch_remap_to_native(const float *beap, const geer_camera *cam, double fov_y, double focal,
                                   double phi_max, const float *fill, float *out, uint8_t *regions, cudaStream_t s);
cudaError_t launch_native_to_beap(const float *native, const geer_camera *cam, double fov_y, double focal,
                                  double phi_max, float *beap, uint8_t *valid, cudaStream_t s);
cudaError_t launch_adam_gaussians(const geer_adam *hp, int64_t n, int32_t sh_degree, float *mean, float *log_scale,
                                  float *quat, float *logit_opacity, float *sh, const float *d_mean,
                                  const float *d_scale, const float *d_quat, const float *d_opacity,
                                  const float *d_sh, float *m, float *v, float *scale, float *opacity,
                                  cudaStream_t s);
size_t densify_scratch_bytes(int64_t n);
cudaError_t launch_densify_accum(const geer_workspace *ws, const float *d_mean, float *accum, float *denom,
                                 cudaStream_t s);
cudaError_t launch_densify_plan(const geer_densify_params *hp, int64_t n, const float *log_scale, const float *logit,
                                const float *accum, const float *denom, void *scratch, unsigned long long *total,
                                cudaStream_t s);
cudaError_t launch_densify_apply(int64_t n, int32_t sh_degree, const float *mean, const float *log_scale,
                                 const float *quat, const float *logit, const float *sh, const float *m,
                                 const float *v, const float *z, void *scratch, int64_t n_out, float *o_mean,
                                 float *o_log_scale, float *o_quat, float *o_logit, float *o_sh, float *o_m,
                                 float *o_v, float *o_scale, float *o_opacity, cudaStream_t s);
cudaError_t launch_opacity_reset(int64_t n, float value, float *logit, float *m_op, float *v_op, float *opacity,
                                 cudaStream_t s);
cudaError_t launch_image_metrics(const float *pred, const float *gt, int width, int height, const uint8_t *regions,
                                 int n_regions, double *acc, cudaStream_t s);
int sort_blocks_per_sm();
int render_bwd_blocks_per_sm(int alpha_model);
int render_train_blocks_per_sm(int alpha_model);

inline int64_t prep_blocks(int64_t n) { return (n + kPrepThreads - 1) / kPrepThreads; }

// The buffer (0 or 1) holding the depth-sorted items after the depth sort: the
// passes whose digit was the same for every key are skipped on the device, so
// the ping-pong parity is known there only (misc as left by the last pass).
__device__ __forceinline__ int depth_sorted_buf(const uint32_t *misc) {
    return misc[kMiscSortSame] ? (int)misc[kMiscSortCur] : 1 - (int)misc[kMiscSortCur];
}

}  // namespace geer
