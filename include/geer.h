/*
 * geer.h -- C ABI of the GB300 (sm_103a) exact ray-Gaussian renderer.
 *
 * The library implements the data-parallel hot path of 3DGEER (arXiv
 * 2505.24053): per-Gaussian preprocessing with Particle Bounding Frustum (PBF)
 * association to the tiles of a Bipolar Equiangular Projection (BEAP) grid,
 * duplication of (tile, depth) keys, a radix sort, per-tile ranges, the
 * closed-form ray integral with front-to-back compositing, and its backward
 * pass (Algorithm 1 "GPU Software Asso. & Render"; App. C gradient cookbook).
 *
 * Conventions for every entry point:
 *  - All pointers to Gaussian data, images and gradients are DEVICE pointers
 *    (cudaMalloc'd or equivalent) owned by the caller. Camera and parameter
 *    structs are HOST pointers, read during the call only.
 *  - `stream` is a cudaStream_t passed as void*. Every call that takes one is
 *    asynchronous on it, except where stated.
 *  - The library never allocates device memory. All scratch lives in the
 *    caller-supplied workspace (geer_workspace_size / geer_workspace_init).
 *    The host-side workspace handle is malloc'ed by geer_workspace_init and
 *    freed by geer_workspace_destroy.
 *  - Argument errors are detected on the host and returned synchronously; no
 *    work is enqueued in that case. Device-side conditions (pair capacity
 *    exceeded, bounded spin timeout) are recorded in a device status word and
 *    read back by geer_last_device_status.
 *  - One workspace must not be used from two streams concurrently.
 *  - Angles are radians. Cameras use OpenCV axes: x right, y down, z forward.
 */
#ifndef GEER_H
#define GEER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GEER_OK = 0,
    GEER_ERR_ARG = 1,         /* invalid argument (null, negative size, bad camera, ...) */
    GEER_ERR_CAPACITY = 2,    /* more (tile, Gaussian) pairs than the workspace holds */
    GEER_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    GEER_ERR_TIMEOUT = 4,     /* a bounded device wait gave up (geer_render_train_l1's unit queue) */
    GEER_ERR_UNSUPPORTED = 5, /* a valid request the library does not implement */
    GEER_ERR_STATE = 6,       /* call out of order (e.g. render before bin_sort) */
    GEER_ERR_BOUNDS = 7       /* checked build: a device bounds guard skipped an access */
} geer_status;

/* Camera models (App. E): pinhole K (tan theta, tan phi, 1); equidistant
 * fisheye r = f phi; Kannala-Brandt r = f phi (1 + k1 phi^2 + ... + k4 phi^8). */
enum { GEER_PINHOLE = 0, GEER_EQUIDISTANT = 1, GEER_KANNALA_BRANDT = 2 };

/* Gaussians (App. B.1): mean mu, scale s (linear, > 0), rotation quaternion q
 * = (w, x, y, z) of any non-zero norm (normalised internally), opacity sigma
 * (activated, in (0, 1]) and real SH coefficients of degree sh_degree <= 3
 * in the 3DGS convention. Device SoA, FP32, contiguous:
 *   mean [n][3], scale [n][3], quat [n][4], opacity [n], sh [n][(deg+1)^2][3].
 * `sh` must be 16-byte aligned. Gaussians with non-finite values, a
 * non-positive scale or a zero quaternion are culled. */
typedef struct {
    const float *mean, *scale, *quat, *opacity, *sh;
    int64_t n;
    int32_t sh_degree;
    int32_t reserved_;
} geer_gaussians;

/* A camera and its BEAP grid (Sec. 3.3). The BEAP image is width x height
 * rays uniform in (theta, phi): pixel (i, j) has theta = ((i + 1/2)/w - 1/2)
 * fov_x and phi = ((j + 1/2)/h - 1/2) fov_y, direction (App. E)
 * (sin theta cos phi, cos theta sin phi, cos theta cos phi). fov_y <= 0 derives
 * the vertical field of view from the camera model: the angle that the same
 * focal length (the one mapping fov_x/2 to w/2) maps to h/2. 0 < fov_x < 2 pi.
 * R_cw, t_cw: world -> camera (x_c = R_cw x_w + t_cw), row-major. bg: colour
 * composited behind the last contributor. */
typedef struct {
    int32_t model;
    int32_t width, height;
    float fov_x, fov_y;
    float k[4];
    float R_cw[9];
    float t_cw[3];
    float bg[3];
} geer_camera;

/* Tile association methods (Sec. 4, association ablation). GEER_ASSOC_PBF:
 * the particle bounding frustum (Sec. 3.2), exact for the alpha_min contour.
 * GEER_ASSOC_EWA / GEER_ASSOC_UT: the splatting bounds it is compared with, a
 * box in the BEAP screen coordinates (atan2(x, z), atan2(y, z)) of the
 * Gaussian's projection, linearised at the mean (EWA, App. H) or through the
 * 7 sigma points of the unscented transform (alpha 1, beta 2, kappa 0); the
 * box is the 3-sigma square of the larger eigenvalue, or with snugbox != 0
 * the bounding box of the alpha_min ellipse, half-sides
 * sqrt(2 ln(sigma/alpha_min) Sigma_ii). Only the association step changes:
 * every mode culls as PBF does (sigma < alpha_min, camera inside the alpha_min
 * contour), and the splatting modes also cull means with z <= 0.2 (their near
 * plane: the projection divides by z). A tile is associated when its
 * rays' angle spans meet the box (rays beyond 90 degrees through the box
 * turned by pi). Every associated pair is still rendered with the exact ray
 * integral. */
enum { GEER_ASSOC_PBF = 0, GEER_ASSOC_EWA = 1, GEER_ASSOC_UT = 2 };

/* Per-ray alpha models (Sec. 4, local affine approximation vs projective-exact
 * integral). GEER_ALPHA_EXACT: the closed-form ray integral (Sec. 3.1).
 * GEER_ALPHA_SPLAT: the local-affine splat of EWA (App. H) on the BEAP screen,
 * alpha = min(alpha_max, sigma exp(-D^T Sigma_2^-1 D / 2)) with D the ray's
 * screen angles (atan2(x, z), atan2(y, z)) minus the mean's (wrapped into
 * [-pi, pi]) and Sigma_2 the EWA covariance of GEER_ASSOC_EWA; Gaussians with
 * z <= 0.2 are culled (the splat divides by z). geer_render_bwd differentiates
 * it (the paper's training-time approximation). It combines with any
 * association method (with PBF, the paper's swap; with EWA, splatting on the
 * BEAP grid). */
enum { GEER_ALPHA_EXACT = 0, GEER_ALPHA_SPLAT = 1 };

/* Rendering parameters. tile_w = tile_h = 16 (BEAP tiles of 16 x 16 rays,
 * each tile a camera sub-frustum, Sec. 3.2). alpha_min: contributions below it
 * are skipped; alpha_max: alpha clamp; T_min: a ray stops before the
 * contributor that would take its transmittance below it (3DGS conventions
 * 1/255, 0.99, 1e-4). lambda_pad: relative padding of the per-Gaussian PBF
 * contour lambda^2 = 2 ln(sigma/alpha_min) (default 1e-3). assoc: a
 * GEER_ASSOC_* method (default PBF); snugbox: 0 or 1, used by EWA and UT;
 * alpha_model: GEER_ALPHA_EXACT (default) or GEER_ALPHA_SPLAT. Calls taking
 * params return GEER_ERR_UNSUPPORTED for tiles other than 16 x 16 and
 * GEER_ERR_ARG for alpha_min or alpha_max outside (0, 1), alpha_max <
 * alpha_min, T_min or lambda_pad outside [0, 1), or an unknown assoc,
 * snugbox or alpha_model. */
typedef struct {
    int32_t tile_w, tile_h;
    float alpha_min, T_min, alpha_max, lambda_pad;
    int32_t assoc, snugbox, alpha_model;
} geer_params;

typedef struct geer_workspace geer_workspace;

/* Human-readable name of a status code. Never returns NULL. */
const char *geer_status_string(geer_status s);

/* Fill *p with the defaults (16, 16, 1/255, 1e-4, 0.99, 1e-3, PBF, 0, EXACT). */
geer_status geer_default_params(geer_params *p);

/* Device bytes needed for a workspace rendering `n_cams` cameras (whose sizes
 * are the capacity: later camera sets must not exceed the total pixel and tile
 * counts nor n_cams) of up to n_gauss Gaussians of SH degree <= sh_degree with
 * up to pair_capacity (super-tile, Gaussian) pairs (see geer_bin_sort). Besides
 * the per-pair, per-Gaussian and per-pixel arrays it holds 16 KB per tile: the
 * forward's record of which warps' rays hit each of the tile's first 2048 list
 * entries, from which the backward skips entries a warp never hit.
 * Host-only; synchronous. */
geer_status geer_workspace_size(const geer_camera *cams, int32_t n_cams, int64_t n_gauss, int32_t sh_degree,
                                int64_t pair_capacity, size_t *bytes);

/* Lay a workspace out in caller-owned device memory dev_mem[bytes] (256-byte
 * aligned) and upload the camera tables (synchronous copies). *ws receives a
 * host handle; release it with geer_workspace_destroy (dev_mem stays the
 * caller's). */
geer_status geer_workspace_init(void *dev_mem, size_t bytes, const geer_camera *cams, int32_t n_cams,
                                int64_t n_gauss, int32_t sh_degree, int64_t pair_capacity,
                                const geer_params *params, geer_workspace **ws);

geer_status geer_workspace_destroy(geer_workspace *ws);

/* Replace the camera set (same capacity limits as at init). The tables are
 * staged in pinned host memory owned by the workspace and copied
 * asynchronously on `stream`; the call returns once they are staged. */
geer_status geer_set_cameras(geer_workspace *ws, const geer_camera *cams, int32_t n_cams, void *stream);

/* Like geer_set_cameras, but camera i is placed at a fixed slot: its tiles start
 * at global tile i * slot_tiles and its pixels at i * slot_pixels of the batched
 * image (rgb and T_final then hold n_slots * slot_pixels rows; rows beyond a
 * camera's w*h are left untouched). active[i] == 0 (active may be NULL = all
 * active) leaves slot i empty: no tiles, no pairs, nothing rendered. With a
 * fixed slot layout every launch of a step has the same configuration, so a
 * step can be captured once in a CUDA graph and replayed with new cameras.
 * Each active camera must fit its slot (tiles and pixels). */
geer_status geer_set_camera_slots(geer_workspace *ws, const geer_camera *cams, int32_t n_slots, const uint8_t *active,
                                  int64_t slot_tiles, int64_t slot_pixels, void *stream);

/* Preprocess (Algorithm 1: CullGaussian, ViewspaceGaussians, PBF_Intersect,
 * PCA_Whitening; Sec. 3.2, App. D): for every (camera, Gaussian) the cull
 * decision, the depth key |mu_c|, the PBF tile ranges, the tile count, the
 * whitening W = S^-1 R^T in the camera frame, o_u, and the view-dependent
 * colour. The Gaussians must have n <= the workspace's n_gauss and
 * sh_degree <= its sh_degree, and stay valid until geer_render_fwd (and
 * geer_render_bwd) have run. */
geer_status geer_preprocess(geer_workspace *ws, const geer_gaussians *g, void *stream);

/* DuplicateWithKeys, SortByKeys, IdentifyFrustumRanges (Algorithm 1), with the
 * Gaussians ordered by depth first: the live (camera, Gaussian) items are
 * sorted by depth (ties by item index), then each item emits one (super-tile,
 * item) pair per super-tile (S x S tiles, S in 4..8) holding an associated tile,
 * in depth order, and a stable radix sort by super-tile id yields every
 * super-tile's depth-ordered list. Each tile's list (its super-tile's list
 * filtered by the association test, i.e. its (tile, Gaussian) pairs in depth
 * order) is read by the render kernels as far as their rays walk it. The pair
 * capacity bounds the number of (super-tile, Gaussian) pairs. If pairs_needed is
 * non-NULL the call synchronises `stream` to read that count, writes it to
 * *pairs_needed and returns GEER_ERR_CAPACITY without sorting when it exceeds
 * the capacity. If NULL the call stays asynchronous; an overflow is then
 * recorded in the device status word and the render calls produce nothing. */
geer_status geer_bin_sort(geer_workspace *ws, int64_t *pairs_needed, void *stream);

/* Render every BEAP ray (Algorithm 1 per-CSF loop: Cano_Ray, Dist,
 * BlendInOrder): o_u, d_u = W d, m_u = o_u x d_u, kappa = |m_u|^2/|d_u|^2,
 * alpha = min(alpha_max, sigma exp(-kappa/2)) (Sec. 3.1), composited front to
 * back in depth order (App. B.1 colour equation) with early termination
 * (with params alpha_model GEER_ALPHA_SPLAT, alpha is the EWA splat instead).
 * rgb: device [sum of h*w over cameras][3] f32, cameras in order, row-major.
 * T_final: device [sum h*w] f32 or NULL. Both caller-owned, overwritten. */
geer_status geer_render_fwd(geer_workspace *ws, float *rgb, float *T_final, void *stream);

/* Backward of geer_render_fwd (App. C two-stage RenderCUDA / PreprocessCUDA):
 * given dL/drgb (same layout as rgb), the gradients of the Gaussians used in
 * the last forward go to d_mean [n][3], d_scale [n][3], d_quat [n][4],
 * d_opacity [n], d_sh [n][(deg+1)^2][3] (device, caller-owned, any of them may
 * be NULL to skip; d_sh 16-byte aligned). accumulate != 0: added (+=) to the
 * buffers' contents; accumulate == 0: written, every row (Gaussians without a
 * gradient get zeros), the buffers' previous contents never read. Must follow
 * geer_render_fwd on the same workspace with the same Gaussians (and the
 * same alpha model). */
geer_status geer_render_bwd(geer_workspace *ws, const geer_gaussians *g, const float *dL_drgb, float *d_mean,
                            float *d_scale, float *d_quat, float *d_opacity, float *d_sh, int32_t accumulate,
                            void *stream);

/* The two stages of geer_render_bwd, callable apart (App. C: RenderCUDA, then
 * PreprocessCUDA), so that a caller can combine the render stage's
 * accumulators across processes before the second stage (a step split by tiles
 * over several GPUs sums them with one all-reduce).
 *
 * geer_render_bwd_tiles: the render stage over the tiles rendered by the last
 * geer_render_fwd. It overwrites the workspace's per-(camera, Gaussian)
 * accumulators (16 f32 each: dL/dsigma, dL/drgb, dL/dW through d_u, dL/do_u)
 * with the sums over those tiles' rays. dL_drgb as for geer_render_bwd.
 * GEER_ERR_STATE before a geer_render_fwd. Asynchronous on `stream`. */
geer_status geer_render_bwd_tiles(geer_workspace *ws, const float *dL_drgb, void *stream);

/* A training step's render with the L1 loss in one launch: geer_render_fwd,
 * geer_l1_loss_grad(rgb, target) and geer_render_bwd_tiles fused (App. C's
 * RenderCUDA backward needs, per ray, only its own pixel's dL/drgb, and the L1
 * gradient sign(rgb - target) / n of a pixel only that pixel). Persistent
 * blocks render the tiles in the render order; a finished tile publishes its
 * backward units in a device queue, and once every tile is taken the blocks
 * walk the published units back, waiting (a bounded poll) for the tiles still
 * rendering, so the backward of the finished tiles fills the SMs that the
 * heaviest tiles' walks leave idle.
 * Outputs as the three calls: rgb and T_final (NULL to skip) as
 * geer_render_fwd, dL_drgb [sum h*w][3] f32 the L1 gradient (n = 3 x pixels
 * values), *loss (device f32, NULL to skip) the mean absolute difference
 * (summed in another order than geer_l1_loss_grad: equal to rounding), and the
 * render-stage accumulators of geer_render_bwd_tiles (equal up to the order of
 * FP32 atomic additions); then geer_preprocess_bwd. target: device, rgb's
 * layout. A tile mask (geer_set_tile_mask) applies as in geer_render_fwd: a
 * caller that splits tiles passes a target that is zero on the other parts'
 * pixels. GEER_ERR_STATE before geer_bin_sort; GEER_ERR_UNSUPPORTED on a
 * forward-only workspace. A queue wait that gave up (it cannot happen while
 * the device makes progress) is reported by geer_last_device_status as
 * GEER_ERR_TIMEOUT. Asynchronous on `stream`. */
geer_status geer_render_train_l1(geer_workspace *ws, const float *target, float *rgb, float *T_final,
                                 float *dL_drgb, float *loss, void *stream);

/* Device address and size (in f32) of the accumulators geer_render_bwd_tiles
 * writes: [n_cams * n][16] f32 inside the workspace memory, n the Gaussian
 * count of the last geer_preprocess. The caller may read and overwrite them
 * (e.g. replace them by their sum over processes) before
 * geer_preprocess_bwd. Host-only; *acc and *n_floats must be non-NULL. */
geer_status geer_grad_accumulators(geer_workspace *ws, float **acc, int64_t *n_floats);

/* The preprocess stage: chains the accumulators to the Gaussians' parameters
 * (through o_u = -W mu_c, W = S^-1 R^T with the normalised quaternion, and the
 * SH colour), summing over cameras, into d_mean .. d_sh as geer_render_bwd does
 * (same layouts, NULL to skip, accumulate as there). g: the Gaussians of the
 * last geer_preprocess. GEER_ERR_STATE unless geer_render_bwd_tiles ran after
 * the last geer_render_fwd. Asynchronous on `stream`. */
geer_status geer_preprocess_bwd(geer_workspace *ws, const geer_gaussians *g, float *d_mean, float *d_scale,
                                float *d_quat, float *d_opacity, float *d_sh, int32_t accumulate, void *stream);

/* Splitting a camera set's tiles over n_parts processes (one GPU each): the
 * (camera, tile) key space is partitioned, every process preprocesses and
 * bins all Gaussians, renders only its own tiles (geer_set_tile_mask), and
 * the render-stage accumulators are summed across processes before
 * geer_preprocess_bwd, which then gives every process the full gradient.
 *
 * geer_tile_owners: owner[t] in [0, n_parts) for every tile of the camera set
 * in the tile order of geer_set_cameras (cameras in order, each one's tiles row
 * by row, ceil(w/16) x ceil(h/16)): tile (cx, cy) of camera c belongs to part
 * (cx + cy + c) mod n_parts, diagonal stripes that give every part a share of
 * every region of every image. owner: HOST int32 [total tiles]. Host-only (no
 * device work); GEER_ERR_ARG for n_parts < 1 or an invalid camera. */
geer_status geer_tile_owners(const geer_camera *cams, int32_t n_cams, int32_t n_parts, int32_t *owner);

/* Restrict geer_render_fwd to the tiles t with mask[t] != 0 (HOST u8 [n_tiles],
 * n_tiles the current camera set's tile count; NULL: all tiles). Rays of the
 * other tiles get rgb = 0 and T_final = 0 and are skipped by the backward, so
 * the renders of a partition of the tiles sum to the full render and their
 * accumulators to the full accumulators. The mask stays in effect until it
 * is replaced or the camera set changes (geer_set_cameras and
 * geer_set_camera_slots clear it). Synchronous (copies the mask and
 * synchronises `stream`). */
geer_status geer_set_tile_mask(geer_workspace *ws, const uint8_t *mask, int64_t n_tiles, void *stream);

/* Synchronise `stream`, then read and clear the device status word: GEER_OK,
 * GEER_ERR_CAPACITY (pairs exceeded capacity) or, in the checked build,
 * GEER_ERR_BOUNDS (a bounds guard skipped an access; geer_bounds_violation
 * tells where). *pairs (may be NULL) receives the last pair count. */
geer_status geer_last_device_status(geer_workspace *ws, int64_t *pairs, void *stream);

/* The checked build. Every kernel index that comes from an earlier kernel's
 * output (a tile from the render order, a super-tile list range, an item id of
 * a sorted pair, a super-tile id of an emitted pair) is guarded: when it lies
 * outside its array the access is skipped (an unrendered tile, an empty list,
 * a record no ray hits, an uncounted pair) instead of reading or writing out
 * of bounds. libgeer.so keeps the guards silent; libgeer_checked.so (the same
 * sources built with GEER_CHECKED=1, the stand-in for a memory checker) also
 * records the first failing guard: its site and index, with the status bit that
 * geer_last_device_status reports as GEER_ERR_BOUNDS.
 *
 * geer_checked_build: 1 in libgeer_checked.so, 0 in libgeer.so. */
int32_t geer_checked_build(void);

/* Synchronise `stream`, then read the first recorded bounds violation: *site
 * (0: none; 1 forward tile, 2 forward list range, 3 forward item, 4 backward
 * tile, 5 backward list range, 6 backward item, 7 duplicated pair's super-tile)
 * and *index (the offending value). A violation read is cleared, with its
 * status bit. Always GEER_OK with *site = 0 in libgeer.so. */
geer_status geer_bounds_violation(geer_workspace *ws, uint32_t *site, int64_t *index, void *stream);

/* Inspection (synchronous): after geer_bin_sort, replace the order in which
 * the forward's blocks take the tiles (order: HOST u32 [n], n the camera set's
 * tile count). Every permutation of the tiles renders the same image; the
 * order only schedules. GEER_ERR_ARG for an entry beyond the current tiles
 * (libgeer.so) or beyond the workspace's tile capacity (libgeer_checked.so,
 * which lets the tiles in between through to exercise its device guards). */
geer_status geer_debug_set_render_order(geer_workspace *ws, const uint32_t *order, int64_t n, void *stream);

/* Debug/inspection (synchronous): copy the per-(camera, Gaussian) preprocess
 * results into HOST buffers, each sized n_cams * n (any may be NULL):
 * ranges [.][8] u16 {X0lo, X0hi, X1lo, X1hi, Y0lo, Y0hi, Y1lo, Y1hi}
 * (X*: tile columns for rows with cos(phi) >= 0 / <= 0, Y*: tile rows for
 * columns with cos(theta) >= 0 / <= 0), tile counts u32, depth keys u32,
 * cull flags u8. */
geer_status geer_debug_preprocess(geer_workspace *ws, uint16_t *ranges, uint32_t *counts, uint32_t *keys,
                                  uint8_t *cull, void *stream);

/* Debug/inspection (synchronous): build every tile's full list and copy up to
 * cap of the (tile, Gaussian) pairs, ordered by tile then depth (keys u64 =
 * tile << 32 | depth bits, values u32 = camera * n + gaussian), into HOST
 * buffers; *count receives the number P of (tile, Gaussian) associations.
 * Returns GEER_ERR_CUDA if the lists do not hold exactly P pairs and
 * GEER_ERR_CAPACITY if P exceeds the workspace's pair capacity. Leaves the
 * render state intact. */
geer_status geer_debug_pairs(geer_workspace *ws, uint64_t *keys, uint32_t *values, int64_t cap, int64_t *count,
                             void *stream);

/* L1 photometric loss of a render against a target image (the training loss of
 * Algorithm 2 instantiated as mean |C - target|): writes dL/drgb =
 * sign(rgb - target) / n_values and, if loss is non-NULL, the loss (device
 * float). rgb, target, dL_drgb: device [n_values] f32. */
geer_status geer_l1_loss_grad(const float *rgb, const float *target, int64_t n_values, float *dL_drgb, float *loss,
                              void *stream);

/* Debug/inspection (synchronous), after geer_render_fwd: per ray (HOST buffers
 * of n_pixels, any may be NULL) the ray-Gaussian evaluations executed and the
 * contributors composited (evals [.][2] u32) and the list entries its backward
 * walks (last u32); per tile (n_tiles) the forward's walk record (walk [.][2]
 * u32: super-tile list position just past the tile's last contributor, and the
 * number of tile-list entries before it). */
geer_status geer_debug_render_state(geer_workspace *ws, uint32_t *evals, uint32_t *last, uint32_t *walk,
                                    void *stream);

/* Measurement (synchronous): after geer_bin_sort, the number of (tile,
 * Gaussian) associations P, of (super-tile, Gaussian) pairs sorted, the radix
 * passes of that sort and the live (camera, Gaussian) items (associated with at
 * least one tile); any pointer may be NULL. */
geer_status geer_pair_counts(geer_workspace *ws, int64_t *tile_pairs, int64_t *super_pairs, int32_t *sort_passes,
                             int64_t *live_items, void *stream);

/* Measurement (synchronous): after geer_bin_sort, the length of every tile's
 * list, i.e. its number of (tile, Gaussian) associations (counts: HOST u32
 * [n_tiles], tiles of the current camera set in order). Leaves the render state
 * intact. GEER_ERR_CAPACITY after a pair-capacity overflow. */
geer_status geer_tile_counts(geer_workspace *ws, uint32_t *counts, void *stream);

/* Measurement (synchronous): totals over all rays of the last geer_render_fwd
 * of the ray-Gaussian evaluations executed (list entries walked up to early
 * termination), of the contributors composited, and (walked_back, may be NULL)
 * of the list entries the backward walks (up to each ray's last contributor). */
geer_status geer_render_counts(geer_workspace *ws, uint64_t *evaluated, uint64_t *applied, uint64_t *walked_back,
                               void *stream);

/* Stage timing. When enabled, the calls above record a pair of CUDA events on
 * their stream around each stage's kernels (stages: see geer_stage_name:
 * preprocess, bin_front, depth_sort, count_pairs, duplicate, tile_sort,
 * render_fwd, render_bwd, preprocess_bwd), keeping the most recent 64 per
 * stage. geer_stage_times synchronises `stream` and writes the mean duration in
 * ms of the recorded occurrences of each stage into ms[0..9] (n >= 10) and
 * their number into counts (may be NULL). Do not enable it while capturing a
 * CUDA graph. */
geer_status geer_enable_timing(geer_workspace *ws, int32_t enable);
/* As geer_enable_timing, recording events for the stages in `mask` only (bit s
 * = stage s, 0: timing off). An event between two kernels keeps the second
 * from launching while the first runs (programmatic dependent launch), so a
 * measurement of whole steps times the long stages only. */
geer_status geer_enable_stage_timing(geer_workspace *ws, uint32_t mask);
geer_status geer_stage_times(geer_workspace *ws, float *ms, int32_t n, int32_t *counts, void *stream);
const char *geer_stage_name(int32_t stage);

/* Resample a BEAP image of camera `cam` (beap_rgb: device [h][w][3] f32, the
 * camera's rows of a geer_render_fwd output) into the camera's native image
 * (native_rgb: device [h][w][3] f32) by bilinear inverse interpolation (App. E).
 * Native intrinsics: square pixels, principal point at the image centre, focal
 * length mapping fov_x/2 to w/2; pinhole x = f tan(theta), equidistant r = f phi,
 * Kannala-Brandt r = f phi_d(phi). Native pixels whose ray falls outside the BEAP
 * grid, or where the distortion cannot be inverted, get fill_rgb (host [3],
 * NULL = black). Asynchronous on `stream`. */
geer_status geer_remap_to_native(const float *beap_rgb, const geer_camera *cam, const float *fill_rgb,
                                 float *native_rgb, void *stream);

/* The supervision of a BEAP render from a native camera image (BEAP ray
 * sampling with ground-truth interpolation, Algorithm 2): each BEAP pixel's ray
 * is projected into the native image (the model and intrinsics of
 * geer_remap_to_native) and the native image (native_rgb: device [h][w][3] f32)
 * is interpolated bilinearly there into beap_rgb (device [h][w][3] f32,
 * overwritten). valid (device [h][w] u8, may be NULL) gets 1, or 0 (and black)
 * where the ray's point is not within half a pixel of the native image or has
 * no projection. Asynchronous on `stream`. */
geer_status geer_native_to_beap(const float *native_rgb, const geer_camera *cam, float *beap_rgb, uint8_t *valid,
                                void *stream);

/* Adam (Kingma and Ba) over the 3DGS parameterisation: learning rates per
 * parameter group (SH degree 0 and the higher degrees apart), beta1, beta2, eps,
 * and the 1-based step count of the bias correction. */
typedef struct {
    float lr_mean, lr_scale, lr_quat, lr_opacity, lr_sh_dc, lr_sh_rest;
    float beta1, beta2, eps;
    int32_t step;
} geer_adam;

/* One Adam step of n Gaussians (the optimiser of Algorithm 2 as 3DGS runs it).
 * Raw parameters (device, caller-owned, updated in place): mean [n][3],
 * log_scale [n][3], quat [n][4], logit_opacity [n], sh [n][(deg+1)^2][3].
 * d_*: the gradients geer_render_bwd produced, with respect to the activated
 * parameters (scale = exp(log_scale), opacity = sigmoid(logit)); the chain rule
 * is applied here. m, v: device [n * (11 + 3 (deg+1)^2)] f32 moments each,
 * zero before the first step, laid out as [mean | log_scale | quat | logit | sh]
 * blocks in those shapes. scale [n][3] and opacity [n] (device, may be NULL)
 * receive the activated values of the updated parameters. Asynchronous on
 * `stream`. */
geer_status geer_adam_step(const geer_adam *hp, int64_t n, int32_t sh_degree, float *mean, float *log_scale,
                           float *quat, float *logit_opacity, float *sh, const float *d_mean, const float *d_scale,
                           const float *d_quat, const float *d_opacity, const float *d_sh, float *m, float *v,
                           float *scale, float *opacity, void *stream);

/* Adaptive density control (Algorithm 2's refinement iterations, the 3DGS
 * rules driven by the gradient of the view-space mean3D instead of the
 * screen-space mean2D, App. G). With g = accum / denom (0 where denom = 0) and
 * s the activated scales, a Gaussian is pruned when sigmoid(logit) <
 * min_opacity or (max_scale > 0) max(s) > max_scale, else densified when
 * g >= grad_threshold: cloned when max(s) <= clone_max_scale (3DGS:
 * percent_dense x scene extent), split otherwise; else kept.
 * Errors of the calls below: GEER_ERR_ARG for invalid thresholds
 * (grad_threshold < 0, clone_max_scale <= 0, min_opacity outside (0, 1),
 * max_scale < 0, any of them not finite), n outside [0, 2^30], a NULL array
 * that the sizes require, a scratch buffer misaligned or too small, n_out
 * outside [0, 2 n]; GEER_ERR_STATE when the workspace has no preprocess yet;
 * GEER_ERR_CUDA when a launch or a copy fails. Nothing is written on an
 * argument error. */
typedef struct {
    float grad_threshold, clone_max_scale, min_opacity, max_scale;
} geer_densify_params;

/* The densification statistics of a step: for every Gaussian that the
 * workspace's last geer_preprocess associated with at least one tile (any of
 * its cameras), accum[i] += |d_mean[i]| and denom[i] += 1 (device [n] f32,
 * caller-owned, zero at the start; n = the workspace's Gaussian count). d_mean:
 * the step's mean gradient (geer_render_bwd); its norm is that of the
 * view-space mean3D gradient, the world-to-camera map being rigid.
 * Asynchronous on `stream`. */
geer_status geer_densify_accumulate(geer_workspace *ws, const float *d_mean, float *accum, float *denom,
                                    void *stream);

/* Device scratch bytes that geer_densify_plan / geer_densify_apply need for n
 * Gaussians. Host-only. */
size_t geer_densify_scratch_bytes(int64_t n);

/* Classify n Gaussians (log_scale [n][3], logit_opacity [n], accum, denom:
 * device) and count the outputs: *n_out (HOST) receives the number of
 * Gaussians after densification (n <= 2^30). The plan stays in scratch (device,
 * caller-owned, geer_densify_scratch_bytes(n) bytes, 16-byte aligned) for
 * geer_densify_apply. Synchronises `stream`. */
geer_status geer_densify_plan(const geer_densify_params *hp, int64_t n, const float *log_scale,
                              const float *logit_opacity, const float *accum, const float *denom, void *scratch,
                              size_t scratch_bytes, int64_t *n_out, void *stream);

/* Write the plan's n_out Gaussians into new arrays (device, caller-owned,
 * disjoint from the inputs): o_mean [n_out][3], o_log_scale [n_out][3], o_quat
 * [n_out][4], o_logit [n_out], o_sh [n_out][(deg+1)^2][3], the Adam moments
 * o_m, o_v in geer_adam_step's layout for n_out, and (may be NULL) the
 * activated o_scale [n_out][3] and o_opacity [n_out]. The outputs follow the
 * originals' order, each original's outputs together: a kept or cloned
 * Gaussian with its moments, a clone's identical copy with zero moments, a
 * split Gaussian's two children with zero moments, child i at
 * mean + R(q) (s * z[i]) with log-scale - ln 1.6 (3DGS: s / (0.8 N), N = 2).
 * z: device [n][2][3] standard normals (drawn by the caller). m, v: the inputs'
 * moments (geer_adam_step layout for n). scratch: the plan's (apply also keeps
 * its output offsets there). Asynchronous on `stream`. */
geer_status geer_densify_apply(int64_t n, int32_t sh_degree, const float *mean, const float *log_scale,
                               const float *quat, const float *logit_opacity, const float *sh, const float *m,
                               const float *v, const float *z, void *scratch, size_t scratch_bytes,
                               int64_t n_out, float *o_mean, float *o_log_scale, float *o_quat, float *o_logit,
                               float *o_sh, float *o_m, float *o_v, float *o_scale, float *o_opacity, void *stream);

/* The 3DGS opacity reset: logit_opacity <- min(logit_opacity, logit(value))
 * (0 < value < 1), and the opacity moments (m, v in geer_adam_step's layout)
 * of the Gaussians it lowered restart at zero; opacity (device [n], may be
 * NULL) receives the activated values. GEER_ERR_ARG for value outside (0, 1),
 * n < 0 or NULL arrays with n > 0. Asynchronous on `stream`. */
geer_status geer_opacity_reset(int64_t n, int32_t sh_degree, float value, float *logit_opacity, float *m, float *v,
                               float *opacity, void *stream);

/* Evaluation regions of the camera's native image (the paper's evaluation of
 * renders reprojected to native fisheye images, appendix on central and
 * peripheral regions): regions (device [h][w] u8, caller-owned, overwritten)
 * gets 0 where the pixel's ray has BEAP angles |theta| <= w / (2f) and
 * |phi| <= h / (2f) (central; f the native focal length of
 * geer_remap_to_native), 1 for the other rays of the BEAP grid (peripheral) and
 * 255 where the pixel has no ray in the grid. Asynchronous on `stream`. */
geer_status geer_native_regions(const geer_camera *cam, uint8_t *regions, void *stream);

/* Image metrics of pred against gt (device [height][width][3] f32, values in
 * [0, 1]) per region: out (HOST [n_regions][5] f64) gets, for each region
 * r < n_regions (1..8), the sum of squared errors over its pixels and the
 * three channels, the sum over its pixels of the SSIM averaged over the
 * channels, its pixel count, its PSNR = 10 log10(1 / MSE) = 10 log10(3 count /
 * sum of squared errors) (+inf for identical images, NaN for an empty region)
 * and its mean SSIM (sum / count; NaN for an empty region). regions: device
 * [height][width] u8 region id per pixel (ids >= n_regions are left out) or
 * NULL (every pixel in region 0). SSIM: 11 x 11 Gaussian window (sigma 1.5,
 * normalised), zero padding, C1 = 0.01^2, C2 = 0.03^2. acc: device scratch of
 * 3 * n_regions f64 (caller-owned). Synchronises `stream`. */
geer_status geer_image_metrics(const float *pred, const float *gt, int32_t width, int32_t height,
                               const uint8_t *regions, int32_t n_regions, double *acc, double *out, void *stream);

/* Render one small camera without allocating anything.
 *
 * For callers that cannot call cudaMalloc or any other allocator at render
 * time: plugins and embedded renderers whose host application owns all device
 * memory (and forbids a library's own allocations), and latency-critical loops
 * that must not synchronise with an allocator or risk an out-of-memory error
 * halfway through a frame. This entry point takes no workspace: every
 * piece of device scratch it needs lives in one fixed array inside the library
 * (28 MiB per GPU that loads the library, held until the process exits), and
 * its host-side state is static too. No paper counterpart: it is a packaging
 * of geer_preprocess + geer_bin_sort + geer_render_fwd for one camera.
 *
 * Limits: n <= 32768 Gaussians, width * height <= 262144 rays,
 * ceil(w/16) * ceil(h/16) <= 2048 tiles, w + h <= 8192, at most 2^19
 * (super-tile, Gaussian) pairs (geer_bin_sort). Larger requests return
 * GEER_ERR_CAPACITY and render nothing.
 * Inputs and outputs as for geer_preprocess / geer_render_fwd (rgb [h*w][3],
 * T_final [h*w] or NULL, device, caller-owned). params may be NULL (defaults).
 *
 * The first call on a device sets that device up (it looks up the address of the
 * scratch array with that device current); make that first call before any
 * stream capture. Every call synchronises `stream` once, to read the pair count
 * back before it sorts.
 * All calls on a device share the one scratch array, which keeps the last
 * call's contents: calls that overlap on the GPU (different streams, or host
 * threads) race and corrupt each other's results; serialise them. */
geer_status geer_render_noalloc(const geer_gaussians *g, const geer_camera *cam, const geer_params *params,
                                float *rgb, float *T_final, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GEER_H */
