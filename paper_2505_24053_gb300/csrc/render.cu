// render.cu -- the per-ray render (Algorithm 1 per-CSF loop: Cano_Ray, Dist,
// BlendInOrder) and its backward (App. C, RenderCUDA stage).
//
// A BEAP tile (a camera sub-frustum) of 16 x 16 rays is processed by 16 / ROWS
// blocks of ROWS x 16 threads, one thread per ray, tiles taken in the order of
// descending pair count (the costliest first). The forward builds the tile's
// depth-ordered list on the fly from its super-tile's list (association test per
// entry), stages the records through shared memory in batches of BATCH and every
// ray walks them front to back with the closed-form ray integral (Sec. 3.1):
//   d_u = W d, m_u = o_u x d_u, kappa = |m_u|^2 / |d_u|^2,
//   alpha = min(alpha_max, sigma exp(-kappa / 2)),
// skipping alpha < alpha_min and Gaussians whose closest approach lies behind
// the camera (o_u . d_u >= 0), stopping before the contributor that would take
// the transmittance below T_min (App. B.1 colour equation, 3DGS thresholds).
#include <algorithm>

#include "geer_internal.cuh"

namespace geer {
namespace {

#ifndef GEER_FWD_ROWS
#define GEER_FWD_ROWS 16
#endif
#ifndef GEER_FWD_BATCH
#define GEER_FWD_BATCH 256
#endif
#ifndef GEER_FWD_UNROLL
#define GEER_FWD_UNROLL 4
#endif
#ifndef GEER_FWD_MINB
#define GEER_FWD_MINB 4  // resident forward blocks per SM the registers must allow
#endif
#ifndef GEER_FWD_BULK
#define GEER_FWD_BULK 0  // 1: the forward stages its records with bulk copies (TMA engine) on an mbarrier
#endif
constexpr uint32_t kBarPolls = 1u << 22;  // bound of a wait on a shared-memory barrier
constexpr int kFwdUnroll = GEER_FWD_UNROLL;
#ifndef GEER_SCAN
#define GEER_SCAN 4
#endif
constexpr int kScan = GEER_SCAN;  // super-list loads in flight per thread in a list fill
#ifndef GEER_BWD_ROWS
#define GEER_BWD_ROWS 16
#endif
#ifndef GEER_BWD_BATCH
#define GEER_BWD_BATCH 256
#endif
#ifndef GEER_BWD_MINB
#define GEER_BWD_MINB 4
#endif
constexpr float kNegHalfLog2e = -0.72134752044448170f;  // -log2(e) / 2

// A load of data written earlier in the same launch (CG: through L2, never a
// stale L1 line) or an ordinary one.
template <bool CG, typename T>
__device__ __forceinline__ T ld_cg(const T *p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

__device__ __forceinline__ int find_cam(const DevCam *cams, int ncams, int t) {
    int c = 0;
    for (int i = 1; i < ncams; ++i)
        if (cams[i].tile_base <= t) c = i;
    return c;
}

// One ray-Gaussian evaluation in the camera frame (Sec. 3.1): d_u = W d,
// m_u = o_u x d_u, kappa = |m_u|^2 / |d_u|^2 and the exponent argument
// log2(sigma) - kappa log2(e) / 2. The forward and the backward share it so that
// both take the same FP32 decisions.
struct Eval {
    float du0, du1, du2, m0, m1, m2, dd, od, kappa, arg;
    bool hit;  // alpha >= alpha_min and the closest approach lies in front of the camera
};

__device__ __forceinline__ Eval evaluate(const float4 &a, const float4 &b, const float4 &c, const float4 &e, float dx,
                                         float dy, float dz, float log2_amin) {
    Eval v;
    v.du0 = a.x * dx + a.y * dy + a.z * dz;
    v.du1 = a.w * dx + b.x * dy + b.y * dz;
    v.du2 = b.z * dx + b.w * dy + c.x * dz;
    v.m0 = c.z * v.du2 - c.w * v.du1;
    v.m1 = c.w * v.du0 - c.y * v.du2;
    v.m2 = c.y * v.du1 - c.z * v.du0;
    const float mm = v.m0 * v.m0 + v.m1 * v.m1 + v.m2 * v.m2;
    v.dd = v.du0 * v.du0 + v.du1 * v.du1 + v.du2 * v.du2;
    v.od = c.y * v.du0 + c.z * v.du1 + c.w * v.du2;
    v.kappa = __fdividef(mm, v.dd);
    v.arg = fmaf(v.kappa, kNegHalfLog2e, e.x);
    v.hit = !(v.arg < log2_amin || v.od >= 0.0f);
    return v;
}

// The splat alpha (GEER_ALPHA_SPLAT, the local-affine model of EWA): the record
// holds the mean's screen angles and the conic (a = theta, phi, A, B; b.x = C);
// (ts, ps) are the ray's screen angles (atan2(x, z), atan2(y, z)). The exponent
// argument is log2(sigma) - D^T conic D log2(e) / 2 with D wrapped into
// [-pi, pi]. Sets arg and hit, and for the backward du0, du1 = D and kappa = q.
__device__ __forceinline__ Eval evaluate_splat(const float4 &a, const float4 &b, const float4 &e, float ts, float ps,
                                               float log2_amin) {
    constexpr float kTwoPi = 6.28318530717959f, kInvTwoPi = 0.159154943091895f;
    float dt = ts - a.x, dp = ps - a.y;
    dt = fmaf(-kTwoPi, rintf(dt * kInvTwoPi), dt);
    dp = fmaf(-kTwoPi, rintf(dp * kInvTwoPi), dp);
    Eval v{};
    const float q = fmaf(a.z * dt, dt, fmaf(2.0f * a.w * dt, dp, b.x * dp * dp));
    v.du0 = dt;
    v.du1 = dp;
    v.kappa = q;
    v.arg = fmaf(q, kNegHalfLog2e, e.x);
    v.hit = !(v.arg < log2_amin);
    return v;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Tile (cx, cy)'s list is its super-tile's depth-ordered list filtered by the
// association test (sranges: the association ranges of the sorted pairs, in
// list order): appends the entries of [pos, end) that pass until s_id holds at
// least `want` entries or the list ends. Each step loads kScan x kThreads
// entries at once (independent loads: a sparse tile's scan is bound by their
// latency) and appends them in sub-steps of kThreads while s_id holds fewer than
// `want`, so that s_id never takes more than want - 1 + kThreads entries; the
// entries of sub-steps it did not take are read again by the next call.
// Block-uniform (pos, end, s_cnt, want are the same in every thread); s_id is
// visible on return. s_wcnt holds kScan x kThreads / 32 counts.
template <int kThreads>
__device__ __forceinline__ void fill_list(const uint32_t *__restrict__ svals, const uint4 *__restrict__ sranges,
                                          const float4 &col, const float4 &row, int cx, int cy, uint32_t &pos,
                                          uint32_t end, int want, uint32_t *s_id, uint32_t *s_pos, int &s_cnt,
                                          uint32_t *s_wcnt) {
    constexpr int kWarps = kThreads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    while (s_cnt < want && pos < end) {
        uint4 raw[kScan];
        uint32_t id[kScan];
#pragma unroll
        for (int r = 0; r < kScan; ++r) {
            const uint32_t i = pos + (uint32_t)(r * kThreads) + threadIdx.x;
            raw[r] = make_uint4(0u, 0u, 0u, 0u);
            id[r] = 0u;
            if (i < end) {
                raw[r] = sranges[i];
                id[r] = svals[i];
            }
        }
        uint32_t bal[kScan];
#pragma unroll
        for (int r = 0; r < kScan; ++r) {
            const uint32_t i = pos + (uint32_t)(r * kThreads) + threadIdx.x;
            bool ok = false;
            if (i < end) {
                int rg[8];
                unpack_ranges(raw[r], rg);
                ok = tile_assoc(col, row, cx, cy, rg);
            }
            bal[r] = __ballot_sync(0xffffffffu, ok);
            if (lane == 0) s_wcnt[r * kWarps + warp] = __popc(bal[r]);
        }
        __syncthreads();
        int cnt = s_cnt;
        uint32_t adv = 0;
#pragma unroll
        for (int r = 0; r < kScan; ++r) {
            if (cnt >= want) break;  // block-uniform: every thread reads the same counts
            uint32_t base = 0, tot = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t c = s_wcnt[r * kWarps + w];
                base += w < warp ? c : 0u;
                tot += c;
            }
            if (bal[r] >> lane & 1u) {
                const int k = cnt + (int)(base + __popc(bal[r] & lanemask_lt()));
                s_id[k] = id[r];
                if (s_pos) s_pos[k] = pos + (uint32_t)(r * kThreads) + threadIdx.x;
            }
            cnt += (int)tot;
            adv += kThreads;
        }
        __syncthreads();
        s_cnt = cnt;
        pos += adv;
    }
}

// Moves the s_cnt - cnt entries not yet consumed (fewer than kThreads) to the front.
template <int kThreads>
__device__ __forceinline__ void shift_list(uint32_t *s_id, uint32_t *s_pos, int cnt, int &s_cnt) {
    const int rem = s_cnt - cnt;
    uint32_t keep = 0, keep_pos = 0;
    if ((int)threadIdx.x < rem) {
        keep = s_id[cnt + threadIdx.x];
        if (s_pos) keep_pos = s_pos[cnt + threadIdx.x];
    }
    __syncthreads();
    if ((int)threadIdx.x < rem) {
        s_id[threadIdx.x] = keep;
        if (s_pos) s_pos[threadIdx.x] = keep_pos;
    }
    s_cnt = rem;
}

// The same filter walking the super-tile list backwards: appends the passing
// entries of [beg, pos) in descending position order (the tile list read back to
// front) until s_id holds at least BATCH entries or pos reaches beg.
template <int kThreads, int BATCH>
__device__ __forceinline__ void fill_list_rev(const uint32_t *__restrict__ svals, const uint4 *__restrict__ sranges,
                                              const float4 &col, const float4 &row, int cx, int cy, uint32_t &pos,
                                              uint32_t beg, uint32_t *s_id, int &s_cnt, uint32_t *s_wcnt) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    while (s_cnt < BATCH && pos > beg) {
        bool ok = false;
        uint32_t id = 0;
        if (pos - beg > threadIdx.x) {
            const uint32_t i = pos - 1 - threadIdx.x;
            int rg[8];
            unpack_ranges(sranges[i], rg);
            ok = tile_assoc(col, row, cx, cy, rg);
            if (ok) id = svals[i];
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, ok);
        if (lane == 0) s_wcnt[warp] = __popc(bal);
        __syncthreads();
        uint32_t base = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            const uint32_t c = s_wcnt[w];
            base += w < warp ? c : 0u;
            tot += c;
        }
        if (ok) s_id[s_cnt + base + __popc(bal & lanemask_lt())] = id;
        __syncthreads();
        s_cnt += (int)tot;
        pos = pos - beg > (uint32_t)kThreads ? pos - kThreads : beg;
    }
}

// Shared-memory working set of one block's walk over its tile's list.
template <int kThreads, int BATCH>
struct WalkSmem {
    float4 rec[BATCH * 4];           // records of the current batch
    uint32_t id[BATCH + kThreads];   // tile-list entries found by the filter (item ids)
    uint32_t pos[BATCH + kThreads];  // their positions in the super-tile list (forward)
    uint2 hit[BATCH];                // per entry: one byte per warp of the tile, nonzero if a ray hit it
    uint32_t wcnt[kScan * kThreads / 32];
    uint32_t maxlast, walkpos;       // the tile's last contributor and its super-list position + 1
    uint32_t nck, next_ck;           // forward: checkpoints recorded, list index of the next one
    uint32_t wacc[kThreads];         // forward: each thread's count of backward steps
    uint32_t ckw[kCkptMax];          // forward: the counts at the checkpoints (work: then the walk's)
    uint32_t ckB[kCkptMax];          // forward: the checkpoints' tile-list indices
    uint32_t work, pend;             // forward: a checkpoint's count of backward steps; its index + 1 while due
    int cam;
    uint64_t bar;                    // forward with bulk staging: the batch's records have landed
};

// Copies item `id`'s 64-byte record into shared memory (4 x 16 B). An id beyond
// the items (a guard failure) stages a record that no ray hits: W = 0 gives
// kappa = 0/0 and o_u . d_u = 0 (the exact integral's test fails), and
// log2(sigma) = -inf fails the splat alpha's.
__device__ __forceinline__ void stage_record(float4 *dst, const Record *__restrict__ rec, uint32_t id, uint64_t items,
                                             uint32_t site, uint32_t *misc) {
    if (in_bounds(id, items, site, misc)) {
        const float4 *src = reinterpret_cast<const float4 *>(rec + id);
#pragma unroll
        for (int k = 0; k < 4; ++k) dst[k] = src[k];
    } else {
        dst[0] = dst[1] = dst[2] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        dst[3] = make_float4(-INFINITY, 0.0f, 0.0f, 0.0f);
    }
}

// A tile's super-tile list range must lie within the sorted pairs; a guard
// failure leaves the tile an empty list.
__device__ __forceinline__ uint2 checked_range(uint2 sr, int64_t cap_pairs, uint32_t site, uint32_t *misc) {
    if (!in_bounds(sr.y, (uint64_t)cap_pairs + 1u, site, misc) || !in_bounds(sr.x, (uint64_t)sr.y + 1u, site, misc))
        return make_uint2(0u, 0u);
    return sr;
}

// Per-ray forward state (n_eval: entries evaluated, set when the walk ends).
struct FwdRay {
    float T, cr, cg, cb;
    uint32_t last, n_eval, n_applied;
    bool done;
};

// Composites list entries [j0, j1) of the staged batch into ray state f, front
// to back (App. B.1 colour equation), until the ray terminates: kFwdUnroll
// entries are evaluated together (independent work for the scheduler on long
// walks), then composited strictly in list order. Entry j of the batch has
// tile-list index n_list + j. hit_b: the ray's warp's hit byte of entry 0 (8
// bytes per entry).
template <bool SPLAT>
__device__ __forceinline__ void walk_entries(const float4 *srec, int j0, int j1, uint32_t n_list, uint8_t *hit_b,
                                             const Params &p, float log2_amin, float dx, float dy, float dz,
                                             FwdRay &f) {
    int j = j0;
    for (; j + kFwdUnroll <= j1 && !f.done; j += kFwdUnroll) {
        Eval v[kFwdUnroll];
        float4 e[kFwdUnroll];
#pragma unroll
        for (int u = 0; u < kFwdUnroll; ++u) {
            const float4 a = srec[(j + u) * 4 + 0];  // W00 W01 W02 W10
            const float4 b = srec[(j + u) * 4 + 1];  // W11 W12 W20 W21
            const float4 c = srec[(j + u) * 4 + 2];  // W22 ou0 ou1 ou2
            e[u] = srec[(j + u) * 4 + 3];            // log2 sigma, r, g, b
            v[u] = SPLAT ? evaluate_splat(a, b, e[u], dx, dy, log2_amin) : evaluate(a, b, c, e[u], dx, dy, dz, log2_amin);
        }
        // after the group's record loads (a byte store may alias them); the
        // same value from every lane of the warp: no race
#pragma unroll
        for (int u = 0; u < kFwdUnroll; ++u)
            if (v[u].hit) hit_b[(j + u) * 8] = 1;
#pragma unroll
        for (int u = 0; u < kFwdUnroll; ++u) {
            if (!v[u].hit) continue;
            const float alpha = fminf(exp2f(v[u].arg), p.alpha_max);
            const float Tn = f.T * (1.0f - alpha);
            if (Tn < p.T_min) {
                f.done = true;
                f.n_eval = n_list + (uint32_t)(j + u) + 1u;  // entries up to this one
                break;
            }
            const float wgt = alpha * f.T;
            f.cr = fmaf(wgt, e[u].y, f.cr);
            f.cg = fmaf(wgt, e[u].z, f.cg);
            f.cb = fmaf(wgt, e[u].w, f.cb);
            f.T = Tn;
            ++f.n_applied;
            f.last = n_list + (uint32_t)(j + u) + 1u;
        }
    }
    for (; j < j1 && !f.done; ++j) {
        const float4 a = srec[j * 4 + 0];
        const float4 b = srec[j * 4 + 1];
        const float4 c = srec[j * 4 + 2];
        const float4 e = srec[j * 4 + 3];
        const Eval v = SPLAT ? evaluate_splat(a, b, e, dx, dy, log2_amin) : evaluate(a, b, c, e, dx, dy, dz, log2_amin);
        if (!v.hit) continue;
        hit_b[j * 8] = 1;
        const float alpha = fminf(exp2f(v.arg), p.alpha_max);
        const float Tn = f.T * (1.0f - alpha);
        if (Tn < p.T_min) {
            f.done = true;
            f.n_eval = n_list + (uint32_t)j + 1u;
            break;
        }
        const float wgt = alpha * f.T;
        f.cr = fmaf(wgt, e.y, f.cr);
        f.cg = fmaf(wgt, e.z, f.cg);
        f.cb = fmaf(wgt, e.w, f.cb);
        f.T = Tn;
        ++f.n_applied;
        f.last = n_list + (uint32_t)j + 1u;
    }
}

// The tile's forward walk (the per-CSF loop of Algorithm 1): its list is the
// super-tile list [sr.x, sr.y) filtered by the association test; batches of
// records are staged in shared memory and each ray composites them front to
// back until it terminates. On return sm.maxlast / sm.walkpos hold the tile's
// walk record: [sr.x, walkpos) of the super-tile list holds tile-list entries
// 0 .. maxlast - 1.
// SPLAT: the splat alpha (GEER_ALPHA_SPLAT) in place of the ray integral;
// (dx, dy) then carry the ray's screen angles.
template <int kThreads, int BATCH, bool SPLAT>
__device__ __forceinline__ void forward_walk(WalkSmem<kThreads, BATCH> &sm, const uint32_t *__restrict__ svals,
                                             const uint4 *__restrict__ sranges, const Record *__restrict__ rec,
                                             const Params &p, const float4 &col, const float4 &row, int cx, int cy,
                                             uint2 sr, float dx, float dy, float dz, uint2 *__restrict__ hit_rec,
                                             uint32_t *__restrict__ id_rec, int64_t hit_entries, uint64_t items,
                                             uint32_t *misc,
                                             float4 *__restrict__ ckpt, uint2 *__restrict__ ckpt_at,
                                             FwdRay &f) {
    const int tid = threadIdx.x;
    uint8_t *const hit_b = reinterpret_cast<uint8_t *>(sm.hit) + (tid >> 5);  // this warp's byte of entry 0
    if (tid == 0) {
        sm.maxlast = 0u;
        sm.walkpos = sr.x;
        sm.nck = 0u;
        sm.next_ck = ckpt ? kCkptFirst : 0xffffffffu;
        sm.work = 0u;
        sm.pend = 0u;
    }
    sm.wacc[tid] = 0u;
    const float log2_amin = log2f(p.alpha_min);
    uint32_t pos = sr.x, n_list = 0;
    int s_cnt = 0, want = BATCH < 64 ? BATCH : 64;
#if GEER_FWD_BULK
    static_assert(BATCH <= kThreads, "one record per thread and batch");
    uint32_t parity = 0;
    if (tid == 0) mbar_init(&sm.bar, kThreads);
#endif
    while (true) {
        if (__syncthreads_count(f.done) == kThreads) break;
        // batches grow 64, 128, ... BATCH: most rays of a dense scene stop early
        fill_list<kThreads>(svals, sranges, col, row, cx, cy, pos, sr.y, want, sm.id, sm.pos, s_cnt, sm.wcnt);
        want = min(2 * want, BATCH);
        const int cnt = min(s_cnt, BATCH);
        if (cnt == 0) break;
#if GEER_FWD_BULK
        // every thread arrives once; thread r < cnt copies record r (64 B) with the
        // TMA engine and announces its bytes
        fence_proxy_async();
        if (tid < cnt) {
            const uint32_t id = sm.id[tid];
            if (in_bounds(id, items, kSiteFwdItem, misc)) {
                mbar_arrive_expect(&sm.bar, (uint32_t)sizeof(Record));
                bulk_g2s(sm.rec + tid * 4, rec + id, (uint32_t)sizeof(Record), &sm.bar);
            } else {
                stage_record(sm.rec + tid * 4, rec, id, items, kSiteFwdItem, misc);
                mbar_arrive_expect(&sm.bar, 0u);
            }
            sm.hit[tid] = make_uint2(0u, 0u);
        } else {
            mbar_arrive_expect(&sm.bar, 0u);
        }
        __syncthreads();
        if (!mbar_wait(&sm.bar, parity, kBarPolls)) atomicOr(misc + kMiscStatus, kStatusTimeout);
        parity ^= 1u;
#else
        for (int r = tid; r < cnt; r += kThreads) {
            stage_record(sm.rec + r * 4, rec, sm.id[r], items, kSiteFwdItem, misc);
            sm.hit[r] = make_uint2(0u, 0u);
        }
        __syncthreads();
#endif
        if (!f.done) walk_entries<SPLAT>(sm.rec, 0, cnt, n_list, hit_b, p, log2_amin, dx, dy, dz, f);
        // a checkpoint for the backward: every ray's (T, C) in front of tile-list
        // entry n_list + cnt and where that entry's search starts in the super-tile list
        // (its state lives in shared memory, advanced by thread 0 after the next
        // barrier: the walk's registers are at their limit)
        const uint32_t nck = sm.nck;
        const bool ck = n_list + (uint32_t)cnt >= sm.next_ck && nck < (uint32_t)kCkptMax;
        if (ck) ckpt[(size_t)nck * kTilePix + tid] = make_float4(f.T, f.cr, f.cg, f.cb);
        // the tile's last contributor so far and where it lies in the super-tile list
        const uint32_t wl = __reduce_max_sync(0xffffffffu, f.last);
        if ((tid & 31) == 0) atomicMax(&sm.maxlast, wl);
        __syncthreads();
        if (ck && tid == 0) {
            ckpt_at[nck] = make_uint2(n_list + (uint32_t)cnt, sm.pos[cnt - 1] + 1u);
            sm.ckB[nck] = n_list + (uint32_t)cnt;
            sm.pend = nck + 1u;
            sm.nck = nck + 1u;
            sm.next_ck = n_list + (uint32_t)cnt + kCkptStride;
        }
        if (tid == 0 && sm.maxlast > n_list) sm.walkpos = sm.pos[sm.maxlast - 1u - n_list] + 1u;
        // the batch's hit bytes, for the backward's skip of entries its warp never hit,
        // and its item ids: the backward reads the tile's list from here without
        // filtering; with checkpoints, the count of the backward's steps (one per
        // entry and warp that hit it), summed over the block at each checkpoint
        uint32_t we = 0;
        for (int r = tid; r < cnt; r += kThreads) {
            const uint2 h = sm.hit[r];
            if (ckpt) we += (uint32_t)(__popc(__vcmpne4(h.x, 0u)) + __popc(__vcmpne4(h.y, 0u))) >> 3;
            if (hit_rec && (int64_t)n_list + r < hit_entries) {
                hit_rec[n_list + r] = h;
                id_rec[n_list + r] = sm.id[r];
            }
        }
        if (ckpt) {  // the thread's count lives in shared memory: the walk's registers are at their limit
            we += sm.wacc[tid];
            sm.wacc[tid] = we;
            if (ck) {
                we = __reduce_add_sync(0xffffffffu, we);
                if ((tid & 31) == 0) atomicAdd(&sm.work, we);
            }
        }
        shift_list<kThreads>(sm.id, sm.pos, cnt, s_cnt);
        // after shift_list's barrier: the checkpoint's count has landed
        if (tid == 0 && sm.pend) {
            sm.ckw[sm.pend - 1u] = sm.work;
            sm.work = 0u;
            sm.pend = 0u;
        }
        n_list += (uint32_t)cnt;
    }
    if (!f.done) f.n_eval = n_list;  // a ray that never terminated evaluated every entry walked
    if (ckpt) {
        const uint32_t we = __reduce_add_sync(0xffffffffu, sm.wacc[tid]);
        if ((tid & 31) == 0) atomicAdd(&sm.work, we);
    }
    __syncthreads();
}

// The block's rays and tile: camera, tile coordinates, ray direction (from the
// per-pixel (sin, cos) tables of the BEAP angles), the tile's association
// table entries and super-tile list. Returns false for a padding tile.
struct TileRay {
    int cx, cy, x, y;
    bool inside;
    float dx, dy, dz;
    float4 col, row;
    uint2 sr;
};

__device__ __forceinline__ bool tile_ray(const DevCam &cam, int t, int row0, const float2 *__restrict__ ptab,
                                         const float4 *__restrict__ ttab, const uint2 *__restrict__ srange, int S,
                                         TileRay &r, int ray) {
    const int lt = t - cam.tile_base;
    if (lt >= cam.tiles_x * cam.tiles_y) return false;  // padding tile of a camera slot
    r.cx = lt % cam.tiles_x;
    r.cy = lt / cam.tiles_x;
    r.x = r.cx * kTile + (ray & (kTile - 1));
    r.y = r.cy * kTile + row0 + (ray / kTile);
    r.inside = r.x < cam.width && r.y < cam.height;
    r.dx = 0.0f;
    r.dy = 0.0f;
    r.dz = 1.0f;
    if (r.inside) {
        const float2 th = ptab[cam.pcol_off + r.x];  // (sin theta, cos theta)
        const float2 ph = ptab[cam.prow_off + r.y];  // (sin phi, cos phi)
        r.dx = th.x * ph.y;
        r.dy = th.y * ph.x;
        r.dz = th.y * ph.y;
    }
    r.col = ttab[cam.tcol_off + r.cx];
    r.row = ttab[cam.trow_off + r.cy];
    r.sr = srange[cam.stile_base + (r.cy / S) * cam.stiles_x + r.cx / S];
    return true;
}

// The L1 loss at one pixel, as geer_l1_loss_grad computes it over the n = 3 x
// pixels values (the mean absolute difference): dL/dC = sign(C - target) / n
// into dL, |C - target| added to acc.
__device__ __forceinline__ void l1_pixel(float c0, float c1, float c2, const float *__restrict__ target,
                                         float *__restrict__ dL, int64_t pix, float inv_m, float &acc) {
    const float c[3] = {c0, c1, c2};
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float d = c[ch] - target[3 * pix + ch];
        dL[3 * pix + ch] = d > 0.0f ? inv_m : (d < 0.0f ? -inv_m : 0.0f);
        acc += fabsf(d);
    }
}

// One tile of the forward (the body of k_render_fwd): the tile's rays walk its
// list and write their colour, transmittance, last contributor and counts, the
// hit and list records, the checkpoints and the backward's unit record. With
// L1, each pixel's L1 gradient against target too (dL; |differences| summed
// into l1acc). Returns the tile's backward unit count in thread 0.
template <int ROWS, int BATCH, bool SPLAT, bool L1>
__device__ __forceinline__ uint32_t fwd_tile(WalkSmem<ROWS * kTile, BATCH> &sm, uint32_t t_id,
                                         const DevCam *__restrict__ cams,
                                         int ncams,
                                         const float2 *__restrict__ ptab,
                                         const float4 *__restrict__ ttab,
                                         int S,
                                         uint2 *__restrict__ tile_walk,
                                         const uint2 *__restrict__ srange,
                                         const uint32_t *__restrict__ svals,
                                         const uint4 *__restrict__ sranges,
                                         const Record *__restrict__ rec,
                                         uint32_t *__restrict__ misc,
                                         Params p,
                                         float *__restrict__ rgb,
                                         float *__restrict__ Tout,
                                         float *__restrict__ Tfin,
                                         uint32_t *__restrict__ last_out,
                                         uint2 *__restrict__ evals,
                                         uint2 *__restrict__ hit,
                                         uint32_t *__restrict__ idrec,
                                         int64_t hit_entries,
                                         const uint8_t *__restrict__ tile_mask,
                                         int64_t ntiles,
                                         uint64_t items,
                                         int64_t cap_pairs,
                                         float4 *__restrict__ ckpt,
                                         uint2 *__restrict__ ckpt_at,
                                         uint32_t *__restrict__ ckpt_cnt,
                                         uint4 *__restrict__ unit_rec,
                                         float4 *__restrict__ Cfin,
                                         const float *__restrict__ target, float *__restrict__ dL, float inv_m,
                                         float &l1acc) {
    constexpr int kThreads = ROWS * kTile;
    if (!in_bounds(t_id, (uint64_t)ntiles, kSiteFwdTile, misc)) return 0u;  // block-uniform
    const int t = (int)t_id;
    if (threadIdx.x == 0) sm.cam = find_cam(cams, ncams, t);
    __syncthreads();
    const DevCam &cam = cams[sm.cam];
    TileRay tr;
    if (!tile_ray(cam, t, 0, ptab, ttab, srange, S, tr, (int)threadIdx.x)) {
        if (threadIdx.x == 0) {
            tile_walk[t] = make_uint2(0u, 0u);
            if (ckpt_cnt) ckpt_cnt[t] = 0u;
            if (unit_rec) unit_rec[t] = make_uint4(0u, 0u, 0u, 0u);
        }
        return 0u;
    }
    tr.sr = checked_range(tr.sr, cap_pairs, kSiteFwdList, misc);
    if (tile_mask && !tile_mask[t]) {  // another part's tile: zeros, nothing for the backward to walk
        if (threadIdx.x == 0) {
            tile_walk[t] = make_uint2(0u, 0u);
            if (ckpt_cnt) ckpt_cnt[t] = 0u;
            if (unit_rec) unit_rec[t] = make_uint4(0u, 0u, 0u, 0u);
        }
        if (tr.inside) {
            const int64_t pix = cam.pix_base + (int64_t)tr.y * cam.width + tr.x;
            rgb[3 * pix + 0] = 0.0f;
            rgb[3 * pix + 1] = 0.0f;
            rgb[3 * pix + 2] = 0.0f;
            if (Tout) Tout[pix] = 0.0f;
            Tfin[pix] = 0.0f;
            last_out[pix] = 0u;
            evals[pix] = make_uint2(0u, 0u);
            if (L1) l1_pixel(0.0f, 0.0f, 0.0f, target, dL, pix, inv_m, l1acc);
        }
        return 0u;
    }
    FwdRay f{1.0f, 0.0f, 0.0f, 0.0f, 0u, 0u, 0u, !tr.inside};
    if (SPLAT) {  // the ray's screen angles
        const float ts = atan2f(tr.dx, tr.dz), ps = atan2f(tr.dy, tr.dz);
        tr.dx = ts;
        tr.dy = ps;
    }
    forward_walk<kThreads, BATCH, SPLAT>(sm, svals, sranges, rec, p, tr.col, tr.row, tr.cx, tr.cy, tr.sr, tr.dx, tr.dy,
                                         tr.dz, hit ? hit + (int64_t)t * hit_entries : nullptr,
                                         hit ? idrec + (int64_t)t * hit_entries : nullptr, hit_entries, items,
                                         misc, ckpt ? ckpt + (size_t)t * kCkptMax * kTilePix : nullptr,
                                         ckpt ? ckpt_at + (size_t)t * kCkptMax : nullptr,
                                         f);
    if (threadIdx.x == 0) {
        tile_walk[t] = make_uint2(sm.walkpos, sm.maxlast);
        if (ckpt_cnt) ckpt_cnt[t] = sm.nck;
    }
    if (tr.inside) {
        const int64_t pix = cam.pix_base + (int64_t)tr.y * cam.width + tr.x;
        const float c0 = fmaf(f.T, cam.bg[0], f.cr), c1 = fmaf(f.T, cam.bg[1], f.cg), c2 = fmaf(f.T, cam.bg[2], f.cb);
        rgb[3 * pix + 0] = c0;
        rgb[3 * pix + 1] = c1;
        rgb[3 * pix + 2] = c2;
        if (Tout) Tout[pix] = f.T;
        Tfin[pix] = f.T;
        last_out[pix] = f.last;
        evals[pix] = make_uint2(f.n_eval, f.n_applied);
        if (Cfin && sm.nck) Cfin[pix] = make_float4(f.cr, f.cg, f.cb, f.T);  // the backward's colour behind
        if (L1) l1_pixel(c0, c1, c2, target, dL, pix, inv_m, l1acc);
    }
    // the backward's units: the checkpoints inside the walk [0, W) split it; thread k
    // writes unit k's schedule bucket (from the steps counted in it), thread
    // kUnitCountByte the number of units
    // (returns the number of units in thread 0)
    uint32_t units = 0;
    if (unit_rec && ((int)threadIdx.x <= kCkptMax || threadIdx.x == kUnitCountByte)) {
        const uint32_t W = sm.maxlast, nk = W > kCkptFirst ? min(sm.nck, (uint32_t)kCkptMax) : 0u;
        uint32_t m = 0;
        for (uint32_t j = 0; j < nk; ++j) m += sm.ckB[j] < W ? 1u : 0u;
        units = W > 0 ? m + 1u : 0u;
        const uint32_t k = threadIdx.x;
        uint8_t *rb = reinterpret_cast<uint8_t *>(unit_rec + t);
        if (k == (uint32_t)kUnitCountByte) {
            rb[k] = (uint8_t)units;
        } else if (k < units) {
            const uint32_t wlo = k == 0 ? 0u : sm.ckw[k - 1], whi = k < m ? sm.ckw[k] : sm.work;
            rb[k] = (uint8_t)order_bucket(max(whi - wlo, 1u));
        }
    }
    return units;
}

template <int ROWS, int BATCH, bool SPLAT>
__global__ void __launch_bounds__(ROWS * kTile, GEER_FWD_MINB) k_render_fwd(const DevCam *__restrict__ cams, int ncams,
                                                            const float2 *__restrict__ ptab,
                                                            const float4 *__restrict__ ttab, int S,
                                                            uint2 *__restrict__ tile_walk,
                                                            const uint32_t *__restrict__ tile_order,
                                                            const uint2 *__restrict__ srange,
                                                            const uint32_t *__restrict__ svals,
                                                            const uint4 *__restrict__ sranges,
                                                            const Record *__restrict__ rec,
                                                            uint32_t *__restrict__ misc, Params p,
                                                            float *__restrict__ rgb,
                                                            float *__restrict__ Tout, float *__restrict__ Tfin,
                                                            uint32_t *__restrict__ last_out,
                                                            uint2 *__restrict__ evals, uint2 *__restrict__ hit,
                                                            uint32_t *__restrict__ idrec, int64_t hit_entries,
                                                            const uint8_t *__restrict__ tile_mask, int64_t ntiles,
                                                            uint64_t items, int64_t cap_pairs,
                                                            float4 *__restrict__ ckpt, uint2 *__restrict__ ckpt_at,
                                                            uint32_t *__restrict__ ckpt_cnt,
                                                            uint4 *__restrict__ unit_rec,
                                                            float4 *__restrict__ Cfin) {
    grid_dep_sync();
    constexpr int kThreads = ROWS * kTile, kParts = kTile / ROWS;
    static_assert(kParts == 1, "one block per tile: the block records the tile's walk");
    __shared__ WalkSmem<kThreads, BATCH> sm;
    if (misc[kMiscStatus] & kStatusCapacity) return;
    float l1acc = 0.0f;
    fwd_tile<ROWS, BATCH, SPLAT, false>(sm, tile_order[blockIdx.x], cams, ncams, ptab, ttab, S, tile_walk, srange, svals, sranges, rec, misc, p, rgb, Tout, Tfin, last_out, evals, hit, idrec, hit_entries, tile_mask, ntiles, items, cap_pairs, ckpt, ckpt_at, ckpt_cnt, unit_rec, Cfin, nullptr, nullptr, 0.0f,
                                        l1acc);
}

// Every tile's full list (no early termination), filtered from its super-tile's
// list exactly as the renders do. With lists == NULL: count[t] = the list's
// length; else lists[off[t] + k] = entry k (off in the same array). For inspection.
__global__ void __launch_bounds__(kTilePix) k_expand_tiles(const DevCam *__restrict__ cams, int ncams,
                                                          const float4 *__restrict__ ttab, int S,
                                                          const uint2 *__restrict__ srange,
                                                          const uint32_t *__restrict__ svals,
                                                          const uint4 *__restrict__ sranges,
                                                          const uint32_t *__restrict__ misc,
                                                          uint32_t *__restrict__ count_or_off,
                                                          uint32_t *__restrict__ lists, int64_t cap) {
    grid_dep_sync();
    __shared__ uint32_t s_id[2 * kTilePix];
    __shared__ uint32_t s_wcnt[kScan * kTilePix / 32];
    __shared__ int s_cam;
    if (misc[kMiscStatus] & kStatusCapacity) return;
    const int t = blockIdx.x, tid = threadIdx.x;
    if (tid == 0) s_cam = find_cam(cams, ncams, t);
    __syncthreads();
    const DevCam &cam = cams[s_cam];
    const int lt = t - cam.tile_base;
    if (lt >= cam.tiles_x * cam.tiles_y) {
        if (!lists && tid == 0) count_or_off[t] = 0u;
        return;
    }
    const int cx = lt % cam.tiles_x, cy = lt / cam.tiles_x;
    const float4 col = ttab[cam.tcol_off + cx], row = ttab[cam.trow_off + cy];
    const uint2 sr = srange[cam.stile_base + (cy / S) * cam.stiles_x + cx / S];
    const int64_t off = lists ? (int64_t)count_or_off[t] : 0;
    uint32_t pos = sr.x, n_list = 0;
    int s_cnt = 0;
    while (true) {
        fill_list<kTilePix>(svals, sranges, col, row, cx, cy, pos, sr.y, kTilePix, s_id, nullptr, s_cnt, s_wcnt);
        const int cnt = min(s_cnt, kTilePix);
        if (cnt == 0) break;
        if (lists)
            for (int r = tid; r < cnt; r += kTilePix)
                if (off + n_list + r < cap) lists[off + n_list + r] = s_id[r];
        __syncthreads();
        shift_list<kTilePix>(s_id, nullptr, cnt, s_cnt);
        n_list += (uint32_t)cnt;
    }
    if (!lists && tid == 0) count_or_off[t] = n_list;
}

// RenderCUDA backward (App. C): reverse traversal of each ray's contributors
// from the last one composited, transmittance recovered as T_i = T_{i+1}/(1-a_i),
// colour behind accumulated back to front. Per (camera, Gaussian) it accumulates
// dL/dsigma, dL/dc, dL/dW through d_u (outer product with the ray direction)
// and dL/do_u (the PreprocessCUDA part chains o_u = -W mu_c).
//
// The 16 values are reduced over the warp (reduce-scatter by shuffles), over the
// block in shared memory, then added to global memory with one set of float4
// atomics per (block, Gaussian). A warp skips list entries beyond the last
// contributor of its rays, and entries that none of its rays hit in the forward
// (the forward's per-warp hit record; the same FP32 evaluation decides both).
// gS: the colour behind the current entry (what lies after it in the list, the
// background included) projected on dL/dC. dL/dalpha needs only this dot product,
// so the ray carries one scalar instead of the three channels.
struct BwdRay {
    float dx, dy, dz, g0, g1, g2, T, gS;
    uint32_t last;
};

// One ray's contribution to the 16 accumulators of the Gaussian in (a, b, c, e)
// (GradAcc order), and the step of the ray's reverse compositing state.
// SPLAT: the splat alpha (r.dx, r.dy the ray's screen angles); its record is
// the centre and conic, and gv[4..8] take dL/d(theta_c, phi_c, A, B, C):
// dq/dtheta_c = -2 (A D0 + B D1), dq/dphi_c = -2 (B D0 + C D1),
// dq/dA = D0^2, dq/dB = 2 D0 D1, dq/dC = D1^2.
template <bool SPLAT>
__device__ __forceinline__ void ray_gradient(BwdRay &r, const float4 &a, const float4 &b, const float4 &c,
                                             const float4 &e, float log2_amin, float alpha_max, float gv[16],
                                             bool &contrib) {
    const Eval v = SPLAT ? evaluate_splat(a, b, e, r.dx, r.dy, log2_amin)
                         : evaluate(a, b, c, e, r.dx, r.dy, r.dz, log2_amin);
    if (!v.hit) return;
    contrib = true;
    const float ae = exp2f(v.arg);
    const float alpha = fminf(ae, alpha_max);
    // approximate reciprocal (within 2 ulp): the correctly rounded one costs more
    // than the rest of this step's transmittance update
    const float inv_om = __fdividef(1.0f, 1.0f - alpha);
    const float Ti = r.T * inv_om;  // transmittance in front of this Gaussian
    const float wgt = Ti * alpha;
    gv[1] = fmaf(r.g0, wgt, gv[1]);
    gv[2] = fmaf(r.g1, wgt, gv[2]);
    gv[3] = fmaf(r.g2, wgt, gv[3]);
    // dL/dalpha = sum_ch g_ch (T_i c_ch - S_ch / (1 - alpha)) = T_i (g . c) - (g . S) / (1 - alpha)
    const float gc = fmaf(r.g0, e.y, fmaf(r.g1, e.z, r.g2 * e.w));
    const float dLda = fmaf(Ti, gc, -r.gS * inv_om);
    r.gS = fmaf(wgt, gc, r.gS);
    r.T = Ti;
    if (ae < alpha_max) {
        gv[0] = fmaf(dLda, exp2f(v.kappa * kNegHalfLog2e), gv[0]);  // dL/dsigma = dL/da e^{-kappa/2}
        const float dLdk = -0.5f * dLda * ae;
        if (SPLAT) {
            const float d0 = v.du0, d1 = v.du1;
            gv[4] = fmaf(-2.0f * dLdk, fmaf(a.z, d0, a.w * d1), gv[4]);
            gv[5] = fmaf(-2.0f * dLdk, fmaf(a.w, d0, b.x * d1), gv[5]);
            gv[6] = fmaf(dLdk, d0 * d0, gv[6]);
            gv[7] = fmaf(2.0f * dLdk, d0 * d1, gv[7]);
            gv[8] = fmaf(dLdk, d1 * d1, gv[8]);
            return;
        }
        // with g_m = 2 m_u / |d_u|^2 (dkappa/dm_u), scaled by dL/dkappa:
        //   dL/dd_u = dL/dkappa (-(2 kappa / |d_u|^2) d_u + g_m x o_u),  dL/do_u = dL/dkappa (d_u x g_m)
        const float h = 2.0f * dLdk * __fdividef(1.0f, v.dd);
        const float gm0 = h * v.m0, gm1 = h * v.m1, gm2 = h * v.m2;
        const float sk = -h * v.kappa;
        const float r0 = sk * v.du0 + (gm1 * c.w - gm2 * c.z);
        const float r1 = sk * v.du1 + (gm2 * c.y - gm0 * c.w);
        const float r2 = sk * v.du2 + (gm0 * c.z - gm1 * c.y);
        gv[13] += v.du1 * gm2 - v.du2 * gm1;
        gv[14] += v.du2 * gm0 - v.du0 * gm2;
        gv[15] += v.du0 * gm1 - v.du1 * gm0;
        gv[4] = fmaf(r0, r.dx, gv[4]); gv[5] = fmaf(r0, r.dy, gv[5]); gv[6] = fmaf(r0, r.dz, gv[6]);
        gv[7] = fmaf(r1, r.dx, gv[7]); gv[8] = fmaf(r1, r.dy, gv[8]); gv[9] = fmaf(r1, r.dz, gv[9]);
        gv[10] = fmaf(r2, r.dx, gv[10]); gv[11] = fmaf(r2, r.dy, gv[11]); gv[12] = fmaf(r2, r.dz, gv[12]);
    }
}

// A backward unit's walk: tile-list entries [lo, walk.y) read back to front,
// filtered as in the forward from super-list positions [plo, walk.x) (walk.x:
// just past entry walk.y - 1; plo: where entry lo's search starts).
template <int kThreads, int BATCH, bool SPLAT, bool CG>
__device__ __forceinline__ void backward_walk(WalkSmem<kThreads, BATCH> &sm, float (*s_acc)[17],
                                              const uint32_t *__restrict__ svals,
                                              const uint4 *__restrict__ sranges, const Record *__restrict__ rec,
                                              const Params &p, const float4 &col, const float4 &row, int cx, int cy,
                                              uint32_t plo, uint32_t lo, uint2 walk, uint32_t warp_last,
                                              uint32_t block_last,
                                              const uint2 *__restrict__ hit_rec,
                                              const uint32_t *__restrict__ id_rec, int64_t hit_entries, int fwarp,
                                              BwdRay &ray, GradAcc *__restrict__ gacc, uint64_t items,
                                              uint32_t *misc) {
    const int tid = threadIdx.x, lane = tid & 31;
    const float log2_amin = log2f(p.alpha_min);
    // entry r of a batch has list index top - 1 - r
    uint32_t pos = walk.x, top = walk.y;
    int s_cnt = 0;
    while (top > lo) {
        // within the forward's record the list is read directly, beyond it filtered again
        const bool direct = id_rec && (int64_t)top <= hit_entries;
        int cnt;
        if (direct) {
            cnt = (int)min((uint32_t)BATCH, top - lo);
        } else {
            fill_list_rev<kThreads, BATCH>(svals, sranges, col, row, cx, cy, pos, plo, sm.id, s_cnt, sm.wcnt);
            cnt = min(s_cnt, BATCH);
            if (cnt == 0) break;
        }
        // entries at or beyond the block's last contributor are not walked
        const int skip = top > block_last ? (int)min((uint32_t)cnt, top - block_last) : 0;
        for (int r = skip + tid; r < cnt; r += kThreads) {
            const uint32_t j = top - 1u - (uint32_t)r;
            uint32_t id;
            if (direct) {
                id = ld_cg<CG>(id_rec + j);
                sm.id[r] = id;
            } else {
                id = sm.id[r];
            }
            // beyond the recorded entries every warp evaluates
            const uint2 h = hit_rec && (int64_t)j < hit_entries ? ld_cg<CG>(hit_rec + j) : make_uint2(~0u, ~0u);
            // an entry no warp hit is never read: its record is not staged
            if (h.x | h.y) stage_record(sm.rec + r * 4, rec, id, items, kSiteBwdItem, misc);
            // transposed to warp-major order: warp w's flags of the batch are contiguous
            uint8_t *hw = reinterpret_cast<uint8_t *>(sm.hit);
#pragma unroll
            for (int w = 0; w < kTileWarps; ++w)
                hw[w * BATCH + r] = (uint8_t)((w < 4 ? h.x : h.y) >> (8 * (w & 3)));
        }
        for (int i = skip * 17 + tid; i < cnt * 17; i += kThreads) (&s_acc[0][0])[i] = 0.0f;
        __syncthreads();
        // this warp's first entry below its rays' last contributor (warp-uniform)
        const int r0 = max(skip, top > warp_last ? (int)min((uint32_t)cnt, top - warp_last) : 0);
        // entries none of this warp's rays hit in the forward are skipped (the same
        // FP32 decisions here would not hit either): 32 entries' flags per ballot
        const uint8_t *hit_w = reinterpret_cast<const uint8_t *>(sm.hit) + fwarp * BATCH;
        for (int base = r0; base < cnt; base += 32) {
            uint32_t todo = __ballot_sync(0xffffffffu, base + lane < cnt && hit_w[base + lane] != 0);
            while (todo) {
                const int r = base + __ffs(todo) - 1;
                todo &= todo - 1u;
                const uint32_t j = top - 1u - (uint32_t)r;
                float gv[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) gv[k] = 0.0f;
                bool contrib = false;
                if (j < ray.last) {
                    const float4 a = sm.rec[r * 4 + 0];
                    const float4 b = sm.rec[r * 4 + 1];
                    const float4 c = sm.rec[r * 4 + 2];
                    const float4 e = sm.rec[r * 4 + 3];
                    ray_gradient<SPLAT>(ray, a, b, c, e, log2_amin, p.alpha_max, gv, contrib);
                }
                if (__any_sync(0xffffffffu, contrib)) {
                    // warp reduce-scatter of the 16 values: lane l ends with the sum of value (l >> 1)
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const bool up = lane & 16;
                        const float send = up ? gv[k] : gv[k + 8];
                        const float keep = up ? gv[k + 8] : gv[k];
                        gv[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const bool up = lane & 8;
                        const float send = up ? gv[k] : gv[k + 4];
                        const float keep = up ? gv[k + 4] : gv[k];
                        gv[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
                    }
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const bool up = lane & 4;
                        const float send = up ? gv[k] : gv[k + 2];
                        const float keep = up ? gv[k + 2] : gv[k];
                        gv[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
                    }
                    {
                        const bool up = lane & 2;
                        const float send = up ? gv[0] : gv[1];
                        const float keep = up ? gv[1] : gv[0];
                        gv[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
                    }
                    gv[0] += __shfl_xor_sync(0xffffffffu, gv[0], 1);
                    if ((lane & 1) == 0) atomicAdd(&s_acc[r][lane >> 1], gv[0]);
                }
            }
        }
        __syncthreads();
        // flush: one Gaussian of the batch per thread, four float4 atomics
        for (int r = skip + tid; r < cnt; r += kThreads) {
            const float *v = s_acc[r];
            bool any = false;
#pragma unroll
            for (int k = 0; k < 16; ++k) any |= v[k] != 0.0f;
            if (any && in_bounds(sm.id[r], items, kSiteBwdItem, misc)) {
                float4 *dst = reinterpret_cast<float4 *>(gacc + sm.id[r]);
                atomicAdd(dst + 0, make_float4(v[0], v[1], v[2], v[3]));
                atomicAdd(dst + 1, make_float4(v[4], v[5], v[6], v[7]));
                atomicAdd(dst + 2, make_float4(v[8], v[9], v[10], v[11]));
                atomicAdd(dst + 3, make_float4(v[12], v[13], v[14], v[15]));
            }
        }
        if (!direct) shift_list<kThreads>(sm.id, nullptr, cnt, s_cnt);
        top -= (uint32_t)cnt;
    }
}

// Backward ray state at the end of the forward: direction, dL/dC, final
// transmittance and last contributor; the colour behind starts with the background.
__device__ __forceinline__ BwdRay bwd_ray(const TileRay &tr, const DevCam &cam, float g0, float g1, float g2, float T,
                                          uint32_t last) {
    BwdRay r;
    r.dx = tr.dx;
    r.dy = tr.dy;
    r.dz = tr.dz;
    r.g0 = g0;
    r.g1 = g1;
    r.g2 = g2;
    r.T = T;
    r.last = last;
    r.gS = T * fmaf(g0, cam.bg[0], fmaf(g1, cam.bg[1], g2 * cam.bg[2]));
    return r;
}

// The backward in units: a tile's walk [0, W) is split at the forward's
// checkpoints B_1 < B_2 < ... below W into the units [0, B_1), [B_1, B_2), ...,
// [B_m, W), each walked back to front by one block. A unit below the top starts
// every ray that walks past it from the checkpoint's state (T in front of
// B_{k+1}, and the colour behind it, C_final - C_checkpoint + T_final bg);
// the top unit starts from the final state. The units are independent, so a
// tile's long walk runs on several SMs at once and its transmittance is
// recovered by division over one unit at most. Persistent blocks take units
// in the order of k_bwd_order (descending length) from a counter.
// One backward unit (the body of k_render_bwd's loop): unit code = tile << 4 | k,
// row part `part` of the tile's rays. CG: read what the forward wrote through
// L2 (the fused kernel reads it in the launch that wrote it).
template <int ROWS, int BATCH, bool SPLAT, bool CG>
__device__ __forceinline__ void bwd_unit(WalkSmem<ROWS * kTile, BATCH> &sm, float (*s_acc)[17], uint32_t code,
                                         int part,
                                         const DevCam *__restrict__ cams,
                                         int ncams,
                                         const float2 *__restrict__ ptab,
                                         const float4 *__restrict__ ttab,
                                         int S,
                                         const uint2 *__restrict__ tile_walk,
                                         const uint2 *__restrict__ srange,
                                         const uint32_t *__restrict__ svals,
                                         const uint4 *__restrict__ sranges,
                                         const Record *__restrict__ rec,
                                         uint32_t *__restrict__ misc,
                                         Params p,
                                         const float *__restrict__ dL_drgb,
                                         const float *__restrict__ Tfin,
                                         const uint32_t *__restrict__ last_in,
                                         const uint2 *__restrict__ hit,
                                         const uint32_t *__restrict__ idrec,
                                         int64_t hit_entries,
                                         GradAcc *__restrict__ gacc,
                                         int64_t ntiles,
                                         uint64_t items,
                                         int64_t cap_pairs,
                                         const float4 *__restrict__ ckpt,
                                         const uint2 *__restrict__ ckpt_at,
                                         const uint32_t *__restrict__ ckpt_cnt,
                                         const float4 *__restrict__ Cfin) {
    constexpr int kThreads = ROWS * kTile;
    const int tray = part * kThreads + (int)threadIdx.x;  // the ray's index in the tile
    const uint32_t t_id = code >> 4, k = code & 15u;
    if (!in_bounds(t_id, (uint64_t)ntiles, kSiteBwdTile, misc)) return;  // block-uniform
    const int t = (int)t_id;
    if (threadIdx.x == 0) sm.cam = find_cam(cams, ncams, t);
    __syncthreads();
    const DevCam &cam = cams[sm.cam];
    TileRay tr;
    if (!tile_ray(cam, t, part * ROWS, ptab, ttab, srange, S, tr, (int)threadIdx.x)) return;
    tr.sr = checked_range(tr.sr, cap_pairs, kSiteBwdList, misc);
    uint2 walk = ld_cg<CG>(tile_walk + t);
    if (!in_bounds(walk.x, (uint64_t)tr.sr.y + 1u, kSiteBwdList, misc)) walk = make_uint2(0u, 0u);
    // the unit: tile-list entries [lo, hi), super-list positions [plo, phi)
    uint32_t lo = 0u, plo = tr.sr.x, hi = walk.y, phi = walk.x;
    bool top = true;
    const uint32_t nck = ckpt_cnt ? min(ld_cg<CG>(ckpt_cnt + t), (uint32_t)kCkptMax) : 0u;
    if (k > 0 && k <= nck) {
        const uint2 a = ld_cg<CG>(ckpt_at + (size_t)t * kCkptMax + k - 1);
        lo = a.x;
        plo = a.y;
    }
    if (k < nck) {
        const uint2 b = ld_cg<CG>(ckpt_at + (size_t)t * kCkptMax + k);
        if (b.x < walk.y) {
            hi = b.x;
            phi = b.y;
            top = false;
        }
    }
    if (!in_bounds(phi, (uint64_t)walk.x + 1u, kSiteBwdList, misc) ||
        !in_bounds(plo, (uint64_t)phi + 1u, kSiteBwdList, misc) || lo >= hi)
        return;
    float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f, T = 1.0f;
    uint32_t last = 0;
    int64_t pix = 0;
    if (tr.inside) {
        pix = cam.pix_base + (int64_t)tr.y * cam.width + tr.x;
        g0 = ld_cg<CG>(dL_drgb + 3 * pix + 0);
        g1 = ld_cg<CG>(dL_drgb + 3 * pix + 1);
        g2 = ld_cg<CG>(dL_drgb + 3 * pix + 2);
        T = ld_cg<CG>(Tfin + pix);
        last = ld_cg<CG>(last_in + pix);
    }
    if (SPLAT) {  // the ray's screen angles
        const float ts = atan2f(tr.dx, tr.dz), ps = atan2f(tr.dy, tr.dz);
        tr.dx = ts;
        tr.dy = ps;
    }
    BwdRay ray = bwd_ray(tr, cam, g0, g1, g2, T, last);
    if (!top && last > hi) {
        // the ray walks past this unit: its state in front of entry hi is the forward's checkpoint
        const float4 c = ld_cg<CG>(ckpt + ((size_t)t * kCkptMax + k) * kTilePix + tray);
        const float4 cf = ld_cg<CG>(Cfin + pix);
        ray.T = c.x;
        const float S0 = fmaf(T, cam.bg[0], cf.x - c.y), S1 = fmaf(T, cam.bg[1], cf.y - c.z),
                    S2 = fmaf(T, cam.bg[2], cf.z - c.w);
        ray.gS = fmaf(g0, S0, fmaf(g1, S1, g2 * S2));
    }
    const uint32_t warp_last = __reduce_max_sync(0xffffffffu, last);
    if ((threadIdx.x & 31) == 0) atomicMax(&sm.maxlast, warp_last);
    __syncthreads();
    const uint32_t block_last = sm.maxlast;
    if (block_last <= lo) return;
    backward_walk<kThreads, BATCH, SPLAT, CG>(sm, s_acc, svals, sranges, rec, p, tr.col, tr.row, tr.cx, tr.cy, plo, lo,
                                          make_uint2(phi, hi), warp_last, block_last,
                                          hit ? hit + (int64_t)t * hit_entries : nullptr,
                                          hit ? idrec + (int64_t)t * hit_entries : nullptr, hit_entries,
                                          tray >> 5, ray, gacc, items, misc);
}

template <int ROWS, int BATCH, bool SPLAT>
__global__ void __launch_bounds__(ROWS * kTile, GEER_BWD_MINB) k_render_bwd(const DevCam *__restrict__ cams, int ncams,
                                                                           const float2 *__restrict__ ptab,
                                                                           const float4 *__restrict__ ttab, int S,
                                                                           const uint2 *__restrict__ tile_walk,
                                                                           const uint32_t *__restrict__ units,
                                                                           const uint2 *__restrict__ srange,
                                                                           const uint32_t *__restrict__ svals,
                                                                           const uint4 *__restrict__ sranges,
                                                                           const Record *__restrict__ rec,
                                                                           uint32_t *__restrict__ misc, Params p,
                                                                           const float *__restrict__ dL_drgb,
                                                                           const float *__restrict__ Tfin,
                                                                           const uint32_t *__restrict__ last_in,
                                                                           const uint2 *__restrict__ hit,
                                                                           const uint32_t *__restrict__ idrec,
                                                                           int64_t hit_entries,
                                                                           GradAcc *__restrict__ gacc, int64_t ntiles,
                                                                           uint64_t items, int64_t cap_pairs,
                                                                           const float4 *__restrict__ ckpt,
                                                                           const uint2 *__restrict__ ckpt_at,
                                                                           const uint32_t *__restrict__ ckpt_cnt,
                                                                           const float4 *__restrict__ Cfin) {
    grid_dep_sync();
    constexpr int kThreads = ROWS * kTile, kParts = kTile / ROWS;
    static_assert(kParts * ROWS == kTile, "a unit's rays are split into kParts blocks of ROWS rows");
    __shared__ WalkSmem<kThreads, BATCH> sm;
    __shared__ float s_acc[BATCH][17];
    __shared__ uint32_t s_unit;
    if (misc[kMiscStatus] & kStatusCapacity) return;
    const uint32_t n_work = misc[kMiscUnits] * (uint32_t)kParts;  // (unit, row part) pairs
    while (true) {
        __syncthreads();  // the previous unit's shared state has been read
        if (threadIdx.x == 0) {
            s_unit = atomicAdd(&misc[kMiscUnitNext], 1u);
            sm.maxlast = 0u;
        }
        __syncthreads();
        const uint32_t w = s_unit;
        if (w >= n_work) break;
        bwd_unit<ROWS, BATCH, SPLAT, false>(sm, s_acc, units[w / kParts], (int)(w % kParts), cams, ncams, ptab, ttab, S, tile_walk, srange, svals, sranges, rec, misc, p, dL_drgb, Tfin, last_in, hit, idrec, hit_entries, gacc, ntiles, items, cap_pairs, ckpt, ckpt_at, ckpt_cnt, Cfin);
    }
}

// Forward, L1 gradient and the render stage of the backward in one persistent
// launch (a training step's render with the per-pixel L1 loss: a tile's
// gradient needs only its own pixels, so its backward can start when its
// forward ends). Blocks take forward tiles in the render order; a finished tile
// publishes its backward units (tile << 4 | k) in a queue. Once every tile is
// taken, blocks take queue slots in order and wait, bounded, for the units of
// tiles still rendering: the backward of the finished tiles fills the SMs the
// heaviest tiles' walks leave idle. A block waits only for work that a running
// block holds. A unit's tile data, written in this launch, is read through L2
// after the slot's acquire.
constexpr uint32_t kQueueEmpty = 0xffffffffu;  // an unpublished queue slot (the host fills the queue with it)
constexpr uint32_t kQueuePolls = 1u << 22;     // bound of a wait for a queue slot (<= ~1 us sleep between polls)

template <int ROWS, int BATCH, bool SPLAT>
__global__ void __launch_bounds__(ROWS * kTile, GEER_BWD_MINB) k_render_train(
    const DevCam *__restrict__ cams, int ncams, const float2 *__restrict__ ptab, const float4 *__restrict__ ttab,
    int S, uint2 *__restrict__ tile_walk, const uint32_t *__restrict__ tile_order, const uint2 *__restrict__ srange,
    const uint32_t *__restrict__ svals, const uint4 *__restrict__ sranges, const Record *__restrict__ rec,
    uint32_t *__restrict__ misc, Params p, float *__restrict__ rgb, float *__restrict__ Tout,
    float *__restrict__ Tfin, uint32_t *__restrict__ last, uint2 *__restrict__ evals, uint2 *__restrict__ hit,
    uint32_t *__restrict__ idrec, int64_t hit_entries, const uint8_t *__restrict__ tile_mask, int64_t ntiles,
    uint64_t items, int64_t cap_pairs, float4 *__restrict__ ckpt, uint2 *__restrict__ ckpt_at,
    uint32_t *__restrict__ ckpt_cnt, uint4 *__restrict__ unit_rec, float4 *__restrict__ Cfin,
    const float *__restrict__ target, float *__restrict__ dL, float inv_m, float *__restrict__ loss,
    GradAcc *__restrict__ gacc, uint32_t *__restrict__ queue, uint32_t queue_cap) {
    grid_dep_sync();
    constexpr int kThreads = ROWS * kTile;
    static_assert(ROWS == kTile, "one block per tile and per unit");
    __shared__ WalkSmem<kThreads, BATCH> sm;
    __shared__ float s_acc[BATCH][17];
    __shared__ uint32_t s_work;
    __shared__ float s_loss;
    if (misc[kMiscStatus] & kStatusCapacity) return;
    float l1acc = 0.0f;
    if (threadIdx.x == 0) s_loss = 0.0f;
    while (true) {  // forward tiles
        __syncthreads();  // the previous tile's shared state has been read
        if (threadIdx.x == 0) s_work = atomicAdd(&misc[kMiscFwdNext], 1u);
        __syncthreads();
        const uint32_t f = s_work;
        if (f >= (uint32_t)ntiles) break;
        const uint32_t t = tile_order[f];
        const uint32_t nu = fwd_tile<ROWS, BATCH, SPLAT, true>(
            sm, t, cams, ncams, ptab, ttab, S, tile_walk, srange, svals, sranges, rec, misc, p, rgb, Tout, Tfin, last,
            evals, hit, idrec, hit_entries, tile_mask, ntiles, items, cap_pairs, ckpt, ckpt_at, ckpt_cnt, unit_rec,
            Cfin, target, dL, inv_m, l1acc);
        __syncthreads();  // every thread's outputs of the tile are written
        if (threadIdx.x == 0) {
            __threadfence();  // release: the tile's outputs before its units
            if (nu) {
                const uint32_t slot = atomicAdd(&misc[kMiscUnitsPub], nu);
                for (uint32_t k = 0; k < nu; ++k)
                    if (slot + k < queue_cap) atomicExch(&queue[slot + k], (t << 4) | k);
            }
            __threadfence();
            atomicAdd(&misc[kMiscFwdDone], 1u);
        }
    }
    // the L1 loss: one atomic per block
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l1acc += __shfl_xor_sync(0xffffffffu, l1acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_loss, l1acc);
    __syncthreads();
    if (threadIdx.x == 0 && loss) atomicAdd(loss, s_loss * inv_m);
    while (true) {  // backward units, in the order they were published
        __syncthreads();  // the previous unit's shared state has been read
        if (threadIdx.x == 0) {
            const uint32_t w = atomicAdd(&misc[kMiscTrainNext], 1u);
            uint32_t code = kQueueEmpty, sleep = 32;
            for (uint32_t it = 0; w < queue_cap; ++it) {
                const uint32_t c = atomicAdd(&queue[w], 0u);
                if (c != kQueueEmpty) {
                    code = c;
                    break;
                }
                // every tile finished and published: slot w beyond the published units stays empty
                if (atomicAdd(&misc[kMiscFwdDone], 0u) >= (uint32_t)ntiles) {
                    __threadfence();  // the final unit count after the last tile's count
                    if (w >= atomicAdd(&misc[kMiscUnitsPub], 0u)) break;
                }
                if (it + 1 == kQueuePolls) {
                    atomicOr(&misc[kMiscStatus], kStatusTimeout);
                    break;
                }
                __nanosleep(sleep);
                sleep = min(sleep * 2u, 1024u);
            }
            __threadfence();  // acquire: the unit's tile data after its slot
            sm.maxlast = 0u;
            s_work = code;
        }
        __syncthreads();
        const uint32_t code = s_work;
        if (code == kQueueEmpty) break;
        bwd_unit<ROWS, BATCH, SPLAT, true>(sm, s_acc, code, 0, cams, ncams, ptab, ttab, S, tile_walk, srange, svals,
                                           sranges, rec, misc, p, dL, Tfin, last, hit, idrec, hit_entries, gacc,
                                           ntiles, items, cap_pairs, ckpt, ckpt_at, ckpt_cnt, Cfin);
    }
}

}  // namespace

cudaError_t launch_render_fwd(const geer_workspace *ws, float *rgb, float *T_final, cudaStream_t s) {
    if (ws->n_tiles == 0) return cudaSuccess;
    constexpr int R = GEER_FWD_ROWS, B = GEER_FWD_BATCH;
    launch_k(ws->params.alpha_model == GEER_ALPHA_EXACT ? k_render_fwd<R, B, false> : k_render_fwd<R, B, true>,
        dim3((unsigned)(ws->n_tiles * (kTile / R))), dim3(R * kTile), 0, s,
        ws->d_cams, ws->n_cams, ws->d_pix_tab, ws->d_tile_tab, ws->super_size, ws->d_tile_walk, ws->d_tile_order,
        ws->d_srange, ws->d_vals[ws->sorted_buf], ws->d_sranges, ws->d_rec, ws->d_misc,
        ws->params, rgb, T_final,
        ws->d_Tfin, ws->d_last, ws->d_evals, ws->d_hit, ws->d_idrec, ws->hit_entries,
        ws->tile_mask_on ? static_cast<const uint8_t *>(ws->d_tile_mask) : nullptr, ws->n_tiles,
        (uint64_t)ws->n_cams * (uint64_t)ws->n_gauss, ws->cap_pairs, ws->d_ckpt, ws->d_ckpt_at, ws->d_ckpt_cnt,
        ws->d_unit_rec, ws->d_Cfin);
    return cudaGetLastError();
}

cudaError_t launch_expand_tiles(const geer_workspace *ws, uint32_t *count_or_off, uint32_t *lists, cudaStream_t s) {
    if (ws->n_tiles == 0) return cudaSuccess;
    launch_k(k_expand_tiles, dim3((unsigned)ws->n_tiles), dim3(kTilePix), 0, s, ws->d_cams, ws->n_cams,
             ws->d_tile_tab, ws->super_size, ws->d_srange, ws->d_vals[ws->sorted_buf], ws->d_sranges, ws->d_misc,
             count_or_off, lists, ws->cap_pairs);
    return cudaGetLastError();
}

cudaError_t launch_render_bwd(const geer_workspace *ws, const float *dL_drgb, cudaStream_t s) {
    if (ws->n_tiles == 0) return cudaSuccess;
    constexpr int R = GEER_BWD_ROWS, B = GEER_BWD_BATCH;
    launch_k(ws->params.alpha_model == GEER_ALPHA_EXACT ? k_render_bwd<R, B, false> : k_render_bwd<R, B, true>,
        dim3((unsigned)std::max(1, ws->bwd_grid)), dim3(R * kTile), 0, s,
        ws->d_cams, ws->n_cams, ws->d_pix_tab, ws->d_tile_tab, ws->super_size, ws->d_tile_walk, ws->d_bwd_order,
        ws->d_srange, ws->d_vals[ws->sorted_buf], ws->d_sranges, ws->d_rec, ws->d_misc,
        ws->params, dL_drgb,
        ws->d_Tfin, ws->d_last, ws->d_hit, ws->d_idrec, ws->hit_entries, ws->d_gacc, ws->n_tiles,
        (uint64_t)ws->n_cams * (uint64_t)ws->n_gauss, ws->cap_pairs, ws->d_ckpt, ws->d_ckpt_at, ws->d_ckpt_cnt,
        ws->d_Cfin);
    return cudaGetLastError();
}

cudaError_t launch_render_train(const geer_workspace *ws, const float *target, float *rgb, float *T_final,
                                float *dL_drgb, float *loss, cudaStream_t s) {
    if (ws->n_tiles == 0) return cudaSuccess;
    constexpr int R = GEER_BWD_ROWS, B = GEER_BWD_BATCH;
    const int64_t m = 3 * ws->n_pixels;  // the L1 mean's value count
    launch_k(ws->params.alpha_model == GEER_ALPHA_EXACT ? k_render_train<R, B, false> : k_render_train<R, B, true>,
        dim3((unsigned)std::max(1, ws->train_grid)), dim3(R * kTile), 0, s,
        ws->d_cams, ws->n_cams, ws->d_pix_tab, ws->d_tile_tab, ws->super_size, ws->d_tile_walk, ws->d_tile_order,
        ws->d_srange, ws->d_vals[ws->sorted_buf], ws->d_sranges, ws->d_rec, ws->d_misc, ws->params, rgb, T_final,
        ws->d_Tfin, ws->d_last, ws->d_evals, ws->d_hit, ws->d_idrec, ws->hit_entries,
        ws->tile_mask_on ? static_cast<const uint8_t *>(ws->d_tile_mask) : nullptr, ws->n_tiles,
        (uint64_t)ws->n_cams * (uint64_t)ws->n_gauss, ws->cap_pairs, ws->d_ckpt, ws->d_ckpt_at, ws->d_ckpt_cnt,
        ws->d_unit_rec, ws->d_Cfin, target, dL_drgb, m > 0 ? 1.0f / (float)m : 0.0f, loss, ws->d_gacc,
        ws->d_bwd_order, (uint32_t)(ws->n_tiles * (kCkptMax + 1)));
    return cudaGetLastError();
}

int render_train_blocks_per_sm(int alpha_model) {
    constexpr int R = GEER_BWD_ROWS, B = GEER_BWD_BATCH;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &b, alpha_model == GEER_ALPHA_EXACT ? k_render_train<R, B, false> : k_render_train<R, B, true>,
            R * kTile, 0) != cudaSuccess)
        b = 1;
    return b < 1 ? 1 : b;
}

int render_bwd_blocks_per_sm(int alpha_model) {
    constexpr int R = GEER_BWD_ROWS, B = GEER_BWD_BATCH;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &b, alpha_model == GEER_ALPHA_EXACT ? k_render_bwd<R, B, false> : k_render_bwd<R, B, true>, R * kTile,
            0) != cudaSuccess)
        b = 1;
    return b < 1 ? 1 : b;
}

}  // namespace geer
