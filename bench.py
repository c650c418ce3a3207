"""Benchmark of the exact ray-Gaussian render hot path on GB300.

Workload (the headline configuration): 1M Gaussians (means uniform in a 4 m cube
3-7 m ahead, log-scales N(-2.5, 0.5), SH degree 3), Kannala-Brandt fisheye
1280x960, 190 deg FoV, k_i ~ U[-0.05, 0.05], BEAP 16x16 tiles, seeded synthetic
data. One step = preprocess (PBF association) + depth sort + duplicate + tile
sort + render of the whole frame + L1 loss gradient against a seeded target +
backward (render and preprocess stages) to all Gaussian parameters.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0). With N > 1 (torchrun), every rank renders its
own replica of the workload (the path has no cross-GPU exchange) and the time
is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import contextlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpix/s fwd and fwd+bwd at 1M Gaussians, 180° fisheye; serving p50/p99 ms"
WORKLOAD = "1M Gaussians (cube 4 m, 3-7 m ahead, SH3), Kannala-Brandt 1280x960 190deg, BEAP 16x16 tiles"
# Algorithmic work of the render kernels, the scope table's counts: 66 flop per
# ray-Gaussian evaluation in the forward (W d, the cross product, two norms, the
# divide, the exponent and the blend, FMAs counted as two), and twice that per
# list entry the backward walks back (re-evaluation, then the gradient terms).
FLOPS_FWD_EVAL = 66
FLOPS_BWD_EVAL = 2 * FLOPS_FWD_EVAL
                   # d_u / o_u / W (80) and its share of the warp reduction (16)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.proc = None
        self.index = index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.strip()]
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 8]
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _oracle_step(orc, scene, cam, pix, target):
    """One oracle step on a pixel sample, the step the GPU times: the FP32 replica
    (cull, keys, ranges), the FP64 render of the pixels and the FP64 gradient of
    their L1 loss against the target."""
    rep = orc.replica(scene, cam)
    out = orc.render_pixels(scene, cam, pix, rep=rep)
    dL = np.sign(out["rgb"] - target[pix[:, 1], pix[:, 0]]) / (3.0 * pix.shape[0])
    orc.render_grad(scene, cam, pix, dL, rep=rep)


def _oracle_probe(orc, scene, cam, target, seed: int):
    """(seconds per step without pixels, seconds per pixel) of the oracle step."""
    t0 = time.perf_counter()
    orc.replica(scene, cam)
    t_rep = time.perf_counter() - t0
    pix = _random_pixels(cam, 4, seed)
    t0 = time.perf_counter()
    _oracle_step(orc, scene, cam, pix, target)
    return t_rep, max((time.perf_counter() - t0 - t_rep) / pix.shape[0], 1e-9)


def _random_pixels(cam, n, seed):
    from paper_2505_24053_gb300 import workloads as wl
    return wl.random_pixels(cam, n, seed)  # seeded sample of distinct pixels


def _oracle_sample(scene, cam, target, seconds: float, seed: int = 7):
    """Time the CPU oracle's training step (render + L1 gradient + backward) on a
    seeded pixel sample sized to ~seconds of work."""
    from oracle import oracle as orc
    t_rep, per_px = _oracle_probe(orc, scene, cam, target, seed)
    n = int(max(4, min(8192, (seconds - t_rep) / per_px)))
    pix = _random_pixels(cam, n, seed + 1)
    t0 = time.perf_counter()
    _oracle_step(orc, scene, cam, pix, target)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": n / dt / 1e6, "unit": "Mpix/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} seeded pixels of the {cam.width}x{cam.height} frame against all {scene.n} Gaussians: "
                      f"FP32 replica pass, FP64 brute-force render and FP64 gradient of their L1 loss, {dt:.1f} s"}


def run_reference(args):
    """The oracle as it stands, timed on the host cores (rank 0 only): each step
    the replica pass, the FP64 render of a seeded pixel sample and the FP64
    gradient of its L1 loss (the GPU step's forward, L1 gradient and backward),
    the sample sized so that the whole run takes about two and a half minutes."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as orc
    from paper_2505_24053_gb300 import workloads as wl
    orc.build()
    scene = wl.config_scene(3)
    cam = wl.config_cameras(3)[0]
    target = wl.l1_target(cam, seed=3)
    t_rep, per_px = _oracle_probe(orc, scene, cam, target, 999)
    budget = 150.0 / (args.steps + args.warmup)
    per_step = int(max(2, min(args.ref_pixels, (budget - t_rep) / per_px)))
    for w in range(args.warmup):
        _oracle_step(orc, scene, cam, wl.random_pixels(cam, per_step, 1000 + w), target)
    t0 = time.perf_counter()
    for k in range(args.steps):
        _oracle_step(orc, scene, cam, wl.random_pixels(cam, per_step, 2000 + k), target)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "pass": "fwd+L1+bwd", "sample_pixels_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} seeded pixels per step against all {scene.n} Gaussians: FP32 "
                                       f"replica pass, FP64 render and FP64 gradient of their L1 loss"},
            "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def aggregate(local_ms: float, pixels_per_rank: int, steps: int, world: int, dist=None, device=None,
              shared: bool = False):
    """Whole-job Mpix/s from per-rank device time: time = max over ranks, work =
    all ranks' pixels (replicas, weak scaling), or, with shared (the tile split:
    the ranks share one frame's pixels, strong scaling), the frame's pixels."""
    t = local_ms
    if world > 1:
        import torch
        x = torch.tensor([local_ms], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    frames = 1 if shared else world
    return frames * pixels_per_rank * steps / (t / 1e3) / 1e6, t


SERVING_MODES = (("concurrent", 1, 2), ("batched", 4, 2), ("one_at_a_time", 1, 1))


def run_serving(args, dev):
    """Workload 4: 2M-Gaussian resident scene, Poisson request stream (pinhole
    1920x1080 70 deg / equidistant 1280x1280 200 deg / Kannala-Brandt 640x480
    150 deg, random poses within 1 m), served by the engine (captured CUDA graphs)
    with one request per launch on two concurrent streams ("concurrent"), with
    batches of up to four cameras on two streams ("batched") and one request at a
    time ("one_at_a_time"), on the same trace: at the workload's 200 req/s and
    at a rate beyond what one request at a time sustains (--serving-sat-rate).
    Per mode: latency percentiles, the sustained completion rate while requests
    keep arriving, the backlog's drain time, and where latency went (queue,
    host launch, GPU, completion noticed) at p50 / p99 / max."""
    import torch

    from paper_2505_24053_gb300 import geer, serve
    from paper_2505_24053_gb300 import workloads as wl

    scene = wl.config_scene(4)
    g = geer.Gaussians.from_scene(scene)
    models = [k[0] for k in wl.SERVING_KINDS]
    warm = args.serving_warmup
    engines = {}
    for name, slots, bufs in SERVING_MODES:
        # capacity in (super-tile, Gaussian) pairs: ~37M for the largest request kind alone
        eng = serve.Engine(g, n_slots=slots, n_buffers=bufs, pair_capacity=slots * 60_000_000)
        calib = wl.serving_requests(24, seed=4, rate_hz=args.serving_rate)
        eng.calibrate([serve.Request(i, t, c, kind=models.index(c.model)) for i, (t, c) in enumerate(calib)])
        eng.prepare()
        engines[name] = eng
    out = {"scene": "2M Gaussians resident (workload-1 distribution, SH degree 3)",
           "mix": "equal mix of pinhole 1920x1080 70deg, equidistant 1280x1280 200deg, Kannala-Brandt 640x480 "
                  "150deg, random poses within 1 m"}
    rates = [(f"{args.serving_rate:g}_req_s", args.serving_rate, args.serving_seconds)]
    if args.serving_sat_rate > 0:
        rates.append((f"{args.serving_sat_rate:g}_req_s", args.serving_sat_rate, args.serving_sat_seconds))
    for label, rate, seconds in rates:
        n_req = int(round(rate * seconds))
        trace = wl.serving_requests(n_req, seed=4, rate_hz=rate)
        res = {"trace": f"Poisson {rate:g} req/s, {n_req} requests over {seconds:g} s (first {warm:g} s excluded)"}
        for name, slots, bufs in SERVING_MODES:
            eng = engines[name]
            reqs = [serve.Request(i, t, c, kind=models.index(c.model)) for i, (t, c) in enumerate(trace)]
            done = eng.run(reqs)
            keep = [r for r in done if r.arrival >= warm]
            st = serve.summarize(keep, max(1e-9, seconds - warm), window=(warm, seconds))
            st.update({"slots": slots, "buffers": bufs, "graphs": True, "failed": len(eng.failed)})
            res[name] = st
        out[label] = res
    engines.clear()
    torch.cuda.empty_cache()
    return out


# (name, association, SnugBox, alpha model): the association methods with the
# exact ray integral, then the render-time splat alpha with PBF association
# (the swap at render time) and with EWA association (splatting on the BEAP grid)
ASSOC_MODES = (("pbf", 0, False, 0), ("ewa", 1, False, 0), ("ewa_snugbox", 1, True, 0), ("ut", 2, False, 0),
               ("ut_snugbox", 2, True, 0), ("pbf_splat_alpha", 0, False, 1), ("ewa_splat_alpha", 1, False, 1))


def _association_ablation(args, geer, wl, g, cams, rgb_pbf, flush, stream):
    """The association ablation: the same forward pass with the tile association
    of PBF or of the splatting bounds (EWA / UT, 3-sigma square or SnugBox), and
    with the render-time splat alpha in place of the ray integral, on the bench
    scene and on an indoor room of the same size (wall surfels and clutter
    around the camera). Per method: associated (tile, Gaussian) pairs per tile,
    the forward stages' times (CUDA events, L2 flushed between steps) and the
    render's PSNR / SSIM against the exact PBF render (what the splatting bounds
    lose: contributions above alpha_min on tiles their boxes miss; what the
    splat alpha changes)."""
    room = geer.Gaussians.from_scene(wl.room_scene(g.n, 6, g.sh_degree))
    tiles = sum(math.ceil(c.width / 16) * math.ceil(c.height / 16) for c in cams)
    return {"tiles": tiles, "steps": 10,
            "scenes": {"bench": _ablate_scene(geer, g, cams, rgb_pbf, flush, stream, tiles),
                       "room": _ablate_scene(geer, room, cams, rgb_pbf, flush, stream, tiles)},
            "room": "room_scene: 80% wall surfels (box 5 x 2.8 x 6 m around the camera), 20% clutter"}


def _ablate_scene(geer, g, cams, rgb_pbf, flush, stream, tiles):
    import torch
    out = {"modes": {}}
    ref = None
    for name, mode, snug, alpha in ASSOC_MODES:
        rr = geer.Renderer(cams, g.n, g.sh_degree, params=geer.params_c(assoc=mode, snugbox=snug, alpha_model=alpha))
        rr.prepare(g)
        img = torch.empty_like(rgb_pbf)
        evs = []
        for k in range(3 + 10):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            rr.ws.preprocess(g)
            ev[1].record(stream)
            rr.ws.bin_sort(sync=False)
            ev[2].record(stream)
            rr.ws.render_fwd(img)
            ev[3].record(stream)
            if k >= 3:
                evs.append(ev)
        torch.cuda.synchronize()
        st, _ = rr.ws.device_status()
        if st != geer.OK:
            raise RuntimeError(f"association ablation ({name}): {geer.status_string(st)}")
        pairs, _ = rr.ws.pair_counts()
        if ref is None:
            ref = img
        c0 = cams[0]
        q = geer.image_metrics(img[:c0.pixels].view(c0.height, c0.width, 3),
                               ref[:c0.pixels].view(c0.height, c0.width, 3))[0]
        out["modes"][name] = {
            "gaussians_per_tile": int(pairs) / tiles, "pairs": int(pairs), "live_items": rr.ws.live_items(),
            "preprocess_ms": statistics.mean(e[0].elapsed_time(e[1]) for e in evs),
            "bin_sort_ms": statistics.mean(e[1].elapsed_time(e[2]) for e in evs),
            "render_fwd_ms": statistics.mean(e[2].elapsed_time(e[3]) for e in evs),
            "fwd_ms": statistics.mean(e[0].elapsed_time(e[3]) for e in evs),
            "psnr_vs_pbf": q["psnr"] if ref is not img else None,
            "ssim_vs_pbf": q["ssim"] if ref is not img else None}
        if ref is not img:
            del rr, img
    torch.cuda.empty_cache()
    return out


def _tile_stats(ws, cams):
    """Gaussians per tile (mean and standard deviation over every tile of the
    cameras: the (tile, Gaussian) associations each tile's list holds, as the
    paper's association tables report them) and the render's device memory: the
    workspace (every buffer the render and its backward use) beside the
    Gaussians' own arrays. Read after the timed steps (synchronous copies)."""
    per_tile = ws.tile_counts().astype(np.float64)
    ntiles = per_tile.size
    return {"gaussians_per_tile_mean": float(per_tile.mean()), "gaussians_per_tile_std": float(per_tile.std()),
            "gaussians_per_tile_max": int(per_tile.max()), "tiles": int(ntiles),
            "workspace_bytes": int(ws.nbytes), "workspace_gb": ws.nbytes / 1e9}


def run(args):
    import torch
    import torch.distributed as dist

    from paper_2505_24053_gb300 import geer, tilesplit
    from paper_2505_24053_gb300 import workloads as wl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    scene = wl.config_scene(args.workload, n=args.gaussians)
    cams = wl.config_cameras(args.workload)
    cam = cams[0]
    g = geer.Gaussians.from_scene(scene)
    r = geer.Renderer(cams, scene.n, scene.sh_degree)
    P = r.prepare(g)  # sizes the pair capacity (synchronous count), then everything stays asynchronous
    ws = r.ws
    pixels = sum(c.pixels for c in cams)
    rgb = torch.empty((pixels, 3), dtype=torch.float32, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # 512 MB > 129 MB L2
    stream = torch.cuda.current_stream()
    grads = {k: torch.zeros_like(v) for k, v in (("mean", g.mean), ("scale", g.scale), ("quat", g.quat),
                                                 ("opacity", g.opacity), ("sh", g.sh))}
    have_bwd = not args.fwd_only
    target = torch.as_tensor(np.concatenate([wl.l1_target(c, seed=3 + i).reshape(-1, 3) for i, c in enumerate(cams)]),
                             device=dev)
    dL = torch.empty_like(rgb)
    loss = torch.empty(1, device=dev)
    split = args.split == "tiles"
    target_step = target
    if split:
        # this rank renders its share of the tiles; the backward's render-stage
        # accumulators are summed over the ranks (NCCL) before its preprocess stage
        ts = tilesplit.TileSplit(ws, rank, world)
        target_step = ts.masked_target(target)

    fused = not args.separate_render

    def backward(gk):
        if split:
            ws.render_bwd_tiles(dL)
            tilesplit.reduce_sum(ws.grad_accumulators(), None, world)
            ws.preprocess_bwd(gk, grads, accumulate=False)
        else:
            ws.render_bwd(gk, dL, grads, accumulate=False)

    def render_step(gk, rgb_out):
        """The step's render: forward, L1 gradient and backward (the gradients written).
        Fused: one launch for the forward, the L1 gradient and the backward's render
        stage (geer_render_train_l1), then its preprocess stage."""
        if fused:
            ws.render_train_l1(target_step, rgb_out, dL)
            if split:
                tilesplit.reduce_sum(ws.grad_accumulators(), None, world)
            ws.preprocess_bwd(gk, grads, accumulate=False)
        else:
            ws.render_fwd(rgb_out)
            geer.l1_loss_grad(rgb_out, target_step, dL)
            backward(gk)

    # ev[0] and ev[3] bracket a step; with detail, ev[1] and ev[2] also mark the
    # end of the preprocess and of the binning (a breakdown run, not the timed one:
    # an event between two kernels keeps the second from launching while the first
    # runs, which the binning's short kernels would pay for)
    def train_step(ev, detail=False):
        ev[0].record(stream)
        ws.preprocess(g)
        if detail:
            ev[1].record(stream)
        ws.bin_sort(sync=False)
        if detail:
            ev[2].record(stream)
        # training step: forward, L1 loss gradient, backward (the step's gradients written)
        render_step(g, rgb)
        ev[3].record(stream)

    def fwd_step(ev, detail=False):
        ev[0].record(stream)
        ws.preprocess(g)
        if detail:
            ev[1].record(stream)
        ws.bin_sort(sync=False)
        if detail:
            ev[2].record(stream)
        ws.render_fwd(rgb)
        ev[3].record(stream)

    def timed(step, clk_sample, steps=None, detail=False):
        steps = args.steps if steps is None else steps
        for _ in range(args.warmup):
            flush.zero_()
            step([torch.cuda.Event(enable_timing=True) for _ in range(4)], detail)
        torch.cuda.synchronize()
        st, _ = ws.device_status()
        if st != geer.OK:
            raise RuntimeError(f"device status after warm-up: {geer.status_string(st)}")
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) if clk_sample else contextlib.nullcontext() as clk:
            t0 = time.perf_counter()
            for k in range(steps):
                flush.zero_()  # between timed steps, outside the step's events
                step(evs[k], detail)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        if world > 1:
            dist.barrier()
        st, _ = ws.device_status()
        if st != geer.OK:
            raise RuntimeError(f"device status after timed steps: {geer.status_string(st)}")
        return evs, wall, clk

    # the timed steps: the library's stage events around the dominant kernel's stage
    # only (the backward render; the forward render without a backward)
    dom_stage = ("render_train" if fused else "render_bwd") if have_bwd else "render_fwd"
    ws.enable_timing(True, stages=(dom_stage, "render_fwd") if have_bwd and fused else (dom_stage,))
    train_evs = None
    if have_bwd:
        train_evs, t_wall, clk = timed(train_step, True)
        dom_stage_ms = {dom_stage: ws.stage_times()[dom_stage][0]}  # the last 64 timed steps
    fwd_evs, fwd_wall, fclk = timed(fwd_step, not have_bwd)
    fwd_stage_ms = ws.stage_times()["render_fwd"][0]  # the forward render in the forward-only steps
    if not have_bwd:
        t_wall, clk = fwd_wall, fclk
        dom_stage_ms = {dom_stage: ws.stage_times()[dom_stage][0]}
    pairs, super_pairs = ws.pair_counts()
    tile_stats = _tile_stats(ws, cams)
    # the breakdown: the same step with every stage's events, in a run of its own
    ws.enable_timing(False)
    ws.enable_timing(True)
    bd_evs, _, _ = timed(train_step if have_bwd else fwd_step, False, steps=min(args.steps, 64), detail=True)
    stage_ms = {k: v[0] for k, v in ws.stage_times().items()}
    stage_ms.update(dom_stage_ms)
    ws.enable_timing(False)
    main_evs = train_evs if have_bwd else fwd_evs
    step_ms = [e[0].elapsed_time(e[3]) for e in main_evs]
    prep_ms = [e[0].elapsed_time(e[1]) for e in bd_evs]
    sort_ms = [e[1].elapsed_time(e[2]) for e in bd_evs]
    rend_ms = [e[2].elapsed_time(e[3]) for e in bd_evs]
    value, total_ms = aggregate(float(sum(step_ms)), pixels, args.steps, world, dist, dev, shared=split)
    fwd_ms = [e[0].elapsed_time(e[3]) for e in fwd_evs]
    fwd_value = pixels / (statistics.mean(fwd_ms) / 1e3) / 1e6
    fwd_render_ms = stage_ms.get("render_fwd") or fwd_stage_ms
    if fused and have_bwd:
        stage_ms["render_fwd"] = fwd_stage_ms

    # end to end through the C ABI with host buffers: every step copies its
    # Gaussians from pinned host memory and reads its image back into pinned host
    # memory. A streaming user's pipeline: uploads run on a copy stream into two
    # device buffers, so step k+1's upload overlaps step k's compute, and each
    # image is read back on a third stream; one timed region spans all steps with
    # every copy inside it (inputs > L2, no flush).
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in
            (scene.mean, scene.scale, scene.quat, scene.opacity, scene.sh)]
    gbuf = [g, geer.Gaussians.from_scene(scene)]
    rgb_buf = [rgb, torch.empty_like(rgb)]
    out_host = [torch.empty((pixels, 3), dtype=torch.float32).pin_memory() for _ in range(2)]
    h2d = sum(h.numel() * 4 for h in host)
    d2h = out_host[0].numel() * 4
    up_s, down_s = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def pipeline(n):
        ev = lambda: torch.cuda.Event()
        up_done, comp_done, down_done = [ev(), ev()], [ev(), ev()], [ev(), ev()]

        def upload(k):
            b = k % 2
            up_s.wait_event(comp_done[b])  # step k - 2, the buffer's last reader, has finished
            with torch.cuda.stream(up_s):
                for h, d in zip(host, (gbuf[b].mean, gbuf[b].scale, gbuf[b].quat, gbuf[b].opacity, gbuf[b].sh)):
                    d.copy_(h, non_blocking=True)
            up_done[b].record(up_s)

        start = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        up_s.wait_event(start)
        upload(0)
        for k in range(n):
            b = k % 2
            if k + 1 < n:
                upload(k + 1)
            stream.wait_event(up_done[b])
            stream.wait_event(down_done[b])  # the image of step k - 2 has been read back
            gk = gbuf[b]
            ws.preprocess(gk)
            ws.bin_sort(sync=False)
            if have_bwd:
                render_step(gk, rgb_buf[b])
            else:
                ws.render_fwd(rgb_buf[b])
            comp_done[b].record(stream)
            down_s.wait_event(comp_done[b])
            with torch.cuda.stream(down_s):
                out_host[b].copy_(rgb_buf[b], non_blocking=True)
            down_done[b].record(down_s)
        for e in down_done + [up_done[(n - 1) % 2]]:
            stream.wait_event(e)
        return start

    pipeline(args.warmup)
    torch.cuda.synchronize()
    e0 = pipeline(args.steps)
    e1 = torch.cuda.Event(enable_timing=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e_evs = [(e0, e1)]
    e2e, e2e_ms = aggregate(sum(a.elapsed_time(b) for a, b in e_evs), pixels, args.steps, world, dist, dev,
                            shared=split)
    if split:
        ws.set_tile_mask(None)  # the measurements below render whole frames

    # remap of the BEAP render to the native camera image: an optional output
    # stage, timed on its own (not part of the step or of Mpix/s)
    native = torch.empty_like(rgb)
    beap_img = rgb[:cam.pixels].view(cam.height, cam.width, 3)
    r_evs = []
    for k in range(3 + 20):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        geer.remap_to_native(beap_img, cam, out=native[:cam.pixels].view(cam.height, cam.width, 3))
        e1.record(stream)
        if k >= 3:
            r_evs.append((e0, e1))
    torch.cuda.synchronize()
    remap_ms = statistics.mean(a.elapsed_time(b) for a, b in r_evs)

    # native-camera evaluation (timed on its own): the evaluation regions of the
    # native image, then PSNR / SSIM per region of the reprojected render against
    # a reference native image (here the reprojected L1 target, for timing)
    nat = native[:cam.pixels].view(cam.height, cam.width, 3)
    ref_nat = geer.remap_to_native(target[:cam.pixels].view(cam.height, cam.width, 3).contiguous(), cam)
    regions = geer.native_regions(cam)
    acc = torch.empty(6, dtype=torch.float64, device=dev)
    reg_evs, met_ms = [], []
    for k in range(3 + 10):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        geer.native_regions(cam, out=regions)
        e1.record(stream)
        if k >= 3:
            reg_evs.append((e0, e1))
    for k in range(3 + 10):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = geer.image_metrics(nat, ref_nat, regions, 2)  # synchronous (the sums copied back)
        e1.record(stream)
        if k >= 3:
            met_ms.append((e0, e1))
    torch.cuda.synchronize()
    regions_ms = statistics.mean(a.elapsed_time(b) for a, b in reg_evs)
    metrics_ms = statistics.mean(a.elapsed_time(b) for a, b in met_ms)

    # rooflines: per stage from algorithmic work and CUDA-event times measured in the timed steps
    evals, applied, walked = ws.render_counts()
    peaks, peak_src = _peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    n_items = scene.n * len(cams)  # (camera, Gaussian) items
    live = ws.live_items()
    sort_passes = ws.sort_passes()
    sh_bytes = 4 * 3 * (scene.sh_degree + 1) ** 2
    g_bytes = 4 * (3 + 3 + 4 + 1) + sh_bytes
    work = {
        # record, ranges, count, key per item; in the training step also the item's
        # backward accumulators zeroed (64 B)
        "preprocess": ("hbm", scene.n * g_bytes + n_items * (64 + 16 + 4 + 4 + (64 if have_bwd else 0))),
        "depth_sort": ("hbm", 4 * 20 * live),
        # per live item: id, tile count and ranges read; 8 B per (super-tile, item) pair written
        "duplicate": ("hbm", live * (4 + 4 + 16) + int(super_pairs) * 8),
        # passes x (read key 4 B + key/value 8 B, write 8 B), and 16 B of ranges gathered + written
        "tile_sort": ("hbm", sort_passes * 20 * int(super_pairs) + 32 * int(super_pairs)),
        "render_fwd": ("alu", FLOPS_FWD_EVAL * evals),
        "render_bwd": ("alu", FLOPS_BWD_EVAL * walked),
        # the fused render: the forward's evaluations and the backward's walked entries
        "render_train": ("alu", FLOPS_FWD_EVAL * evals + FLOPS_BWD_EVAL * walked),
        # the step writes its gradients: parameters and accumulators read, gradients written
        "preprocess_bwd": ("hbm", scene.n * g_bytes * 2 + n_items * 64),
    }
    stages = {}
    for name, (bound, amount) in work.items():
        t = stage_ms.get(name, 0.0)
        if t <= 0:
            continue
        if bound == "hbm":
            ach = amount / (t / 1e3) / 1e9
            stages[name] = {"ms": t, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                            "frac": ach / hbm_peak, "algorithmic_bytes": amount}
        else:
            ach = amount / (t / 1e3) / 1e12
            stages[name] = {"ms": t, "bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                            "frac": ach / fp32_peak, "algorithmic_flops": amount}
    kernel_of = {"render_fwd": "k_render_fwd", "render_bwd": "k_render_bwd", "render_train": "k_render_train",
                 "preprocess": "k_preprocess",
                 "preprocess_bwd": "k_preprocess_bwd", "duplicate": "k_duplicate"}
    single = {k: v for k, v in stages.items() if k in kernel_of}
    dom = max(single, key=lambda k: single[k]["ms"])
    traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        import hashlib
        with open(prof) as f:
            tr = json.load(f).get(kernel_of[dom])
        if tr:
            src = os.path.join(ROOT, "paper_2505_24053_gb300", "csrc", tr["source"])
            if hashlib.sha1(open(src, "rb").read()).hexdigest() == tr["source_sha1"]:
                traffic = tr["bytes_per_launch"]
    # a full training step (Algorithm 2 with the 3DGS optimiser): fwd, L1, bwd and
    # one Adam step over the raw parameters (log-scale, logit-opacity), timed on
    # its own; the Gaussians move from step to step as training does
    op = np.clip(scene.opacity.astype(np.float64), 1e-6, 1 - 1e-6)
    adam = geer.Adam(scene.mean, np.log(scene.scale), scene.quat, np.log(op / (1 - op)).astype(np.float32),
                     scene.sh, scene.sh_degree, lr_mean=1e-3)
    tgrads = {k: torch.empty_like(v) for k, v in grads.items()}
    tr_evs = []
    for k in range(args.warmup + max(10, args.steps // 4)):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        ga = adam.gaussians
        ws.preprocess(ga)
        ws.bin_sort(sync=False)
        if fused:
            ws.render_train_l1(target, rgb, dL)
            ws.preprocess_bwd(ga, tgrads, accumulate=False)
        else:
            ws.render_fwd(rgb)
            geer.l1_loss_grad(rgb, target, dL)
            ws.render_bwd(ga, dL, tgrads, accumulate=False)
        ev[1].record(stream)
        adam.step(tgrads)
        ev[2].record(stream)
        if k >= args.warmup:
            tr_evs.append(ev)
    torch.cuda.synchronize()
    train_ms = statistics.mean(e[0].elapsed_time(e[2]) for e in tr_evs)
    adam_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in tr_evs)
    per_g = 11 + 3 * (scene.sh_degree + 1) ** 2
    adam_bytes = scene.n * per_g * 28 + scene.n * 16  # p, g, m, v read; p, m, v written; activated scale + opacity
    adam_gbs = adam_bytes / (adam_ms / 1e3) / 1e9

    assoc = _association_ablation(args, geer, wl, g, cams, rgb, flush, stream) if not args.no_ablation else None

    # a refinement iteration at this size (Algorithm 2, 3DGS density control):
    # plan (classify + count, synchronous) and apply over the trained Gaussians,
    # with statistics drawn so that about 10% are densified; timed on its own
    dens = None
    if not args.no_ablation:
        drng = torch.Generator(device=dev).manual_seed(9)
        accum = torch.rand(adam.n, device=dev, generator=drng) * 2.2e-4  # g >= 2e-4 for ~9%
        denom = torch.ones(adam.n, device=dev)
        zd = torch.randn((adam.n, 2, 3), device=dev, generator=drng)
        n_in = adam.n
        base = {k: v.clone() for k, v in adam.raw.items()}
        m0, v0 = adam.m.clone(), adam.v.clone()
        d_ms = []
        for k in range(3 + 5):
            adam.raw = {k2: v2.clone() for k2, v2 in base.items()}
            adam.m, adam.v, adam.n = m0.clone(), v0.clone(), n_in
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            n_out = adam.densify(accum, denom, zd, grad_threshold=2e-4, clone_max_scale=0.08, min_opacity=0.005)
            e1.record(stream)
            if k >= 3:
                d_ms.append((e0, e1))
        torch.cuda.synchronize()
        dms = statistics.mean(a.elapsed_time(c) for a, c in d_ms)
        row = 4 * (11 + 3 * (scene.sh_degree + 1) ** 2)  # raw parameters, one Gaussian
        # read: parameters + 2 moment rows + statistics and normals (4 + 4 + 24 B, plan reads 16 B) per input;
        # written: parameters + 2 moment rows + activated scale and opacity (16 B) per output
        dbytes = n_in * (3 * row + 48) + n_out * (3 * row + 16)
        dens = {"ms": dms, "n_in": n_in, "n_out": n_out, "bound": "hbm", "algorithmic_bytes": dbytes,
                "achieved": dbytes / (dms / 1e3) / 1e9, "peak": hbm_peak,
                "frac": dbytes / (dms / 1e3) / 1e9 / hbm_peak,
                "note": "geer_densify_plan (classify, scan, synchronous count) + geer_densify_apply + the new "
                        "tensors' allocation, timed on its own; not in value"}

    remap_gbs = 24 * cam.pixels / (remap_ms / 1e3) / 1e9  # 12 B read + 12 B written per native pixel
    remap = {"ms": remap_ms, "bound": "hbm", "achieved": remap_gbs, "peak": hbm_peak, "unit": "GB/s",
             "frac": remap_gbs / hbm_peak, "algorithmic_bytes": 24 * cam.pixels,
             "note": "BEAP -> native Kannala-Brandt resampling, timed separately, not in value"}
    d = stages[dom]
    roofline = {"bound": d["bound"], "kernel": kernel_of[dom], "achieved": d["achieved"],
                "peak": d["peak"], "unit": d["unit"], "frac": d["frac"], "traffic": traffic,
                "kernel_ms": d["ms"],
                "peak_source": (f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz "
                                f"(max SM clock, {peak_src})") if d["bound"] == "alu"
                               else f"copy bandwidth, {peak_src}",
                "work": {"evaluations": evals, "applied": applied, "walked_back": walked}}
    tiles = math.ceil(cam.width / 16) * math.ceil(cam.height / 16)
    # preprocess, live scan, compact, 4 depth passes x 2, gather, pair scan, emit, offsets,
    # super-tile sort passes x 2, render forward (+ L1 gradient, backward order, render backward,
    # preprocess backward): 22 per training step with one super-tile pass, as the ncu launch list shows
    launches_per_step = 16 + 2 * sort_passes + ((1 if fused else 4) if have_bwd else 0)

    line = {
        "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if split else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.workload == 3 else f"workload {args.workload}",
                   "pass": "fwd+L1+bwd" if have_bwd else "fwd", "gaussians": scene.n,
                   "pixels_per_gpu": pixels, "pairs": int(pairs), "super_pairs": int(super_pairs),
                   "parallelism": (f"tile split x{world}: each rank renders 1/{world} of the tiles, the "
                                   f"backward's render-stage accumulators all-reduced (NCCL)") if split
                                  else f"replicas x{world}",
                   "l2": "512 MB buffer written between timed steps (outside step events); inputs 236 MB > L2"},
        "fwd_only": {"value": fwd_value, "unit": "Mpix/s", "ms": statistics.mean(fwd_ms)},
        "stages_ms": {"preprocess": statistics.mean(prep_ms), "bin_sort": statistics.mean(sort_ms),
                      "render_fwd": fwd_render_ms,
                      "render_fwd_l1_bwd": statistics.mean(rend_ms) if have_bwd else None},
        "roofline": roofline,
        "association": tile_stats,
        "stages": stages,
        "remap": remap,
        "train_step": {
            "value": pixels / (train_ms / 1e3) / 1e6, "unit": "Mpix/s", "ms": train_ms,
            "adam": {"ms": adam_ms, "bound": "hbm", "achieved": adam_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": adam_gbs / hbm_peak, "algorithmic_bytes": adam_bytes},
            "densify": dens,
            "note": "fwd + L1 + bwd (gradients written) + one Adam step over mean, log-scale, quat, "
                    "logit-opacity and SH (geer_adam_step), timed on its own; not in value"},
        "evaluation": {
            "regions_ms": regions_ms, "metrics_ms": metrics_ms,
            "metrics_gbs": (25 * cam.pixels) / (metrics_ms / 1e3) / 1e9,
            "pixels": {"central": res[0]["count"], "peripheral": res[1]["count"]},
            "note": "native evaluation regions and per-region PSNR/SSIM (11x11 Gaussian window) of the "
                    "reprojected render, timed on their own with CUDA events (metrics: the kernel, its "
                    "accumulator reset and the 48 B copy back; 24 B of images + 1 B region read per "
                    "pixel); not in value"},
        "association_ablation": assoc,
        "e2e": {"value": e2e, "unit": "Mpix/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "pipeline": "H2D of step k+1 on a copy stream during step k (two device buffers), D2H on a "
                            "third stream; one timed region over all steps; inputs > L2, no flush"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
        "wall_s_timed": t_wall,
    }
    if args.serving_seconds > 0 and world == 1:
        line["serving"] = run_serving(args, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _oracle_sample(scene, cam, wl.l1_target(cam, seed=3), args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="geer", choices=["geer", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fwd-only", action="store_true", help="time the forward render only")
    ap.add_argument("--separate-render", action="store_true",
                    help="the training step's render as three calls (forward, L1 gradient, backward) "
                         "instead of the fused launch")
    ap.add_argument("--no-ablation", action="store_true", help="skip the association ablation")
    ap.add_argument("--serving-seconds", type=float, default=8.0, help="serving trace length (0: skip)")
    ap.add_argument("--serving-warmup", type=float, default=1.0)
    ap.add_argument("--serving-rate", type=float, default=200.0)
    ap.add_argument("--serving-sat-rate", type=float, default=700.0,
                    help="second, saturating serving trace (0: skip)")
    ap.add_argument("--serving-sat-seconds", type=float, default=5.0)
    ap.add_argument("--ref-pixels", type=int, default=24)
    ap.add_argument("--split", default="replicas", choices=["replicas", "tiles"],
                    help="N > 1: independent replicas (weak scaling) or one frame's tiles split over the ranks with "
                         "the gradient accumulators all-reduced (strong scaling)")
    ap.add_argument("--gaussians", type=int, default=None,
                    help="scene size override (the workload's distribution with fewer Gaussians; profiling)")
    ap.add_argument("--workload", type=int, default=3, choices=[1, 2, 3, 5],
                    help="3 = the headline configuration; 1, 2 = smaller cases for profiling")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run(args)


if __name__ == "__main__":
    main()
