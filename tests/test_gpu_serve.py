"""Serving engine on the GPU: continuous batching through captured CUDA graphs.

Each request's image rendered in a mixed batch (fixed camera slots, graph
replay) must equal the same request rendered alone through the workspace path
(bit for bit: per-ray order depends only on depth keys and Gaussian indices).
"""
import math

import numpy as np
import pytest
import torch

from paper_2505_24053_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_2505_24053_gb300 import geer, serve
    scene = wl.cube_scene(200_000, 41, 3)
    g = geer.Gaussians.from_scene(scene)
    return geer, serve, scene, g


def _trace(n, seed, rate=400.0):
    rng = np.random.default_rng(seed)
    kinds = [(wl.PINHOLE, 480, 270, 70.0, None), (wl.EQUIDISTANT, 320, 320, 200.0, None),
             (wl.KANNALA_BRANDT, 160, 120, 150.0, 44)]
    t, out = 0.0, []
    from paper_2505_24053_gb300.serve import Request
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        k = int(rng.integers(0, 3))
        model, w, h, fov, ks = kinds[k]
        R, tc = wl.random_pose(rng)
        cam = wl.Camera(model, w, h, math.radians(fov), k=wl.kb_coeffs(ks) if ks else (0, 0, 0, 0), R_cw=R, t_cw=tc)
        out.append(Request(i, t, cam, kind=k))
    return out


def test_mixed_batches_equal_single_renders(env):
    geer, serve, scene, g = env
    eng = serve.Engine(g, n_slots=4, n_buffers=2, pair_capacity=20_000_000, max_width=480, max_height=320)
    eng.prepare()
    reqs = _trace(14, 1)
    done = eng.run(reqs, keep_images=True, realtime=False)
    assert len(done) == len(reqs)
    assert len({r.batch for r in done}) < len(reqs)  # really batched
    for r in done:
        alone = geer.Renderer([r.camera], scene.n, scene.sh_degree)
        img = alone.images(alone.forward(g))[0]
        assert torch.equal(r.image, img), r.rid


def test_realtime_trace_and_latency(env):
    geer, serve, scene, g = env
    eng = serve.Engine(g, n_slots=4, n_buffers=2, pair_capacity=20_000_000, max_width=480, max_height=320)
    eng.prepare()
    reqs = _trace(120, 2, rate=300.0)
    done = eng.run(reqs)
    s = serve.summarize(done, reqs[-1].arrival)
    assert s["requests"] == 120
    assert all(r.latency_ms is not None and r.latency_ms > 0 for r in done)
    assert s["p50_ms"] <= s["p99_ms"] < 5000


def test_capacity_overflow_splits_batches(env):
    geer, serve, scene, g = env
    # a pair capacity that fits one request but not four: batches must be split and retried
    eng = serve.Engine(g, n_slots=4, n_buffers=1, pair_capacity=2_500_000, max_width=480, max_height=320,
                       use_graphs=False)
    eng.prepare()
    reqs = _trace(8, 3)
    eng.scheduler.estimates = {0: 1, 1: 1, 2: 1}   # deliberately too low: the device status catches it
    done = eng.run(reqs, keep_images=True, realtime=False)
    assert sorted(r.rid for r in done) == list(range(8))
    for r in done[:3]:
        alone = geer.Renderer([r.camera], scene.n, scene.sh_degree)
        assert torch.equal(r.image, alone.images(alone.forward(g))[0])


def test_overflowing_warmup_does_not_leak_into_requests(env):
    geer, serve, scene, g = env
    # a capacity far below what even one request needs for the warm-up cameras of
    # the other tests, but enough for the small requests served here
    eng = serve.Engine(g, n_slots=2, n_buffers=2, pair_capacity=1_500_000, max_width=480, max_height=320)
    for b in eng.buffers:  # force an overflow in each buffer before preparation
        b.load([serve.Request(-1, 0.0, eng.capacity_camera)])
        b.step_body()
        b.stream.synchronize()
    eng.prepare()
    reqs = [r for r in _trace(30, 5) if r.kind == 2][:4]
    done = eng.run(reqs, realtime=False)
    assert len(done) == len(reqs) and not eng.failed
