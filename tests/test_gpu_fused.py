"""The fused training render (geer_render_train_l1) against the separate calls
and the FP64 oracle.

One launch renders the tiles, takes the per-pixel L1 gradient and walks the
finished tiles' backward units back from a device queue. It must equal
geer_render_fwd + geer_l1_loss_grad + geer_render_bwd_tiles:
- the image, the final transmittance and the L1 gradient bit for bit (the same
  kernels' arithmetic on the same pixels);
- the loss to rounding (a sum in another order);
- the render-stage accumulators to 1e-5 relative and the parameter gradients
  to 1e-4 (FP32 atomics add in another order; the chain to the quaternion
  cancels terms of ~1e-10, so reordered sums move it by up to ~2e-5);
and its gradient must match the oracle's at the backward tests' 1e-3.
Scenes: small cameras (the oracle), the stack of faint Gaussians whose walks
pass the 2048-entry hit record and several checkpoints, a tile-masked part,
and the full-size fisheye workload.
"""
import math

import numpy as np
import pytest
import torch

from paper_2505_24053_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

BLOCKS = ("mean", "scale", "quat", "opacity", "sh")


@pytest.fixture(scope="module")
def geer():
    from paper_2505_24053_gb300 import geer
    geer.lib()
    return geer


def _grads_like(g):
    return {k: torch.empty_like(v) for k, v in (("mean", g.mean), ("scale", g.scale), ("quat", g.quat),
                                                 ("opacity", g.opacity), ("sh", g.sh))}


def _rel(a, b):
    a, b = a.double().ravel(), b.double().ravel()
    nb = float(b.norm())
    return float((a - b).norm()) / nb if nb > 0 else float(a.abs().max())


def _separate(geer, ws, g, target, npix):
    rgb = torch.empty((npix, 3), device="cuda")
    T = torch.empty(npix, device="cuda")
    ws.preprocess(g)
    ws.bin_sort()
    ws.render_fwd(rgb, T)
    loss, dL = geer.l1_loss_grad(rgb, target)
    ws.render_bwd_tiles(dL)
    acc = ws.grad_accumulators().clone()
    grads = _grads_like(g)
    ws.preprocess_bwd(g, grads, accumulate=False)
    torch.cuda.synchronize()
    return rgb, T, dL, float(loss.item()), acc, grads


def _fused(geer, ws, g, target, npix):
    rgb = torch.empty((npix, 3), device="cuda")
    T = torch.empty(npix, device="cuda")
    dL = torch.empty((npix, 3), device="cuda")
    loss = torch.empty(1, device="cuda")
    ws.preprocess(g)
    ws.bin_sort()
    ws.render_train_l1(target, rgb, dL, loss, T)
    acc = ws.grad_accumulators().clone()
    grads = _grads_like(g)
    ws.preprocess_bwd(g, grads, accumulate=False)
    torch.cuda.synchronize()
    assert ws.device_status()[0] == geer.OK
    return rgb, T, dL, float(loss.item()), acc, grads


def _check_equal(sep, fus, tol=1e-5, grad_tol=1e-4):
    rgb0, T0, dL0, loss0, acc0, g0 = sep
    rgb1, T1, dL1, loss1, acc1, g1 = fus
    assert torch.equal(rgb0, rgb1) and torch.equal(T0, T1) and torch.equal(dL0, dL1)
    assert loss1 == pytest.approx(loss0, rel=1e-5)
    assert _rel(acc1, acc0) <= tol
    for k in BLOCKS:
        assert _rel(g1[k], g0[k]) <= grad_tol, k


def _target(npix, seed):
    return torch.as_tensor(np.random.default_rng(seed).uniform(0, 1, (npix, 3)).astype(np.float32), device="cuda")


CAMS = [
    ("kb190", [wl.Camera(wl.KANNALA_BRANDT, 48, 40, math.radians(190), k=wl.kb_coeffs(3))]),
    ("two_cams", [wl.Camera(wl.EQUIDISTANT, 36, 36, math.radians(180)),
                  wl.Camera(wl.PINHOLE, 30, 20, math.radians(50),
                            R_cw=wl.pose(wl.rot_y(0.3), (0.2, -0.1, 0.0))[0],
                            t_cw=wl.pose(wl.rot_y(0.3), (0.2, -0.1, 0.0))[1], bg=(0.3, 0.5, 0.7))]),
]


@pytest.mark.parametrize("name,cams", CAMS, ids=[c[0] for c in CAMS])
def test_fused_matches_separate_and_oracle(geer, orc, name, cams):
    full = wl.config_scene(3)
    scene = full.subset(np.arange(1500))
    g = geer.Gaussians.from_scene(scene)
    npix = sum(c.pixels for c in cams)
    target = _target(npix, 7)
    ws = geer.Workspace(cams, scene.n, scene.sh_degree, 1_000_000)
    sep = _separate(geer, ws, g, target, npix)
    fus = _fused(geer, ws, g, target, npix)
    _check_equal(sep, fus)
    # the fused gradient against the FP64 oracle's, for the L1 gradient the kernel wrote
    dL = fus[2].cpu().numpy().astype(np.float64)
    ref, off = None, 0
    for cam in cams:
        gr = orc.render_grad(scene, cam, wl.all_pixels(cam), dL[off:off + cam.pixels])
        off += cam.pixels
        ref = gr if ref is None else {k: ref[k] + gr[k] for k in ref}
    for k in BLOCKS:
        a, b = fus[5][k].cpu().numpy().astype(np.float64).ravel(), ref[k].ravel()
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        mx = np.abs(a - b).max() / np.abs(b).max()
        assert rel <= 1e-3 and mx <= 1e-3, (name, k, rel, mx)


def test_fused_walks_past_the_hit_record_and_checkpoints(geer):
    """3000 faint Gaussians stacked on the axis of a 16x16 pinhole: the centre
    rays composite ~2270 entries, past the hit record and eight checkpoints, so
    the queue holds nine units of the tile."""
    n = 3000
    rng = np.random.default_rng(11)
    mean = np.stack([rng.normal(0, 0.02, n), rng.normal(0, 0.02, n), rng.uniform(2.0, 5.0, n)], 1)
    scene = wl.Scene(mean.astype(np.float32), rng.uniform(0.9, 1.1, (n, 3)).astype(np.float32),
                     rng.standard_normal((n, 4)).astype(np.float32),
                     rng.uniform(0.00415, 0.00425, n).astype(np.float32),
                     rng.normal(0, 0.3, (n, 1, 3)).astype(np.float32), 0)
    cams = [wl.Camera(wl.PINHOLE, 16, 16, math.radians(10))]
    g = geer.Gaussians.from_scene(scene)
    target = _target(256, 12)
    ws = geer.Workspace(cams, scene.n, scene.sh_degree, 1_000_000)
    sep = _separate(geer, ws, g, target, 256)
    _, last, walk = ws.debug_render_state()
    assert walk[0, 1] > 2048
    fus = _fused(geer, ws, g, target, 256)
    _check_equal(sep, fus)


def test_fused_with_a_tile_mask_and_repeated(geer):
    """A part of a 2-way tile split (its target zero on the other part's
    pixels), then the whole image again, twice: the queue and its counters
    start afresh on every call."""
    from paper_2505_24053_gb300 import tilesplit
    scene = wl.cube_scene(20000, 7, 3)
    cams = [wl.Camera(wl.KANNALA_BRANDT, 160, 128, math.radians(190), k=wl.kb_coeffs(3))]
    g = geer.Gaussians.from_scene(scene)
    npix = cams[0].pixels
    target = _target(npix, 5)
    ws = geer.Workspace(cams, scene.n, scene.sh_degree, 4_000_000)
    split = tilesplit.TileSplit(ws, 1, 2)
    tm = split.masked_target(target)
    _check_equal(_separate(geer, ws, g, tm, npix), _fused(geer, ws, g, tm, npix))
    ws.set_tile_mask(None)
    sep = _separate(geer, ws, g, target, npix)
    _check_equal(sep, _fused(geer, ws, g, target, npix))
    _check_equal(sep, _fused(geer, ws, g, target, npix))


def test_fused_full_size_workload3(geer):
    """The 1M-Gaussian 190 deg fisheye workload of the bench: 4800 tiles, units
    published while the heaviest tiles still render."""
    scene = wl.config_scene(3)
    cams = wl.config_cameras(3)
    g = geer.Gaussians.from_scene(scene)
    npix = sum(c.pixels for c in cams)
    target = _target(npix, 3)
    r = geer.Renderer(cams, scene.n, scene.sh_degree)
    r.prepare(g)
    sep = _separate(geer, r.ws, g, target, npix)
    _check_equal(sep, _fused(geer, r.ws, g, target, npix))


def test_fused_errors(geer):
    scene = wl.cube_scene(500, 3, 0)
    cams = [wl.Camera(wl.PINHOLE, 32, 32, math.radians(60))]
    g = geer.Gaussians.from_scene(scene)
    ws = geer.Workspace(cams, scene.n, scene.sh_degree, 100_000)
    x = torch.zeros((cams[0].pixels, 3), device="cuda")
    with pytest.raises(geer.GeerError) as e:
        ws.render_train_l1(x, x.clone(), x.clone())  # before bin_sort
    assert e.value.status == geer.ERR_STATE


def test_fused_repeated_without_a_new_binning(geer):
    """The step's preprocess zeroes the accumulators and its binning resets the
    unit queue; a fused render that follows another render stage without a new
    preprocess or binning must reset them itself: the same results every time."""
    scene = wl.cube_scene(20000, 7, 3)
    cams = [wl.Camera(wl.KANNALA_BRANDT, 160, 128, math.radians(190), k=wl.kb_coeffs(3))]
    g = geer.Gaussians.from_scene(scene)
    npix = cams[0].pixels
    target = _target(npix, 8)
    ws = geer.Workspace(cams, scene.n, scene.sh_degree, 4_000_000)
    sep = _separate(geer, ws, g, target, npix)  # leaves the queue holding the separate backward's unit order
    runs = []
    for _ in range(2):  # twice after the same binning
        rgb, dL = torch.empty((npix, 3), device="cuda"), torch.empty((npix, 3), device="cuda")
        loss = torch.empty(1, device="cuda")
        ws.render_train_l1(target, rgb, dL, loss)
        acc = ws.grad_accumulators().clone()
        grads = _grads_like(g)
        ws.preprocess_bwd(g, grads, accumulate=False)
        torch.cuda.synchronize()
        assert ws.device_status()[0] == geer.OK
        runs.append((rgb, sep[1], dL, float(loss.item()), acc, grads))
    for run in runs:
        rgb, T, dL, loss, acc, grads = run
        assert torch.equal(rgb, sep[0]) and torch.equal(dL, sep[2])
        assert loss == pytest.approx(sep[3], rel=1e-5)
        assert _rel(acc, sep[4]) <= 1e-5
        for k in BLOCKS:
            assert _rel(grads[k], sep[5][k]) <= 1e-4, k
