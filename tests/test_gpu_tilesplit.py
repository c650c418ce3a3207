"""The tile split on one GPU: the parts of a partition of the tiles, rendered and
differentiated one after the other, must sum to the full step.

Each part renders only its tiles (zeros elsewhere) and its backward's render
stage sums only its tiles' rays; the sum of the parts' images is the full
image (bit for bit: every pixel is rendered by one part, identically), and the
sum of their accumulators, chained by the preprocess stage, is the full
gradient within the gradient tolerance (FP32 atomics sum in another order).
The processes of a multi-GPU run exchange exactly these accumulators."""
import math

import numpy as np
import pytest
import torch

from paper_2505_24053_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def env():
    from paper_2505_24053_gb300 import geer, tilesplit
    scene = wl.cube_scene(20000, 7, 3)
    R, t = wl.pose(wl.rot_y(0.3) @ wl.rot_x(-0.1), (0.2, -0.1, 0.4))
    cams = [wl.Camera(wl.KANNALA_BRANDT, 160, 128, math.radians(190), k=wl.kb_coeffs(3)),
            wl.Camera(wl.PINHOLE, 96, 72, math.radians(70), R_cw=R, t_cw=t, bg=(0.2, 0.3, 0.4))]
    return geer, tilesplit, scene, cams


def _grads(g):
    return {k: torch.empty_like(v) for k, v in (("mean", g.mean), ("scale", g.scale), ("quat", g.quat),
                                                 ("opacity", g.opacity), ("sh", g.sh))}


def _full(geer, scene, cams, g, target):
    ws = geer.Workspace(cams, scene.n, scene.sh_degree, 4_000_000)
    npix = sum(c.pixels for c in cams)
    rgb = torch.empty((npix, 3), device="cuda")
    T = torch.empty(npix, device="cuda")
    ws.preprocess(g)
    ws.bin_sort()
    ws.render_fwd(rgb, T)
    loss, dL = geer.l1_loss_grad(rgb, target)
    grads = _grads(g)
    ws.render_bwd_tiles(dL)
    acc = ws.grad_accumulators().clone()
    ws.preprocess_bwd(g, grads, accumulate=False)
    # the two stages equal the one-call backward (the same kernels; FP32 atomics
    # may sum in another order)
    one = _grads(g)
    ws.render_bwd(g, dL, one, accumulate=False)
    torch.cuda.synchronize()
    for k in one:
        assert _rel(one[k], grads[k]) <= 1e-5, k
    return ws, rgb, T, float(loss.item()), acc, grads


def _rel(a, b):
    a, b = a.double().ravel(), b.double().ravel()
    return float((a - b).norm() / max(float(b.norm()), 1e-30))


@pytest.mark.parametrize("world", [2, 3])
def test_tile_parts_sum_to_the_full_step(env, world):
    geer, tilesplit, scene, cams = env
    g = geer.Gaussians.from_scene(scene)
    npix = sum(c.pixels for c in cams)
    target = torch.as_tensor(np.random.default_rng(5).uniform(0, 1, (npix, 3)).astype(np.float32), device="cuda")
    ws_full, rgb_full, T_full, loss_full, acc_full, grads_full = _full(geer, scene, cams, g, target)

    ws = geer.Workspace(cams, scene.n, scene.sh_degree, 4_000_000)
    owners = geer.tile_owners(cams, world)
    pix_owner = torch.as_tensor(tilesplit.pixel_owners(cams, world), device="cuda")
    rgb_sum = torch.zeros_like(rgb_full)
    T_sum = torch.zeros_like(T_full)
    acc_sum = torch.zeros_like(acc_full)
    loss_sum = 0.0
    for part in range(world):
        split = tilesplit.TileSplit(ws, part, world)
        assert np.array_equal(split.pixel_mask.cpu().numpy() != 0, (pix_owner == part).cpu().numpy())
        rgb = torch.full_like(rgb_full, -7.0)
        T = torch.full_like(T_full, -7.0)
        ws.preprocess(g)
        ws.bin_sort()
        ws.render_fwd(rgb, T)
        own = pix_owner == part
        # this part's pixels as in the full render, the others zero
        assert torch.equal(rgb[own], rgb_full[own])
        assert torch.equal(T[own], T_full[own])
        assert torch.all(rgb[~own] == 0) and torch.all(T[~own] == 0)
        loss, dL = geer.l1_loss_grad(rgb, split.masked_target(target))
        assert torch.all(dL[~own] == 0)
        ws.render_bwd_tiles(dL)
        acc_sum += ws.grad_accumulators()
        rgb_sum += rgb
        T_sum += T
        loss_sum += float(loss.item())
        # only this part's rays were walked
        ev, last, walk = ws.debug_render_state()
        assert np.all(ev[~own.cpu().numpy()] == 0) and np.all(last[~own.cpu().numpy()] == 0)
        assert np.all(walk[owners != part] == 0)
    assert torch.equal(rgb_sum, rgb_full) and torch.equal(T_sum, T_full)
    assert loss_sum == pytest.approx(loss_full, rel=1e-5)
    assert _rel(acc_sum, acc_full) <= 1e-5
    # the summed accumulators in place of the last part's, then the preprocess stage
    ws.grad_accumulators().copy_(acc_sum)
    grads = _grads(g)
    ws.preprocess_bwd(g, grads, accumulate=False)
    torch.cuda.synchronize()
    for k in grads:
        assert _rel(grads[k], grads_full[k]) <= GRAD_TOL, k
        scale = float(grads_full[k].abs().max())
        assert float((grads[k] - grads_full[k]).abs().max()) <= GRAD_TOL * scale, k
    # clearing the mask renders every tile again
    ws.set_tile_mask(None)
    rgb = torch.empty_like(rgb_full)
    ws.render_fwd(rgb)
    assert torch.equal(rgb, rgb_full)


def test_tile_split_step_of_one_rank_is_the_full_step(env):
    geer, tilesplit, scene, cams = env
    g = geer.Gaussians.from_scene(scene)
    npix = sum(c.pixels for c in cams)
    target = torch.as_tensor(np.random.default_rng(6).uniform(0, 1, (npix, 3)).astype(np.float32), device="cuda")
    _, rgb_full, _, loss_full, _, grads_full = _full(geer, scene, cams, g, target)
    ws = geer.Workspace(cams, scene.n, scene.sh_degree, 4_000_000)
    split = tilesplit.TileSplit(ws, 0, 1)
    rgb, dL, grads = torch.empty_like(rgb_full), torch.empty_like(rgb_full), _grads(g)
    loss = split.step(g, split.masked_target(target), rgb, dL, grads)
    torch.cuda.synchronize()
    assert torch.equal(rgb, rgb_full)
    assert float(loss.item()) == pytest.approx(loss_full, rel=1e-6)
    for k in grads:
        assert _rel(grads[k], grads_full[k]) <= GRAD_TOL, k


def test_stage_errors(env):
    geer, tilesplit, scene, cams = env
    g = geer.Gaussians.from_scene(scene)
    ws = geer.Workspace(cams, scene.n, scene.sh_degree, 4_000_000)
    ws.preprocess(g)
    ws.bin_sort()
    with pytest.raises(geer.GeerError) as e:
        ws.preprocess_bwd(g, _grads(g))
    assert e.value.status == geer.ERR_STATE
    with pytest.raises(geer.GeerError) as e:
        ws.set_tile_mask(np.ones(3, np.uint8))  # not the camera set's tile count
    assert e.value.status == geer.ERR_ARG
