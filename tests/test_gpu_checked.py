"""The checked build (libgeer_checked.so, GEER_CHECKED=1): the stand-in for a
memory checker on this GPU. Its bounds guards skip an out-of-range access and
record the first one (site and index) next to the device status word.

- Without violations it renders and differentiates exactly as libgeer.so.
- A tile index planted in the render schedule (geer_debug_set_render_order,
  host input) beyond the camera set's tiles is recorded by the forward's tile
  guard, the block is skipped and every other tile renders as before;
  libgeer.so refuses the same schedule on the host. The planted index stays
  within the workspace's tile capacity, so no access could leave the
  workspace's arrays even without the guard.
- The fused training render with the checked build: no violation on a
  normal step, and the planted schedule entry recorded and skipped there
  too, with the launch ending (its unit queue does not wait for the skipped
  tile).
"""
import math

import numpy as np
import pytest
import torch

from paper_2505_24053_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SITE_FWD_TILE = 1


@pytest.fixture(scope="module")
def libs():
    from paper_2505_24053_gb300 import geer
    plain, checked = geer.lib(), geer.lib(checked=True)
    assert plain.geer_checked_build() == 0 and checked.geer_checked_build() == 1
    return geer, plain, checked


SCENE = wl.cube_scene(3000, 5, 1)
BIG = wl.Camera(wl.PINHOLE, 128, 96, math.radians(60))          # 8 x 6 = 48 tiles of capacity
SMALL = wl.Camera(wl.EQUIDISTANT, 64, 48, math.radians(180))    # 4 x 3 = 12 tiles rendered


def _workspace(geer, L):
    ws = geer.Workspace([BIG], SCENE.n, SCENE.sh_degree, 1 << 20, library=L)
    ws.set_cameras([SMALL])
    g = geer.Gaussians.from_scene(SCENE)
    ws.preprocess(g)
    ws.bin_sort()
    return ws, g


def test_checked_build_matches_the_plain_build(libs):
    geer, plain, checked = libs
    out = {}
    for name, L in (("plain", plain), ("checked", checked)):
        ws, g = _workspace(geer, L)
        rgb = torch.empty((SMALL.pixels, 3), device="cuda")
        ws.render_fwd(rgb)
        w = torch.as_tensor(np.random.default_rng(3).normal(0, 1, (SMALL.pixels, 3)).astype(np.float32),
                            device="cuda")
        grads = {k: torch.empty_like(v) for k, v in (("mean", g.mean), ("scale", g.scale), ("quat", g.quat),
                                                     ("opacity", g.opacity), ("sh", g.sh))}
        ws.render_bwd(g, w, grads, accumulate=False)
        assert ws.device_status()[0] == geer.OK
        assert ws.bounds_violation() == (0, 0)
        out[name] = (rgb.cpu(), {k: v.cpu() for k, v in grads.items()})
    assert torch.equal(out["plain"][0], out["checked"][0])
    for k, a in out["plain"][1].items():
        b = out["checked"][1][k]
        assert float((a - b).abs().max()) <= 1e-5 * float(a.abs().max()) + 1e-12, k


def test_render_order_is_only_a_schedule(libs):
    geer, plain, _ = libs
    ws, _ = _workspace(geer, plain)
    rgb = torch.empty((SMALL.pixels, 3), device="cuda")
    ws.render_fwd(rgb)
    ref = rgb.clone()
    ws.set_render_order(np.random.default_rng(1).permutation(12))
    rgb.fill_(-1.0)
    ws.render_fwd(rgb)
    assert torch.equal(rgb, ref)


def test_planted_tile_index_is_recorded_and_skipped(libs):
    geer, plain, checked = libs
    order = np.arange(12, dtype=np.uint32)
    order[5] = 12 + 3  # beyond the 12 tiles rendered, within the 48 of capacity
    # libgeer.so refuses it on the host: nothing is launched
    ws, _ = _workspace(geer, plain)
    with pytest.raises(geer.GeerError) as e:
        ws.set_render_order(order)
    assert e.value.status == geer.ERR_ARG
    # libgeer_checked.so passes it to the device, whose guard records and skips it
    ws, _ = _workspace(geer, checked)
    rgb = torch.empty((SMALL.pixels, 3), device="cuda")
    ws.render_fwd(rgb)
    ref = rgb.clone().view(SMALL.height, SMALL.width, 3)
    ws.set_render_order(order)
    rgb.fill_(-1.0)
    ws.render_fwd(rgb)
    st, _ = ws.device_status()
    assert st == geer.ERR_BOUNDS
    assert ws.bounds_violation() == (SITE_FWD_TILE, 15)
    assert ws.bounds_violation() == (0, 0) and ws.device_status()[0] == geer.OK
    img = rgb.view(SMALL.height, SMALL.width, 3)
    skipped = torch.zeros((SMALL.height, SMALL.width), dtype=torch.bool, device="cuda")
    skipped[16:32, 16:32] = True  # tile 5 = (1, 1) of a 4-wide grid was taken out of the schedule
    assert torch.all(img[skipped] == -1.0)
    assert torch.equal(img[~skipped], ref[~skipped])


def test_checked_build_fused_render(libs):
    """The fused training render (forward, L1 gradient and the backward's render
    stage in one launch) records no violation and matches the plain build."""
    geer, plain, checked = libs
    target = torch.as_tensor(np.random.default_rng(4).uniform(0, 1, (SMALL.pixels, 3)).astype(np.float32),
                             device="cuda")
    out = {}
    for name, L in (("plain", plain), ("checked", checked)):
        ws, g = _workspace(geer, L)
        rgb, dL = torch.empty((SMALL.pixels, 3), device="cuda"), torch.empty((SMALL.pixels, 3), device="cuda")
        ws.render_train_l1(target, rgb, dL)
        grads = {k: torch.empty_like(v) for k, v in (("mean", g.mean), ("scale", g.scale), ("quat", g.quat),
                                                     ("opacity", g.opacity), ("sh", g.sh))}
        ws.preprocess_bwd(g, grads, accumulate=False)
        assert ws.device_status()[0] == geer.OK
        assert ws.bounds_violation() == (0, 0)
        out[name] = (rgb.cpu(), dL.cpu(), {k: v.cpu() for k, v in grads.items()})
    assert torch.equal(out["plain"][0], out["checked"][0]) and torch.equal(out["plain"][1], out["checked"][1])
    for k, a in out["plain"][2].items():
        b = out["checked"][2][k]
        assert float((a - b).abs().max()) <= 1e-4 * float(a.abs().max()) + 1e-12, k


def test_planted_tile_index_in_the_fused_render(libs):
    """The same planted schedule entry in the fused render: the guard records it,
    the block counts the tile as finished with no units, and the launch ends
    (the backward's queue never waits for the skipped tile)."""
    geer, _, checked = libs
    order = np.arange(12, dtype=np.uint32)
    order[5] = 12 + 3
    ws, g = _workspace(geer, checked)
    target = torch.zeros((SMALL.pixels, 3), device="cuda")
    rgb, dL = torch.full((SMALL.pixels, 3), -1.0, device="cuda"), torch.empty((SMALL.pixels, 3), device="cuda")
    ws.set_render_order(order)
    ws.render_train_l1(target, rgb, dL)
    torch.cuda.synchronize()
    st, _ = ws.device_status()
    assert st == geer.ERR_BOUNDS  # not ERR_TIMEOUT: the queue drained
    assert ws.bounds_violation() == (SITE_FWD_TILE, 15)
    img = rgb.view(SMALL.height, SMALL.width, 3)
    skipped = torch.zeros((SMALL.height, SMALL.width), dtype=torch.bool, device="cuda")
    skipped[16:32, 16:32] = True
    assert torch.all(img[skipped] == -1.0) and torch.all(img[~skipped] >= 0.0)
