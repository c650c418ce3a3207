"""GPU parity of the splatting association modes (EWA, UT, each with and
without SnugBox) against the FP64 oracle (oracle/splat.py, pinned in
tests/test_oracle_splat.py), through the C ABI.

- Masks: the GPU's boxes are FP32, the oracle's FP64, so a tile may differ only
  where a box edge lies within delta of the tile's edge ray: the oracle's mask
  of the box shrunk by delta lies inside the GPU's mask, and the GPU's inside
  the oracle's mask of the box grown by delta (delta = 2e-5 rad + 1e-4 of the
  box's larger half-side). The GPU's per-item tile counts equal its masks'
  sizes exactly.
- Render and backward: on every tile whose association is the same under the
  shrunk and grown boxes, the pixels match the brute-force oracle render over
  that tile's associated Gaussians (within 2e-4 of an admissible result, as in
  the PBF forward tests), and the gradients of a loss on those pixels match the
  oracle's (relative L2 and max error 1e-3, as in the PBF backward tests).
- Splat alpha (the local-affine model): pixels within 2e-4 of the FP64 splat
  render (mean 1e-5) away from alpha_min / T_min decisions; its gradient within
  1e-3 (relative L2 and max) of the FP64 oracle gradient.
"""
import math

import numpy as np
import pytest
import torch

from paper_2505_24053_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def geer():
    from paper_2505_24053_gb300 import geer
    geer.lib()
    assert torch.cuda.is_available()
    return geer


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    return oracle


@pytest.fixture(scope="module")
def S():
    from oracle import splat
    return splat


def _scene(seed, n, deg, near_frac=0.1, spread=2.5):
    """Far Gaussians around the camera plus a share of near, large ones (whose
    boxes reach past 90 degrees and wrap)."""
    rng = np.random.default_rng(seed)
    n_near = int(n * near_frac)
    mean = rng.uniform(-spread, spread, (n, 3))
    mean[:n_near] = rng.normal(0, 0.5, (n_near, 3)) + (0, 0, 0.7)
    log_s = rng.normal(-1.8, 0.5, (n, 3))
    log_s[:n_near] = rng.normal(-1.0, 0.3, (n_near, 3))
    quat = rng.standard_normal((n, 4))
    opacity = 1 / (1 + np.exp(-rng.normal(0.5, 1.5, n)))
    sh = rng.normal(0, 0.3, (n, (deg + 1) ** 2, 3))
    return wl.Scene(mean.astype(np.float32), np.exp(log_s).astype(np.float32), quat.astype(np.float32),
                    opacity.astype(np.float32), sh.astype(np.float32), deg)


def _delta(boxes):
    return np.array([0.0 if b is None else 2e-5 + 1e-4 * max(b[1] - b[0], b[3] - b[2]) * 0.5 for b in boxes])


MODES = [("ewa", 1, False), ("ewa_snug", 1, True), ("ut", 2, False), ("ut_snug", 2, True)]
_R, _t = wl.pose(wl.rot_y(math.radians(25)) @ wl.rot_x(math.radians(-10)), (0.3, -0.2, 0.4))
MASK_CAMS = [
    ("pinhole90", wl.Camera(wl.PINHOLE, 150, 100, math.radians(90))),
    ("equi190_posed", wl.Camera(wl.EQUIDISTANT, 112, 96, math.radians(190), R_cw=_R, t_cw=_t)),
    ("equi200", wl.Camera(wl.EQUIDISTANT, 128, 120, math.radians(200))),
    ("kb190", wl.Camera(wl.KANNALA_BRANDT, 160, 120, math.radians(190), k=wl.kb_coeffs(3))),
]


@pytest.mark.parametrize("mname,mode,snug", MODES, ids=[m[0] for m in MODES])
@pytest.mark.parametrize("cname,cam", MASK_CAMS, ids=[c[0] for c in MASK_CAMS])
def test_splat_masks_match_oracle(geer, orc, S, cname, cam, mname, mode, snug):
    scene = _scene(len(cname) * 7 + mode, 1500, 1)
    r = geer.Renderer([cam], scene.n, scene.sh_degree, params=geer.params_c(assoc=mode, snugbox=snug))
    r.prepare(geer.Gaussians.from_scene(scene))
    _, _, ranges, counts = r.ws.debug_preprocess()
    got = orc.assoc_mask(cam, ranges).astype(bool)
    assert np.array_equal(got.reshape(scene.n, -1).sum(1), counts), "tile counts vs ranges"
    boxes = S.scene_boxes(cam, scene, mode, snug)
    d = _delta(boxes)
    lo = S.scene_masks(cam, boxes, -d)
    hi = S.scene_masks(cam, boxes, d)
    miss = (lo & ~got).reshape(scene.n, -1).any(1)
    extra = (got & ~hi).reshape(scene.n, -1).any(1)
    assert not miss.any(), (cname, mname, np.flatnonzero(miss)[:5])
    assert not extra.any(), (cname, mname, np.flatnonzero(extra)[:5])
    live = np.array([b is not None for b in boxes])
    assert live.sum() > scene.n // 4 and got.sum() > 2 * scene.n




def _tiles(cam):
    for cy in range((cam.height + 15) // 16):
        for cx in range((cam.width + 15) // 16):
            ii, jj = np.meshgrid(np.arange(16 * cx, min(16 * cx + 16, cam.width)),
                                 np.arange(16 * cy, min(16 * cy + 16, cam.height)))
            yield cx, cy, np.stack([ii.ravel(), jj.ravel()], 1).astype(np.int32)


RENDER_CASES = [
    ("pinhole_ewa", wl.Camera(wl.PINHOLE, 64, 48, math.radians(70), bg=(0.2, 0.3, 0.4)), 1, False),
    ("equi200_ut", wl.Camera(wl.EQUIDISTANT, 48, 48, math.radians(200)), 2, False),
    ("kb190_ewa_snug", wl.Camera(wl.KANNALA_BRANDT, 64, 48, math.radians(190), k=wl.kb_coeffs(3)), 1, True),
    ("pinhole_ut_snug", wl.Camera(wl.PINHOLE, 50, 37, math.radians(80)), 2, True),
]


@pytest.mark.parametrize("name,cam,mode,snug", RENDER_CASES, ids=[c[0] for c in RENDER_CASES])
def test_splat_render_and_backward_match_oracle(geer, orc, S, name, cam, mode, snug):
    scene = _scene(len(name), 400, 2, near_frac=0.03, spread=3.0)
    key = orc.replica(scene, cam)[1]  # depth keys: the splatting modes cull a superset of PBF's Gaussians
    boxes = S.scene_boxes(cam, scene, mode, snug)
    d = _delta(boxes)
    lo, hi = S.scene_masks(cam, boxes, -d), S.scene_masks(cam, boxes, d)
    r = geer.Renderer([cam], scene.n, scene.sh_degree, params=geer.params_c(assoc=mode, snugbox=snug))
    g = geer.Gaussians.from_scene(scene)
    rgb = r.forward(g)
    img = rgb.cpu().numpy().reshape(cam.height, cam.width, 3)
    rng = np.random.default_rng(3)
    dL = rng.normal(0, 1, (cam.height, cam.width, 3))
    ref = None
    checked = 0
    for cx, cy, pix in _tiles(cam):
        if (lo[:, cy, cx] != hi[:, cy, cx]).any():
            dL[pix[:, 1], pix[:, 0]] = 0.0  # an ambiguous tile: left out of both sides
            continue
        rep = ((~hi[:, cy, cx]).astype(np.uint8), key)
        out = orc.render_pixels(scene, cam, pix, rep=rep)
        ok, err, _, und = orc.match_pixels(img[pix[:, 1], pix[:, 0]].astype(np.float64), out, 2e-4,
                                           cond_limit=np.inf)
        assert ok.all() and und.sum() == 0, (name, cx, cy, err.max())
        gr = orc.render_grad(scene, cam, pix, dL[pix[:, 1], pix[:, 0]], rep=rep)
        ref = gr if ref is None else {k: ref[k] + gr[k] for k in ref}
        checked += pix.shape[0]
    assert checked >= cam.pixels // 2, (name, checked)
    grads = r.backward(g, torch.as_tensor(dL.reshape(-1, 3), dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    for k in ("mean", "scale", "quat", "opacity", "sh"):
        a = grads[k].cpu().numpy().astype(np.float64).ravel()
        b = ref[k].ravel()
        nb = np.linalg.norm(b)
        assert nb > 0, (name, k)
        assert np.linalg.norm(a - b) / nb <= 1e-3 and np.abs(a - b).max() <= 1e-3 * np.abs(b).max(), (name, k)


SPLAT_ALPHA_CASES = [
    ("pinhole_pbf", wl.Camera(wl.PINHOLE, 64, 48, math.radians(70), bg=(0.2, 0.3, 0.4)), 0),
    ("equi200_pbf", wl.Camera(wl.EQUIDISTANT, 64, 64, math.radians(200)), 0),
    ("kb190_ewa", wl.Camera(wl.KANNALA_BRANDT, 64, 48, math.radians(190), k=wl.kb_coeffs(3)), 1),
    ("equi190_posed_ut", wl.Camera(wl.EQUIDISTANT, 64, 64, math.radians(190), R_cw=_R, t_cw=_t), 2),
]


@pytest.mark.parametrize("name,cam,assoc", SPLAT_ALPHA_CASES, ids=[c[0] for c in SPLAT_ALPHA_CASES])
def test_splat_alpha_render_matches_oracle(geer, orc, S, name, cam, assoc):
    """The render-time splat alpha (GEER_ALPHA_SPLAT) with PBF association (the
    FP32 replica's, bit-exact) or EWA association (tiles where the delta
    sandwich is ambiguous left out): every pixel within 2e-4 of the FP64 splat
    render, mean error <= 1e-5, except pixels with an alpha or a transmittance
    within 1e-3 (relative) of alpha_min / T_min."""
    scene = _scene(len(name) + 11, 400, 2, near_frac=0.03, spread=3.0)
    _, key, ranges, _ = orc.replica(scene, cam)
    ty, tx = (cam.height + 15) // 16, (cam.width + 15) // 16
    if assoc == 0:
        mask = orc.assoc_mask(cam, ranges).astype(bool)
        amb = np.zeros((ty, tx), bool)
    else:
        boxes = S.scene_boxes(cam, scene, assoc, False)
        d = _delta(boxes)
        lo, mask = S.scene_masks(cam, boxes, -d), S.scene_masks(cam, boxes, d)
        amb = (lo != mask).any(0)
    r = geer.Renderer([cam], scene.n, scene.sh_degree, params=geer.params_c(assoc=assoc, alpha_model=geer.ALPHA_SPLAT))
    img = r.forward(geer.Gaussians.from_scene(scene)).cpu().numpy().astype(np.float64)
    pix = wl.all_pixels(cam)
    pix = pix[~amb[pix[:, 1] // 16, pix[:, 0] // 16]]
    ref, near = S.splat_render(scene, cam, pix, mask, key)
    err = np.abs(img.reshape(cam.height, cam.width, 3)[pix[:, 1], pix[:, 0]] - ref)[~near]
    assert near.sum() < 0.02 * len(pix) and len(err) > cam.pixels // 2, (name, near.sum(), len(err))
    assert err.max() <= 2e-4 and err.mean() <= 1e-5, (name, err.max(), err.mean())
    assert np.abs(ref - np.asarray(cam.bg)).max() > 0.2, name


SPLAT_GRAD_CASES = [
    ("pinhole_pbf", wl.Camera(wl.PINHOLE, 48, 40, math.radians(60), bg=(0.2, 0.3, 0.4))),
    ("kb190_posed_pbf", wl.Camera(wl.KANNALA_BRANDT, 48, 40, math.radians(190), k=wl.kb_coeffs(3), R_cw=_R, t_cw=_t)),
    ("equi200_pbf", wl.Camera(wl.EQUIDISTANT, 48, 48, math.radians(200))),
]


@pytest.mark.parametrize("name,cam", SPLAT_GRAD_CASES, ids=[c[0] for c in SPLAT_GRAD_CASES])
def test_splat_alpha_backward_matches_oracle(geer, orc, S, name, cam):
    """geer_render_bwd with the splat alpha (the training-time approximation)
    against the FP64 oracle gradient (pinned by finite differences): relative
    L2 and max error 1e-3 per parameter block, as for the exact backward; pixels
    with an alpha or transmittance within 1e-3 of alpha_min / T_min carry no
    loss gradient."""
    scene = _scene(len(name) + 21, 120, 1, near_frac=0.0, spread=2.0)
    _, key, ranges, _ = orc.replica(scene, cam)
    mask = orc.assoc_mask(cam, ranges).astype(bool)
    pix = wl.all_pixels(cam)
    _, near = S.splat_render(scene, cam, pix, mask, key)
    rng = np.random.default_rng(4)
    dL = rng.normal(0, 1, (len(pix), 3))
    dL[near] = 0.0
    ref = S.splat_render_grad(scene, cam, pix, mask, key, dL)
    r = geer.Renderer([cam], scene.n, scene.sh_degree, params=geer.params_c(alpha_model=geer.ALPHA_SPLAT))
    g = geer.Gaussians.from_scene(scene)
    r.forward(g)
    dev = torch.zeros((cam.pixels, 3), dtype=torch.float32, device="cuda")
    dev[torch.as_tensor(pix[:, 1] * cam.width + pix[:, 0], device="cuda")] = torch.as_tensor(dL, dtype=torch.float32,
                                                                                           device="cuda")
    grads = r.backward(g, dev)
    torch.cuda.synchronize()
    for k in ("mean", "scale", "quat", "opacity", "sh"):
        a = grads[k].cpu().numpy().astype(np.float64).ravel()
        b = ref[k].ravel()
        nb = np.linalg.norm(b)
        assert nb > 0, (name, k)
        rel, mx = np.linalg.norm(a - b) / nb, np.abs(a - b).max() / np.abs(b).max()
        assert rel <= 1e-3 and mx <= 1e-3, (name, k, rel, mx)


def test_training_with_the_splat_alpha(geer):
    """The training-time approximation: a scene trained with the splat alpha in
    both the forward and the backward still fits its target."""
    cam = wl.Camera(wl.PINHOLE, 64, 48, math.radians(70))
    rng = np.random.default_rng(8)
    n = 300
    mean = np.stack([rng.uniform(-1.5, 1.5, n), rng.uniform(-1.0, 1.0, n), rng.uniform(3, 5, n)], 1).astype(np.float32)
    log_s = rng.normal(-2.0, 0.3, (n, 3)).astype(np.float32)
    quat = rng.standard_normal((n, 4)).astype(np.float32)
    logit = rng.normal(1.0, 0.5, n).astype(np.float32)
    sh = rng.normal(0, 0.4, (n, 1, 3)).astype(np.float32)
    true = geer.Gaussians(mean, np.exp(log_s), quat, 1 / (1 + np.exp(-logit)), sh, 0)
    params = geer.params_c(alpha_model=geer.ALPHA_SPLAT)
    r = geer.Renderer([cam], n, 0, params=params)
    target = r.forward(true).clone()
    adam = geer.Adam(mean + rng.normal(0, 0.05, mean.shape).astype(np.float32), log_s, quat, logit - 1.0,
                     rng.normal(0, 0.4, sh.shape).astype(np.float32), 0, lr_mean=2e-3)
    losses = []
    for _ in range(80):
        rgb = r.forward(adam.gaussians)
        loss, dL = geer.l1_loss_grad(rgb, target)
        losses.append(float(loss))
        adam.step(r.backward(adam.gaussians, dL))
    assert losses[-1] < 0.6 * losses[0], (losses[0], losses[-1])
