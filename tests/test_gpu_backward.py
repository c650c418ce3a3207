"""GPU backward (render + preprocess stages) against the FP64 oracle gradient.

The oracle's analytic gradient is itself pinned to central finite differences
(tests/test_oracle_grad.py). Tolerance, per parameter block (mean, scale, quat,
opacity, sh): relative L2 error <= 1e-3 and max abs error <= 1e-3 x max |grad|
(FP32 arithmetic, order-nondeterministic atomics; a ray whose alpha_min or
T_min decision falls inside the FP32 rounding band may take the other branch).
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


def _scene(seed, n, deg, zlo=2.0, zhi=5.0, spread=1.2, log_s=-1.6):
    rng = np.random.default_rng(seed)
    mean = np.stack([rng.uniform(-spread, spread, n), rng.uniform(-spread, spread, n), rng.uniform(zlo, zhi, n)], 1)
    s = np.exp(rng.normal(log_s, 0.4, (n, 3)))
    quat = rng.standard_normal((n, 4))
    opacity = rng.uniform(0.05, 0.999, n)
    sh = rng.normal(0, 0.3, (n, (deg + 1) ** 2, 3))
    return wl.Scene(mean.astype(np.float32), s.astype(np.float32), quat.astype(np.float32),
                    opacity.astype(np.float32), sh.astype(np.float32), deg)


def _gpu_grads(geer, scene, cams, dLdC=None, target=None):
    r = geer.Renderer(cams, scene.n, scene.sh_degree)
    g = geer.Gaussians.from_scene(scene)
    rgb = r.forward(g)
    if target is not None:
        _, dL = geer.l1_loss_grad(rgb, torch.as_tensor(target, device="cuda").reshape(rgb.shape))
    else:
        dL = torch.as_tensor(dLdC, dtype=torch.float32, device="cuda")
    grads = r.backward(g, dL)
    torch.cuda.synchronize()
    return rgb.cpu().numpy(), dL.cpu().numpy(), {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}


def _oracle_grads(orc, scene, cams, dL):
    tot = None
    off = 0
    for cam in cams:
        pix = wl.all_pixels(cam)
        g = orc.render_grad(scene, cam, pix, dL[off:off + cam.pixels].astype(np.float64))
        off += cam.pixels
        tot = g if tot is None else {k: tot[k] + g[k] for k in tot}
    return tot


def _compare(gpu, ref, label):
    for k in BLOCKS:
        a, b = gpu[k].ravel(), ref[k].ravel()
        nb = np.linalg.norm(b)
        if nb == 0:
            assert np.abs(a).max() == 0, (label, k)
            continue
        rel = np.linalg.norm(a - b) / nb
        mx = np.abs(a - b).max() / np.abs(b).max()
        assert rel <= 1e-3 and mx <= 1e-3, (label, k, rel, mx)


CAMS = [
    ("pinhole", [wl.Camera(wl.PINHOLE, 40, 32, math.radians(70), bg=(0.3, 0.5, 0.7))]),
    ("kb190", [wl.Camera(wl.KANNALA_BRANDT, 48, 40, math.radians(190), k=wl.kb_coeffs(3))]),
    ("two_cams", [wl.Camera(wl.EQUIDISTANT, 36, 36, math.radians(180)),
                  wl.Camera(wl.PINHOLE, 30, 20, math.radians(50),
                            R_cw=wl.pose(wl.rot_y(0.3), (0.2, -0.1, 0.0))[0],
                            t_cw=wl.pose(wl.rot_y(0.3), (0.2, -0.1, 0.0))[1])]),
]


@pytest.mark.parametrize("name,cams", CAMS, ids=[c[0] for c in CAMS])
def test_backward_matches_oracle_tiny(geer, orc, name, cams):
    scene = _scene(len(name), 64, 2)
    pixels = sum(c.pixels for c in cams)
    dLdC = np.random.default_rng(5).normal(0, 1, (pixels, 3)).astype(np.float32)
    rgb, dL, g = _gpu_grads(geer, scene, cams, dLdC=dLdC)
    ref = _oracle_grads(orc, scene, cams, dL)
    _compare(g, ref, name)


@pytest.mark.parametrize("deg", [0, 1, 3])
@pytest.mark.parametrize("name,cams", CAMS[1:], ids=[c[0] for c in CAMS[1:]])
def test_backward_sh_degrees(geer, orc, name, cams, deg):
    """Every SH degree through the one-camera and the several-camera variants of
    the per-Gaussian backward."""
    scene = _scene(31 + deg, 48, deg)
    pixels = sum(c.pixels for c in cams)
    dLdC = np.random.default_rng(6 + deg).normal(0, 1, (pixels, 3)).astype(np.float32)
    rgb, dL, g = _gpu_grads(geer, scene, cams, dLdC=dLdC)
    ref = _oracle_grads(orc, scene, cams, dL)
    _compare(g, ref, f"{name}-deg{deg}")


def test_backward_beyond_the_hit_record(geer, orc):
    """Rays walking more than the 2048 list entries whose per-warp hit bytes the
    forward records: 3000 broad, faint Gaussians (alpha just above alpha_min)
    stacked on the axis of a 16x16 pinhole, so that the centre rays composite
    ~2270 of them before T falls below T_min. The backward evaluates every entry
    beyond the record. The walk is split into units at the forward's
    checkpoints (every ~256 entries from entry 192), each starting from the
    forward's own transmittance, so the reverse recovery T_i = T_(i+1) / (1 - a_i)
    runs over at most ~512 steps (relative error <= 512 * 3 * 2^-24 ~ 1e-4):
    the common 1e-3 tolerance holds."""
    n = 3000
    rng = np.random.default_rng(11)
    mean = np.stack([rng.normal(0, 0.02, n), rng.normal(0, 0.02, n), rng.uniform(2.0, 5.0, n)], 1)
    scale = rng.uniform(0.9, 1.1, (n, 3))  # anisotropic: the rotation matters
    scene = wl.Scene(mean.astype(np.float32), scale.astype(np.float32),
                     rng.standard_normal((n, 4)).astype(np.float32),
                     rng.uniform(0.00415, 0.00425, n).astype(np.float32),
                     rng.normal(0, 0.3, (n, 1, 3)).astype(np.float32), 0)
    cam = wl.Camera(wl.PINHOLE, 16, 16, math.radians(10))
    dLdC = np.random.default_rng(12).normal(0, 1, (cam.pixels, 3)).astype(np.float32)
    r = geer.Renderer([cam], scene.n, scene.sh_degree)
    g = geer.Gaussians.from_scene(scene)
    r.forward(g)
    _, last, walk = r.ws.debug_render_state()
    assert last.max() > 2048 and walk[0, 1] > 2048, (last.max(), walk[0])
    grads = r.backward(g, torch.as_tensor(dLdC, device="cuda"))
    torch.cuda.synchronize()
    gpu = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}
    ref = orc.render_grad(scene, cam, wl.all_pixels(cam), dLdC.astype(np.float64))
    for k in BLOCKS:
        a, b = gpu[k].ravel(), ref[k].ravel()
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        mx = np.abs(a - b).max() / np.abs(b).max()
        assert rel <= 1e-3 and mx <= 1e-3, (k, rel, mx)


def test_backward_workload3_subset_l1(geer, orc):
    """The workload-3 gradient check: 2048 Gaussians of the 1M scene, 64x64
    Kannala-Brandt 190 deg camera, L1 loss against the seeded target."""
    full = wl.config_scene(3)
    scene = full.subset(np.arange(2048))
    cam = wl.Camera(wl.KANNALA_BRANDT, 64, 64, math.radians(190), k=wl.kb_coeffs(3))
    target = wl.l1_target(cam, seed=3)
    rgb, dL, g = _gpu_grads(geer, scene, [cam], target=target)
    # the L1 gradient kernel
    diff = rgb.reshape(-1) - target.reshape(-1)
    assert np.array_equal(dL.reshape(-1), (np.sign(diff) / diff.size).astype(np.float32))
    ref = _oracle_grads(orc, scene, [cam], dL)
    _compare(g, ref, "workload3-subset")


def test_l1_loss_value(geer):
    rng = np.random.default_rng(2)
    a = torch.as_tensor(rng.uniform(0, 1, 3001).astype(np.float32), device="cuda")
    b = torch.as_tensor(rng.uniform(0, 1, 3001).astype(np.float32), device="cuda")
    loss, grad = geer.l1_loss_grad(a, b)
    assert float(loss) == pytest.approx(float((a - b).abs().mean()), rel=1e-5)


def test_autograd_and_accumulation(geer):
    scene = _scene(9, 128, 1)
    cam = wl.Camera(wl.EQUIDISTANT, 40, 40, math.radians(160))
    r = geer.Renderer([cam], scene.n, scene.sh_degree)
    params = [torch.tensor(x, device="cuda", requires_grad=True) for x in
              (scene.mean, scene.scale, scene.quat, scene.opacity, scene.sh)]
    rgb = geer.render(r, *params, sh_degree=scene.sh_degree)
    w = torch.randn_like(rgb)
    (rgb * w).sum().backward()
    g = geer.Gaussians.from_scene(scene)
    r2 = geer.Renderer([cam], scene.n, scene.sh_degree)
    r2.forward(g)
    direct = r2.backward(g, w)

    def close(a, b, k):
        # the float atomics sum in a run-dependent order: equal up to rounding
        # relative to the block's scale (an entry may itself be a cancelling sum)
        scale = float(b.abs().max())
        assert float((a - b).abs().max()) <= 1e-5 * scale + 1e-9, (k, float((a - b).abs().max()), scale)

    for p, k in zip(params, BLOCKS):
        close(p.grad, direct[k], k)
    # geer_render_bwd accumulates
    r2.backward(g, w, direct)
    for p, k in zip(params, BLOCKS):
        close(direct[k], 2 * p.grad, k)


def test_overwrite_writes_every_row(geer):
    """accumulate == 0 writes every gradient row (zeros where a Gaussian has no
    gradient: here the half behind the camera) and never reads the buffers (they
    start as NaN); equal to accumulating into zeros up to the atomics' order."""
    scene = _scene(21, 300, 3, zlo=-6.0, zhi=4.0)
    cam = wl.Camera(wl.PINHOLE, 48, 40, math.radians(80))
    r = geer.Renderer([cam], scene.n, scene.sh_degree)
    g = geer.Gaussians.from_scene(scene)
    rgb = r.forward(g)
    w = torch.randn_like(rgb)
    shapes = (("mean", g.mean), ("scale", g.scale), ("quat", g.quat), ("opacity", g.opacity), ("sh", g.sh))
    acc = {k: torch.zeros_like(v) for k, v in shapes}
    r.ws.render_bwd(g, w, acc, accumulate=True)
    out = {k: torch.full_like(v, float("nan")) for k, v in shapes}
    r.ws.render_bwd(g, w, out, accumulate=False)
    torch.cuda.synchronize()
    behind = torch.as_tensor(scene.mean[:, 2] < -3.0, device="cuda")  # beyond any extent
    assert int(behind.sum()) > 50
    for k in BLOCKS:
        a, b = out[k], acc[k]
        assert not torch.isnan(a).any(), k
        assert float(a[behind].abs().max()) == 0.0, k
        scale = float(b.abs().max())
        assert float((a - b).abs().max()) <= 1e-5 * scale + 1e-9, (k, float((a - b).abs().max()), scale)


def _sparse_dl(cams, per_cam, seed):
    rng = np.random.default_rng(seed)
    pixels = sum(c.pixels for c in cams)
    dL = np.zeros((pixels, 3), np.float32)
    picks, off = [], 0
    for ci, cam in enumerate(cams):
        pix = wl.random_pixels(cam, per_cam, seed + ci)
        rows = off + pix[:, 1] * cam.width + pix[:, 0]
        dL[rows] = rng.normal(0, 1, (per_cam, 3)).astype(np.float32)
        picks.append(pix)
        off += cam.pixels
    return dL, picks


@pytest.mark.parametrize("cfg,per_cam", [(3, 48), (5, 6)])
def test_backward_full_size_sampled_pixels(geer, orc, cfg, per_cam):
    """Full-size workloads 3 (1M Gaussians, KB 190) and 5 (6M, four 210 deg cameras)
    in the bench's launch configuration; dL/dC is non-zero on seeded sample
    pixels only, so the oracle's gradient over those pixels is the exact answer."""
    scene = wl.config_scene(cfg)
    cams = wl.config_cameras(cfg)
    dL, picks = _sparse_dl(cams, per_cam, 700 + cfg)
    _, _, g = _gpu_grads(geer, scene, cams, dLdC=dL)
    ref = None
    off = 0
    for cam, pix in zip(cams, picks):
        rows = off + pix[:, 1] * cam.width + pix[:, 0]
        gi = orc.render_grad(scene, cam, pix, dL[rows].astype(np.float64))
        ref = gi if ref is None else {k: ref[k] + gi[k] for k in ref}
        off += cam.pixels
    _compare(g, ref, f"workload{cfg}")



@pytest.mark.parametrize("cfg,n_tiles,per_tile", [(3, 32, 8), (5, 32, 8)])
def test_backward_heaviest_tiles_full_size(geer, orc, cfg, n_tiles, per_tile):
    """The backward on the full-size workloads' hardest rays: dL/dC is non-zero on
    256 rays of the tiles with the longest walks (and on any ray walking past the
    hit record), in the bench's launch configuration; the oracle's gradient over
    those rays is the exact answer, checked at the 1e-3 tolerance."""
    from heavy_pixels import heavy_pixels
    scene = wl.config_scene(cfg)
    cams = wl.config_cameras(cfg)
    r = geer.Renderer(cams, scene.n, scene.sh_degree)
    g = geer.Gaussians.from_scene(scene)
    r.forward(g)
    picks, walks, beyond = heavy_pixels(r.ws, cams, n_tiles, per_tile, seed=950 + cfg)
    assert sum(len(p) for p in picks) >= n_tiles * per_tile
    rng = np.random.default_rng(960 + cfg)
    dL = np.zeros((r.pixels, 3), np.float32)
    off, rows_all = 0, []
    for cam, pix in zip(cams, picks):
        rows = off + pix[:, 1] * cam.width + pix[:, 0]
        dL[rows] = rng.normal(0, 1, (len(rows), 3)).astype(np.float32)
        rows_all.append(rows)
        off += cam.pixels
    grads = r.backward(g, torch.as_tensor(dL, device="cuda"))
    torch.cuda.synchronize()
    gpu = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}
    ref = None
    for cam, pix, rows in zip(cams, picks, rows_all):
        if len(pix) == 0:
            continue
        gi = orc.render_grad(scene, cam, pix, dL[rows].astype(np.float64))
        ref = gi if ref is None else {k: ref[k] + gi[k] for k in ref}
    print(f"workload {cfg}: {sum(len(p) for p in picks)} rays of the {n_tiles} heaviest tiles "
          f"(walks {int(walks.min())}..{int(walks.max())}), {beyond} rays beyond the hit record")
    _compare(gpu, ref, f"workload{cfg}/heavy")
