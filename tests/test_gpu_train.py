"""GPU training-step pieces against the FP64 oracle (oracle/training.py, pinned
in tests/test_oracle_training.py), and a synthetic training run.

Sampling: FP32 projection against FP64; a BEAP pixel's validity may only differ
where its point lies within 1e-3 px of the half-pixel edge of the native image
or its ray within 1e-5 rad of the end of the projection's invertible range
(decided pixel by pixel from the oracle's coordinates), values within 1e-3 on a
random image (position error x image gradient) and 1e-5 on a linear one.
Adam: FP32 against FP64, moments within 1e-5 relative, parameters within
1e-6 + 1e-5 relative."""
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
    return geer


@pytest.fixture(scope="module")
def T():
    from oracle import training
    return training


CAMS = [
    ("pinhole", wl.Camera(wl.PINHOLE, 41, 29, math.radians(65))),
    ("equi180", wl.Camera(wl.EQUIDISTANT, 48, 37, math.radians(180))),
    ("kb190", wl.Camera(wl.KANNALA_BRANDT, 64, 48, math.radians(190), k=wl.kb_coeffs(3))),
]


@pytest.mark.parametrize("name,cam", CAMS, ids=[c[0] for c in CAMS])
def test_native_to_beap_matches_oracle(geer, T, name, cam):
    rng = np.random.default_rng(len(name))
    native = rng.uniform(0, 1, (cam.height, cam.width, 3)).astype(np.float32)
    out, valid = geer.native_to_beap(torch.as_tensor(native, device="cuda"), cam)
    ref, rvalid, uv, pmargin = T.native_to_beap(cam, native, coords=True)
    out, valid = out.cpu().numpy(), valid.cpu().numpy()
    both = (valid == 1) & (rvalid == 1)
    # every pixel whose validity differs lies within FP32 rounding of a decision edge
    u, v = uv[..., 0], uv[..., 1]
    w, h = cam.width, cam.height
    with np.errstate(invalid="ignore"):
        edge_px = np.minimum.reduce([np.abs(u + 0.5), np.abs(u - (w - 0.5)), np.abs(v + 0.5),
                                     np.abs(v - (h - 0.5))])
    near = (np.nan_to_num(edge_px, nan=np.inf) <= 1e-3) | (np.abs(np.nan_to_num(pmargin, nan=np.inf)) <= 1e-5)
    differ = valid != rvalid
    assert not (differ & ~near).any(), (name, np.argwhere(differ & ~near)[:5])
    assert np.abs(out[both] - ref[both]).max() < 1e-3, name
    assert np.all(out[valid == 0] == 0.0)
    # exact on a linear image: only the FP32 position error remains
    jj, ii = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    lin = (0.004 * ii[..., None] + 0.003 * jj[..., None] + np.array([0.1, 0.2, 0.3])).astype(np.float32)
    out2, _ = geer.native_to_beap(torch.as_tensor(lin, device="cuda"), cam)
    ref2, _ = T.native_to_beap(cam, lin)
    assert np.abs(out2.cpu().numpy()[both] - ref2[both]).max() < 1e-5, name


def _dev(d):
    return {k: torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float32, device="cuda") for k, v in d.items()}


@pytest.mark.parametrize("n", [1000, 1001])  # 128-bit path (n % 4 == 0) and element path
def test_adam_step_matches_oracle(geer, T, n):
    rng = np.random.default_rng(7)
    deg = 3
    k = (deg + 1) ** 2
    raw = {"mean": rng.normal(0, 1, (n, 3)), "log_scale": rng.normal(-2, 0.5, (n, 3)), "quat": rng.normal(0, 1, (n, 4)),
           "logit_opacity": rng.normal(0, 1.5, n), "sh": rng.normal(0, 0.3, (n, k, 3))}
    raw = {key: v.astype(np.float32) for key, v in raw.items()}
    # the rates and betas as the ABI holds them (FP32): 1 - beta2 in FP32 differs
    # from 1 - 0.999 by 1.3e-5 relative
    hp = {kk: float(np.float32(vv)) for kk, vv in dict(geer.ADAM_DEFAULTS, lr_mean=1e-3, eps=1e-15).items()}
    adam = geer.Adam(raw["mean"], raw["log_scale"], raw["quat"], raw["logit_opacity"], raw["sh"], deg, **hp)
    zero = {key: np.zeros_like(v, np.float64) for key, v in raw.items()}
    ref_raw, ref_m, ref_v = {key: v.astype(np.float64) for key, v in raw.items()}, zero, dict(zero)
    for step in range(1, 4):
        grad = {"mean": rng.normal(0, 1, (n, 3)), "scale": rng.normal(0, 1, (n, 3)), "quat": rng.normal(0, 1, (n, 4)),
                "opacity": rng.normal(0, 1, n), "sh": rng.normal(0, 1, (n, k, 3))}
        grad = {key: v.astype(np.float32) for key, v in grad.items()}
        adam.step(_dev(grad))
        ref_raw, ref_m, ref_v, act = T.adam_gaussians(hp, ref_raw, grad, ref_m, ref_v, step)
    torch.cuda.synchronize()
    sizes = [3 * n, 3 * n, 4 * n, n, 3 * k * n]
    m = np.split(adam.m.cpu().numpy().astype(np.float64), np.cumsum(sizes)[:-1])
    v = np.split(adam.v.cpu().numpy().astype(np.float64), np.cumsum(sizes)[:-1])
    for idx, key in enumerate(T.GROUPS):
        got = adam.raw[key].cpu().numpy().astype(np.float64).ravel()
        want = ref_raw[key].ravel()
        assert np.all(np.abs(got - want) <= 1e-6 + 1e-5 * np.abs(want)), key
        assert np.all(np.abs(m[idx] - ref_m[key].ravel()) <= 1e-5 * np.abs(ref_m[key].ravel()) + 1e-7), key
        assert np.all(np.abs(v[idx] - ref_v[key].ravel()) <= 1e-5 * np.abs(ref_v[key].ravel()) + 1e-9), key
    assert np.allclose(adam.gaussians.scale.cpu().numpy(), act["scale"], rtol=1e-5, atol=1e-7)
    assert np.allclose(adam.gaussians.opacity.cpu().numpy(), act["opacity"], rtol=1e-5, atol=1e-7)


def test_training_reduces_the_loss(geer):
    """Algorithm 2 on a synthetic scene: the ground truth is the GEER render of a
    'true' scene reprojected to a native pinhole image, supervised back at the
    BEAP rays; a perturbed copy trained with L1 loss and Adam for 80 steps
    reaches well below its initial loss."""
    cam = wl.Camera(wl.PINHOLE, 64, 48, math.radians(70))
    rng = np.random.default_rng(3)
    n = 300
    mean = np.stack([rng.uniform(-1.5, 1.5, n), rng.uniform(-1.0, 1.0, n), rng.uniform(3, 5, n)], 1).astype(np.float32)
    log_s = rng.normal(-2.0, 0.3, (n, 3)).astype(np.float32)
    quat = rng.standard_normal((n, 4)).astype(np.float32)
    logit = rng.normal(1.0, 0.5, n).astype(np.float32)
    sh = rng.normal(0, 0.4, (n, 1, 3)).astype(np.float32)
    true = geer.Gaussians(mean, np.exp(log_s), quat, 1 / (1 + np.exp(-logit)), sh, 0)
    r = geer.Renderer([cam], n, 0)
    gt_beap = r.forward(true).clone()
    native = geer.remap_to_native(gt_beap.view(cam.height, cam.width, 3), cam)
    target, valid = geer.native_to_beap(native, cam)
    assert bool(valid.all())
    target = target.view(-1, 3)
    adam = geer.Adam(mean + rng.normal(0, 0.05, mean.shape).astype(np.float32), log_s, quat,
                     logit - 1.0, rng.normal(0, 0.4, sh.shape).astype(np.float32), 0, lr_mean=2e-3)
    losses = []
    for _ in range(80):
        rgb = r.forward(adam.gaussians)
        loss, dL = geer.l1_loss_grad(rgb, target)
        losses.append(float(loss))
        adam.step(r.backward(adam.gaussians, dL))
    assert losses[-1] < 0.6 * losses[0], (losses[0], losses[-1])


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    return oracle


@pytest.fixture(scope="module")
def DN():
    from oracle import densify
    return densify


def _moments(rng, n, k):
    return rng.normal(0, 1, n * (11 + 3 * k)).astype(np.float32), rng.uniform(0, 1, n * (11 + 3 * k)).astype(np.float32)


def _split_groups(flat, n, k):
    sizes = [3 * n, 3 * n, 4 * n, n, 3 * k * n]
    parts = np.split(np.asarray(flat, np.float64), np.cumsum(sizes)[:-1])
    shapes = [(n, 3), (n, 3), (n, 4), (n,), (n, k, 3)]
    return {key: p.reshape(s) for key, p, s in zip(("mean", "log_scale", "quat", "logit_opacity", "sh"), parts, shapes)}


@pytest.mark.parametrize("n,max_scale", [(3000, 0.0), (1001, 0.2)])  # ragged blocks; big-Gaussian pruning
def test_densify_matches_oracle(geer, DN, n, max_scale):
    """Plan and apply against the FP64 oracle: the same actions (FP32 decisions
    on both sides), kept and cloned rows and their moments bit for bit, clone
    copies and split children with zero moments, children's means within 1e-6
    (relative) and log-scales within 1e-6."""
    rng = np.random.default_rng(n)
    deg, k = 1, 4
    raw = {"mean": rng.normal(0, 1, (n, 3)), "log_scale": rng.normal(-3.5, 0.8, (n, 3)),
           "quat": rng.normal(0, 1, (n, 4)), "logit_opacity": rng.normal(-1, 3, n), "sh": rng.normal(0, 0.3, (n, k, 3))}
    raw = {key: v.astype(np.float32) for key, v in raw.items()}
    accum = rng.uniform(0, 1e-3, n).astype(np.float32)
    denom = rng.integers(0, 5, n).astype(np.float32)
    z = rng.standard_normal((n, 2, 3)).astype(np.float32)
    m, v = _moments(rng, n, k)
    hp = dict(grad_threshold=2e-4, clone_max_scale=0.03, min_opacity=0.005, max_scale=max_scale)
    act, near = DN.classify(hp, raw["log_scale"], raw["logit_opacity"], accum, denom)
    assert not near.any() and len(set(act.tolist())) == 4
    adam = geer.Adam(raw["mean"], raw["log_scale"], raw["quat"], raw["logit_opacity"], raw["sh"], deg)
    adam.m.copy_(torch.as_tensor(m))
    adam.v.copy_(torch.as_tensor(v))
    dev = lambda a: torch.as_tensor(a, device="cuda")
    no = adam.densify(dev(accum), dev(denom), dev(z), **hp)
    r2, m2, v2, actv, act2 = DN.apply(hp, raw, _split_groups(m, n, k), _split_groups(v, n, k), accum, denom, z)
    assert no == r2["mean"].shape[0] and np.array_equal(act, act2)
    torch.cuda.synchronize()
    got = {key: t.cpu().numpy().astype(np.float64) for key, t in adam.raw.items()}
    gm, gv = _split_groups(adam.m.cpu().numpy(), no, k), _split_groups(adam.v.cpu().numpy(), no, k)
    per = np.array([0, 1, 2, 2])[act]
    new = np.zeros(no, bool)  # rows whose parameters are computed (split children)
    off = np.concatenate([[0], np.cumsum(per)])
    new[off[:-1][act == DN.SPLIT]] = True
    new[off[:-1][act == DN.SPLIT] + 1] = True
    for key in got:
        same = ~new if key in ("mean", "log_scale") else np.ones(no, bool)
        assert np.array_equal(got[key][same], r2[key][same]), key
        assert np.array_equal(gm[key], m2[key]) and np.array_equal(gv[key], v2[key]), key
    assert np.all(np.abs(got["mean"][new] - r2["mean"][new]) <= 1e-6 * (1 + np.abs(r2["mean"][new])))
    assert np.all(np.abs(got["log_scale"][new] - r2["log_scale"][new]) <= 1e-6 * np.abs(r2["log_scale"][new]))
    assert np.allclose(adam.gaussians.scale.cpu().numpy(), actv["scale"], rtol=1e-6)
    assert np.allclose(adam.gaussians.opacity.cpu().numpy(), actv["opacity"], rtol=1e-6, atol=1e-7)


def test_densify_statistics_and_opacity_reset_match_oracle(geer, orc, DN):
    """geer_densify_accumulate adds |d_mean| for the Gaussians the preprocess
    associated with a tile (visibility from the FP32 replica's tile counts);
    geer_opacity_reset caps the logits and zeroes the changed moments."""
    cam = wl.Camera(wl.EQUIDISTANT, 96, 80, math.radians(180))
    rng = np.random.default_rng(11)
    n = 2000
    scene = wl.Scene(rng.uniform(-3, 3, (n, 3)).astype(np.float32),
                     np.exp(rng.normal(-2.5, 0.5, (n, 3))).astype(np.float32),
                     rng.standard_normal((n, 4)).astype(np.float32), rng.uniform(0.01, 0.99, n).astype(np.float32),
                     rng.normal(0, 0.3, (n, 1, 3)).astype(np.float32), 0)
    r = geer.Renderer([cam], n, 0)
    r.prepare(geer.Gaussians.from_scene(scene))
    visible = orc.replica(scene, cam)[3] > 0
    assert 0 < visible.sum() < n
    accum = torch.zeros(n, device="cuda")
    denom = torch.zeros(n, device="cuda")
    ref_a, ref_d = np.zeros(n), np.zeros(n)
    for step in range(2):
        d_mean = rng.normal(0, 1e-3, (n, 3)).astype(np.float32)
        geer.densify_accumulate(r.ws, torch.as_tensor(d_mean, device="cuda"), accum, denom)
        ref_a, ref_d = DN.accumulate(ref_a, ref_d, d_mean, visible)
    torch.cuda.synchronize()
    assert np.allclose(accum.cpu().numpy(), ref_a, rtol=1e-6, atol=0) and np.array_equal(denom.cpu().numpy(), ref_d)
    logit = rng.normal(-3, 3, n).astype(np.float32)
    adam = geer.Adam(scene.mean, np.log(scene.scale), scene.quat, logit, scene.sh, 0)
    m, v = _moments(rng, n, 1)
    adam.m.copy_(torch.as_tensor(m))
    adam.v.copy_(torch.as_tensor(v))
    adam.opacity_reset(0.01)
    l2, m_op, v_op = DN.opacity_reset(logit, m[10 * n:11 * n], v[10 * n:11 * n])
    torch.cuda.synchronize()
    assert np.allclose(adam.raw["logit_opacity"].cpu().numpy(), l2, rtol=1e-6, atol=1e-6)
    gm = adam.m.cpu().numpy()
    assert np.array_equal(gm[10 * n:11 * n], m_op.astype(np.float32)) and np.array_equal(gm[:10 * n], m[:10 * n])
    assert np.array_equal(adam.v.cpu().numpy()[10 * n:11 * n], v_op.astype(np.float32))
    assert np.allclose(adam.gaussians.opacity.cpu().numpy(), 1 / (1 + np.exp(-l2)), rtol=1e-5)


def test_training_with_densification(geer):
    """Algorithm 2 with refinement iterations: every 20 steps the Gaussians are
    densified from their view-space mean3D statistics (the threshold at the
    statistics' 80th percentile, so that some are cloned or split) and the
    renderer is rebuilt for the new count; the loss still falls well below its
    initial value and the count grows."""
    cam = wl.Camera(wl.PINHOLE, 64, 48, math.radians(70))
    rng = np.random.default_rng(5)
    n = 300
    mean = np.stack([rng.uniform(-1.5, 1.5, n), rng.uniform(-1.0, 1.0, n), rng.uniform(3, 5, n)], 1).astype(np.float32)
    log_s = rng.normal(-2.0, 0.3, (n, 3)).astype(np.float32)
    quat = rng.standard_normal((n, 4)).astype(np.float32)
    logit = rng.normal(1.0, 0.5, n).astype(np.float32)
    sh = rng.normal(0, 0.4, (n, 1, 3)).astype(np.float32)
    true = geer.Gaussians(mean, np.exp(log_s), quat, 1 / (1 + np.exp(-logit)), sh, 0)
    target = geer.Renderer([cam], n, 0).forward(true).clone()
    adam = geer.Adam(mean + rng.normal(0, 0.05, mean.shape).astype(np.float32), log_s, quat, logit - 1.0,
                     rng.normal(0, 0.4, sh.shape).astype(np.float32), 0, lr_mean=2e-3)
    r = geer.Renderer([cam], adam.n, 0)
    accum = torch.zeros(adam.n, device="cuda")
    denom = torch.zeros(adam.n, device="cuda")
    losses, counts = [], [adam.n]
    gen = torch.Generator(device="cuda").manual_seed(0)
    for it in range(1, 81):
        rgb = r.forward(adam.gaussians)
        loss, dL = geer.l1_loss_grad(rgb, target)
        losses.append(float(loss))
        grads = r.backward(adam.gaussians, dL)
        geer.densify_accumulate(r.ws, grads["mean"], accum, denom)
        adam.step(grads)
        if it % 20 == 0 and it < 80:
            avg = (accum / denom.clamp(min=1)).cpu().numpy()
            thr = float(np.quantile(avg[avg > 0], 0.8))
            z = torch.randn((adam.n, 2, 3), device="cuda", generator=gen)
            adam.densify(accum, denom, z, grad_threshold=thr, clone_max_scale=0.15, min_opacity=0.005)
            counts.append(adam.n)
            r = geer.Renderer([cam], adam.n, 0)
            accum = torch.zeros(adam.n, device="cuda")
            denom = torch.zeros(adam.n, device="cuda")
    assert counts[-1] > counts[0], counts
    assert losses[-1] < 0.6 * losses[0], (losses[0], losses[-1])


def test_densify_edge_cases(geer, DN):
    """No Gaussians; every Gaussian pruned (no outputs); every Gaussian split
    (twice as many, all moments zero)."""
    dev = lambda a: torch.as_tensor(np.asarray(a, np.float32), device="cuda")
    empty = geer.Adam(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 4)), np.zeros(0), np.zeros((0, 1, 3)), 0)
    assert empty.densify(dev(np.zeros(0)), dev(np.zeros(0)), dev(np.zeros((0, 2, 3)))) == 0
    rng = np.random.default_rng(2)
    n = 700
    mean, log_s, quat = rng.normal(0, 1, (n, 3)), np.full((n, 3), -1.0), rng.normal(0, 1, (n, 4))
    sh = rng.normal(0, 0.3, (n, 1, 3))
    pruned = geer.Adam(mean, log_s, quat, np.full(n, -9.0), sh, 0)
    assert pruned.densify(dev(np.ones(n)), dev(np.ones(n)), dev(rng.standard_normal((n, 2, 3)))) == 0
    assert pruned.gaussians.n == 0 and pruned.m.numel() == 0
    split = geer.Adam(mean, log_s, quat, np.full(n, 2.0), sh, 0)
    split.m.fill_(1.0)
    z = rng.standard_normal((n, 2, 3)).astype(np.float32)
    assert split.densify(dev(np.ones(n)), dev(np.ones(n)), dev(z), clone_max_scale=0.01) == 2 * n
    torch.cuda.synchronize()
    assert not split.m.any() and not split.v.any()
    raw = {"mean": mean, "log_scale": log_s, "quat": quat, "logit_opacity": np.full(n, 2.0), "sh": sh}
    raw = {k: v.astype(np.float32) for k, v in raw.items()}
    zero = {k: np.zeros_like(v) for k, v in raw.items()}
    r2, _, _, _, act = DN.apply(dict(geer.DENSIFY_DEFAULTS, clone_max_scale=0.01), raw, zero, zero, np.ones(n),
                                np.ones(n), z)
    assert (act == DN.SPLIT).all()
    got = split.raw["mean"].cpu().numpy()
    assert np.all(np.abs(got - r2["mean"]) <= 1e-6 * (1 + np.abs(r2["mean"])))
