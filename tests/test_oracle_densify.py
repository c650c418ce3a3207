"""Pins of the density-control oracle (oracle/densify.py): split children are
samples of their Gaussian, the classification on cases clearly on either side
of each threshold, the output bookkeeping (counts, copies, moments), the
statistics and the opacity reset."""
import math

import numpy as np

from oracle import densify as D
from oracle.training import GROUPS

HP = dict(grad_threshold=2e-4, clone_max_scale=0.05, min_opacity=0.005, max_scale=0.0)


def _raw(rng, n, deg=1):
    k = (deg + 1) ** 2
    return {"mean": rng.normal(0, 1, (n, 3)), "log_scale": rng.normal(-3, 0.7, (n, 3)),
            "quat": rng.normal(0, 1, (n, 4)), "logit_opacity": rng.normal(0, 2, n), "sh": rng.normal(0, 0.3, (n, k, 3))}


def _like(raw, rng=None):
    return {k: (rng.normal(0, 1, v.shape) if rng is not None else np.zeros_like(v)) for k, v in raw.items()}


def test_split_children_are_samples_of_the_gaussian():
    """Splitting one anisotropic, rotated Gaussian many times: the children's
    means have the Gaussian's mean and covariance R diag(s^2) R^T (Monte Carlo,
    4e4 children), their scales are s / 1.6 (3DGS: s / (0.8 N), N = 2)."""
    rng = np.random.default_rng(1)
    n = 20000
    q = rng.normal(0, 1, 4)
    s = np.array([0.3, 0.1, 0.05])
    raw = {"mean": np.tile([1.0, -2.0, 3.0], (n, 1)), "log_scale": np.tile(np.log(s), (n, 1)),
           "quat": np.tile(q, (n, 1)), "logit_opacity": np.full(n, 2.0), "sh": np.zeros((n, 1, 3))}
    accum, denom = np.full(n, 1.0), np.ones(n)
    z = rng.standard_normal((n, 2, 3))
    r2, m2, v2, act, a = D.apply(HP, raw, _like(raw), _like(raw), accum, denom, z)
    assert (a == D.SPLIT).all() and r2["mean"].shape == (2 * n, 3)
    R = D._rot(q)
    cov = np.cov(r2["mean"].T)
    want = R @ np.diag(s * s) @ R.T
    assert np.abs(cov - want).max() < 0.03 * s[0] ** 2
    assert np.abs(r2["mean"].mean(0) - [1.0, -2.0, 3.0]).max() < 4 * s[0] / math.sqrt(2 * n)
    assert np.allclose(np.exp(r2["log_scale"]) * 1.6, s)
    assert not any(m2[k].any() or v2[k].any() for k in GROUPS)


def test_classification_on_clear_cases():
    g_hi, g_lo = 3e-4, 1e-4
    cases = [  # (accum, denom, max scale, opacity) -> action
        (g_hi * 4, 4, 0.01, 0.5, D.CLONE), (g_hi * 4, 4, 0.2, 0.5, D.SPLIT), (g_lo * 4, 4, 0.2, 0.5, D.KEEP),
        (g_hi, 1, 0.01, 0.001, D.PRUNE), (0.0, 0, 0.01, 0.5, D.KEEP), (g_hi * 2, 2, 0.01, 0.004, D.PRUNE),
        (g_lo, 1, 0.03, 0.006, D.KEEP),
    ]
    log_scale = np.array([[math.log(c[2]), math.log(c[2]) - 1, math.log(c[2]) - 2] for c in cases])
    logit = np.array([math.log(c[3] / (1 - c[3])) for c in cases])
    act, near = D.classify(HP, log_scale, logit, [c[0] for c in cases], [c[1] for c in cases])
    assert list(act) == [c[4] for c in cases] and not near.any()
    big = dict(HP, max_scale=0.1)
    act2, _ = D.classify(big, log_scale, logit, [c[0] for c in cases], [c[1] for c in cases])
    assert list(act2) == [D.CLONE, D.PRUNE, D.PRUNE, D.PRUNE, D.KEEP, D.PRUNE, D.KEEP]


def test_outputs_bookkeeping():
    """Outputs in the originals' order: kept and cloned Gaussians with their
    moments, clones as identical copies with zero moments, split children in
    place of their parent; the count is the sum of the per-action outputs."""
    rng = np.random.default_rng(3)
    n = 500
    raw = _raw(rng, n)
    m, v = _like(raw, rng), _like(raw, rng)
    accum = rng.uniform(0, 8e-4, n)
    denom = rng.integers(0, 4, n).astype(np.float64)
    z = rng.standard_normal((n, 2, 3))
    r2, m2, v2, actv, act = D.apply(HP, raw, m, v, accum, denom, z)
    per = np.array([0, 1, 2, 2])[act]
    assert r2["mean"].shape[0] == per.sum() and len(set(act)) == 4
    off = np.concatenate([[0], np.cumsum(per)])
    for g in range(n):
        o = off[g]
        if act[g] in (D.KEEP, D.CLONE):
            for k in GROUPS:
                assert np.array_equal(r2[k][o], raw[k][g]) and np.array_equal(m2[k][o], m[k][g])
                assert np.array_equal(v2[k][o], v[k][g])
        if act[g] == D.CLONE:
            for k in GROUPS:
                assert np.array_equal(r2[k][o + 1], raw[k][g]) and not m2[k][o + 1].any() and not v2[k][o + 1].any()
        if act[g] == D.SPLIT:
            for i in range(2):
                for k in ("quat", "logit_opacity", "sh"):
                    assert np.array_equal(r2[k][o + i], raw[k][g])
                assert not any(m2[k][o + i].any() for k in GROUPS)
    assert np.allclose(actv["scale"], np.exp(r2["log_scale"]))
    assert np.allclose(actv["opacity"], 1 / (1 + np.exp(-r2["logit_opacity"])))


def test_statistics_and_opacity_reset():
    accum, denom = np.zeros(4), np.zeros(4)
    d = np.array([[3.0, 4.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 2.0], [5.0, 5.0, 5.0]])
    accum, denom = D.accumulate(accum, denom, d, [True, False, True, True])
    accum, denom = D.accumulate(accum, denom, 2 * d, [True, True, False, False])
    assert np.allclose(accum, [15.0, 2.0, 2.0, math.sqrt(75)]) and np.array_equal(denom, [2, 1, 1, 1])
    logit = np.array([-8.0, -4.6, 0.0, 3.0])  # logit(0.01) = -4.595
    cap = math.log(0.01 / 0.99)
    l2, m2, v2 = D.opacity_reset(logit, np.ones(4), np.ones(4))
    assert np.allclose(l2, [-8.0, -4.6, cap, cap]) and list(m2) == [1, 1, 0, 0] and list(v2) == [1, 1, 0, 0]
    assert np.allclose(1 / (1 + np.exp(-l2[2:])), 0.01)
