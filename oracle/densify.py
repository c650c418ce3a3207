"""Adaptive density control of the training loop (Algorithm 2, "Optimize" at
refinement iterations), FP64 numpy.

TEST INFRASTRUCTURE: imported only by the tests; the product path never
imports it.

The paper refines the Gaussians as 3DGS does, driven by the gradient of the
view-space mean3D instead of 3DGS's screen-space mean2D (App. G,
implementation details). Plain definitions:

- accumulate(accum, denom, d_mean, visible): for every Gaussian visible in the
  step's view (associated with at least one tile), accum += |dL/dmu_c| and
  denom += 1. mu_c = R_cw mu + t_cw is rigid, so |dL/dmu_c| = |dL/dmu|.
- classify(...): per Gaussian, with g = accum / denom (0 where denom = 0),
  s = exp(log-scale), sigma = sigmoid(logit):
    prune  (0 outputs)  sigma < min_opacity, or max_scale > 0 and max(s) > max_scale;
    clone  (2 outputs)  g >= grad_threshold and max(s) <= clone_max_scale;
    split  (2 outputs)  g >= grad_threshold and max(s) >  clone_max_scale;
    keep   (1 output)   otherwise.
  (3DGS densifies first and prunes the result, which prunes a low-opacity
  Gaussian's copies with it: the same set.)
- apply(...): the outputs in the originals' order, each original's outputs
  together. keep: the Gaussian and its Adam moments. clone: the Gaussian with
  its moments, then an identical copy with zero moments. split: two children
  with zero moments, child i (i = 0, 1) at mean + R(q) (s * z_i) (z_i ~ N(0, I),
  passed in), log-scale = log-scale - ln(1.6) (3DGS: s / (0.8 N), N = 2), the
  other parameters copied. The activated scale and opacity of the outputs are
  returned as well. The statistics restart at zero.
- opacity_reset(logit, m, v): logit <- min(logit, logit(0.01)), the opacity
  moments of the Gaussians whose logit changed restart at zero (3DGS).

Where floating point decides an integer (the action), the comparisons are
taken in FP32 on FP32 inputs, as the kernel takes them: g = accum / denom in
FP32, the largest log-scale against ln of the scale thresholds and the logit
against logit(min_opacity) (ln and logit of the FP32 parameters taken in FP64,
rounded to FP32). `near` marks Gaussians within 1e-5 (relative) of a threshold.
"""
from __future__ import annotations

import math

import numpy as np

from .training import GROUPS

PRUNE, KEEP, CLONE, SPLIT = 0, 1, 2, 3
SPLIT_LOG_SHRINK = math.log(1.6)


def accumulate(accum, denom, d_mean, visible):
    accum = np.asarray(accum, np.float64).copy()
    denom = np.asarray(denom, np.float64).copy()
    v = np.asarray(visible, bool)
    accum[v] += np.linalg.norm(np.asarray(d_mean, np.float64)[v], axis=1)
    denom[v] += 1.0
    return accum, denom


def _rot(q):
    q = np.asarray(q, np.float64)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def classify(hp: dict, log_scale, logit, accum, denom):
    """(action [n] in {PRUNE, KEEP, CLONE, SPLIT}, near [n])."""
    f = np.float32
    accum = np.asarray(accum, f)
    denom = np.asarray(denom, f)
    g = np.where(denom > 0, accum / np.where(denom > 0, denom, f(1)), f(0)).astype(f)
    ls_max = np.asarray(log_scale, f).max(axis=1)
    logit = np.asarray(logit, f)
    # thresholds: the FP32 parameters, their logs / logits taken in FP64 and rounded to FP32
    h32 = lambda key: float(f(hp[key]))
    thr_g = f(h32("grad_threshold"))
    lc = f(math.log(h32("clone_max_scale")))
    lo = f(math.log(h32("min_opacity") / (1.0 - h32("min_opacity"))))
    big = hp.get("max_scale", 0.0) > 0
    lb = f(math.log(h32("max_scale"))) if big else f(np.inf)
    prune = (logit < lo) | (big & (ls_max > lb))
    dens = g >= thr_g
    act = np.where(prune, PRUNE, np.where(dens, np.where(ls_max <= lc, CLONE, SPLIT), KEEP))
    rel = lambda a, b: np.abs(a.astype(np.float64) - float(b)) <= 1e-5 * max(abs(float(b)), 1e-30)
    near = rel(g, thr_g) | rel(ls_max, lc) | rel(logit, lo) | (big & rel(ls_max, lb))
    return act, near


def apply(hp: dict, raw: dict, m: dict, v: dict, accum, denom, z):
    """Densify and prune. raw / m / v: dicts over GROUPS (m, v shaped like raw);
    z: [n, 2, 3] standard normals. Returns (raw', m', v', activated
    {scale, opacity}, action)."""
    act, _ = classify(hp, raw["log_scale"], raw["logit_opacity"], accum, denom)
    raw = {k: np.asarray(raw[k], np.float64) for k in GROUPS}
    m = {k: np.asarray(m[k], np.float64) for k in GROUPS}
    v = {k: np.asarray(v[k], np.float64) for k in GROUPS}
    out = {k: [] for k in GROUPS}
    om = {k: [] for k in GROUPS}
    ov = {k: [] for k in GROUPS}

    def emit(src: dict, mm: dict | None, vv: dict | None, g: int):
        for k in GROUPS:
            out[k].append(src[k])
            om[k].append(np.zeros_like(raw[k][g]) if mm is None else mm[k][g])
            ov[k].append(np.zeros_like(raw[k][g]) if vv is None else vv[k][g])

    for g in range(len(act)):
        row = {k: raw[k][g] for k in GROUPS}
        if act[g] == PRUNE:
            continue
        if act[g] in (KEEP, CLONE):
            emit(row, m, v, g)
        if act[g] == CLONE:
            emit(row, None, None, g)
        if act[g] == SPLIT:
            s = np.exp(raw["log_scale"][g])
            R = _rot(raw["quat"][g])
            for i in range(2):
                child = dict(row)
                child["mean"] = raw["mean"][g] + R @ (s * np.asarray(z[g, i], np.float64))
                child["log_scale"] = raw["log_scale"][g] - SPLIT_LOG_SHRINK
                emit(child, None, None, g)
    shape = {k: raw[k].shape[1:] for k in GROUPS}
    stack = lambda lst, k: np.array(lst, np.float64).reshape((-1,) + shape[k])
    r2 = {k: stack(out[k], k) for k in GROUPS}
    m2 = {k: stack(om[k], k) for k in GROUPS}
    v2 = {k: stack(ov[k], k) for k in GROUPS}
    actv = {"scale": np.exp(r2["log_scale"]), "opacity": 1.0 / (1.0 + np.exp(-r2["logit_opacity"]))}
    return r2, m2, v2, actv, act


def opacity_reset(logit, m_op, v_op, value: float = 0.01):
    logit = np.asarray(logit, np.float64)
    cap = math.log(value / (1 - value))
    changed = logit > cap
    return np.minimum(logit, cap), np.where(changed, 0.0, m_op), np.where(changed, 0.0, v_op)
