"""Pin of the oracle's analytic gradients (App. C cookbook) against FP64 central
finite differences of the oracle's forward render.

Inputs are FP32, so each step h is a power of two that keeps x +- h exact. A
coordinate is skipped when the +-h renders take different discrete decisions
(contributor count, depth order, cull) or straddle a kink (alpha_max or colour
clamp); the number skipped is bounded. The central-difference error must shrink
like O(h^2) on a two-step ladder.
"""
import math

import numpy as np
import pytest

from paper_2505_24053_gb300 import workloads as wl


def _scene(seed, n=10, deg=2):
    rng = np.random.default_rng(seed)
    mean = np.stack([rng.uniform(-0.8, 0.8, n), rng.uniform(-0.6, 0.6, n), rng.uniform(3, 5, n)], 1)
    log_s = rng.normal(-1.3, 0.3, (n, 3))
    quat = rng.standard_normal((n, 4))
    opacity = rng.uniform(0.2, 0.999, n)
    opacity[0] = 0.9999  # alpha_max clamp somewhere
    nb = (deg + 1) ** 2
    sh = rng.normal(0, 0.4, (n, nb, 3))
    return wl.Scene(mean.astype(np.float32), np.exp(log_s).astype(np.float32), quat.astype(np.float32),
                    opacity.astype(np.float32), sh.astype(np.float32), deg)


def _loss_and_state(orc, scene, cam, pix, w):
    out = orc.render_pixels(scene, cam, pix)
    rep = orc.replica(scene, cam)
    return float((out["rgb"] * w).sum()), out["ncontrib"].copy(), np.argsort(rep[1], kind="stable"), rep[0].copy()


def _pow2_step(x, rel):
    # power of two near rel * max(1, |x|): x +- h is exact in FP32 for |x| >= its ulp scale
    return 2.0 ** math.floor(math.log2(rel * max(1.0, abs(float(x)))))


@pytest.mark.parametrize("seed", [1, 2])
def test_oracle_gradient_matches_central_differences(orc, seed):
    cam = wl.Camera(wl.KANNALA_BRANDT, 20, 16, math.radians(100), k=(0.01, -0.02, 0.005, 0.0),
                    bg=(0.3, 0.6, 0.9))
    scene = _scene(seed)
    pix = wl.all_pixels(cam)
    rng = np.random.default_rng(100 + seed)
    w = rng.normal(0, 1, (pix.shape[0], 3))
    g = orc.render_grad(scene, cam, pix, w)
    base_L, base_nc, base_ord, base_cull = _loss_and_state(orc, scene, cam, pix, w)

    fields = [("mean", scene.mean), ("scale", scene.scale), ("quat", scene.quat), ("opacity", scene.opacity),
              ("sh", scene.sh)]
    checked = skipped = 0
    worst = 0.0
    ladder = []
    for name, arr in fields:
        flat = arr.reshape(-1)
        gflat = g[name].reshape(-1)
        for idx in range(flat.size):
            x0 = flat[idx]
            h = _pow2_step(x0, 2.0 ** -11)
            vals = {}
            ok = True
            for sgn in (1, -1, 2, -2):
                flat[idx] = np.float32(float(x0) + math.copysign(h * (0.5 if abs(sgn) == 2 else 1.0), sgn))
                L, nc, ordr, cull = _loss_and_state(orc, scene, cam, pix, w)
                if not (np.array_equal(nc, base_nc) and np.array_equal(ordr, base_ord)
                        and np.array_equal(cull, base_cull)):
                    ok = False
                vals[sgn] = L
            flat[idx] = x0
            if not ok:
                skipped += 1
                continue
            fwd = (vals[1] - base_L) / h
            bwd = (base_L - vals[-1]) / h
            if abs(fwd - bwd) > 2e-2 * (abs(fwd) + abs(bwd)) + 1e-7:
                skipped += 1  # kink (clamp) between the two sides
                continue
            fd1 = (vals[1] - vals[-1]) / (2 * h)
            fd2 = (vals[2] - vals[-2]) / h
            an = gflat[idx]
            scale = max(1e-6, abs(an), abs(fd2))
            e1, e2 = abs(fd1 - an), abs(fd2 - an)
            assert e2 <= 2e-5 * scale + 1e-9, (name, idx, an, fd1, fd2)
            # O(h^2) ladder, where truncation (not round-off) dominates
            if e1 > 1e-6 * scale:
                ladder.append(e2 / e1)
            worst = max(worst, e2 / scale)
            checked += 1
    assert checked > 150 and skipped < 0.15 * (checked + skipped), (checked, skipped)
    ladder = np.array(ladder)
    assert ladder.size > 20 and np.mean(ladder < 0.4) > 0.9, (ladder.size, np.median(ladder))
