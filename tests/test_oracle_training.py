"""Pins of the training-step oracle (oracle/training.py): ground-truth sampling
at BEAP rays against the C oracle's App. E projection, and Adam closed forms."""
import math

import numpy as np
import pytest

from paper_2505_24053_gb300 import workloads as wl

from oracle import oracle as orc
from oracle import training as T


def _beap_ray(cam, i, j):
    th = ((i + 0.5) / cam.width - 0.5) * cam.fov_x
    ph = ((j + 0.5) / cam.height - 0.5) * orc.fov_y(cam)
    return np.array([math.sin(th) * math.cos(ph), math.cos(th) * math.sin(ph), math.cos(th) * math.cos(ph)])


@pytest.mark.parametrize("cam", [wl.Camera(wl.PINHOLE, 21, 15, math.radians(60)),
                                 wl.Camera(wl.EQUIDISTANT, 24, 19, math.radians(160)),
                                 wl.Camera(wl.KANNALA_BRANDT, 26, 20, math.radians(170), k=(0.03, -0.01, 0.0, 0.0))],
                         ids=["pinhole", "equi160", "kb170"])
def test_linear_image_is_sampled_at_the_projection(cam):
    """On a native image linear in the pixel coordinates, bilinear interpolation
    is exact: each supervised BEAP pixel equals the linear function at the
    native point of its ray, taken from the C oracle's App. E projection
    (pixel centres at integer + 1/2)."""
    a, b, c = np.array([0.011, -0.004, 0.002]), np.array([0.003, 0.009, -0.006]), np.array([0.2, 0.5, 0.1])
    jj, ii = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    native = ii[..., None] * a + jj[..., None] * b + c
    beap, valid = T.native_to_beap(cam, native)
    checked = 0
    for j in range(cam.height):
        for i in range(cam.width):
            d = _beap_ray(cam, i, j)
            if d[2] <= 0:
                continue
            xp, yp = orc.project(cam, d)
            u, v = xp - 0.5, yp - 0.5
            if 0 <= u <= cam.width - 1 and 0 <= v <= cam.height - 1:
                assert valid[j, i] == 1
                assert np.abs(beap[j, i] - (u * a + v * b + c)).max() < 1e-12, (i, j)
                checked += 1
    assert checked > cam.pixels // 2


def test_centre_ray_samples_the_image_centre():
    cam = wl.Camera(wl.EQUIDISTANT, 25, 17, math.radians(150))
    native = np.random.default_rng(0).uniform(0, 1, (17, 25, 3))
    beap, valid = T.native_to_beap(cam, native)
    assert valid[8, 12] == 1 and np.abs(beap[8, 12] - native[8, 12]).max() < 1e-12


def _params(rng, n, deg):
    k = (deg + 1) ** 2
    raw = {"mean": rng.normal(0, 1, (n, 3)), "log_scale": rng.normal(-2, 0.5, (n, 3)),
           "quat": rng.normal(0, 1, (n, 4)), "logit_opacity": rng.normal(0, 1, n), "sh": rng.normal(0, 0.3, (n, k, 3))}
    grad = {"mean": rng.normal(0, 1, (n, 3)), "scale": rng.normal(0, 1, (n, 3)), "quat": rng.normal(0, 1, (n, 4)),
            "opacity": rng.normal(0, 1, n), "sh": rng.normal(0, 1, (n, k, 3))}
    return raw, grad


HP = {"lr_mean": 1e-3, "lr_scale": 5e-3, "lr_quat": 1e-3, "lr_opacity": 0.05, "lr_sh_dc": 2.5e-3,
      "lr_sh_rest": 2.5e-3 / 20, "beta1": 0.9, "beta2": 0.999, "eps": 0.0}


def test_adam_first_steps_move_each_parameter_by_its_rate():
    """With eps = 0 the bias-corrected first step is m^ / sqrt(v^) = g / |g|: each
    raw parameter moves by exactly -lr sign(g), the chain rule through exp and
    sigmoid keeping the sign; a gradient that stays the same keeps that step."""
    rng = np.random.default_rng(1)
    raw, grad = _params(rng, 7, 1)
    zero = {k: np.zeros_like(v) for k, v in raw.items()}
    r1, m1, v1, act = T.adam_gaussians(HP, raw, grad, zero, zero, 1)
    sign = {"mean": np.sign(grad["mean"]), "log_scale": np.sign(grad["scale"]), "quat": np.sign(grad["quat"]),
            "logit_opacity": np.sign(grad["opacity"]), "sh": np.sign(grad["sh"])}
    lr = {"mean": HP["lr_mean"], "log_scale": HP["lr_scale"], "quat": HP["lr_quat"], "logit_opacity": HP["lr_opacity"]}
    for key in lr:
        assert np.abs((raw[key] - r1[key]) - lr[key] * sign[key]).max() < 1e-12, key
    dsh = raw["sh"] - r1["sh"]
    assert np.abs(dsh[:, 0] - HP["lr_sh_dc"] * sign["sh"][:, 0]).max() < 1e-12
    assert np.abs(dsh[:, 1:] - HP["lr_sh_rest"] * sign["sh"][:, 1:]).max() < 1e-12
    assert np.allclose(act["scale"], np.exp(r1["log_scale"]))
    assert np.allclose(act["opacity"], 1 / (1 + np.exp(-r1["logit_opacity"])))
    # second step, the same gradient in the chain-ruled (raw) parameters: the same move
    raw_g = {"mean": grad["mean"], "log_scale": grad["scale"] * np.exp(raw["log_scale"]), "quat": grad["quat"],
             "logit_opacity": grad["opacity"] * (lambda s: s * (1 - s))(1 / (1 + np.exp(-raw["logit_opacity"]))),
             "sh": grad["sh"]}
    g2 = {"mean": raw_g["mean"], "scale": raw_g["log_scale"] / np.exp(r1["log_scale"]), "quat": raw_g["quat"],
          "opacity": raw_g["logit_opacity"] / ((lambda s: s * (1 - s))(1 / (1 + np.exp(-r1["logit_opacity"])))),
          "sh": raw_g["sh"]}
    r2, _, _, _ = T.adam_gaussians(HP, r1, g2, m1, v1, 2)
    for key in lr:
        assert np.abs((r1[key] - r2[key]) - lr[key] * sign[key]).max() < 1e-12, key


def test_adam_without_gradient_does_not_move():
    rng = np.random.default_rng(2)
    raw, grad = _params(rng, 5, 0)
    zero = {k: np.zeros_like(v) for k, v in raw.items()}
    g0 = {k: np.zeros_like(v) for k, v in grad.items()}
    r1, m1, v1, _ = T.adam_gaussians(dict(HP, eps=1e-15), raw, g0, zero, zero, 1)
    for key in raw:
        assert np.array_equal(r1[key], raw[key]) and not m1[key].any() and not v1[key].any()
