"""Training-step pieces (Algorithm 2 on synthetic scenes), FP64 numpy.

TEST INFRASTRUCTURE: imported only by the tests; the product path never
imports it. Plain definitions:

- native_to_beap(cam, native): the supervision of a BEAP render from a native
  camera image (BEAP ray sampling with ground-truth interpolation). Each BEAP
  pixel's ray d (its BEAP angles theta_i, phi_j, Sec. 3.3: d = (sin theta cos phi,
  cos theta sin phi, cos theta cos phi)) is projected into the native image
  (App. E, with the native intrinsics of the remap: square pixels, principal
  point at the centre, focal length f mapping fov_x / 2 to w / 2): pinhole
  (x, y) = f (d_x, d_y) / d_z for d_z > 0; fisheye, with the polar angle
  p = atan2(sqrt(d_x^2 + d_y^2), d_z), (x, y) = f p_d(p) (d_x, d_y) / sqrt(d_x^2 + d_y^2)
  (p_d the Kannala-Brandt polynomial, identity for equidistant) for p within the
  increasing branch of p_d. The pixel coordinate is (x + w/2, y + h/2) with pixel
  centres at integer + 1/2; the value is the bilinear interpolation of the
  native image at (x + w/2 - 1/2, y + h/2 - 1/2) (clamped to the image) when
  that point lies within half a pixel of it; otherwise the BEAP pixel has no
  supervision (valid 0).
- adam_gaussians(hp, raw, grad, m, v, step): one Adam step (Kingma and Ba) of
  the 3DGS parameterisation: mean, log-scale (scale = exp), quaternion,
  logit-opacity (opacity = sigmoid) and SH, each with its learning rate (SH
  degree-0 and higher coefficients apart). The renderer's gradients are with
  respect to the activated scale and opacity; the chain rule gives
  dL/dlog_scale = dL/dscale * scale and dL/dlogit = dL/dopacity * o (1 - o).
  m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
  p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as orc

GROUPS = ("mean", "log_scale", "quat", "logit_opacity", "sh")


PINHOLE, EQUIDISTANT, KANNALA_BRANDT = 0, 1, 2  # camera model codes (the ABI's)


def _kb_coeffs(cam):
    """The camera's distortion coefficients as the ABI holds them (FP32)."""
    if cam.model == KANNALA_BRANDT:
        return [float(np.float32(x)) for x in cam.k]
    return [0.0, 0.0, 0.0, 0.0]


def _pd(p, k):
    p2 = p * p
    return p * (1 + p2 * (k[0] + p2 * (k[1] + p2 * (k[2] + p2 * k[3]))))


def _phi_max(k, steps=4096):
    """End of the increasing branch of p_d on [0, pi]."""
    prev = 0.0
    for s in range(1, steps + 1):
        ph = math.pi * s / steps
        val = _pd(ph, k)
        if not val > prev:
            return math.pi * (s - 1) / steps
        prev = val
    return math.pi


def native_to_beap(cam, native: np.ndarray, coords: bool = False):
    """(beap [h, w, 3] float64, valid [h, w] uint8) of a native image [h, w, 3].
    With coords=True also the native coordinates (u, v) of each BEAP pixel's
    ray [h, w, 2] (NaN where the ray has no projection) and, for the fisheye
    models, the ray's angle off the axis minus the end of the invertible range
    [h, w] (NaN for the pinhole)."""
    w, h = cam.width, cam.height
    fx = cam.fov_x
    fy = orc.fov_y(cam)
    f = orc.native_focal(cam)
    pinhole = cam.model == PINHOLE
    k = _kb_coeffs(cam)
    pmax = None if pinhole else _phi_max(k)
    native = np.asarray(native, np.float64)
    out = np.zeros((h, w, 3))
    valid = np.zeros((h, w), np.uint8)
    uv = np.full((h, w, 2), np.nan)
    pmargin = np.full((h, w), np.nan)
    for j in range(h):
        ph = ((j + 0.5) / h - 0.5) * fy
        for i in range(w):
            th = ((i + 0.5) / w - 0.5) * fx
            d = np.array([math.sin(th) * math.cos(ph), math.cos(th) * math.sin(ph), math.cos(th) * math.cos(ph)])
            if pinhole:
                if not d[2] > 0:
                    continue
                x, y = f * d[0] / d[2], f * d[1] / d[2]
            else:
                rho = math.hypot(d[0], d[1])
                p = math.atan2(rho, d[2])
                pmargin[j, i] = p - pmax
                if p > pmax:
                    continue
                if rho > 0:
                    s = f * _pd(p, k) / rho
                    x, y = s * d[0], s * d[1]
                else:
                    x, y = 0.0, 0.0
            u, v = x + 0.5 * w - 0.5, y + 0.5 * h - 0.5
            uv[j, i] = (u, v)
            if not (-0.5 <= u <= w - 0.5 and -0.5 <= v <= h - 0.5):
                continue
            uc, vc = min(max(u, 0.0), w - 1.0), min(max(v, 0.0), h - 1.0)
            x0, y0 = min(int(uc), max(w - 2, 0)), min(int(vc), max(h - 2, 0))
            x1, y1 = min(x0 + 1, w - 1), min(y0 + 1, h - 1)
            ax, ay = uc - x0, vc - y0
            top = native[y0, x0] + ax * (native[y0, x1] - native[y0, x0])
            bot = native[y1, x0] + ax * (native[y1, x1] - native[y1, x0])
            out[j, i] = top + ay * (bot - top)
            valid[j, i] = 1
    if coords:
        return out, valid, uv, pmargin
    return out, valid


def adam_gaussians(hp: dict, raw: dict, grad: dict, m: dict, v: dict, step: int):
    """One Adam step; returns (raw', m', v', activated {scale, opacity}). grad holds
    the renderer's gradients (mean, scale, quat, opacity, sh)."""
    raw = {key: np.asarray(val, np.float64) for key, val in raw.items()}
    scale = np.exp(raw["log_scale"])
    opac = 1.0 / (1.0 + np.exp(-raw["logit_opacity"]))
    g = {"mean": np.asarray(grad["mean"], np.float64),
         "log_scale": np.asarray(grad["scale"], np.float64) * scale,
         "quat": np.asarray(grad["quat"], np.float64),
         "logit_opacity": np.asarray(grad["opacity"], np.float64) * opac * (1.0 - opac),
         "sh": np.asarray(grad["sh"], np.float64)}
    b1, b2, eps = hp["beta1"], hp["beta2"], hp["eps"]
    lr = {"mean": hp["lr_mean"], "log_scale": hp["lr_scale"], "quat": hp["lr_quat"],
          "logit_opacity": hp["lr_opacity"]}
    out_raw, out_m, out_v = {}, {}, {}
    for key in GROUPS:
        mm = b1 * np.asarray(m[key], np.float64) + (1 - b1) * g[key]
        vv = b2 * np.asarray(v[key], np.float64) + (1 - b2) * g[key] ** 2
        if key == "sh":
            rate = np.full(raw["sh"].shape, hp["lr_sh_rest"])
            rate[:, 0, :] = hp["lr_sh_dc"]
        else:
            rate = lr[key]
        step_ = rate * (mm / (1 - b1 ** step)) / (np.sqrt(vv / (1 - b2 ** step)) + eps)
        out_raw[key] = raw[key] - step_
        out_m[key], out_v[key] = mm, vv
    act = {"scale": np.exp(out_raw["log_scale"]), "opacity": 1.0 / (1.0 + np.exp(-out_raw["logit_opacity"]))}
    return out_raw, out_m, out_v, act
