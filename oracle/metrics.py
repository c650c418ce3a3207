"""Native-camera evaluation: image metrics and evaluation regions, FP64 numpy.

TEST INFRASTRUCTURE: imported only by the tests and the benchmark's checks; the
product path never imports it. Plain, slow definitions written from the
paper's evaluation protocol and the standard metric definitions:

- native_regions(cam): per native pixel 0 (central), 1 (peripheral) or 255 (no
  ray of the BEAP grid). Renders are reprojected to the native camera image for
  evaluation (Sec. 5, implementation details); the central part holds the rays
  whose BEAP angles satisfy |theta| <= w / (2 f_x) and |phi| <= h / (2 f_y), f the
  native focal length, the peripheral part the rest (App., central and
  peripheral regions of the ScanNet++ evaluation). The ray of each native pixel
  comes from the C oracle's inverse projection (App. E).
- ssim_map(x, y): structural similarity of two images in [0, 1] per pixel and
  channel (Wang et al. 2004, the form 3DGS-style training and evaluation use):
  local means, variances and covariance under an 11 x 11 Gaussian window
  (sigma 1.5, normalised to sum 1) with zero padding,
  SSIM = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)),
  C1 = 0.01^2, C2 = 0.03^2.
- region_metrics(pred, gt, regions, n): per region, the sum of squared errors
  over its pixels and channels, the sum over its pixels of the channel-mean
  SSIM and its pixel count; psnr(sse, count) = 10 log10(1 / MSE), MSE over the
  region's pixels and 3 channels.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as orc

WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def native_regions(cam) -> np.ndarray:
    """[h, w] uint8: 0 central, 1 peripheral, 255 without a ray in the BEAP grid."""
    dummy = np.zeros((cam.height, cam.width, 3), np.float32)
    _, uv = orc.remap_to_native(cam, dummy, coords=True)
    w, h = cam.width, cam.height
    fy = orc.fov_y(cam)
    f = orc.native_focal(cam)
    u, v = uv[..., 0], uv[..., 1]
    valid = np.isfinite(u) & (u >= -0.5) & (u <= w - 0.5) & (v >= -0.5) & (v <= h - 0.5)
    # the BEAP angles of the ray (the grid maps them linearly to (u, v))
    theta = (np.where(valid, u, 0.0) + 0.5 - 0.5 * w) / w * cam.fov_x
    phi = (np.where(valid, v, 0.0) + 0.5 - 0.5 * h) / h * fy
    central = (np.abs(theta) <= w / (2.0 * f)) & (np.abs(phi) <= h / (2.0 * f))
    out = np.full((h, w), 255, np.uint8)
    out[valid & central] = 0
    out[valid & ~central] = 1
    return out


def gaussian_window(size: int = WINDOW, sigma: float = SIGMA) -> np.ndarray:
    k = np.arange(size) - size // 2
    g = np.exp(-(k ** 2) / (2.0 * sigma ** 2))
    g = g / g.sum()
    return np.outer(g, g)


def local_sum(img: np.ndarray, win: np.ndarray) -> np.ndarray:
    """Sum of win-weighted neighbours of each pixel of a 2-D image, zero padding."""
    r = win.shape[0] // 2
    pad = np.pad(img, r)
    view = np.lib.stride_tricks.sliding_window_view(pad, win.shape)
    return np.einsum("ijkl,kl->ij", view, win)


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """[h, w, c] SSIM of two [h, w, c] images, per pixel and channel."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    win = gaussian_window()
    out = np.empty_like(x)
    for ch in range(x.shape[2]):
        a, b = x[..., ch], y[..., ch]
        mu_a, mu_b = local_sum(a, win), local_sum(b, win)
        s_aa = local_sum(a * a, win) - mu_a * mu_a
        s_bb = local_sum(b * b, win) - mu_b * mu_b
        s_ab = local_sum(a * b, win) - mu_a * mu_b
        out[..., ch] = ((2 * mu_a * mu_b + C1) * (2 * s_ab + C2)) / ((mu_a ** 2 + mu_b ** 2 + C1) * (s_aa + s_bb + C2))
    return out


def region_metrics(pred: np.ndarray, gt: np.ndarray, regions: np.ndarray | None, n: int) -> np.ndarray:
    """[n, 3]: (sum of squared errors, sum of channel-mean SSIM, pixel count) per region;
    regions None: every pixel in region 0."""
    pred = np.asarray(pred, np.float64)
    gt = np.asarray(gt, np.float64)
    h, w = pred.shape[:2]
    reg = np.zeros((h, w), np.int64) if regions is None else np.asarray(regions, np.int64)
    se = ((pred - gt) ** 2).sum(axis=2)
    ss = ssim_map(pred, gt).mean(axis=2)
    out = np.zeros((n, 3))
    for r in range(n):
        m = reg == r
        out[r] = (se[m].sum(), ss[m].sum(), m.sum())
    return out


def psnr(sse: float, count: float) -> float:
    return 10.0 * math.log10(1.0 / (sse / (3.0 * count)))
