"""GPU resampling of a BEAP image into the native camera image (App. E camera
models) against the FP64 oracle, through geer_remap_to_native.

Tolerance: the kernel finds each native pixel's ray and BEAP coordinate in
FP32. Its coordinate error is a few ulp of the coordinate (2e-3 px up to
2048 px) plus the direction's absolute error (<= 1e-6) times the conditioning
of the BEAP angles: theta = atan2(x, z) loses precision as x^2 + z^2 -> 0
(the poles at +-y, where every theta is the same ray) and phi = atan(y / z) as
y^2 + z^2 -> 0 (at +-x), so
  du = 2e-3 + w / FoV_x * 1e-6 / sqrt(x^2 + z^2),
  dv = 2e-3 + h / FoV_y * 1e-6 / sqrt(y^2 + z^2)      (unit direction),
and a colour may differ by max(du, dv) times the image's local slope (the
largest difference between neighbours around the sampled cell) plus 1e-5.
Pixels with max(du, dv) > 0.5 px (within about 1e-4 rad of a pole), where the
coordinate itself is ill-conditioned, must hold a value that bilinear
interpolation can produce within max(du, dv) + 1 px of the oracle's
coordinate (between the smallest and the largest BEAP value there). A pixel
may switch between fill and interpolation only where the oracle puts it within
max(du, dv) of the grid's edge or where it has no ray (the end of the
distortion's invertible range), and its value is then the fill colour or such
an interpolated value. Every pixel is decided on its own: no share of the
pixels is excused.
"""
import math

import numpy as np
import pytest
import torch

from paper_2505_24053_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FILL = (0.25, 0.5, 0.75)

CAMS = [
    ("pinhole70", wl.Camera(wl.PINHOLE, 320, 240, math.radians(70))),
    ("pinhole_odd", wl.Camera(wl.PINHOLE, 97, 61, math.radians(120))),
    ("equi200", wl.Camera(wl.EQUIDISTANT, 256, 256, math.radians(200))),
    ("equi180_wide", wl.Camera(wl.EQUIDISTANT, 300, 170, math.radians(180))),
    ("kb190", wl.Camera(wl.KANNALA_BRANDT, 320, 240, math.radians(190), k=wl.kb_coeffs(3))),
    ("kb150", wl.Camera(wl.KANNALA_BRANDT, 320, 240, math.radians(150), k=wl.kb_coeffs(44))),
    ("serving_equi1280", wl.Camera(wl.EQUIDISTANT, 1280, 1280, math.radians(200))),
]


@pytest.fixture(scope="module")
def geer():
    from paper_2505_24053_gb300 import geer
    geer.lib()
    return geer


def _local_slope(img):
    """Per cell (y, x): largest |difference| between the 3x3 neighbours' values."""
    h, w, _ = img.shape
    pad = np.pad(img.astype(np.float64), ((1, 2), (1, 2), (0, 0)), mode="edge")
    win = np.stack([pad[dy:dy + h, dx:dx + w] for dy in range(4) for dx in range(4)], 0)
    return (win.max(0) - win.min(0)).max(-1)


@pytest.mark.parametrize("name,cam", CAMS, ids=[c[0] for c in CAMS])
def test_remap_matches_oracle(geer, orc, name, cam):
    beap = wl.beap_image(cam, seed=len(name))
    ref, uv = orc.remap_to_native(cam, beap, fill=FILL, coords=True)
    out = geer.remap_to_native(torch.as_tensor(beap, device="cuda"), cam, fill=FILL)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    h, w = cam.height, cam.width
    u, v = uv[..., 0], uv[..., 1]
    has = np.isfinite(u)
    inside = has & (u >= -0.5) & (u <= w - 0.5) & (v >= -0.5) & (v <= h - 0.5)
    slope = _local_slope(beap)
    xs = np.clip(np.floor(np.nan_to_num(u)), 0, w - 1).astype(int)
    ys = np.clip(np.floor(np.nan_to_num(v)), 0, h - 1).astype(int)
    # BEAP direction of the oracle's coordinate (sin t cos p, cos t sin p, cos t cos p), normalised
    th = (np.nan_to_num(u) + 0.5 - w / 2) / w * np.float32(cam.fov_x)
    ph = (np.nan_to_num(v) + 0.5 - h / 2) / h * orc.fov_y(cam)
    norm = np.sqrt(np.cos(ph) ** 2 + (np.cos(th) * np.sin(ph)) ** 2)
    rho_x = np.abs(np.cos(ph)) / norm          # sqrt(x^2 + z^2)
    rho_y = np.abs(np.cos(th)) / norm          # sqrt(y^2 + z^2)
    with np.errstate(divide="ignore"):
        du = 2e-3 + w / np.float32(cam.fov_x) * 1e-6 / rho_x
        dv = 2e-3 + h / orc.fov_y(cam) * 1e-6 / rho_y
    delta = np.maximum(du, dv)
    pole = has & (delta > 0.5)
    tol = 1e-5 + delta * slope[ys, xs]
    err = np.abs(got - ref).max(-1)
    bad = (err > tol) & ~pole
    edge = (~has) | (np.minimum.reduce([np.abs(u + 0.5), np.abs(u - (w - 0.5)), np.abs(v + 0.5),
                                        np.abs(v - (h - 0.5))]) <= np.maximum(delta, 0.01))
    assert not (bad & ~edge).any(), (name, np.argwhere(bad & ~edge)[:5], err[bad & ~edge].max())

    def interpolable(j, i, radius):
        # a value bilinear interpolation can give near the oracle's coordinate
        x0, x1 = int(max(0, math.floor(u[j, i] - radius))), int(min(w - 1, math.ceil(u[j, i] + radius)))
        y0, y1 = int(max(0, math.floor(v[j, i] - radius))), int(min(h - 1, math.ceil(v[j, i] + radius)))
        win = beap[y0:y1 + 1, x0:x1 + 1].reshape(-1, 3).astype(np.float64)
        return x0 <= x1 and y0 <= y1 and np.all(got[j, i] >= win.min(0) - 1e-6) and np.all(
            got[j, i] <= win.max(0) + 1e-6)

    fill64 = np.float32(FILL).astype(np.float64)
    for j, i in np.argwhere(bad):  # edge pixels: the fill colour or an interpolated value
        if np.array_equal(got[j, i], fill64):
            continue
        assert has[j, i] and interpolable(j, i, min(delta[j, i], 4.0) + 1.0), (name, j, i, got[j, i])
    for j, i in np.argwhere(pole):  # ill-conditioned coordinate: an interpolated value near it
        assert np.array_equal(got[j, i], fill64) and not inside[j, i] or interpolable(
            j, i, min(delta[j, i], 4.0) + 1.0), (name, j, i, got[j, i], delta[j, i])
    # outside the BEAP grid: exactly the fill colour
    far = has & ~inside & ~edge & ~pole
    assert np.array_equal(got[far], np.broadcast_to(np.float32(FILL).astype(np.float64), got[far].shape))
    assert inside.sum() > 0.3 * cam.pixels


def test_remap_empty_and_bad_args(geer):
    cam = wl.Camera(wl.PINHOLE, 0, 0, math.radians(60))
    empty = torch.empty((0, 3), device="cuda")
    with pytest.raises(geer.GeerError):
        geer.remap_to_native(empty, cam)
    cam = wl.Camera(wl.PINHOLE, 16, 16, math.radians(200))   # pinhole beyond 180 deg
    img = torch.zeros((16, 16, 3), device="cuda")
    with pytest.raises(geer.GeerError):
        geer.remap_to_native(img, cam)
