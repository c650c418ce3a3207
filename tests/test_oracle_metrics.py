"""Pins of the evaluation oracle (oracle/metrics.py): closed forms of SSIM,
PSNR and the central / peripheral regions, independent of its own code."""
import math

import numpy as np
import pytest

from paper_2505_24053_gb300 import workloads as wl

from oracle import metrics as M


def _g1():
    k = np.arange(11) - 5
    g = np.exp(-(k ** 2) / (2 * 1.5 ** 2))
    return g / g.sum()


def test_window_is_a_normalised_symmetric_gaussian():
    win = M.gaussian_window()
    assert win.shape == (11, 11)
    assert abs(win.sum() - 1.0) < 1e-14
    assert np.allclose(win, win.T) and np.allclose(win, win[::-1, ::-1])
    # centre weight: 1 / (sum_k exp(-k^2 / 4.5))^2
    s = sum(math.exp(-(k * k) / 4.5) for k in range(-5, 6))
    assert abs(win[5, 5] - 1.0 / (s * s)) < 1e-15


def test_ssim_of_identical_images_is_one():
    x = np.random.default_rng(0).uniform(0, 1, (20, 17, 3))
    assert np.abs(M.ssim_map(x, x) - 1.0).max() < 1e-12


def test_ssim_of_constant_images_closed_form():
    """Constant images a and b: in the interior the variances vanish and
    SSIM = (2ab + C1) / (a^2 + b^2 + C1); at a corner the zero padding leaves a
    window mass m = (sum of the window's inner half)^2 inside, so mu = a m and
    s_ab = ab m (1 - m), which gives its own closed form."""
    h, w, a, b = 24, 21, 0.8, 0.3
    x = np.full((h, w, 3), a)
    y = np.full((h, w, 3), b)
    s = M.ssim_map(x, y)
    inner = (2 * a * b + M.C1) / (a * a + b * b + M.C1)
    assert np.abs(s[5:-5, 5:-5] - inner).max() < 1e-13
    m = _g1()[5:].sum() ** 2
    corner = ((2 * a * b * m * m + M.C1) * (2 * a * b * m * (1 - m) + M.C2)) / \
             (((a * a + b * b) * m * m + M.C1) * ((a * a + b * b) * m * (1 - m) + M.C2))
    for (i, j) in ((0, 0), (0, w - 1), (h - 1, 0), (h - 1, w - 1)):
        assert abs(s[i, j, 1] - corner) < 1e-13


def test_ssim_is_symmetric_and_at_most_one():
    rng = np.random.default_rng(1)
    x, y = rng.uniform(0, 1, (2, 15, 19, 3))
    a, b = M.ssim_map(x, y), M.ssim_map(y, x)
    assert np.abs(a - b).max() < 1e-14
    assert a.max() <= 1.0 + 1e-12


def test_ssim_matches_an_explicit_window_loop():
    """A few pixels by a direct double loop over the window (zero outside)."""
    rng = np.random.default_rng(2)
    x, y = rng.uniform(0, 1, (2, 13, 16, 3))
    g = _g1()
    s = M.ssim_map(x, y)
    for (i, j, ch) in ((0, 0, 0), (3, 7, 1), (12, 15, 2), (6, 2, 0)):
        sums = np.zeros(5)
        for di in range(-5, 6):
            for dj in range(-5, 6):
                ii, jj = i + di, j + dj
                if 0 <= ii < 13 and 0 <= jj < 16:
                    wgt = g[di + 5] * g[dj + 5]
                    a, b = x[ii, jj, ch], y[ii, jj, ch]
                    sums += wgt * np.array([a, b, a * a, b * b, a * b])
        ma, mb = sums[0], sums[1]
        va, vb, cab = sums[2] - ma * ma, sums[3] - mb * mb, sums[4] - ma * mb
        ref = ((2 * ma * mb + M.C1) * (2 * cab + M.C2)) / ((ma * ma + mb * mb + M.C1) * (va + vb + M.C2))
        assert abs(s[i, j, ch] - ref) < 1e-12


def test_psnr_of_a_constant_offset():
    gt = np.random.default_rng(3).uniform(0.2, 0.7, (9, 11, 3))
    for d in (0.1, 0.01, 1e-3):
        m = M.region_metrics(gt + d, gt, None, 1)[0]
        assert m[2] == 99
        assert abs(M.psnr(m[0], m[2]) - (-20.0 * math.log10(d))) < 1e-9


def test_region_metrics_split_by_region():
    rng = np.random.default_rng(4)
    x, y = rng.uniform(0, 1, (2, 10, 12, 3))
    reg = rng.integers(0, 3, (10, 12)).astype(np.uint8)
    reg[0, 0] = 255  # no region: counted nowhere
    per = M.region_metrics(x, y, reg, 3)
    whole = M.region_metrics(x, y, None, 1)[0]
    se = ((x - y) ** 2).sum(axis=2)
    assert per[:, 2].sum() == 119
    assert abs(per[:, 0].sum() + se[0, 0] - whole[0]) < 1e-12


def test_pinhole_pixels_are_all_central():
    """Pinhole: a pixel's BEAP angles are atan(u), atan(v) with |u| <= w / (2f),
    |v| <= h / (2f), and |atan t| < |t|: every pixel is central."""
    cam = wl.Camera(wl.PINHOLE, 40, 30, math.radians(70))
    assert np.all(M.native_regions(cam) == 0)


@pytest.mark.parametrize("fov", [150, 180, 200])
def test_equidistant_pixels_in_the_grid_are_all_central(fov):
    """Equidistant fisheye: the native focal maps fov_x / 2 to w / 2, so
    w / (2f) = fov_x / 2 and h / (2f) = fov_y / 2, the BEAP grid's own half
    angles: every pixel with a ray in the grid is central, and the middle row has
    rays in the grid; the split is symmetric under flips."""
    cam = wl.Camera(wl.EQUIDISTANT, 48, 37, math.radians(fov))
    reg = M.native_regions(cam)
    assert set(np.unique(reg)) <= {0, 255}
    assert np.all(reg[(cam.height - 1) // 2] == 0)
    assert np.array_equal(reg, reg[::-1]) and np.array_equal(reg, reg[:, ::-1])


def _kb(p, k):
    p2 = p * p
    return p * (1 + p2 * (k[0] + p2 * (k[1] + p2 * (k[2] + p2 * k[3]))))


def test_barrel_fisheye_middle_row_split():
    """Kannala-Brandt with barrel distortion (phi_d(phi) < phi): w / (2f) =
    phi_d(fov_x / 2) < fov_x / 2. A middle-row pixel at image radius u (focal
    units) has polar angle = BEAP theta = phi_d^-1(|u|); it is central exactly
    when that is <= phi_d(fov_x / 2). The inverse is taken here by bisection on
    the polynomial (not the oracle's inverse)."""
    k = (-0.06, 0.0, 0.0, 0.0)
    fov = math.radians(190)
    cam = wl.Camera(wl.KANNALA_BRANDT, 64, 49, fov, k=k)
    reg = M.native_regions(cam)
    f = (cam.width / 2) / _kb(fov / 2, k)
    bound = _kb(fov / 2, k)
    mid = (cam.height - 1) // 2
    for i in range(cam.width):
        u = abs(i + 0.5 - cam.width / 2) / f
        lo, hi = 0.0, fov / 2 + 0.2
        for _ in range(80):
            m = 0.5 * (lo + hi)
            lo, hi = (m, hi) if _kb(m, k) < u else (lo, m)
        theta = 0.5 * (lo + hi)
        if abs(theta - bound) < 1e-9:
            continue
        assert reg[mid, i] == (0 if theta <= bound else 1), (i, theta, bound, reg[mid, i])
    assert (reg == 1).any() and reg[mid, cam.width // 2] == 0
    assert np.array_equal(reg, reg[::-1]) and np.array_equal(reg, reg[:, ::-1])
