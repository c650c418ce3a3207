"""GPU native-camera evaluation (evaluation regions and image metrics) against
the FP64 oracle (oracle/metrics.py, pinned in tests/test_oracle_metrics.py).

Regions: the GPU inverts each native pixel's ray in FP32 (Newton), the oracle
in FP64 (bisection); a pixel may only differ where its ray lies within rounding
of a region boundary (the central half angles or the BEAP grid's edge).
Metrics: FP32 window sums against FP64; squared errors and SSIM sums within
1e-5 relative (SSIM: 1e-5 per pixel), counts exact."""
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
def M():
    from oracle import metrics
    return metrics


def _oracle_angles(orc, cam):
    """(theta, phi, u, v) of each native pixel's ray in the oracle (NaN without a ray)."""
    _, uv = orc.remap_to_native(cam, np.zeros((cam.height, cam.width, 3), np.float32), coords=True)
    u, v = uv[..., 0], uv[..., 1]
    th = (u + 0.5 - 0.5 * cam.width) / cam.width * cam.fov_x
    ph = (v + 0.5 - 0.5 * cam.height) / cam.height * orc.fov_y(cam)
    return th, ph, u, v


CAMS = [
    ("pinhole", wl.Camera(wl.PINHOLE, 40, 30, math.radians(70))),
    ("equi180", wl.Camera(wl.EQUIDISTANT, 48, 37, math.radians(180))),
    ("equi200", wl.Camera(wl.EQUIDISTANT, 51, 40, math.radians(200))),
    ("kb190_barrel", wl.Camera(wl.KANNALA_BRANDT, 64, 49, math.radians(190), k=(-0.06, 0.0, 0.0, 0.0))),
    ("kb190_full", wl.Camera(wl.KANNALA_BRANDT, 1280, 960, math.radians(190), k=wl.kb_coeffs(3))),
]


@pytest.mark.parametrize("name,cam", CAMS, ids=[c[0] for c in CAMS])
def test_native_regions_match_oracle(geer, orc, M, name, cam):
    gpu = geer.native_regions(cam).cpu().numpy()
    ref = M.native_regions(cam)
    bad = np.nonzero(gpu != ref)
    # decided pixel by pixel: each disagreement lies within rounding of a boundary
    if bad[0].size:
        th, ph, u, v = _oracle_angles(orc, cam)
        f = orc.native_focal(cam)
        for j, i in zip(*bad):
            margin = min(abs(abs(th[j, i]) - cam.width / (2 * f)), abs(abs(ph[j, i]) - cam.height / (2 * f)),
                         abs(u[j, i] + 0.5), abs(u[j, i] - cam.width + 0.5), abs(v[j, i] + 0.5),
                         abs(v[j, i] - cam.height + 0.5))
            assert margin < 1e-4, (name, j, i, gpu[j, i], ref[j, i], margin)


@pytest.mark.parametrize("h,w", [(23, 37), (48, 64), (240, 320), (17, 5)])
def test_image_metrics_match_oracle(geer, M, h, w):
    rng = np.random.default_rng(h * 1000 + w)
    gt = rng.uniform(0, 1, (h, w, 3)).astype(np.float32)
    # a prediction correlated with the reference: SSIM well away from 0 and 1
    pred = np.clip(gt + rng.normal(0, 0.08, gt.shape), 0, 1).astype(np.float32)
    reg = rng.integers(0, 3, (h, w)).astype(np.uint8)
    reg[rng.uniform(0, 1, (h, w)) < 0.1] = 255
    res = geer.image_metrics(torch.as_tensor(pred, device="cuda"), torch.as_tensor(gt, device="cuda"),
                             torch.as_tensor(reg, device="cuda"), 3)
    ref = M.region_metrics(pred, gt, reg, 3)
    for r in range(3):
        assert res[r]["count"] == int(ref[r, 2])
        assert abs(res[r]["sse"] - ref[r, 0]) <= 1e-5 * ref[r, 0] + 1e-9, (r, res[r]["sse"], ref[r, 0])
        assert abs(res[r]["ssim_sum"] - ref[r, 1]) <= 1e-5 * ref[r, 2], (r, res[r]["ssim_sum"], ref[r, 1])
        # PSNR and mean SSIM from the library: 10 log10(1 / MSE) and the mean (R20)
        assert res[r]["psnr"] == pytest.approx(10 * math.log10(3 * ref[r, 2] / ref[r, 0]), abs=1e-4)
        assert res[r]["ssim"] == pytest.approx(ref[r, 1] / ref[r, 2], abs=1e-5)


def test_image_metrics_identical_images(geer):
    x = torch.rand(50, 70, 3, device="cuda")
    (res,) = geer.image_metrics(x, x.clone())
    assert res["count"] == 3500 and res["sse"] == 0.0
    assert abs(res["ssim"] - 1.0) < 1e-6 and res["psnr"] == float("inf")


def test_evaluation_of_a_render_against_the_oracle(geer, orc, M):
    """End to end: the GEER BEAP render of a small scene reprojected to a barrel
    Kannala-Brandt 190 deg native image, evaluated per region against the
    oracle's own render reprojected by the oracle. The GPU metrics equal the
    oracle's metrics of the same two images, and the two pipelines agree to
    FP32 rounding (PSNR > 60 dB, SSIM > 0.9999 in both regions)."""
    cam = CAMS[3][1]
    rng = np.random.default_rng(8)
    n = 400
    mean = np.stack([rng.uniform(-3, 3, n), rng.uniform(-3, 3, n), rng.uniform(-1, 5, n)], 1)
    scene = wl.Scene(mean.astype(np.float32), np.exp(rng.normal(-1.4, 0.4, (n, 3))).astype(np.float32),
                     rng.standard_normal((n, 4)).astype(np.float32), rng.uniform(0.1, 0.95, n).astype(np.float32),
                     rng.normal(0, 0.3, (n, 4, 3)).astype(np.float32), 1)
    r = geer.Renderer([cam], scene.n, scene.sh_degree)
    rgb = r.forward(geer.Gaussians.from_scene(scene))
    pred = geer.remap_to_native(rgb.view(cam.height, cam.width, 3), cam)
    beap_ref = orc.render_pixels(scene, cam, wl.all_pixels(cam))["rgb"].reshape(cam.height, cam.width, 3)
    gt = orc.remap_to_native(cam, beap_ref.astype(np.float32))
    regions = geer.native_regions(cam)
    res = geer.image_metrics(pred, torch.as_tensor(gt.astype(np.float32), device="cuda"), regions, 2)
    ref = M.region_metrics(pred.cpu().numpy(), gt.astype(np.float32), regions.cpu().numpy(), 2)
    for k in range(2):
        assert res[k]["count"] == int(ref[k, 2]) > 0
        assert abs(res[k]["sse"] - ref[k, 0]) <= 1e-4 * ref[k, 0] + 1e-12
        assert abs(res[k]["ssim_sum"] - ref[k, 1]) <= 1e-5 * ref[k, 2]
        assert res[k]["psnr"] > 60.0 and res[k]["ssim"] > 0.9999, (k, res[k])
