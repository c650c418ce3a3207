"""Pins of the splatting association bounds (oracle/splat.py): closed forms on
the optical axis, Monte Carlo moments of the true angle distribution, the
ellipse geometry of the boxes, and a per-ray brute force of the tile masks."""
import math

import numpy as np
import pytest

from paper_2505_24053_gb300 import workloads as wl

from oracle import oracle as orc
from oracle import splat as S

AMIN = 1.0 / 255.0


def _cam(model=wl.PINHOLE, w=64, h=48, fov=math.radians(70), **kw):
    return wl.Camera(model, w, h, fov, **kw)


def _quat_of(rng):
    q = rng.standard_normal(4)
    return q / np.linalg.norm(q)


@pytest.mark.parametrize("z,s", [(3.0, 0.1), (1.0, 0.25), (10.0, 0.02)])
def test_ewa_on_axis_isotropic(z, s):
    """On the axis J = I / z, so an isotropic Gaussian projects to variance s^2 / z^2
    in both angles, whatever its rotation: the 3DGS square has half-side 3 s / z
    and SnugBox sqrt(2 ln(sigma / alpha_min)) s / z."""
    cam = _cam()
    q = _quat_of(np.random.default_rng(1))
    box = S.splat_box(cam, (0, 0, z), (s, s, s), q, 0.8, S.EWA, False)
    assert np.allclose(box, (-3 * s / z, 3 * s / z, -3 * s / z, 3 * s / z), rtol=1e-12, atol=1e-15)
    e = math.sqrt(2 * math.log(0.8 / AMIN)) * s / z
    assert np.allclose(S.splat_box(cam, (0, 0, z), (s, s, s), q, 0.8, S.EWA, True), (-e, e, -e, e), rtol=1e-12)


@pytest.mark.parametrize("z,s", [(3.0, 0.1), (1.0, 0.25), (0.5, 0.14)])  # camera outside the contour
def test_ut_on_axis_isotropic(z, s):
    """Axis-aligned on the axis: the two sigma points along x sit at angles
    +-atan(sqrt(3) s / z), the rest at 0, so the mean angle is 0 and the variance
    2 / 6 atan(sqrt(3) s / z)^2: the square has half-side sqrt(3) atan(sqrt(3) s / z)
    (3 s / z for small s / z, the EWA value)."""
    cam = _cam()
    box = S.splat_box(cam, (0, 0, z), (s, s, s), (1, 0, 0, 0), 0.8, S.UT, False)
    e = math.sqrt(3.0) * math.atan(math.sqrt(3.0) * s / z)
    assert np.allclose(box, (-e, e, -e, e), rtol=1e-12, atol=1e-15)


def _angle_samples(cam, mu, scale, quat, n, seed):
    rng = np.random.default_rng(seed)
    mu_c, Rc = S.camera_frame(cam, mu)
    M = Rc @ S._rot(quat)
    t = mu_c + (rng.standard_normal((n, 3)) * np.asarray(scale)) @ M.T
    return np.stack([np.arctan2(t[:, 0], t[:, 2]), np.arctan2(t[:, 1], t[:, 2])], 1)


CASES = [((0.9, -0.5, 2.0), (0.03, 0.01, 0.02)), ((-1.4, 0.8, 1.5), (0.01, 0.04, 0.015)),
         ((2.5, 2.0, 0.8), (0.02, 0.005, 0.01))]


@pytest.mark.parametrize("mu,s", CASES)
def test_ewa_covariance_is_the_small_gaussian_limit(mu, s):
    """For a small Gaussian (s / |mu| ~ 1e-3) the angles of its samples are
    linear in the offset: their covariance is J Sigma_c J^T (Monte Carlo with
    4e5 samples, 1.5% on each entry relative to the larger diagonal)."""
    R_cw, t_cw = wl.pose(wl.rot_z(0.4), (0.1, -0.2, 0.05))
    cam = _cam(R_cw=R_cw, t_cw=t_cw)
    q = _quat_of(np.random.default_rng(len(mu)))
    scale = np.asarray(s) * 1e-1
    c, S2 = S.screen_cov(cam, mu, scale, q, S.EWA)
    a = _angle_samples(cam, mu, scale, q, 400000, 3)
    emp = np.cov(a.T)
    assert np.abs(emp - S2).max() < 0.015 * max(S2[0, 0], S2[1, 1])
    assert np.abs(a.mean(0) - c).max() < 3 * math.sqrt(max(S2[0, 0], S2[1, 1]) / 400000) + 1e-9


@pytest.mark.parametrize("mu,s", CASES)
def test_ut_moments_match_monte_carlo(mu, s):
    """At s / |mu| ~ 1e-2 the angle map is visibly nonlinear: the UT mean and
    covariance track the Monte Carlo moments of the true angle distribution
    (1e6 samples) closer than the linearised EWA moments do, and both converge
    to the same values as the Gaussian shrinks."""
    cam = _cam()
    q = _quat_of(np.random.default_rng(7 + len(mu)))
    scale = np.asarray(s) * 3.0
    cu, Su = S.screen_cov(cam, mu, scale, q, S.UT)
    ce, Se = S.screen_cov(cam, mu, scale, q, S.EWA)
    a = _angle_samples(cam, mu, scale, q, 1000000, 11)
    mc_mean, mc_cov = a.mean(0), np.cov(a.T)
    sd = math.sqrt(max(mc_cov[0, 0], mc_cov[1, 1]))
    assert np.abs(cu - mc_mean).max() < 0.01 * sd
    assert np.abs(cu - mc_mean).max() < np.abs(ce - mc_mean).max()
    assert np.abs(Su - mc_cov).max() < 0.03 * sd * sd
    small = np.asarray(s) * 1e-3
    cu2, Su2 = S.screen_cov(cam, mu, small, q, S.UT)
    ce2, Se2 = S.screen_cov(cam, mu, small, q, S.EWA)
    assert np.abs(Su2 - Se2).max() < 1e-4 * max(Se2[0, 0], Se2[1, 1])
    assert np.abs(cu2 - ce2).max() < 1e-3 * math.sqrt(max(Se2[0, 0], Se2[1, 1]))


@pytest.mark.parametrize("mode", [S.EWA, S.UT])
def test_boxes_bound_their_ellipses(mode):
    """SnugBox is the bounding box of the ellipse where sigma exp(-v^T Sigma_2^-1 v / 2)
    = alpha_min; the 3DGS square's half-side is 3 sqrt(max over unit u of
    u^T Sigma_2 u). Both checked on the ellipse / the unit circle traced densely."""
    cam = _cam(wl.EQUIDISTANT, 64, 64, math.radians(180))
    rng = np.random.default_rng(5)
    for _ in range(5):
        mu = rng.uniform(-1, 1, 3) + (0, 0, 2.5)
        s = rng.uniform(0.05, 0.4, 3)
        q = _quat_of(rng)
        sigma = rng.uniform(0.05, 0.99)
        c, S2 = S.screen_cov(cam, mu, s, q, mode)
        t = np.linspace(0, 2 * np.pi, 200001)
        L = np.linalg.cholesky(S2)
        v = (L @ np.stack([np.cos(t), np.sin(t)])) * math.sqrt(2 * math.log(sigma / AMIN))
        dens = sigma * np.exp(-0.5 * np.einsum("in,ij,jn->n", v, np.linalg.inv(S2), v))
        assert np.allclose(dens, AMIN, rtol=1e-9)
        snug = S.splat_box(cam, mu, s, q, sigma, mode, True)
        assert np.allclose([c[0] + v[0].min(), c[0] + v[0].max(), c[1] + v[1].min(), c[1] + v[1].max()], snug,
                           rtol=0, atol=1e-9 * (1 + abs(snug[1] - snug[0])))
        u = np.stack([np.cos(t), np.sin(t)])
        lam = np.einsum("in,ij,jn->n", u, S2, u).max()
        sq = S.splat_box(cam, mu, s, q, sigma, mode, False)
        assert math.isclose(sq[1] - c[0], 3 * math.sqrt(lam), rel_tol=1e-9)


def test_culling():
    cam = _cam()
    s, q = (0.1, 0.1, 0.1), (1, 0, 0, 0)
    for mode in (S.EWA, S.UT):
        small = (0.04, 0.04, 0.04)  # the camera outside the contour
        assert S.splat_box(cam, (0, 0, 0.2), small, q, 0.5, mode, False) is None
        assert S.splat_box(cam, (0, 0, 0.2000001), small, q, 0.5, mode, False) is not None
        assert S.splat_box(cam, (0, 0, -3), s, q, 0.5, mode, False) is None
        assert S.splat_box(cam, (0, 0, 3), s, q, 0.5 * AMIN, mode, False) is None
        assert S.splat_box(cam, (0, 0, 3), s, q, AMIN, mode, False) is None  # contour of radius 0
        assert S.splat_box(cam, (0, 0, 3), s, q, 1.01 * AMIN, mode, False) is not None
        # the camera inside the contour: culled as in the PBF pipeline (lambda = 3.2 here)
        assert S.splat_box(cam, (0, 0, 0.5), (0.2, 0.2, 0.2), q, 0.5, mode, False) is None
        assert S.splat_box(cam, (0, 0, 0.5), (0.1, 0.1, 0.1), q, 0.5, mode, False) is not None
        assert not S.box_mask(cam, None).any()


def test_camera_inside_matches_the_replica():
    """The FP64 camera-inside test takes the FP32 replica's decision away from
    the contour (|u|^2 / lambda^2 outside [0.999, 1.001])."""
    rng = np.random.default_rng(9)
    n = 400
    mean = rng.normal(0, 0.6, (n, 3)).astype(np.float32)
    scale = np.exp(rng.normal(-1.5, 0.5, (n, 3))).astype(np.float32)
    quat = rng.standard_normal((n, 4)).astype(np.float32)
    op = rng.uniform(0.01, 0.99, n).astype(np.float32)
    scene = wl.Scene(mean, scale, quat, op, np.zeros((n, 1, 3), np.float32), 0)
    cam = _cam()
    cull = orc.replica(scene, cam)[0]
    both = 0
    for g in range(n):
        mu_c, Rc = S.camera_frame(cam, mean[g])
        u = (Rc @ S._rot(quat[g])).T @ mu_c / scale[g].astype(np.float64)
        r = float(u @ u) / (2 * math.log(op[g] / AMIN) * 1.001)
        if abs(r - 1) < 1e-3:
            continue
        inside = S.camera_inside(cam, mean[g], scale[g], quat[g], float(op[g]))
        assert inside == bool(cull[g]), g
        both += inside
    assert 20 < both < n - 20


def test_meets_on_circle():
    assert S.meets_on_circle(0.1, 0.2, 0.15, 0.3)
    assert not S.meets_on_circle(0.1, 0.2, 0.25, 0.3)
    # wrapped: [3.0, 3.5] reaches -2.78
    assert S.meets_on_circle(-2.9, -2.8, 3.0, 3.5)
    assert not S.meets_on_circle(-2.7, -2.6, 3.0, 3.5)
    assert S.meets_on_circle(-1.0, -0.9, -7.0, -0.2 - 2 * math.pi + 2 * math.pi)
    assert S.meets_on_circle(5.0, 5.1, -100.0, 100.0)


def _pixel_mask(cam, box, grow):
    """Tiles holding a pixel whose ray's screen angles (atan2(x, z), atan2(y, z))
    lie in the box grown by `grow`, modulo 2 pi."""
    ty, tx = (cam.height + 15) // 16, (cam.width + 15) // 16
    m = np.zeros((ty, tx), bool)
    lo_t, hi_t, lo_p, hi_p = box[0] - grow, box[1] + grow, box[2] - grow, box[3] + grow
    for j in range(cam.height):
        for i in range(cam.width):
            _, d = orc.pixel_ray(cam, i, j)
            at, ap = math.atan2(d[0], d[2]), math.atan2(d[1], d[2])
            if S.meets_on_circle(at, at, lo_t, hi_t) and S.meets_on_circle(ap, ap, lo_p, hi_p):
                m[j // 16, i // 16] = True
    return m


@pytest.mark.parametrize("cam", [_cam(wl.PINHOLE, 70, 50, math.radians(90)),
                                 _cam(wl.EQUIDISTANT, 75, 61, math.radians(200), fov_y=math.radians(200))],
                         ids=["pinhole90", "equi200"])
def test_masks_against_per_ray_brute_force(cam):
    """Every tile with a ray inside the box is associated; every associated tile
    (away from the rows and columns where cos(angle) changes sign) has a ray
    within one pixel pitch of the box. Random Gaussians, some near and large
    enough that their boxes pass 90 degrees and wrap past pi."""
    rng = np.random.default_rng(21)
    fy = orc.fov_y(cam)
    pitch = max(cam.fov_x / cam.width, fy / cam.height) * 1.0001
    has0c, has1c = S.cos_flags(cam.width, cam.fov_x)
    has0r, has1r = S.cos_flags(cam.height, fy)
    clean = ~((has0r & has1r)[:, None] | (has0c & has1c)[None, :])
    checked = 0
    for k in range(24):
        near = k % 4 == 0
        mu = rng.normal(0, 0.6 if near else 1.5, 3) + (0, 0, 0.6 if near else 3.0)
        s = rng.uniform(0.2, 0.8, 3) if near else rng.uniform(0.05, 0.3, 3)
        for mode in (S.EWA, S.UT):
            box = S.splat_box(cam, mu, s, _quat_of(rng), 0.7, mode, k % 2 == 1)
            if box is None:
                continue
            mask = S.box_mask(cam, box)
            inner = _pixel_mask(cam, box, 0.0)
            outer = _pixel_mask(cam, box, pitch)
            assert not (inner & ~mask).any(), (k, mode)
            exact = S.box_mask(cam, box, one_interval=False)
            assert not (exact & ~mask).any(), (k, mode)  # one-interval filling only adds tiles
            assert not (exact & ~outer & clean).any(), (k, mode)
            checked += int(mask.sum())
    assert checked > 50


def _f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


@pytest.mark.parametrize("mu", [(0.8, -0.4, 3.0), (2.5, 1.0, 0.8), (-0.3, 2.2, 1.1)])
def test_splat_alpha_is_the_small_gaussian_limit_of_the_integral(mu):
    """The splat alpha linearises the angle map at the mean: for rays through a
    Gaussian (offsets up to ~2.5 sigma) it approaches the exact ray integral's
    alpha (the C oracle's kappa, pinned by quadrature) linearly in s / |mu|,
    the error shrinking tenfold for a tenfold smaller Gaussian."""
    cam = _cam(wl.EQUIDISTANT, 64, 64, math.radians(200))
    rng = np.random.default_rng(4)
    mu = _f32(mu)
    q = _f32(_quat_of(rng))
    M = S._rot(q)
    errs = []
    for sc in (1e-2, 1e-3, 1e-4):
        s = _f32(np.array([1.0, 0.5, 0.7]) * sc * np.linalg.norm(mu))
        e = 0.0
        for _ in range(150):
            t = mu + M @ (rng.normal(0, 1.2, 3) * s)
            d = t / np.linalg.norm(t)
            kap, _, _ = orc.kappa(mu, s, q, np.zeros(3), d)
            e = max(e, abs(S.splat_alpha(cam, mu, s, q, 0.8, d) - 0.8 * math.exp(-0.5 * kap)))
        errs.append(e)
    assert 5 < errs[0] / errs[1] < 20 and 5 < errs[1] / errs[2] < 20, errs
    assert errs[2] < 1e-4, errs


def _small_scene(k):
    """120 Gaussians 3-6 m ahead whose offsets and sizes scale with k, seen by a
    pinhole whose tan(FoV / 2) scales with k: the same image at every k, the
    angular sizes (and the linearisation error) proportional to k."""
    rng = np.random.default_rng(8)
    n = 120
    z = rng.uniform(3.0, 6.0, n)
    mean = np.stack([rng.uniform(-0.12, 0.12, n) * z * k, rng.uniform(-0.1, 0.1, n) * z * k, z], 1)
    scale = np.exp(rng.normal(0, 0.3, (n, 3))) * 0.006 * z[:, None] * k
    scene = wl.Scene(mean.astype(np.float32), scale.astype(np.float32), rng.standard_normal((n, 4)).astype(np.float32),
                     rng.uniform(0.2, 0.9, n).astype(np.float32), rng.normal(0, 0.5, (n, 4, 3)).astype(np.float32), 1)
    return scene, _cam(wl.PINHOLE, 48, 40, 2 * math.atan(k * math.tan(math.radians(8))))


def test_splat_render_converges_to_the_exact_render():
    """The splat render of a scene (PBF association from the FP32 replica)
    differs from the exact oracle's render (orc.render_pixels) only by the
    linearisation error: at angular sizes ~5e-3 rad by < 1e-2, and ten times
    smaller Gaussians (same image) cut the difference at least fivefold. A wrong
    depth order, compositing rule, colour or association would not vanish."""
    errs = []
    for k in (1.0, 0.1):
        scene, cam = _small_scene(k)
        cull, key, ranges, _ = orc.replica(scene, cam)
        mask = orc.assoc_mask(cam, ranges).astype(bool)
        pix = wl.all_pixels(cam)
        # pixels with an alpha within the models' difference (~0.05 k relative) of
        # alpha_min or T_min may take the other branch: left out
        got, near = S.splat_render(scene, cam, pix, mask, key, margin=0.05 * k)
        ref = orc.render_pixels(scene, cam, pix)["rgb"]
        assert np.abs(ref - np.asarray(cam.bg)).max() > 0.3  # the scene covers the image visibly
        assert near.sum() < 0.1 * len(pix)
        errs.append(np.abs(got - ref)[~near])
    assert errs[0].max() < 1e-2, errs[0].max()
    assert errs[1].max() < errs[0].max() / 5 and errs[1].mean() < errs[0].mean() / 5, \
        (errs[0].max(), errs[1].max(), errs[0].mean(), errs[1].mean())


def test_splat_render_gradient_matches_finite_differences():
    """The splat render's gradient (analytic compositing and splat, FP64 central
    differences for the parameter-to-splat map) equals central differences of
    the splat render itself, parameter by parameter, on a few Gaussians and
    pixels away from the alpha_min / T_min decisions."""
    cam = _cam(wl.PINHOLE, 32, 32, math.radians(30))
    rng = np.random.default_rng(12)
    n = 5
    z = rng.uniform(3.0, 4.0, n)
    mean = np.stack([rng.uniform(-0.15, 0.15, n) * z, rng.uniform(-0.15, 0.15, n) * z, z], 1)
    scale = np.exp(rng.normal(0, 0.3, (n, 3))) * 0.12
    scene = wl.Scene(mean.astype(np.float32), scale.astype(np.float32), rng.standard_normal((n, 4)).astype(np.float32),
                     rng.uniform(0.3, 0.8, n).astype(np.float32), rng.normal(0, 0.5, (n, 4, 3)).astype(np.float32), 1)
    cull, key, ranges, _ = orc.replica(scene, cam)
    mask = orc.assoc_mask(cam, ranges).astype(bool)
    pix = wl.random_pixels(cam, 40, 3)
    _, near = S.splat_render(scene, cam, pix, mask, key, margin=1e-2)
    pix = pix[~near]
    dLdC = rng.normal(0, 1, (len(pix), 3))
    got = S.splat_render_grad(scene, cam, pix, mask, key, dLdC)

    def loss(sc):
        rgb, _ = S.splat_render(sc, cam, pix, mask, key)
        return float((rgb * dLdC).sum())

    def with_param(field, g, idx, val):
        arrs = {f: np.asarray(getattr(scene, f), np.float64).copy() for f in ("mean", "scale", "quat", "opacity", "sh")}
        a = arrs[field][g].reshape(-1) if field != "opacity" else arrs[field]
        if field == "opacity":
            a[g] = val
        else:
            a[idx] = val
            arrs[field][g] = a.reshape(arrs[field][g].shape)
        return wl.Scene(arrs["mean"], arrs["scale"], arrs["quat"], arrs["opacity"], arrs["sh"], scene.sh_degree)

    checked = 0
    for field, size in (("mean", 3), ("scale", 3), ("quat", 4), ("opacity", 1), ("sh", 12)):
        for g in range(n):
            for idx in range(size):
                base = float(np.asarray(getattr(scene, field), np.float64)[g].reshape(-1)[idx]) if field != "opacity" \
                    else float(scene.opacity[g])
                h = 1e-5 * max(abs(base), 0.1)
                fd = (loss(with_param(field, g, idx, base + h)) - loss(with_param(field, g, idx, base - h))) / (2 * h)
                an = got[field][g].reshape(-1)[idx] if field != "opacity" else got["opacity"][g]
                assert abs(an - fd) <= 1e-5 + 1e-4 * abs(fd), (field, g, idx, an, fd)
                checked += abs(fd) > 1e-6
    assert checked > 30
