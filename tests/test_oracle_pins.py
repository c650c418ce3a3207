"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: numerical
quadrature and minimisation, scipy's spherical harmonics, closed forms of
special cases, geometric invariants and brute force on tiny scenes.
"""
import math
import zlib

import numpy as np
import pytest
from scipy import integrate, optimize, special
from scipy.spatial.transform import Rotation

from paper_2505_24053_gb300 import workloads as wl


def _sigma_inv(q_wxyz, s):
    # covariance from scipy's rotation (scalar-last quaternion), Sec. 3.1 / App. B.1
    R = Rotation.from_quat([q_wxyz[1], q_wxyz[2], q_wxyz[3], q_wxyz[0]]).as_matrix()
    Sig = R @ np.diag(np.asarray(s, np.float64) ** 2) @ R.T
    return np.linalg.inv(Sig), Sig


def _random_gaussian_ray(rng, aniso):
    mu = rng.uniform(-3, 3, 3).astype(np.float32)
    q = rng.standard_normal(4).astype(np.float32)
    base = math.exp(rng.uniform(-3, 0))
    if aniso == "needle":
        s = np.array([base, base * 1e-4 ** rng.uniform(0.3, 1), base], np.float32)
    elif aniso == "disk":
        s = np.array([base, base, base * 1e-4 ** rng.uniform(0.3, 1)], np.float32)
    else:
        s = np.exp(rng.uniform(-3, 0, 3)).astype(np.float32)
    o = rng.uniform(-8, 8, 3)
    # aim near the Gaussian so that kappa is moderate
    tgt = mu.astype(np.float64) + rng.normal(0, 2.0 * float(s.max()), 3)
    d = tgt - o
    d /= np.linalg.norm(d)
    return mu, s, q, o, d


@pytest.mark.parametrize("aniso", ["general", "needle", "disk"])
def test_kappa_equals_ray_integral_by_quadrature(orc, aniso):
    """Sec. 3.1 / App. B.2: sigma e^{-kappa/2} is the integral of the canonical
    isotropic density (1/rho) exp(-|u|^2/2), rho = sqrt(2 pi), along the canonical
    ray r_u(t) = o_u + t d_u with |d_u| = 1 (the measure-preserving reading)."""
    rng = np.random.default_rng(11 + len(aniso))
    checked = 0
    for _ in range(400):
        mu, s, q, o, d = _random_gaussian_ray(rng, aniso)
        kap, tstar, _ = orc.kappa(mu, s, q, o, d)
        if kap > 60:
            continue
        Sinv, _ = _sigma_inv(q, s)
        wd = math.sqrt(d @ Sinv @ d)        # |W d|: canonical speed of the world ray
        v0 = o - mu.astype(np.float64)

        def f(t):
            x = v0 + t * d
            return math.exp(-0.5 * (x @ Sinv @ x)) * wd / math.sqrt(2 * math.pi)

        # the integrand is a Gaussian in t of width 1/wd centred at the closest point
        tc = optimize.minimize_scalar(lambda t: (v0 + t * d) @ Sinv @ (v0 + t * d),
                                      bracket=(-1e3, 0.0, 1e3), tol=1e-14).x
        w = 1.0 / wd
        val, _ = integrate.quad(f, tc - 40 * w, tc + 40 * w, points=[tc], epsabs=0, epsrel=1e-12, limit=400)
        # the test side evaluates x^T Sigma^-1 x in expanded form, which loses
        # digits for 1e-4 needles and disks; 1e-6 still catches any formula slip
        assert val == pytest.approx(math.exp(-0.5 * kap), rel=1e-6, abs=1e-13)
        # closest approach parameter
        assert tstar == pytest.approx(tc, rel=1e-6, abs=1e-6 * w)
        checked += 1
    assert checked > 200


def test_kappa_is_min_mahalanobis_and_scale_invariant(orc):
    """kappa = min_t (o + t d - mu)^T Sigma^-1 (o + t d - mu) (App. B.2), >= 0 and
    invariant under d -> c d, c > 0."""
    rng = np.random.default_rng(5)
    for _ in range(300):
        mu, s, q, o, d = _random_gaussian_ray(rng, "general")
        kap, _, _ = orc.kappa(mu, s, q, o, d)
        Sinv, _ = _sigma_inv(q, s)
        v0 = o - mu.astype(np.float64)
        res = optimize.minimize_scalar(lambda t: (v0 + t * d) @ Sinv @ (v0 + t * d),
                                       bracket=(-1e3, 0.0, 1e3), tol=1e-14)
        assert kap >= 0
        assert kap == pytest.approx(res.fun, rel=1e-7, abs=1e-9)
        k2, _, _ = orc.kappa(mu, s, q, o, 7.5 * d)
        assert k2 == pytest.approx(kap, rel=1e-12, abs=1e-14)


def test_isotropic_kappa_is_point_line_distance(orc):
    """Theorem (App. B.3): for an isotropic Gaussian of radius r, kappa = D^2 / r^2
    with D the perpendicular distance from the centre to the ray."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        mu = rng.uniform(-2, 2, 3).astype(np.float32)
        r = np.float32(math.exp(rng.uniform(-3, 1)))
        q = rng.standard_normal(4).astype(np.float32)
        o = rng.uniform(-5, 5, 3)
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        D = np.linalg.norm(np.cross(mu.astype(np.float64) - o, d))
        kap, _, _ = orc.kappa(mu, np.array([r, r, r], np.float32), q, o, d)
        assert kap == pytest.approx(D * D / (float(r) ** 2), rel=1e-10)


def _real_sh_scipy(l, m, direction):
    x, y, z = direction
    polar = math.acos(max(-1.0, min(1.0, z)))
    az = math.atan2(y, x)
    Y = special.sph_harm_y(l, abs(m), polar, az)  # complex, Condon-Shortley phase included
    if m == 0:
        return Y.real
    if m > 0:
        return math.sqrt(2) * Y.real
    return math.sqrt(2) * Y.imag


def test_sh_basis_matches_scipy(orc):
    """SH colour of App. B.1 follows 3DGS: real SH with the Condon-Shortley phase,
    index l^2 + l + m. Checked against scipy's complex harmonics."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        Y = orc.sh_basis(3, v)
        for l in range(4):
            for m in range(-l, l + 1):
                assert Y[l * l + l + m] == pytest.approx(_real_sh_scipy(l, m, v), abs=1e-12)
    # known low-order values (3DGS signs): Y_00 = 1/(2 sqrt pi), Y_1,-1 = -sqrt(3/4pi) y
    v = np.array([0.36, 0.48, 0.8])
    Y = orc.sh_basis(1, v)
    assert Y[0] == pytest.approx(0.5 / math.sqrt(math.pi), abs=1e-15)
    assert Y[1] == pytest.approx(-math.sqrt(3 / (4 * math.pi)) * 0.48, abs=1e-15)
    assert Y[2] == pytest.approx(math.sqrt(3 / (4 * math.pi)) * 0.8, abs=1e-15)
    assert Y[3] == pytest.approx(-math.sqrt(3 / (4 * math.pi)) * 0.36, abs=1e-15)


def test_sh_basis_orthonormal(orc):
    """Gauss-Legendre x uniform-azimuth quadrature of Y_a Y_b over the sphere = delta_ab."""
    xs, ws = np.polynomial.legendre.leggauss(16)
    naz = 32
    G = np.zeros((16, 16))
    for z, wz in zip(xs, ws):
        st = math.sqrt(1 - z * z)
        for k in range(naz):
            a = 2 * math.pi * k / naz
            Y = orc.sh_basis(3, np.array([st * math.cos(a), st * math.sin(a), z]))
            G += np.outer(Y, Y) * wz * (2 * math.pi / naz)
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_colour_is_sh_plus_half_clamped(orc):
    """Colour at direction (mu - o)/|mu - o| (App. B.1), 3DGS offset 0.5 and clamp at 0."""
    rng = np.random.default_rng(8)
    for _ in range(50):
        sh = rng.normal(0, 0.6, (16, 3)).astype(np.float32)
        mu = rng.uniform(-3, 3, 3).astype(np.float32)
        o = rng.uniform(-3, 3, 3)
        v = mu - o
        v /= np.linalg.norm(v)
        raw_ref = np.array([sum(float(sh[l * l + l + m, c]) * _real_sh_scipy(l, m, v)
                                for l in range(4) for m in range(-l, l + 1)) + 0.5 for c in range(3)])
        rgb, raw = orc.colour(3, sh, mu, o)
        assert np.allclose(raw, raw_ref, atol=1e-12)
        assert np.allclose(rgb, np.maximum(raw_ref, 0), atol=1e-12)


def test_beap_grid_equiangular(orc):
    """BEAP (Sec. 3.3): rays are uniform in (theta, phi) with pitch FoV/w, symmetric
    about the optical axis; the direction of App. E has tan theta = x/z and
    tan phi = y/z (pinhole reading, App. E) -- checked for |angles| < 90 deg."""
    cam = wl.Camera(wl.EQUIDISTANT, 40, 24, math.radians(170))
    fx = float(np.float32(cam.fov_x))  # the camera carries FP32 angles
    fy = orc.fov_y(cam)
    assert fy == pytest.approx(fx * 24 / 40, rel=1e-14)
    th = []
    for i in range(cam.width):
        o, d = orc.pixel_ray(cam, i, 5)
        assert np.allclose(o, 0)
        assert np.linalg.norm(d) == pytest.approx(1.0, abs=1e-14)
        th.append(math.atan2(d[0], d[2]))
    th = np.array(th)
    assert np.allclose(np.diff(th), fx / cam.width, atol=1e-12)
    assert np.allclose(th + th[::-1], 0, atol=1e-12)
    ph = np.array([math.atan2(orc.pixel_ray(cam, 3, j)[1][1], orc.pixel_ray(cam, 3, j)[1][2])
                   for j in range(cam.height)])
    assert np.allclose(np.diff(ph), fy / cam.height, atol=1e-12)
    # beyond 90 deg (FoV 210): the dihedral angle about the y axis keeps increasing
    wide = wl.Camera(wl.EQUIDISTANT, 42, 8, math.radians(210))
    a = np.unwrap([math.atan2(orc.pixel_ray(wide, i, 4)[1][0], orc.pixel_ray(wide, i, 4)[1][2])
                   for i in range(42)])
    assert np.allclose(np.diff(a), float(np.float32(math.radians(210))) / 42, atol=1e-12)


def test_fov_y_models(orc):
    """FoV_y of the BEAP grid: equidistant is Kannala-Brandt with k = 0; for
    Kannala-Brandt the focal length that maps FoV_x/2 to w/2 maps FoV_y/2 to h/2."""
    for fov in (120, 180, 200):
        e = wl.Camera(wl.EQUIDISTANT, 1280, 960, math.radians(fov))
        k0 = wl.Camera(wl.KANNALA_BRANDT, 1280, 960, math.radians(fov))
        assert orc.fov_y(k0) == pytest.approx(orc.fov_y(e), rel=1e-12)
    cam = wl.Camera(wl.KANNALA_BRANDT, 1280, 960, math.radians(190), k=wl.kb_coeffs(3))
    fy = orc.fov_y(cam)
    k = cam.k

    def dist(p):
        return p * (1 + k[0] * p ** 2 + k[1] * p ** 4 + k[2] * p ** 6 + k[3] * p ** 8)

    f = 640 / dist(float(np.float32(cam.fov_x)) / 2)
    assert f * dist(fy / 2) == pytest.approx(480.0, rel=1e-12)
    pin = wl.Camera(wl.PINHOLE, 1920, 1080, math.radians(70))
    f = 960 / math.tan(float(np.float32(math.radians(70))) / 2)
    assert f * math.tan(orc.fov_y(pin) / 2) == pytest.approx(540.0, rel=1e-12)


def _ellipsoid_extreme_angles(mu_c, A, lam):
    """Extreme dihedral angles (about y: atan2(x,z); about x: atan2(y,z)) of the
    surface mu_c + lam A u, |u| = 1: dense grid over the sphere, then a local
    refinement from the best grid point."""
    ref = (math.atan2(mu_c[0], mu_c[2]), math.atan2(mu_c[1], mu_c[2]))

    def pts(p0, p1):
        u = np.stack([np.sin(p0) * np.cos(p1), np.sin(p0) * np.sin(p1), np.cos(p0)], -1)
        return mu_c + lam * (u @ A.T)

    def ang(x, axis):
        a = np.arctan2(x[..., axis], x[..., 2])
        return (a - ref[axis] + math.pi) % (2 * math.pi) - math.pi + ref[axis]

    g0, g1 = np.meshgrid(np.linspace(0, math.pi, 301), np.linspace(0, 2 * math.pi, 601), indexing="ij")
    P = pts(g0, g1)
    out = []
    for axis in (0, 1):
        a = ang(P, axis)
        res = []
        for sgn in (1.0, -1.0):
            k = np.unravel_index(np.argmin(sgn * a), a.shape)
            r = optimize.minimize(lambda p: sgn * float(ang(pts(p[0], p[1]), axis)), [g0[k], g1[k]],
                                  method="Nelder-Mead", options=dict(xatol=1e-13, fatol=1e-16, maxiter=5000))
            res.append(sgn * r.fun)
        out.append((res[0], res[1]))
    return out


def test_pbf_arcs_tangent_and_conservative(orc):
    """Sec. 3.2 / App. D: the PBF planes are tangent to the lambda-ellipsoid, so its
    angular bounds equal the extreme dihedral angles of the ellipsoid surface.
    The FP32 replica's arcs (mirror transform: tau = tan(angle/2)) must contain
    the true extremes and be no wider than the FP32 margin."""
    rng = np.random.default_rng(21)
    cam = wl.Camera(wl.EQUIDISTANT, 64, 64, math.radians(180))
    checked = 0
    for trial in range(40):
        mu = rng.uniform(-6, 6, 3).astype(np.float32)
        mu[2] = np.float32(abs(mu[2]) + 1.0) if trial % 3 else np.float32(-abs(mu[2]) - 1.0)
        q = rng.standard_normal(4).astype(np.float32)
        s = np.exp(rng.uniform(-3.5, -1.0, 3)).astype(np.float32)
        sigma = np.float32(rng.uniform(0.05, 1.0))
        out = orc.replica_arcs(cam, mu, s, q, sigma)
        lam = math.sqrt(float(out[6]))
        if np.linalg.norm(mu) < 4 * lam * float(s.max()):
            continue
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        A = R @ np.diag(s.astype(np.float64))
        ext = _ellipsoid_extreme_angles(mu.astype(np.float64), A, lam)
        for (lo_t, hi_t), kind, lo, hi in ((ext[0], out[0], out[1], out[2]), (ext[1], out[3], out[4], out[5])):
            if kind == 3:  # axis pierces the ellipsoid: must really be so
                continue
            a_lo, a_hi = 2 * math.atan(lo), 2 * math.atan(hi)
            if kind == 2:
                a_lo -= 0  # [lo, pi) u (-pi, hi]: compare on the unwrapped circle
                a_hi += 2 * math.pi
                ref = (lo_t + hi_t) / 2
                if ref < 0:
                    a_lo -= 2 * math.pi
                    a_hi -= 2 * math.pi
            width = hi_t - lo_t
            assert a_lo <= lo_t + 1e-9 and a_hi >= hi_t - 1e-9, (trial, a_lo, lo_t, a_hi, hi_t)
            # tight: widened only by the FP32 margin (~1e-5 rad) and rounding
            assert lo_t - a_lo < 2e-5 + 1e-4 * width and a_hi - hi_t < 2e-5 + 1e-4 * width
            checked += 1
    assert checked >= 30


def test_lambda2_bounds_alpha_threshold(orc):
    """The association contour lambda^2 >= 2 ln(sigma / alpha_min) (so every ray with
    sigma e^{-kappa/2} >= alpha_min crosses it) and is at most 0.2% larger."""
    cam = wl.Camera(wl.PINHOLE, 16, 16, 1.0)
    for sigma in np.concatenate([np.linspace(0.0040, 1.0, 400), [1 / 255 * 1.0001, 0.5, 0.999999]]):
        out = orc.replica_arcs(cam, np.array([0, 0, 5], np.float32), np.array([.1, .1, .1], np.float32),
                               np.array([1, 0, 0, 0], np.float32), np.float32(sigma))
        exact = 2 * math.log(float(np.float32(sigma)) / float(np.float32(1 / 255)))
        if exact <= 0:
            continue
        assert out[6] >= exact
        assert out[6] <= exact * 1.002 + 1e-6


def _tiny_scene(rng, n, deg, spread, behind=True):
    mean = rng.uniform(-spread, spread, (n, 3))
    if not behind:
        mean[:, 2] = np.abs(mean[:, 2]) + 0.3
    log_s = rng.normal(-1.6, 0.7, (n, 3))
    quat = rng.standard_normal((n, 4))
    opacity = 1 / (1 + np.exp(-rng.normal(0.5, 1.5, n)))
    nb = (deg + 1) ** 2
    sh = rng.normal(0, 0.3, (n, nb, 3))
    return wl.Scene(mean.astype(np.float32), np.exp(log_s).astype(np.float32), quat.astype(np.float32),
                    opacity.astype(np.float32), sh.astype(np.float32), deg)


TINY_CAMS = [
    ("pinhole", wl.Camera(wl.PINHOLE, 64, 48, math.radians(60))),
    ("equidistant180", wl.Camera(wl.EQUIDISTANT, 64, 64, math.radians(180))),
    ("equidistant200sq", wl.Camera(wl.EQUIDISTANT, 56, 56, math.radians(200))),
    ("kb190", wl.Camera(wl.KANNALA_BRANDT, 64, 48, math.radians(190), k=wl.kb_coeffs(3))),
    ("equidistant210", wl.Camera(wl.EQUIDISTANT, 61, 37, math.radians(210))),
]


@pytest.mark.parametrize("name,cam", TINY_CAMS, ids=[c[0] for c in TINY_CAMS])
def test_pbf_zero_misses_brute_force(orc, name, cam):
    """Sec. 3.2: a Gaussian is assigned to a camera sub-frustum iff its PBF meets it.
    On tiny scenes, every (pixel, Gaussian) with FP64 alpha >= 1/255 in front of
    the camera must have the Gaussian associated with the pixel's tile."""
    rng = np.random.default_rng(zlib.crc32(name.encode()) % 1000)
    scene = _tiny_scene(rng, 64, 1, 3.0)
    R, t = wl.random_pose(rng)
    cam = wl.Camera(cam.model, cam.width, cam.height, cam.fov_x, k=cam.k, R_cw=R, t_cw=t)
    cull, key, ranges, count = orc.replica(scene, cam)
    mask = orc.assoc_mask(cam, ranges)
    assert np.array_equal(mask.reshape(scene.n, -1).sum(1), count)
    pairs = 0
    for j in range(cam.height):
        for i in range(cam.width):
            ids = orc.pixel_contributors(scene, cam, cull, i, j)
            for g in ids:
                pairs += 1
                assert mask[g, j // 16, i // 16], (name, i, j, g)
    assert pairs > 200
    # association is not trivially everything
    assert mask.mean() < 0.8


def _render_full(orc, scene, cam):
    pix = wl.all_pixels(cam)
    out = orc.render_pixels(scene, cam, pix)
    return out["rgb"].reshape(cam.height, cam.width, 3), out


def test_single_isotropic_gaussian_image(orc):
    """One isotropic Gaussian: each pixel is c a + (1 - a) bg with a = min(0.99,
    sigma exp(-D^2/(2 r^2))) when a >= 1/255 (App. B.1 colour equation, Theorem
    App. B.3). Rays from tan theta = x/z, tan phi = y/z (pinhole geometry)."""
    cam = wl.Camera(wl.PINHOLE, 32, 24, math.radians(50), bg=(1.0, 0.9, 0.8))
    mu = np.array([[0.3, -0.2, 4.0]], np.float32)
    r = np.float32(0.35)
    rgb = np.array([0.2, 0.7, 0.4])
    dc = (rgb - 0.5) * 2 * math.sqrt(math.pi)
    scene = wl.Scene(mu, np.full((1, 3), r, np.float32), np.array([[0.3, 0.5, -0.1, 0.8]], np.float32),
                     np.array([0.8], np.float32), dc.reshape(1, 1, 3).astype(np.float32), 0)
    img, _ = _render_full(orc, scene, cam)
    fy = orc.fov_y(cam)
    for j in range(cam.height):
        for i in range(cam.width):
            th = ((i + 0.5) / cam.width - 0.5) * float(np.float32(cam.fov_x))
            ph = ((j + 0.5) / cam.height - 0.5) * fy
            d = np.array([math.tan(th), math.tan(ph), 1.0])
            d /= np.linalg.norm(d)
            D = np.linalg.norm(np.cross(mu[0].astype(np.float64), d))
            a = 0.8 * math.exp(-0.5 * D * D / float(r) ** 2)
            exp_c = np.array(cam.bg, np.float64)
            if a >= 1 / 255:
                a = min(a, 0.99)
                colour = dc.astype(np.float32).astype(np.float64) * 0.5 / math.sqrt(math.pi) + 0.5
                exp_c = colour * a + (1 - a) * np.array(cam.bg)
            assert np.allclose(img[j, i], exp_c, atol=1e-12), (i, j)


def test_compositing_invariants(orc):
    """Order/compositing invariants of App. B.1: T in [0,1] and non-increasing in the
    number of contributors; sigma -> 0 gives the background; permuting the input
    leaves the image unchanged; q -> -q changes nothing; swapping two scale axes
    with a matching 90 deg rotation changes nothing; a Gaussian behind the
    camera changes nothing."""
    rng = np.random.default_rng(4)
    cam = wl.Camera(wl.EQUIDISTANT, 24, 20, math.radians(160), bg=(0.1, 0.2, 0.3))
    scene = _tiny_scene(rng, 48, 2, 2.5, behind=False)
    img, out = _render_full(orc, scene, cam)
    assert np.all(out["T"] >= 0) and np.all(out["T"] <= 1)
    assert img.min() >= 0

    zero = scene.subset(np.arange(scene.n))
    zero.opacity[:] = 1e-4
    img0, _ = _render_full(orc, zero, cam)
    assert np.allclose(img0, np.array(cam.bg)[None, None, :], atol=0)

    perm = rng.permutation(scene.n)
    imgp, _ = _render_full(orc, scene.subset(perm), cam)
    assert np.allclose(imgp, img, atol=1e-12)

    neg = scene.subset(np.arange(scene.n))
    neg.quat[:] = -neg.quat
    imgn, _ = _render_full(orc, neg, cam)
    assert np.allclose(imgn, img, atol=1e-12)

    # swap scale axes x<->y and post-multiply R by a 90 deg rotation about z
    sw = scene.subset(np.arange(scene.n))
    sw.scale[:] = scene.scale[:, [1, 0, 2]]
    Rz = Rotation.from_euler("z", 90, degrees=True)
    for g in range(scene.n):
        q = scene.quat[g]
        r = Rotation.from_quat([q[1], q[2], q[3], q[0]]) * Rz
        x, y, z, w = r.as_quat()
        sw.quat[g] = [w, x, y, z]
    imgs, _ = _render_full(orc, sw, cam)
    assert np.allclose(imgs, img, atol=1e-5)

    # add a Gaussian straight behind the camera
    extra = wl.Scene(np.concatenate([scene.mean, [[0.1, 0.0, -3.0]]]).astype(np.float32),
                     np.concatenate([scene.scale, [[0.5, 0.5, 0.5]]]).astype(np.float32),
                     np.concatenate([scene.quat, [[1, 0, 0, 0]]]).astype(np.float32),
                     np.concatenate([scene.opacity, [0.9]]).astype(np.float32),
                     np.concatenate([scene.sh, np.zeros((1,) + scene.sh.shape[1:])]).astype(np.float32), 2)
    imge, _ = _render_full(orc, extra, cam)
    assert np.allclose(imge, img, atol=1e-12)


def test_transmittance_monotone_along_contributors(orc):
    """Along a pixel's sorted contributors T never increases, and the final T is the
    product of (1 - a_i) over the applied contributors."""
    rng = np.random.default_rng(9)
    cam = wl.Camera(wl.PINHOLE, 16, 16, math.radians(40))
    scene = _tiny_scene(rng, 200, 0, 1.0, behind=False)
    scene.mean[:, 2] += 4
    pix = wl.all_pixels(cam)
    base = orc.render_pixels(scene, cam, pix)
    # T_final is non-increasing as more Gaussians (a superset) are added in depth order
    rep = orc.replica(scene, cam)
    order = np.argsort(rep[1], kind="stable")
    prev = np.ones(pix.shape[0])
    for k in (10, 40, 100, 200):
        sub = scene.subset(np.sort(order[:k]))
        T = orc.render_pixels(sub, cam, pix)["T"]
        stopped = base["T"] < 2e-4
        assert np.all((T <= prev + 1e-15) | stopped)
        prev = T
    assert np.allclose(prev, base["T"])


REMAP_CAMS = [
    wl.Camera(wl.PINHOLE, 48, 36, math.radians(70)),
    wl.Camera(wl.EQUIDISTANT, 40, 40, math.radians(180)),
    wl.Camera(wl.KANNALA_BRANDT, 64, 48, math.radians(190), k=wl.kb_coeffs(3)),
    wl.Camera(wl.KANNALA_BRANDT, 40, 30, math.radians(150), k=wl.kb_coeffs(44)),
]


@pytest.mark.parametrize("cam", REMAP_CAMS, ids=["pinhole", "equi180", "kb190", "kb150"])
def test_native_rays_invert_the_app_e_projection(orc, cam):
    """App. E projects a ray to (f tan theta, f tan phi) + c (pinhole) or
    (f phi_d / r)(tan theta, tan phi) + c (fisheye): the oracle's native pixel rays
    must project back onto their pixel centres."""
    checked = 0
    for j in range(cam.height):
        for i in range(cam.width):
            d = orc.native_ray(cam, i, j)
            if d is None or d[2] < math.cos(math.radians(85)):
                continue
            assert np.linalg.norm(d) == pytest.approx(1.0, abs=1e-12)
            xp, yp = orc.project(cam, d)
            assert xp == pytest.approx(i + 0.5, abs=1e-8) and yp == pytest.approx(j + 0.5, abs=1e-8)
            checked += 1
    assert checked > 0.5 * cam.pixels or cam.model != wl.PINHOLE


def test_remap_of_a_linear_beap_image_is_exact(orc):
    """Bilinear interpolation reproduces a BEAP image linear in (column, row): the
    native image then equals that linear function at each native ray's BEAP
    coordinate, computed here from atan2 / the BEAP equation directly."""
    cam = wl.Camera(wl.EQUIDISTANT, 40, 32, math.radians(180))
    fy = orc.fov_y(cam)
    fx = float(np.float32(cam.fov_x))
    jj, ii = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    beap = np.stack([0.01 * ii + 0.02 * jj, 0.5 - 0.01 * jj, 0.003 * ii], -1).astype(np.float64)
    out = orc.remap_to_native(cam, beap.astype(np.float32), fill=(9, 9, 9))
    for j in range(cam.height):
        for i in range(cam.width):
            d = orc.native_ray(cam, i, j)
            if d is None or d[2] <= 0:
                continue
            u = math.atan2(d[0], d[2]) / fx * cam.width + cam.width / 2 - 0.5
            v = math.atan(d[1] / d[2]) / fy * cam.height + cam.height / 2 - 0.5
            if not (0 <= u <= cam.width - 1 and 0 <= v <= cam.height - 1):
                continue
            exp = [0.01 * u + 0.02 * v, 0.5 - 0.01 * v, 0.003 * u]
            assert np.allclose(out[j, i], exp, atol=1e-6), (i, j)


# ---------------------------------------------------------------------------
# The depth key (Algorithm 1 sorts by "frustum id + depth"; the depth is read as
# the distance from the camera centre to the Gaussian's mean, since view z
# orders Gaussians wrongly beyond 90 degrees off axis). The replica's FP32 key
# decides every pixel's compositing order on both sides, so it is pinned here
# against the geometry alone and against an order-sensitive image.

_U32 = 2.0 ** -24


def _posed_camera(rng, model, fov_deg, w=40, h=36):
    R_wc = wl.rot_y(rng.uniform(-math.pi, math.pi)) @ wl.rot_x(rng.uniform(-0.6, 0.6)) @ wl.rot_z(
        rng.uniform(-0.5, 0.5))
    centre = rng.uniform(-4, 4, 3)
    R, t = wl.pose(R_wc, centre)
    return wl.Camera(model, w, h, math.radians(fov_deg), R_cw=R, t_cw=t), centre


def _key_bound(R, t, mu, D):
    """Error bound of an FP32 evaluation of |R mu + t| against the FP64 distance D
    from mu to the camera centre o = -R^T t: each component of R mu + t is a
    sum of four rounded terms (gamma_4 of their magnitudes), R differs from a
    rotation by its FP32 rounding (|I - R R^T| |t| and the spread of R's
    singular values times D), and the norm adds three roundings of D."""
    R64, t64, mu64 = R.astype(np.float64), t.astype(np.float64), mu.astype(np.float64)
    g4 = 4 * _U32 / (1 - 4 * _U32)
    comp = g4 * (np.abs(mu64) @ np.abs(R64).T + np.abs(t64)[None, :])
    E = np.eye(3) - R64 @ R64.T
    sv = np.linalg.svd(R64, compute_uv=False)
    rot = np.linalg.norm(E, 2) * np.linalg.norm(t64) + max(abs(sv[0] - 1), abs(sv[-1] - 1)) * D
    return np.linalg.norm(comp, axis=1) + rot + 3 * _U32 * D


def _key_violations(keys_f32, R, t, mu):
    o = -R.astype(np.float64).T @ t.astype(np.float64)
    D = np.linalg.norm(mu.astype(np.float64) - o[None, :], axis=1)
    err = np.abs(keys_f32.astype(np.float64) - D)
    return err > _key_bound(R, t, mu, D), err / np.spacing(keys_f32).astype(np.float64)


@pytest.mark.parametrize("model,fov", [(wl.EQUIDISTANT, 200), (wl.EQUIDISTANT, 210), (wl.KANNALA_BRANDT, 190),
                                       (wl.PINHOLE, 90)])
def test_depth_key_is_distance_to_camera_centre(orc, model, fov):
    """For posed cameras (rotated, translated; fields of view up to 210 degrees)
    and Gaussians all around the camera centre, behind it included, the replica's
    key equals the FP64 distance |mu - o| (o = -R_cw^T t_cw, the camera centre)
    within the FP32 error bound of its evaluation. View z, a dropped t_cw and a
    transposed R_cw each violate it."""
    rng = np.random.default_rng(1000 + fov + model)
    cam, centre = _posed_camera(rng, model, fov, w=40, h=36 if model != wl.KANNALA_BRANDT else 30)
    if model == wl.KANNALA_BRANDT:
        cam.k = wl.kb_coeffs(5)
    n = 4000
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    mu = (centre[None, :] + d * rng.uniform(0.3, 30.0, (n, 1))).astype(np.float32)
    scene = wl.Scene(mu, np.full((n, 3), 0.02, np.float32), np.tile(np.float32([[1, 0, 0, 0]]), (n, 1)),
                     np.full(n, 0.8, np.float32), np.zeros((n, 1, 3), np.float32), 0)
    cull, key, _, _ = orc.replica(scene, cam)
    live = cull == 0
    assert live.sum() == n  # none inside its contour, all opaque enough
    keys = key.view(np.float32)
    bad, ulps = _key_violations(keys, cam.R_cw, cam.t_cw, mu)
    assert not bad.any(), f"{int(bad.sum())} keys off the distance (max {ulps.max():.1f} ulp)"
    assert np.median(ulps) <= 1.0
    # behind-the-camera Gaussians exist and are keyed by their distance, not their z
    mc = mu.astype(np.float64) @ cam.R_cw.astype(np.float64).T + cam.t_cw.astype(np.float64)
    assert (mc[:, 2] < 0).sum() > n // 4

    # planted mistakes in the key alone fail the same check
    Rf, tf = cam.R_cw.astype(np.float32), cam.t_cw.astype(np.float32)
    m = mu @ Rf.T + tf
    planted = {
        "view z": m[:, 2].astype(np.float32),
        "no t_cw": np.linalg.norm(mu @ Rf.T, axis=1).astype(np.float32),
        "R_cw transposed": np.linalg.norm(mu @ Rf + tf, axis=1).astype(np.float32),
    }
    for name, k in planted.items():
        assert _key_violations(k, cam.R_cw, cam.t_cw, mu)[0].mean() > 0.5, name


def _ray_pair_scene(o, d, t_near, t_far, rgb_near, rgb_far, sigma=0.9, r=0.05):
    """Two isotropic Gaussians centred on the ray o + t d (t_near < t_far)."""
    mu = np.stack([o + t_near * d, o + t_far * d]).astype(np.float32)
    dc = (np.stack([rgb_near, rgb_far]) - 0.5) * 2 * math.sqrt(math.pi)
    return wl.Scene(mu, np.full((2, 3), r, np.float32), np.float32([[1, 0, 0, 0], [0.6, 0.0, 0.8, 0.0]]),
                    np.full(2, sigma, np.float32), dc.reshape(2, 1, 3).astype(np.float32), 0)


def _composite_expected(scene, o, d, bg, alpha_max=0.99):
    """App. B.1's colour equation over the two Gaussians in the order of their
    distance along the ray, with alpha = min(alpha_max, sigma exp(-D^2 / (2 r^2)))
    from the point-line distance D (App. B.3 Theorem, isotropic case)."""
    mu = scene.mean.astype(np.float64)
    t = (mu - o[None, :]) @ d
    order = np.argsort(t)
    C, T = np.zeros(3), 1.0
    for g in order:
        D = np.linalg.norm(np.cross(mu[g] - o, d))
        a = min(alpha_max, float(scene.opacity[g]) * math.exp(-0.5 * D * D / float(scene.scale[g, 0]) ** 2))
        colour = scene.sh[g, 0].astype(np.float64) * 0.5 / math.sqrt(math.pi) + 0.5
        C += T * a * colour
        T *= 1 - a
    return C + T * np.asarray(bg, np.float64), T


@pytest.mark.parametrize("theta_px", [39, 41, 1])
def test_depth_order_decides_the_composited_colour(orc, theta_px):
    """Two nearly opaque Gaussians on one ray of a rotated, translated 210 degree
    camera, the ray 92.5 to 102.5 degrees off the optical axis (beside and behind
    the image plane): the nearer one's colour dominates, as App. B.1's front-to-back
    equation gives. View z orders this pair the other way round, and an image
    composited in that order is far from the expected one."""
    rng = np.random.default_rng(77 + theta_px)
    cam, _ = _posed_camera(rng, wl.EQUIDISTANT, 210, w=42, h=20)
    cam.bg = (0.2, 0.3, 0.9)
    i, j = theta_px, 10
    o, d = orc.pixel_ray(cam, i, j)
    d = d / np.linalg.norm(d)
    dc_ = d @ cam.R_cw.astype(np.float64).T  # ray direction in the camera frame
    assert dc_[2] < 0 and abs(math.atan2(dc_[0], dc_[2])) > math.radians(92)
    scene = _ray_pair_scene(o, d, 1.5, 3.0, np.array([0.95, 0.05, 0.05]), np.array([0.05, 0.95, 0.05]))
    expected, T = _composite_expected(scene, o, d, cam.bg)
    pix = np.array([[i, j]], np.int32)
    rep = orc.replica(scene, cam)
    out = orc.render_pixels(scene, cam, pix, rep=rep)
    assert out["ncontrib"][0] == 2
    assert np.allclose(out["rgb"][0], expected, atol=1e-9)
    assert math.isclose(out["T"][0], T, abs_tol=1e-12)
    assert expected[0] > 0.85 > expected[1]  # the near (red) Gaussian dominates

    # the view-z key orders the pair the other way round here, and that image fails
    mc = scene.mean.astype(np.float64) @ cam.R_cw.astype(np.float64).T + cam.t_cw.astype(np.float64)
    viewz = mc[:, 2].astype(np.float32)
    assert viewz[1] < viewz[0]  # ascending view z puts the far Gaussian first
    planted = (rep[0], np.argsort(np.argsort(viewz)).astype(np.uint32))  # keys ordered as view z
    out_z = orc.render_pixels(scene, cam, pix, rep=planted)
    assert np.abs(out_z["rgb"][0] - expected).max() > 0.5
