"""Splatting-style association bounds (the association ablation), FP64 numpy.

TEST INFRASTRUCTURE: imported only by the tests and the benchmark's CPU leg;
the product path never imports it.

The paper sets its PBF association against the projection-based bounds of EWA
splatting and of the unscented transform (UT), either as the 3-sigma square of
3DGS or with SnugBox, in the same pipeline (Sec. 4, association runtime table;
App. H, EWA splatting preliminaries). On the BEAP grid the screen coordinates of a point
t = (x, y, z) in front of the camera are its BEAP angles
  theta = atan2(x, z), phi = atan2(y, z)
(a BEAP ray d = (sin theta cos phi, cos theta sin phi, cos theta cos phi) has
exactly these for |theta|, |phi| < 90 degrees, Sec. 3.3).

- EWA: the affine approximation of that map at the camera-frame mean mu_c (its
  Jacobian J, rows d theta / dt = (z, 0, -x) / (x^2 + z^2) and
  d phi / dt = (0, z, -y) / (y^2 + z^2)) carries Sigma_c = M diag(s^2) M^T
  (M = R_cw R) to Sigma_2 = J Sigma_c J^T about (theta, phi)(mu_c).
- UT: the 2n + 1 = 7 sigma points mu_c and mu_c +- sqrt(3) s_k M[:, k]
  (n = 3, alpha = 1, beta = 2, kappa = 0: lambda = 0, mean weights 0 and 1/6,
  covariance weights 2 and 1/6) are mapped exactly; each point's angles are
  taken in the branch within pi of the mean's angles; Sigma_2 and the centre
  are their weighted covariance and mean.
- The box: a square of half-side 3 sqrt(largest eigenvalue of Sigma_2), or with
  SnugBox the bounding box of the ellipse where the density reaches alpha_min,
  half-sides sqrt(2 ln(sigma / alpha_min) Sigma_2[i, i]).
- Culling: the pipeline's own (Algorithm 1, CullGaussian: sigma < alpha_min or
  the camera inside the contour lambda^2 = 2 ln(sigma / alpha_min) (1 + 1e-3)),
  plus the splatting near plane, mean with z <= 0.2 (the projection divides by
  z). Only the association step differs from the PBF pipeline. For a whole scene
  the camera-inside decision is the FP32 replica's (oracle.replica), the
  precision the kernel takes it in; splat_box alone takes it in FP64.

The splat alpha (the local-affine model the paper swaps in at render time,
Sec. 4): alpha = sigma exp(-D^T Sigma_2^-1 D / 2) with Sigma_2 the EWA
covariance above and D the ray's screen angles (atan2(x, z), atan2(y, z)) of
its camera-frame direction minus the mean's, wrapped into [-pi, pi]; Gaussians
below the near plane or with a singular Sigma_2 are culled. splat_render
composites these alphas exactly as the exact renderer does (contributors with
alpha >= alpha_min among the Gaussians associated with the pixel's tile, in
depth-key order, alpha clamped at alpha_max, stop before T < T_min, background
behind). splat_render_grad is its gradient: the compositing and the splat's
centre and conic differentiated analytically per pixel, the map from a
Gaussian's parameters to its centre, conic and colour by FP64 central
differences of screen_cov and of an FP64 colour (the oracle's SH basis).

Tiles: a column tile spans the angles [theta(i0), theta(i1)] of its first and
last pixel, theta(i) = ((i + 1/2) / w - 1/2) fov_x. X0 holds the columns whose
span meets the theta box on the circle, X1 those whose span meets the box
turned by pi (a ray with cos(phi) < 0 has atan2(x, z) = theta + pi); Y0 and Y1
likewise for rows. Each of these sets is one interval of tiles (the
association ranges hold one interval per arc, as PBF's do): a set split in two,
which a box through pi meeting both ends of a wide axis makes, takes the whole
axis. The association is the same flagged product as PBF's: tile (cx, cy) is
taken when (its row has a ray with cos(phi) >= 0 and cx in X0, or one with
cos(phi) < 0 and cx in X1) and (the same with columns and Y0, Y1).
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as orc

PBF, EWA, UT = 0, 1, 2
NEAR = 0.2
TWO_PI = 2.0 * math.pi


def _rot(q):
    q = np.asarray(q, np.float64)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _wrap(a):
    """a mod 2 pi in (-pi, pi]."""
    r = math.fmod(a + math.pi, TWO_PI)
    if r <= 0.0:
        r += TWO_PI
    return r - math.pi


def camera_frame(cam, mu):
    Rc = np.asarray(cam.R_cw, np.float64).reshape(3, 3)
    return Rc @ np.asarray(mu, np.float64) + np.asarray(cam.t_cw, np.float64), Rc


def screen_cov(cam, mu, scale, quat, mode: int):
    """(centre (theta, phi), Sigma_2 [2, 2]) of one Gaussian, or None below the near plane."""
    mu_c, Rc = camera_frame(cam, mu)
    if not mu_c[2] > NEAR:
        return None
    M = Rc @ _rot(quat)
    s = np.asarray(scale, np.float64)
    x, y, z = mu_c
    c0 = np.array([math.atan2(x, z), math.atan2(y, z)])
    if mode == EWA:
        J = np.array([[z / (x * x + z * z), 0.0, -x / (x * x + z * z)],
                      [0.0, z / (y * y + z * z), -y / (y * y + z * z)]])
        return c0, J @ (M @ np.diag(s * s) @ M.T) @ J.T
    if mode != UT:
        raise ValueError(mode)
    pts = [mu_c] + [mu_c + sg * math.sqrt(3.0) * s[k] * M[:, k] for k in range(3) for sg in (1.0, -1.0)]
    p = np.array([[c0[0] + _wrap(math.atan2(t[0], t[2]) - c0[0]),
                   c0[1] + _wrap(math.atan2(t[1], t[2]) - c0[1])] for t in pts])
    wm = np.array([0.0] + [1.0 / 6.0] * 6)
    wc = np.array([2.0] + [1.0 / 6.0] * 6)
    centre = wm @ p
    d = p - centre
    return centre, np.einsum("i,ij,ik->jk", wc, d, d)


def camera_inside(cam, mu, scale, quat, sigma, alpha_min: float = 1.0 / 255.0, pad: float = 1e-3) -> bool:
    """The camera (origin) lies inside the Gaussian's contour |S^-1 M^T mu_c|^2 <= lambda^2."""
    mu_c, Rc = camera_frame(cam, mu)
    u = (Rc @ _rot(quat)).T @ mu_c / np.asarray(scale, np.float64)
    return float(u @ u) <= 2.0 * math.log(sigma / alpha_min) * (1.0 + pad)


def splat_box(cam, mu, scale, quat, sigma, mode: int, snug: bool, alpha_min: float = 1.0 / 255.0,
              inside=None):
    """(theta_lo, theta_hi, phi_lo, phi_hi) of one Gaussian, or None when culled
    (inside: a camera-inside decision taken elsewhere, else FP64 here)."""
    if not sigma > alpha_min:
        return None
    if camera_inside(cam, mu, scale, quat, sigma, alpha_min) if inside is None else inside:
        return None
    r = screen_cov(cam, mu, scale, quat, mode)
    if r is None:
        return None
    centre, S2 = r
    if snug:
        e = np.sqrt(2.0 * math.log(sigma / alpha_min) * np.maximum(np.diag(S2), 0.0))
    else:
        e = np.full(2, 3.0 * math.sqrt(max(np.linalg.eigvalsh(S2).max(), 0.0)))
    return centre[0] - e[0], centre[0] + e[0], centre[1] - e[1], centre[1] + e[1]


def beap_angle(i: int, n: int, fov: float) -> float:
    return ((i + 0.5) / n - 0.5) * fov


def meets_on_circle(a: float, b: float, lo: float, hi: float) -> bool:
    """[a, b] (width < 2 pi) meets [lo, hi] taken modulo 2 pi."""
    if hi - lo >= TWO_PI:
        return True
    return any(b >= lo + TWO_PI * k and a <= hi + TWO_PI * k for k in range(-3, 4))


def _one_interval(m: np.ndarray) -> np.ndarray:
    idx = np.flatnonzero(m)
    if idx.size and idx[-1] - idx[0] + 1 != idx.size:
        return np.ones_like(m)
    return m


def axis_sets(lo: float, hi: float, n_pix: int, fov: float, one_interval: bool = True):
    """(direct, turned) membership [tiles] of one axis for the angle box [lo, hi]."""
    tiles = (n_pix + 15) // 16
    direct = np.zeros(tiles, bool)
    turned = np.zeros(tiles, bool)
    for c in range(tiles):
        a, b = beap_angle(16 * c, n_pix, fov), beap_angle(min(16 * c + 15, n_pix - 1), n_pix, fov)
        direct[c] = meets_on_circle(a, b, lo, hi)
        turned[c] = meets_on_circle(a, b, lo + math.pi, hi + math.pi)
    if one_interval:
        return _one_interval(direct), _one_interval(turned)
    return direct, turned


def cos_flags(n_pix: int, fov: float):
    """(has0, has1) per tile: some ray with cos >= 0 / with cos <= 0 (1e-12 slack)."""
    tiles = (n_pix + 15) // 16
    has0 = np.zeros(tiles, bool)
    has1 = np.zeros(tiles, bool)
    for c in range(tiles):
        for i in range(16 * c, min(16 * c + 16, n_pix)):
            cs = math.cos(beap_angle(i, n_pix, fov))
            has0[c] |= cs > -1e-12
            has1[c] |= cs < 1e-12
    return has0, has1


def box_mask(cam, box, grow: float = 0.0, one_interval: bool = True) -> np.ndarray:
    """Association mask [tiles_y, tiles_x] of one box, its sides moved out by grow
    (in by -grow); one_interval=False keeps the exact split sets."""
    ty, tx = (cam.height + 15) // 16, (cam.width + 15) // 16
    if box is None:
        return np.zeros((ty, tx), bool)
    fy = orc.fov_y(cam)
    t0, t1, p0, p1 = box[0] - grow, box[1] + grow, box[2] - grow, box[3] + grow
    if t1 < t0 or p1 < p0:
        return np.zeros((ty, tx), bool)
    x0, x1 = axis_sets(t0, t1, cam.width, cam.fov_x, one_interval)
    y0, y1 = axis_sets(p0, p1, cam.height, fy, one_interval)
    c_has0, c_has1 = cos_flags(cam.width, cam.fov_x)
    r_has0, r_has1 = cos_flags(cam.height, fy)
    cols_ok = (r_has0[:, None] & x0[None, :]) | (r_has1[:, None] & x1[None, :])
    rows_ok = (c_has0[None, :] & y0[:, None]) | (c_has1[None, :] & y1[:, None])
    return cols_ok & rows_ok


def scene_boxes(cam, scene, mode: int, snug: bool, alpha_min: float = 1.0 / 255.0):
    """Boxes of a scene's Gaussians, the pipeline's cull taken from the FP32 replica."""
    cull = orc.replica(scene, cam, alpha_min=alpha_min)[0]
    return [None if cull[g] else
            splat_box(cam, scene.mean[g], scene.scale[g], scene.quat[g], float(scene.opacity[g]), mode, snug,
                      alpha_min, inside=False) for g in range(scene.n)]


def scene_masks(cam, boxes, grow=0.0) -> np.ndarray:
    """[n, tiles_y, tiles_x] association masks of the boxes; grow: a scalar or one
    value per box."""
    grow = np.broadcast_to(np.asarray(grow, np.float64), (len(boxes),))
    return np.stack([box_mask(cam, b, float(d)) for b, d in zip(boxes, grow)]) if boxes else \
        np.zeros((0, 0, 0), bool)


def _wrap_pi(a):
    return (a + math.pi) % TWO_PI - math.pi


def splat_alpha(cam, mu, scale, quat, sigma, d_cam):
    """Splat alpha (unclamped) of one Gaussian for a camera-frame ray direction."""
    r = screen_cov(cam, mu, scale, quat, EWA)
    if r is None:
        return 0.0
    c, S2 = r
    dv = np.array([_wrap_pi(math.atan2(d_cam[0], d_cam[2]) - c[0]), _wrap_pi(math.atan2(d_cam[1], d_cam[2]) - c[1])])
    return float(sigma) * math.exp(-0.5 * float(dv @ np.linalg.solve(S2, dv)))


def splat_render(scene, cam, pix, mask, key, alpha_min=1.0 / 255.0, T_min=1e-4, alpha_max=0.99, margin=1e-3):
    """Splat-alpha render of the listed pixels ([m, 2] column, row). mask: the
    association [n, tiles_y, tiles_x]; key: depth keys [n] (ties by index); the
    pipeline's cull is the FP32 replica's. Returns (rgb [m, 3], near [m]): near
    marks pixels with an alpha within `margin` (relative) of alpha_min or a
    transmittance within it of T_min, where FP32 may take the other branch."""
    Rc = np.asarray(cam.R_cw, np.float64).reshape(3, 3)
    o_w = -Rc.T @ np.asarray(cam.t_cw, np.float64)
    cull = orc.replica(scene, cam, alpha_min=alpha_min)[0]
    n = scene.n
    live = np.zeros(n, bool)
    centre = np.zeros((n, 2))
    conic = np.zeros((n, 2, 2))
    rgb = np.zeros((n, 3))
    for g in range(n):
        if cull[g]:
            continue
        r = screen_cov(cam, scene.mean[g], scene.scale[g], scene.quat[g], EWA)
        if r is None or not np.linalg.det(r[1]) > 0:
            continue
        live[g] = True
        centre[g], conic[g] = r[0], np.linalg.inv(r[1])
        rgb[g] = _colour64(scene.sh_degree, scene.sh[g], scene.mean[g], o_w)
    order = np.lexsort((np.arange(n), np.asarray(key, np.int64)))
    out = np.zeros((len(pix), 3))
    near = np.zeros(len(pix), bool)
    bg = np.asarray(cam.bg, np.float64)
    for m, (i, j) in enumerate(np.asarray(pix)):
        _, d_w = orc.pixel_ray(cam, int(i), int(j))
        d = Rc @ d_w
        ts, ps = math.atan2(d[0], d[2]), math.atan2(d[1], d[2])
        cand = order[live[order] & mask[order, j // 16, i // 16]]
        dv = np.stack([_wrap_pi(ts - centre[cand, 0]), _wrap_pi(ps - centre[cand, 1])], 1)
        q = np.einsum("ki,kij,kj->k", dv, conic[cand], dv)
        a = np.asarray(scene.opacity, np.float64)[cand] * np.exp(-0.5 * q)
        near[m] = bool(np.any(np.abs(a / alpha_min - 1.0) < margin))
        T, C = 1.0, np.zeros(3)
        for k in np.flatnonzero(a >= alpha_min):
            al = min(a[k], alpha_max)
            Tn = T * (1.0 - al)
            near[m] |= abs(Tn / T_min - 1.0) < margin
            if Tn < T_min:
                break
            C += T * al * rgb[cand[k]]
            T = Tn
        out[m] = C + T * bg
    return out, near


def _colour64(deg, sh, mu, o):
    """FP64 colour max(0, sum_k Y_k(dir) sh_k + 1/2), dir = (mu - o) / |mu - o| (the
    oracle's SH basis, pinned to scipy's harmonics)."""
    v = np.asarray(mu, np.float64) - o
    Y = orc.sh_basis(deg, v / np.linalg.norm(v))
    return np.maximum(Y @ np.asarray(sh, np.float64).reshape(-1, 3) + 0.5, 0.0)


def _splat_features(cam, mu, scale, quat, sigma_unused=None):
    """(theta_c, phi_c, A, B, C) of one Gaussian: the EWA centre and the conic."""
    c, S2 = screen_cov(cam, mu, scale, quat, EWA)
    K = np.linalg.inv(S2)
    return np.array([c[0], c[1], K[0, 0], K[0, 1], K[1, 1]])


def splat_render_grad(scene, cam, pix, mask, key, dLdC, alpha_min=1.0 / 255.0, T_min=1e-4, alpha_max=0.99,
                      rel_step=1e-6):
    """Gradient of sum(dLdC * C) over the listed pixels of the splat render:
    dict of mean [n, 3], scale [n, 3], quat [n, 4], opacity [n], sh [n, K, 3]."""
    Rc = np.asarray(cam.R_cw, np.float64).reshape(3, 3)
    o_w = -Rc.T @ np.asarray(cam.t_cw, np.float64)
    cull = orc.replica(scene, cam, alpha_min=alpha_min)[0]
    n, deg = scene.n, scene.sh_degree
    nb = (deg + 1) ** 2
    f64 = lambda a: np.asarray(a, np.float64)
    live = np.zeros(n, bool)
    feat = np.zeros((n, 5))
    rgb = np.zeros((n, 3))
    for g in range(n):
        if cull[g]:
            continue
        r = screen_cov(cam, scene.mean[g], scene.scale[g], scene.quat[g], EWA)
        if r is None or not np.linalg.det(r[1]) > 0:
            continue
        live[g] = True
        feat[g] = _splat_features(cam, scene.mean[g], scene.scale[g], scene.quat[g])
        rgb[g] = _colour64(deg, scene.sh[g], scene.mean[g], o_w)
    order = np.lexsort((np.arange(n), np.asarray(key, np.int64)))
    sig = f64(scene.opacity)
    g_feat = np.zeros((n, 5))
    g_sig = np.zeros(n)
    g_rgb = np.zeros((n, 3))
    bg = f64(cam.bg)
    for m, (i, j) in enumerate(np.asarray(pix)):
        _, d_w = orc.pixel_ray(cam, int(i), int(j))
        d = Rc @ d_w
        ts, ps = math.atan2(d[0], d[2]), math.atan2(d[1], d[2])
        cand = order[live[order] & mask[order, j // 16, i // 16]]
        steps = []  # (gaussian, alpha_raw, alpha, T before, d0, d1, q)
        T = 1.0
        for g in cand:
            d0, d1 = _wrap_pi(ts - feat[g, 0]), _wrap_pi(ps - feat[g, 1])
            q = feat[g, 2] * d0 * d0 + 2 * feat[g, 3] * d0 * d1 + feat[g, 4] * d1 * d1
            ar = sig[g] * math.exp(-0.5 * q)
            if ar < alpha_min:
                continue
            al = min(ar, alpha_max)
            if T * (1 - al) < T_min:
                break
            steps.append((g, ar, al, T, d0, d1, q))
            T *= 1 - al
        gC = f64(dLdC[m])
        S = T * bg  # what lies behind the current contributor, walking back
        for g, ar, al, Tk, d0, d1, q in reversed(steps):
            g_rgb[g] += Tk * al * gC
            dLda = float(gC @ (Tk * rgb[g] - S / (1 - al)))
            S = S + Tk * al * rgb[g]
            if ar < alpha_max:
                g_sig[g] += dLda * math.exp(-0.5 * q)
                dLdq = -0.5 * dLda * ar
                A, B, C = feat[g, 2:]
                g_feat[g] += dLdq * np.array([-2 * (A * d0 + B * d1), -2 * (B * d0 + C * d1), d0 * d0, 2 * d0 * d1,
                                              d1 * d1])
    out = dict(mean=np.zeros((n, 3)), scale=np.zeros((n, 3)), quat=np.zeros((n, 4)), opacity=g_sig,
               sh=np.zeros((n, nb, 3)))
    for g in np.flatnonzero(live & ((np.abs(g_feat).sum(1) > 0) | (np.abs(g_rgb).sum(1) > 0))):
        mu, s, qt, sh = f64(scene.mean[g]), f64(scene.scale[g]), f64(scene.quat[g]), f64(scene.sh[g])

        def central(fun, x, k, h):
            xp, xm = x.copy(), x.copy()
            xp[k] += h
            xm[k] -= h
            return (fun(xp) - fun(xm)) / (2 * h)

        for k in range(3):
            h = rel_step * max(1.0, abs(mu[k]))
            dfe = central(lambda x: _splat_features(cam, x, s, qt), mu, k, h)
            dco = central(lambda x: _colour64(deg, sh, x, o_w), mu, k, h)
            out["mean"][g, k] = g_feat[g] @ dfe + g_rgb[g] @ dco
            h = rel_step * s[k]
            out["scale"][g, k] = g_feat[g] @ central(lambda x: _splat_features(cam, mu, x, qt), s, k, h)
        for k in range(4):
            out["quat"][g, k] = g_feat[g] @ central(lambda x: _splat_features(cam, mu, s, x), qt, k, rel_step)
        for k in range(nb):
            for ch in range(3):
                flat = sh.reshape(-1).copy()
                idx = 3 * k + ch
                out["sh"][g, k, ch] = g_rgb[g] @ central(lambda x: _colour64(deg, x, mu, o_w), flat, idx, 1e-4)
    return out

