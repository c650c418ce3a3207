"""ctypes wrapper of the CPU oracle (geer_oracle.c).

TEST INFRASTRUCTURE: imported only by the tests, by the smoke check and by the
benchmark's CPU-baseline leg. The product path never imports this module.

`build()` compiles the oracle with gcc (OpenMP, -ffp-contract=off: the FP32
replica must not contract multiply-adds) into oracle/_build/.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "geer_oracle.c")
LIB = os.path.join(HERE, "_build", "libgeer_oracle.so")
MAX_ALT = 8


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-Wall", "-o", LIB, SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return LIB


class CameraC(C.Structure):
    _fields_ = [("model", C.c_int32), ("width", C.c_int32), ("height", C.c_int32),
                ("fov_x", C.c_float), ("fov_y", C.c_float), ("k", C.c_float * 4),
                ("R_cw", C.c_float * 9), ("t_cw", C.c_float * 3), ("bg", C.c_float * 3)]


class GaussiansC(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("pad_", C.c_int32),
                ("mean", C.c_void_p), ("scale", C.c_void_p), ("quat", C.c_void_p),
                ("opacity", C.c_void_p), ("sh", C.c_void_p)]


class ParamsC(C.Structure):
    _fields_ = [("alpha_min", C.c_float), ("T_min", C.c_float), ("alpha_max", C.c_float),
                ("lambda_pad", C.c_float)]


DEFAULT_PARAMS = dict(alpha_min=1.0 / 255.0, T_min=1e-4, alpha_max=0.99, lambda_pad=1e-3)

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        _lib.orc_fov_y.restype = C.c_double
        _lib.orc_fov_y.argtypes = [P]
        _lib.orc_pixel_ray.argtypes = [P, C.c_int, C.c_int, P, P]
        _lib.orc_kappa.restype = C.c_double
        _lib.orc_kappa.argtypes = [P, P, P, P, P, P, P]
        _lib.orc_sh_basis.argtypes = [C.c_int, P, P]
        _lib.orc_colour.argtypes = [C.c_int, P, P, P, P, P]
        _lib.orc_replica.argtypes = [P, P, P, P, P, P, P]
        _lib.orc_assoc_mask.argtypes = [P, C.c_int64, P, P]
        _lib.orc_replica_arcs.argtypes = [P, P, P, P, P, C.c_float, P]
        _lib.orc_render_pixels.argtypes = [P, P, P, P, P, C.c_int64, P, P, P, P, P, P, P, P]
        _lib.orc_pixel_contributors.restype = C.c_int64
        _lib.orc_pixel_contributors.argtypes = [P, P, P, P, C.c_int32, C.c_int32, P, C.c_int64]
        _lib.orc_render_grad.argtypes = [P, P, P, P, P, C.c_int64, P, P, P, P, P, P, P]
        _lib.orc_native_focal.restype = C.c_double
        _lib.orc_native_focal.argtypes = [P]
        _lib.orc_project.argtypes = [P, P, P, P]
        _lib.orc_native_ray.restype = C.c_int
        _lib.orc_native_ray.argtypes = [P, C.c_int, C.c_int, P]
        _lib.orc_remap_to_native.argtypes = [P, P, P, P, P]
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def camera_c(cam) -> CameraC:
    c = CameraC()
    c.model, c.width, c.height = int(cam.model), int(cam.width), int(cam.height)
    c.fov_x, c.fov_y = float(cam.fov_x), float(cam.fov_y)
    for i in range(4):
        c.k[i] = float(cam.k[i])
    R = np.asarray(cam.R_cw, np.float32).ravel()
    t = np.asarray(cam.t_cw, np.float32).ravel()
    for i in range(9):
        c.R_cw[i] = float(R[i])
    for i in range(3):
        c.t_cw[i] = float(t[i])
        c.bg[i] = float(cam.bg[i])
    return c


class _SceneC:
    """Keeps the contiguous arrays alive while the C struct points at them."""

    def __init__(self, scene):
        self.arrays = [np.ascontiguousarray(a, np.float32) for a in
                       (scene.mean, scene.scale, scene.quat, scene.opacity, scene.sh)]
        g = GaussiansC()
        g.n = scene.n
        g.sh_degree = scene.sh_degree
        g.mean, g.scale, g.quat, g.opacity, g.sh = [a.ctypes.data for a in self.arrays]
        self.c = g


def params_c(**kw) -> ParamsC:
    d = dict(DEFAULT_PARAMS)
    d.update(kw)
    p = ParamsC()
    p.alpha_min, p.T_min, p.alpha_max, p.lambda_pad = (d["alpha_min"], d["T_min"], d["alpha_max"],
                                                       d["lambda_pad"])
    return p


def fov_y(cam) -> float:
    c = camera_c(cam)
    return lib().orc_fov_y(C.byref(c))


def pixel_ray(cam, i: int, j: int):
    c = camera_c(cam)
    o = np.zeros(3)
    d = np.zeros(3)
    lib().orc_pixel_ray(C.byref(c), i, j, _ptr(o), _ptr(d))
    return o, d


def kappa(mu, s, q, o, d):
    mu, s, q = (np.ascontiguousarray(x, np.float32) for x in (mu, s, q))
    o, d = (np.ascontiguousarray(x, np.float64) for x in (o, d))
    ts = C.c_double()
    on = C.c_double()
    k = lib().orc_kappa(_ptr(mu), _ptr(s), _ptr(q), _ptr(o), _ptr(d), C.byref(ts), C.byref(on))
    return k, ts.value, on.value


def sh_basis(deg: int, direction) -> np.ndarray:
    d = np.ascontiguousarray(direction, np.float64)
    Y = np.zeros(16)
    lib().orc_sh_basis(deg, _ptr(d), _ptr(Y))
    return Y[: (deg + 1) ** 2]


def colour(deg: int, sh_g, mu, o):
    sh_g = np.ascontiguousarray(sh_g, np.float32)
    mu = np.ascontiguousarray(mu, np.float32)
    o = np.ascontiguousarray(o, np.float64)
    rgb = np.zeros(3)
    raw = np.zeros(3)
    lib().orc_colour(deg, _ptr(sh_g), _ptr(mu), _ptr(o), _ptr(rgb), _ptr(raw))
    return rgb, raw


def replica(scene, cam, **params):
    """FP32 replica: (cull u8[n], key u32[n], ranges u16[n,8], count u32[n])."""
    sc = _SceneC(scene)
    c = camera_c(cam)
    p = params_c(**params)
    n = scene.n
    cull = np.zeros(n, np.uint8)
    key = np.zeros(n, np.uint32)
    ranges = np.zeros((n, 8), np.uint16)
    count = np.zeros(n, np.uint32)
    lib().orc_replica(C.byref(sc.c), C.byref(c), C.byref(p), _ptr(cull), _ptr(key), _ptr(ranges), _ptr(count))
    return cull, key, ranges, count


def assoc_mask(cam, ranges: np.ndarray) -> np.ndarray:
    c = camera_c(cam)
    ranges = np.ascontiguousarray(ranges, np.uint16)
    ncols = (cam.width + 15) // 16
    nrows = (cam.height + 15) // 16
    mask = np.zeros((ranges.shape[0], nrows, ncols), np.uint8)
    lib().orc_assoc_mask(C.byref(c), ranges.shape[0], _ptr(ranges), _ptr(mask))
    return mask


def replica_arcs(cam, mu, s, q, sigma, **params):
    c = camera_c(cam)
    p = params_c(**params)
    mu, s, q = (np.ascontiguousarray(x, np.float32) for x in (mu, s, q))
    out = np.zeros(7, np.float32)
    lib().orc_replica_arcs(C.byref(c), C.byref(p), _ptr(mu), _ptr(s), _ptr(q), float(sigma), _ptr(out))
    return out


def render_pixels(scene, cam, pix: np.ndarray, rep=None, **params):
    """Brute-force render of the listed pixels ([m,2] int32 column,row).

    Returns a dict with rgb [m,3], T [m], alt [m,MAX_ALT,4], nalt [m], cond [m],
    ncontrib [m], flags [m]."""
    if rep is None:
        rep = replica(scene, cam, **params)
    cull, key = rep[0], rep[1]
    sc = _SceneC(scene)
    c = camera_c(cam)
    p = params_c(**params)
    pix = np.ascontiguousarray(pix, np.int32)
    m = pix.shape[0]
    out = dict(rgb=np.zeros((m, 3)), T=np.zeros(m), alt=np.zeros((m, MAX_ALT, 4)),
               nalt=np.zeros(m, np.int32), cond=np.zeros(m), ncontrib=np.zeros(m, np.int32),
               flags=np.zeros(m, np.int32))
    lib().orc_render_pixels(C.byref(sc.c), C.byref(c), C.byref(p), _ptr(cull), _ptr(key), m, _ptr(pix),
                            _ptr(out["rgb"]), _ptr(out["T"]), _ptr(out["alt"]), _ptr(out["nalt"]),
                            _ptr(out["cond"]), _ptr(out["ncontrib"]), _ptr(out["flags"]))
    return out


def pixel_contributors(scene, cam, cull, i: int, j: int, cap: int = 1 << 16, **params):
    sc = _SceneC(scene)
    c = camera_c(cam)
    p = params_c(**params)
    ids = np.zeros(cap, np.int64)
    cull = np.ascontiguousarray(cull, np.uint8)
    n = lib().orc_pixel_contributors(C.byref(sc.c), C.byref(c), C.byref(p), _ptr(cull), i, j, _ptr(ids), cap)
    return ids[: min(n, cap)]


def render_grad(scene, cam, pix: np.ndarray, dLdC: np.ndarray, rep=None, **params):
    """FP64 analytic gradients of sum(dLdC * C) over the listed pixels."""
    if rep is None:
        rep = replica(scene, cam, **params)
    sc = _SceneC(scene)
    c = camera_c(cam)
    p = params_c(**params)
    pix = np.ascontiguousarray(pix, np.int32)
    dLdC = np.ascontiguousarray(dLdC, np.float64)
    n = scene.n
    nb = (scene.sh_degree + 1) ** 2
    g = dict(mean=np.zeros((n, 3)), scale=np.zeros((n, 3)), quat=np.zeros((n, 4)), opacity=np.zeros(n),
             sh=np.zeros((n, nb, 3)))
    lib().orc_render_grad(C.byref(sc.c), C.byref(c), C.byref(p), _ptr(rep[0]), _ptr(rep[1]), pix.shape[0],
                          _ptr(pix), _ptr(dLdC), _ptr(g["mean"]), _ptr(g["scale"]), _ptr(g["quat"]),
                          _ptr(g["opacity"]), _ptr(g["sh"]))
    return g


def match_pixels(gpu_rgb: np.ndarray, orc: dict, tol: float = 2e-4, cond_limit: float = 1e-4):
    """Compare GPU pixels [m,3] with the oracle's admissible results.

    A pixel passes if some admissible result is within tol (or tol + 2 cond for
    pixels whose FP32 conditioning bound cond exceeds cond_limit) on every
    channel. Returns (ok mask, err vs the best admissible result [m,3],
    ill-conditioned mask, undecidable mask)."""
    m = gpu_rgb.shape[0]
    alt = orc["alt"][:, :, :3]
    valid = np.arange(MAX_ALT)[None, :] < orc["nalt"][:, None]
    diff = np.abs(alt - gpu_rgb[:, None, :]).max(axis=2)
    diff = np.where(valid, diff, np.inf)
    best = diff.argmin(axis=1)
    err = np.abs(alt[np.arange(m), best] - gpu_rgb)
    ill = orc["cond"] > cond_limit
    lim = np.where(ill, tol + 2.0 * orc["cond"], tol)
    undecidable = orc["flags"] != 0
    ok = (err.max(axis=1) <= lim) | undecidable
    return ok, err, ill, undecidable


def native_focal(cam) -> float:
    c = camera_c(cam)
    return lib().orc_native_focal(C.byref(c))


def project(cam, d):
    """App. E forward projection of a camera-frame direction to native pixel coordinates."""
    c = camera_c(cam)
    d = np.ascontiguousarray(d, np.float64)
    xp, yp = C.c_double(), C.c_double()
    lib().orc_project(C.byref(c), _ptr(d), C.byref(xp), C.byref(yp))
    return xp.value, yp.value


def native_ray(cam, i: int, j: int):
    c = camera_c(cam)
    d = np.zeros(3)
    ok = lib().orc_native_ray(C.byref(c), i, j, _ptr(d))
    return (d if ok else None)


def remap_to_native(cam, beap: np.ndarray, fill=(0.0, 0.0, 0.0), coords: bool = False):
    """Native image [h,w,3] (and, with coords=True, each native pixel's BEAP (u, v), NaN without a ray)."""
    c = camera_c(cam)
    beap = np.ascontiguousarray(beap, np.float32)
    f = np.ascontiguousarray(fill, np.float32)
    out = np.zeros((cam.height, cam.width, 3))
    uv = np.zeros((cam.height, cam.width, 2)) if coords else None
    lib().orc_remap_to_native(C.byref(c), _ptr(beap), _ptr(f), _ptr(out), _ptr(uv) if coords else None)
    return (out, uv) if coords else out
