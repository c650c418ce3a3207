"""Seeded synthetic workloads for the exact ray-Gaussian renderer.

This module only draws random inputs (Gaussian parameters, camera intrinsics and
poses). It holds none of the rendering arithmetic, so both the CUDA path and the
CPU oracle can take their inputs from it.

Workloads (stand-ins for the paper's MipNeRF360 / ScanNet++ / ZipNeRF scenes,
which are not available here):

  1  4096 Gaussians, means uniform in [-2,2]^2 x [3,7] m, log-scale ~ N(-2.5, 0.5)
     per axis, uniform random unit quaternions, opacity = sigmoid(N(0,1)), SH
     degree 0 (DC colour uniform in [0,1]); pinhole 128x128, 60 deg.
  2  500k Gaussians in a spherical shell r ~ U[18,22] m around the camera,
     log-scale ~ N(-4, 0.7), opacity = sigmoid(N(0,1.5)), SH degree 3 (DC colour
     uniform in [0,1], higher bands ~ N(0, 0.2)); equidistant fisheye 1024x1024,
     180 deg.
  3  1M Gaussians of the workload-1 distribution with SH degree 3;
     Kannala-Brandt 1280x960, 190 deg, k_i ~ U[-0.05, 0.05]; an L1 target image
     ~ U[0,1] per BEAP pixel.
  4  2M-Gaussian resident scene (workload-1 distribution, SH degree 3) and a
     Poisson request stream (200 req/s) of pinhole 1920x1080 70 deg, equidistant
     1280x1280 200 deg and Kannala-Brandt 640x480 150 deg cameras with random
     poses within 1 m of the origin.
  5  6M Gaussians in a 100 x 10 x 100 m slab (y is the thin, vertical axis),
     log-scale ~ N(-3.5, 1), SH degree 3; four equidistant fisheye cameras
     1920x1536, 210 deg, yaw 0/90/180/270 deg at the origin.

Besides these, room_scene() draws an indoor room of wall surfels and clutter
around the camera, the structure of trained indoor fisheye scenes, for the
association ablation (it has no counterpart among the numbered workloads).

The DC SH coefficient is drawn uniformly in [-sqrt(pi), sqrt(pi)], which is the
range that makes the degree-0 colour uniform in [0, 1] under the 3DGS colour
convention (colour = Y_00 * dc + 1/2, Y_00 = 1/(2 sqrt(pi))).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PINHOLE, EQUIDISTANT, KANNALA_BRANDT = 0, 1, 2


@dataclass
class Camera:
    model: int
    width: int
    height: int
    fov_x: float                      # radians, horizontal
    fov_y: float = 0.0                # radians; <= 0: derived from the model
    k: tuple = (0.0, 0.0, 0.0, 0.0)   # Kannala-Brandt k1..k4
    R_cw: np.ndarray = field(default_factory=lambda: np.eye(3, dtype=np.float32))
    t_cw: np.ndarray = field(default_factory=lambda: np.zeros(3, dtype=np.float32))
    bg: tuple = (1.0, 1.0, 1.0)

    @property
    def pixels(self) -> int:
        return self.width * self.height


@dataclass
class Scene:
    mean: np.ndarray      # [n,3] f32
    scale: np.ndarray     # [n,3] f32, linear
    quat: np.ndarray      # [n,4] f32, (w,x,y,z)
    opacity: np.ndarray   # [n] f32, activated
    sh: np.ndarray        # [n,(deg+1)^2,3] f32
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.mean[idx].copy(), self.scale[idx].copy(), self.quat[idx].copy(),
                     self.opacity[idx].copy(), self.sh[idx].copy(), self.sh_degree)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _sh(rng, n, deg):
    nb = (deg + 1) ** 2
    sh = np.zeros((n, nb, 3))
    sh[:, 0, :] = rng.uniform(-math.sqrt(math.pi), math.sqrt(math.pi), (n, 3))
    if nb > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.2, (n, nb - 1, 3))
    return sh


def _pack(mean, log_s, quat, opacity, sh, deg) -> Scene:
    f = np.float32
    return Scene(np.ascontiguousarray(mean, f), np.ascontiguousarray(np.exp(log_s), f),
                 np.ascontiguousarray(quat, f), np.ascontiguousarray(opacity, f),
                 np.ascontiguousarray(sh, f), deg)


def cube_scene(n: int, seed: int, deg: int) -> Scene:
    """Workload-1 distribution: cube [-2,2]^2 x [3,7] m, log s ~ N(-2.5, 0.5)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mean = np.stack([rng.uniform(-2, 2, n), rng.uniform(-2, 2, n), rng.uniform(3, 7, n)], 1)
    log_s = rng.normal(-2.5, 0.5, (n, 3))
    quat = _quats(rng, n)
    opacity = _sigmoid(rng.normal(0.0, 1.0, n))
    return _pack(mean, log_s, quat, opacity, _sh(rng, n, deg), deg)


def shell_scene(n: int, seed: int, deg: int = 3) -> Scene:
    """Workload-2 distribution: shell r ~ U[18,22] m, log s ~ N(-4, 0.7)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    mean = v * rng.uniform(18.0, 22.0, (n, 1))
    log_s = rng.normal(-4.0, 0.7, (n, 3))
    quat = _quats(rng, n)
    opacity = _sigmoid(rng.normal(0.0, 1.5, n))
    return _pack(mean, log_s, quat, opacity, _sh(rng, n, deg), deg)


def slab_scene(n: int, seed: int, deg: int = 3) -> Scene:
    """Workload-5 distribution: x, z in [-50, 50], y in [-5, 5] m, log s ~ N(-3.5, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mean = np.stack([rng.uniform(-50, 50, n), rng.uniform(-5, 5, n), rng.uniform(-50, 50, n)], 1)
    log_s = rng.normal(-3.5, 1.0, (n, 3))
    quat = _quats(rng, n)
    opacity = _sigmoid(rng.normal(0.0, 1.0, n))
    return _pack(mean, log_s, quat, opacity, _sh(rng, n, deg), deg)


def _quat_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Hamilton products of quaternion arrays (w, x, y, z) [n, 4]."""
    aw, ax, ay, az = a.T
    bw, bx, by, bz = b.T
    return np.stack([aw * bw - ax * bx - ay * by - az * bz, aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx, aw * bz + ax * by - ay * bx + az * bw], 1)


def _quats_with_axis(rng, normal: np.ndarray) -> np.ndarray:
    """Quaternions whose rotation takes the local z axis to +-normal (unit, [n, 3]),
    spun by a uniform angle about it."""
    n = normal * np.where(normal[:, 2:3] < 0, -1.0, 1.0)  # an ellipsoid is symmetric in its axis' sign
    axis = np.stack([-n[:, 1], n[:, 0], np.zeros(len(n))], 1)  # e_z x n
    s = np.linalg.norm(axis, axis=1, keepdims=True)
    ang = np.arctan2(s[:, 0], n[:, 2])
    axis = np.where(s > 1e-12, axis / np.maximum(s, 1e-300), np.array([1.0, 0.0, 0.0]))
    align = np.concatenate([np.cos(ang / 2)[:, None], np.sin(ang / 2)[:, None] * axis], 1)
    spin_a = rng.uniform(0, 2 * math.pi, len(n))
    spin = np.stack([np.cos(spin_a / 2), np.zeros(len(n)), np.zeros(len(n)), np.sin(spin_a / 2)], 1)
    return _quat_mul(align, spin)


def room_scene(n: int, seed: int, deg: int = 3, half=(2.5, 1.4, 3.0)) -> Scene:
    """An indoor room around the camera (a stand-in for the structure of trained
    indoor fisheye scenes): 80% flat surfels on the six walls of a box of half
    extents `half` centred at the origin (area-weighted; thin axis along the wall
    normal tilted by N(0, 0.15) rad; in-plane log-scales ~ N(-3, 0.8), normal
    log-scale ~ N(-5.5, 0.5); 1 cm of jitter off the wall) and 20% clutter inside
    70% of the box (log-scales ~ N(-3, 0.7) per axis, random rotations); opacity
    = sigmoid(N(1, 1.5)), SH of the other workloads."""
    rng = np.random.Generator(np.random.PCG64(seed))
    hx, hy, hz = half
    n_s = int(round(0.8 * n))
    n_c = n - n_s
    areas = np.array([hy * hz, hy * hz, hx * hz, hx * hz, hx * hy, hx * hy])
    face = rng.choice(6, size=n_s, p=areas / areas.sum())
    ax = face // 2  # 0: x walls, 1: floor / ceiling, 2: front / back
    sign = np.where(face % 2 == 0, -1.0, 1.0)
    h = np.array(half)
    mean_s = rng.uniform(-1, 1, (n_s, 3)) * h
    mean_s[np.arange(n_s), ax] = sign * h[ax] + rng.normal(0, 0.01, n_s)
    normal = np.zeros((n_s, 3))
    normal[np.arange(n_s), ax] = 1.0
    normal += rng.normal(0, 0.15, (n_s, 3))
    normal /= np.linalg.norm(normal, axis=1, keepdims=True)
    q_s = _quats_with_axis(rng, normal)
    log_s_s = np.stack([rng.normal(-3.0, 0.8, n_s), rng.normal(-3.0, 0.8, n_s), rng.normal(-5.5, 0.5, n_s)], 1)
    mean_c = rng.uniform(-0.7, 0.7, (n_c, 3)) * h
    log_s_c = rng.normal(-3.0, 0.7, (n_c, 3))
    q_c = _quats(rng, n_c)
    mean = np.concatenate([mean_s, mean_c])
    log_s = np.concatenate([log_s_s, log_s_c])
    quat = np.concatenate([q_s, q_c])
    opacity = _sigmoid(rng.normal(1.0, 1.5, n))
    return _pack(mean, log_s, quat, opacity, _sh(rng, n, deg), deg)


def rot_y(yaw: float) -> np.ndarray:
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])


def rot_x(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])


def rot_z(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])


def pose(R_wc: np.ndarray, centre) -> tuple[np.ndarray, np.ndarray]:
    """World->camera (R_cw, t_cw) of a camera with camera->world rotation R_wc at centre."""
    R_cw = np.asarray(R_wc, np.float64).T
    t_cw = -R_cw @ np.asarray(centre, np.float64)
    return R_cw.astype(np.float32), t_cw.astype(np.float32)


def random_pose(rng) -> tuple[np.ndarray, np.ndarray]:
    """Centre uniform in the 1 m ball; yaw U[+-30], pitch U[+-15], roll U[+-10] deg."""
    while True:
        c = rng.uniform(-1, 1, 3)
        if c @ c <= 1.0:
            break
    yaw = math.radians(rng.uniform(-30, 30))
    pitch = math.radians(rng.uniform(-15, 15))
    roll = math.radians(rng.uniform(-10, 10))
    return pose(rot_y(yaw) @ rot_x(pitch) @ rot_z(roll), c)


def kb_coeffs(seed: int) -> tuple:
    rng = np.random.Generator(np.random.PCG64(seed))
    return tuple(float(np.float32(v)) for v in rng.uniform(-0.05, 0.05, 4))


def config_cameras(cfg: int) -> list[Camera]:
    deg = math.radians
    if cfg == 1:
        return [Camera(PINHOLE, 128, 128, deg(60))]
    if cfg == 2:
        return [Camera(EQUIDISTANT, 1024, 1024, deg(180))]
    if cfg == 3:
        return [Camera(KANNALA_BRANDT, 1280, 960, deg(190), k=kb_coeffs(3))]
    if cfg == 5:
        cams = []
        for yaw in (0, 90, 180, 270):
            R, t = pose(rot_y(math.radians(yaw)), (0, 0, 0))
            cams.append(Camera(EQUIDISTANT, 1920, 1536, deg(210), R_cw=R, t_cw=t))
        return cams
    raise ValueError(cfg)


def config_scene(cfg: int, n: int | None = None) -> Scene:
    if cfg == 1:
        return cube_scene(n or 4096, 1, 0)
    if cfg == 2:
        return shell_scene(n or 500_000, 2, 3)
    if cfg == 3:
        return cube_scene(n or 1_000_000, 3, 3)
    if cfg == 4:
        return cube_scene(n or 2_000_000, 4, 3)
    if cfg == 5:
        return slab_scene(n or 6_000_000, 5, 3)
    raise ValueError(cfg)


def l1_target(cam: Camera, seed: int = 3) -> np.ndarray:
    """Seeded L1 target image ~ U[0,1], [h, w, 3] f32, one value per BEAP pixel."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(0, 1, (cam.height, cam.width, 3)).astype(np.float32)


SERVING_KINDS = (
    (PINHOLE, 1920, 1080, 70.0, None),
    (EQUIDISTANT, 1280, 1280, 200.0, None),
    (KANNALA_BRANDT, 640, 480, 150.0, 44),
)


def serving_requests(n: int, seed: int = 4, rate_hz: float = 200.0) -> list[tuple[float, Camera]]:
    """Poisson arrivals at rate_hz; each request is one camera drawn from the three kinds."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for _ in range(n):
        t += rng.exponential(1.0 / rate_hz)
        model, w, h, fov, kseed = SERVING_KINDS[int(rng.integers(0, 3))]
        R, tc = random_pose(rng)
        k = kb_coeffs(kseed) if kseed is not None else (0.0, 0.0, 0.0, 0.0)
        out.append((t, Camera(model, w, h, math.radians(fov), k=k, R_cw=R, t_cw=tc)))
    return out


def random_pixels(cam: Camera, count: int, seed: int) -> np.ndarray:
    """Seeded sample of distinct pixel coordinates, [count, 2] int32 (column, row)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    count = min(count, cam.pixels)
    flat = rng.choice(cam.pixels, size=count, replace=False)
    return np.stack([flat % cam.width, flat // cam.width], 1).astype(np.int32)


def all_pixels(cam: Camera) -> np.ndarray:
    j, i = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    return np.stack([i.ravel(), j.ravel()], 1).astype(np.int32)


def beap_image(cam: Camera, seed: int) -> np.ndarray:
    """Seeded synthetic BEAP image [h, w, 3] f32 in [0, 1]: smooth low-frequency
    waves plus a small per-pixel noise, the input of a BEAP -> native resampling."""
    rng = np.random.Generator(np.random.PCG64(seed))
    j, i = np.meshgrid(np.arange(cam.height) / cam.height, np.arange(cam.width) / cam.width, indexing="ij")
    ph = rng.uniform(0, 2 * math.pi, (3, 2))
    fr = rng.uniform(1.0, 4.0, (3, 2))
    img = np.stack([0.5 + 0.25 * np.sin(2 * math.pi * fr[c, 0] * i + ph[c, 0])
                    + 0.2 * np.cos(2 * math.pi * fr[c, 1] * j + ph[c, 1]) for c in range(3)], -1)
    img += rng.uniform(-0.05, 0.05, img.shape)
    return np.clip(img, 0.0, 1.0).astype(np.float32)
