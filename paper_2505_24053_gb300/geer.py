"""Python binding of the C ABI in include/geer.h (argument marshalling only).

Every step of the render runs in libgeer.so's CUDA kernels; torch supplies device
memory and the current stream. There is no CPU fallback: if the library is
missing the first call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

OK, ERR_ARG, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_STATE, ERR_BOUNDS = range(8)
PINHOLE, EQUIDISTANT, KANNALA_BRANDT = 0, 1, 2


class GeerError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


class CameraC(C.Structure):
    _fields_ = [("model", C.c_int32), ("width", C.c_int32), ("height", C.c_int32),
                ("fov_x", C.c_float), ("fov_y", C.c_float), ("k", C.c_float * 4),
                ("R_cw", C.c_float * 9), ("t_cw", C.c_float * 3), ("bg", C.c_float * 3)]


class GaussiansC(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("scale", C.c_void_p), ("quat", C.c_void_p), ("opacity", C.c_void_p),
                ("sh", C.c_void_p), ("n", C.c_int64), ("sh_degree", C.c_int32), ("reserved_", C.c_int32)]


class ParamsC(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("alpha_min", C.c_float), ("T_min", C.c_float),
                ("alpha_max", C.c_float), ("lambda_pad", C.c_float), ("assoc", C.c_int32), ("snugbox", C.c_int32),
                ("alpha_model", C.c_int32)]


EXPORTS = ["geer_status_string", "geer_default_params", "geer_workspace_size", "geer_workspace_init",
           "geer_workspace_destroy", "geer_set_cameras", "geer_preprocess", "geer_bin_sort", "geer_render_fwd",
           "geer_render_bwd", "geer_last_device_status", "geer_debug_preprocess", "geer_debug_pairs",
           "geer_render_counts", "geer_l1_loss_grad", "geer_render_noalloc", "geer_set_camera_slots",
           "geer_enable_timing", "geer_stage_times", "geer_stage_name", "geer_remap_to_native",
           "geer_native_regions", "geer_image_metrics", "geer_native_to_beap", "geer_adam_step",
           "geer_pair_counts", "geer_debug_render_state", "geer_densify_accumulate", "geer_densify_scratch_bytes",
           "geer_densify_plan", "geer_densify_apply", "geer_opacity_reset", "geer_render_bwd_tiles",
           "geer_grad_accumulators", "geer_preprocess_bwd", "geer_tile_owners", "geer_set_tile_mask",
           "geer_tile_counts", "geer_checked_build", "geer_bounds_violation", "geer_debug_set_render_order",
           "geer_enable_stage_timing", "geer_render_train_l1"]

_lib = None
N_STAGES = 10  # the stages geer_stage_name names (geer_stage_times fills that many)


_lib_checked = None


def library_path(checked: bool = False) -> str:
    return _build.LIB_CHECKED if checked else _build.LIB


def lib(build_if_missing: bool = True, checked: bool = False):
    """Load libgeer.so, or with checked=True libgeer_checked.so (the build whose
    bounds guards record their first violation), building it in-tree first if
    it is missing."""
    global _lib, _lib_checked
    if checked and _lib_checked is not None:
        return _lib_checked
    if not checked and _lib is not None:
        return _lib
    path = library_path(checked)
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{os.path.basename(path)} not built ({path}); run paper_2505_24053_gb300/build.py")
        _build.build(checked=checked)
    L = C.CDLL(path)
    P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
    L.geer_status_string.restype = C.c_char_p
    L.geer_status_string.argtypes = [C.c_int]
    L.geer_stage_name.restype = C.c_char_p
    L.geer_stage_name.argtypes = [C.c_int32]
    sigs = {
        "geer_default_params": [P],
        "geer_workspace_size": [P, I32, I64, I32, I64, P],
        "geer_workspace_init": [P, C.c_size_t, P, I32, I64, I32, I64, P, P],
        "geer_workspace_destroy": [P],
        "geer_set_cameras": [P, P, I32, P],
        "geer_preprocess": [P, P, P],
        "geer_bin_sort": [P, P, P],
        "geer_render_fwd": [P, P, P, P],
        "geer_render_bwd": [P, P, P, P, P, P, P, P, I32, P],
        "geer_last_device_status": [P, P, P],
        "geer_debug_preprocess": [P, P, P, P, P, P],
        "geer_debug_pairs": [P, P, P, I64, P, P],
        "geer_render_counts": [P, P, P, P, P],
        "geer_enable_timing": [P, I32],
        "geer_stage_times": [P, P, I32, P, P],
        "geer_remap_to_native": [P, P, P, P, P],
        "geer_native_regions": [P, P, P],
        "geer_native_to_beap": [P, P, P, P, P],
        "geer_adam_step": [P, I64, I32, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P],
        "geer_image_metrics": [P, P, I32, I32, P, I32, P, P, P],
        "geer_pair_counts": [P, P, P, P, P, P],
        "geer_debug_render_state": [P, P, P, P, P],
        "geer_l1_loss_grad": [P, P, I64, P, P, P],
        "geer_render_noalloc": [P, P, P, P, P, P],
        "geer_set_camera_slots": [P, P, I32, P, I64, I64, P],
        "geer_densify_accumulate": [P, P, P, P, P],
        "geer_densify_plan": [P, I64, P, P, P, P, P, C.c_size_t, P, P],
        "geer_densify_apply": [I64, I32, P, P, P, P, P, P, P, P, P, C.c_size_t, I64, P, P, P, P, P, P, P, P, P, P],
        "geer_opacity_reset": [I64, I32, C.c_float, P, P, P, P, P],
        "geer_render_bwd_tiles": [P, P, P],
        "geer_render_train_l1": [P, P, P, P, P, P, P],
        "geer_grad_accumulators": [P, P, P],
        "geer_preprocess_bwd": [P, P, P, P, P, P, P, I32, P],
        "geer_tile_owners": [P, I32, I32, P],
        "geer_set_tile_mask": [P, P, I64, P],
        "geer_tile_counts": [P, P, P],
        "geer_bounds_violation": [P, P, P, P],
        "geer_debug_set_render_order": [P, P, I64, P],
        "geer_enable_stage_timing": [P, C.c_uint32],
    }
    for name, args in sigs.items():
        f = getattr(L, name)
        f.restype = C.c_int
        f.argtypes = args
    L.geer_densify_scratch_bytes.restype = C.c_size_t
    L.geer_densify_scratch_bytes.argtypes = [I64]
    L.geer_checked_build.restype = C.c_int32
    L.geer_checked_build.argtypes = []
    if checked:
        _lib_checked = L
    else:
        _lib = L
    return L


def status_string(s: int) -> str:
    return lib().geer_status_string(int(s)).decode()


def _check(status: int, what: str):
    if status != OK:
        raise GeerError(status, what)


def camera_c(cam) -> CameraC:
    """Convert a workloads.Camera (or any object with the same fields)."""
    c = CameraC()
    c.model, c.width, c.height = int(cam.model), int(cam.width), int(cam.height)
    c.fov_x, c.fov_y = float(cam.fov_x), float(getattr(cam, "fov_y", 0.0) or 0.0)
    k = getattr(cam, "k", (0, 0, 0, 0))
    for i in range(4):
        c.k[i] = float(k[i])
    R = np.asarray(getattr(cam, "R_cw", np.eye(3)), np.float32).ravel()
    t = np.asarray(getattr(cam, "t_cw", np.zeros(3)), np.float32).ravel()
    bg = getattr(cam, "bg", (1.0, 1.0, 1.0))
    for i in range(9):
        c.R_cw[i] = float(R[i])
    for i in range(3):
        c.t_cw[i] = float(t[i])
        c.bg[i] = float(bg[i])
    return c


def cameras_c(cams):
    arr = (CameraC * len(cams))()
    for i, cam in enumerate(cams):
        arr[i] = camera_c(cam)
    return arr


ASSOC_PBF, ASSOC_EWA, ASSOC_UT = 0, 1, 2  # tile association methods (GEER_ASSOC_*)
ALPHA_EXACT, ALPHA_SPLAT = 0, 1  # per-ray alpha models (GEER_ALPHA_*)


def params_c(alpha_min=1 / 255, T_min=1e-4, alpha_max=0.99, lambda_pad=1e-3, assoc: int = ASSOC_PBF,
             snugbox: bool = False, alpha_model: int = ALPHA_EXACT) -> ParamsC:
    p = ParamsC()
    p.tile_w = p.tile_h = 16
    p.alpha_min, p.T_min, p.alpha_max, p.lambda_pad = alpha_min, T_min, alpha_max, lambda_pad
    p.assoc, p.snugbox, p.alpha_model = int(assoc), int(bool(snugbox)), int(alpha_model)
    return p


class Gaussians:
    """Device-resident Gaussians (contiguous FP32 CUDA tensors)."""

    def __init__(self, mean, scale, quat, opacity, sh, sh_degree: int):
        def dev(x):
            t = torch.as_tensor(x, dtype=torch.float32)
            if t.device.type != "cuda":
                t = t.cuda()
            return t.contiguous()

        self.mean, self.scale, self.quat, self.opacity, self.sh = (dev(x) for x in (mean, scale, quat, opacity, sh))
        self.sh_degree = int(sh_degree)
        self.n = int(self.mean.shape[0])

    @classmethod
    def from_scene(cls, scene):
        return cls(scene.mean, scene.scale, scene.quat, scene.opacity, scene.sh, scene.sh_degree)

    def c_struct(self) -> GaussiansC:
        g = GaussiansC()
        g.mean, g.scale, g.quat = self.mean.data_ptr(), self.scale.data_ptr(), self.quat.data_ptr()
        g.opacity, g.sh = self.opacity.data_ptr(), self.sh.data_ptr()
        g.n, g.sh_degree = self.n, self.sh_degree
        return g


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Workspace:
    """A geer workspace in a torch-owned device buffer."""

    def __init__(self, cams, n_gauss: int, sh_degree: int, pair_capacity: int, params: ParamsC | None = None,
                 device=None, library=None):
        L = self._L = library or lib()
        self.cams = list(cams)
        self._cams_c = cameras_c(self.cams)
        self.n_gauss, self.sh_degree, self.pair_capacity = int(n_gauss), int(sh_degree), int(pair_capacity)
        self.params = params or params_c()
        nbytes = C.c_size_t()
        _check(L.geer_workspace_size(self._cams_c, len(self.cams), self.n_gauss, self.sh_degree, self.pair_capacity,
                                     C.byref(nbytes)), "geer_workspace_size")
        self.nbytes = int(nbytes.value)
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device or "cuda")
        base = self.buf.data_ptr()
        aligned = (base + 255) & ~255
        self._handle = C.c_void_p()
        torch.cuda.current_stream().synchronize()
        _check(L.geer_workspace_init(C.c_void_p(aligned), self.nbytes, self._cams_c, len(self.cams), self.n_gauss,
                                     self.sh_degree, self.pair_capacity, C.byref(self.params),
                                     C.byref(self._handle)), "geer_workspace_init")
        self.pixels = sum(c.width * c.height for c in self.cams)

    def __del__(self):
        h = getattr(self, "_handle", None)
        L = getattr(self, "_L", None)
        if h is not None and h.value and L is not None:
            L.geer_workspace_destroy(h)
            self._handle = None

    @property
    def handle(self):
        return self._handle

    def set_cameras(self, cams, stream=None):
        self.cams = list(cams)
        self._cams_c = cameras_c(self.cams)
        _check(self._L.geer_set_cameras(self._handle, self._cams_c, len(self.cams), _stream(stream)),
               "geer_set_cameras")
        self.pixels = sum(c.width * c.height for c in self.cams)

    def set_camera_slots(self, cams, active, slot_tiles: int, slot_pixels: int, stream=None):
        """Place camera i at fixed slot i (see geer_set_camera_slots); active: list of bools."""
        arr = cameras_c(cams)
        act = (C.c_uint8 * len(cams))(*[1 if a else 0 for a in active])
        _check(self._L.geer_set_camera_slots(self._handle, arr, len(cams), act, int(slot_tiles), int(slot_pixels),
                                           _stream(stream)), "geer_set_camera_slots")
        self.cams = list(cams)
        self._slots = (list(active), int(slot_tiles), int(slot_pixels))

    def preprocess(self, g: Gaussians, stream=None):
        self._g = g
        self._gc = g.c_struct()
        _check(self._L.geer_preprocess(self._handle, C.byref(self._gc), _stream(stream)), "geer_preprocess")

    def bin_sort(self, sync: bool = True, stream=None) -> int | None:
        """Duplicate, sort and range. With sync=True returns the pair count and
        raises GeerError(ERR_CAPACITY) if it exceeds the capacity."""
        if sync:
            need = C.c_int64()
            st = self._L.geer_bin_sort(self._handle, C.byref(need), _stream(stream))
            self.last_pairs = int(need.value)
            _check(st, "geer_bin_sort")
            return self.last_pairs
        _check(self._L.geer_bin_sort(self._handle, None, _stream(stream)), "geer_bin_sort")
        return None

    def render_fwd(self, rgb: torch.Tensor, T: torch.Tensor | None = None, stream=None):
        _check(self._L.geer_render_fwd(self._handle, C.c_void_p(rgb.data_ptr()),
                                     C.c_void_p(T.data_ptr()) if T is not None else None, _stream(stream)),
               "geer_render_fwd")

    def render_bwd(self, g: Gaussians, dL_drgb: torch.Tensor, grads: dict, accumulate: bool = True, stream=None):
        """Gradients into grads' tensors: added to them (accumulate) or written."""
        gc = g.c_struct()

        def ptr(name):
            t = grads.get(name)
            return C.c_void_p(t.data_ptr()) if t is not None else None

        _check(self._L.geer_render_bwd(self._handle, C.byref(gc), C.c_void_p(dL_drgb.data_ptr()), ptr("mean"),
                                     ptr("scale"), ptr("quat"), ptr("opacity"), ptr("sh"), 1 if accumulate else 0,
                                     _stream(stream)),
               "geer_render_bwd")

    def render_train_l1(self, target: torch.Tensor, rgb: torch.Tensor, dL_drgb: torch.Tensor,
                        loss: torch.Tensor | None = None, T_final: torch.Tensor | None = None, stream=None):
        """Forward, L1 gradient against target and the backward's render stage in
        one launch (geer_render_train_l1): rgb, dL_drgb, loss (a device f32 [1],
        or None) and the accumulators, as render_fwd + l1_loss_grad +
        render_bwd_tiles; then preprocess_bwd."""
        _check(self._L.geer_render_train_l1(self._handle, C.c_void_p(target.data_ptr()), C.c_void_p(rgb.data_ptr()),
                                          C.c_void_p(T_final.data_ptr()) if T_final is not None else None,
                                          C.c_void_p(dL_drgb.data_ptr()),
                                          C.c_void_p(loss.data_ptr()) if loss is not None else None,
                                          _stream(stream)),
               "geer_render_train_l1")

    def render_bwd_tiles(self, dL_drgb: torch.Tensor, stream=None):
        """The render stage of the backward (geer_render_bwd_tiles): the
        per-(camera, Gaussian) accumulators over the rendered tiles' rays."""
        _check(self._L.geer_render_bwd_tiles(self._handle, C.c_void_p(dL_drgb.data_ptr()), _stream(stream)),
               "geer_render_bwd_tiles")

    def grad_accumulators(self) -> torch.Tensor:
        """The render stage's accumulators [n_cams * n, 16] f32 as a view of the
        workspace's own memory (reading or replacing them, e.g. by an all-reduce
        over processes, acts on the workspace)."""
        ptr = C.c_void_p()
        n = C.c_int64()
        _check(self._L.geer_grad_accumulators(self._handle, C.byref(ptr), C.byref(n)), "geer_grad_accumulators")
        off = int(ptr.value or 0) - self.buf.data_ptr()
        nbytes = 4 * int(n.value)
        if n.value == 0:
            return torch.empty((0, 16), dtype=torch.float32, device=self.buf.device)
        assert 0 <= off and off + nbytes <= self.buf.numel()
        return self.buf[off:off + nbytes].view(torch.float32).view(-1, 16)

    def preprocess_bwd(self, g: Gaussians, grads: dict, accumulate: bool = True, stream=None):
        """The preprocess stage of the backward (geer_preprocess_bwd) from the accumulators."""
        gc = g.c_struct()

        def ptr(name):
            t = grads.get(name)
            return C.c_void_p(t.data_ptr()) if t is not None else None

        _check(self._L.geer_preprocess_bwd(self._handle, C.byref(gc), ptr("mean"), ptr("scale"), ptr("quat"),
                                         ptr("opacity"), ptr("sh"), 1 if accumulate else 0, _stream(stream)),
               "geer_preprocess_bwd")

    def set_tile_mask(self, mask, stream=None):
        """Render only the tiles with mask != 0 (host array of the camera set's
        tile count), or all tiles with mask=None (geer_set_tile_mask)."""
        if mask is None:
            _check(self._L.geer_set_tile_mask(self._handle, None, 0, _stream(stream)), "geer_set_tile_mask")
            return
        m = np.ascontiguousarray(np.asarray(mask).astype(np.uint8))
        _check(self._L.geer_set_tile_mask(self._handle, C.c_void_p(m.ctypes.data), int(m.size), _stream(stream)),
               "geer_set_tile_mask")

    def bounds_violation(self, stream=None):
        """(site, index) of the first failing bounds guard since the last read
        ((0, 0) if none; always none outside the checked build)."""
        site, index = C.c_uint32(), C.c_int64()
        _check(self._L.geer_bounds_violation(self._handle, C.byref(site), C.byref(index), _stream(stream)),
               "geer_bounds_violation")
        return int(site.value), int(index.value)

    def set_render_order(self, order, stream=None):
        """Replace the forward's tile schedule (geer_debug_set_render_order)."""
        o = np.ascontiguousarray(np.asarray(order, np.uint32))
        _check(self._L.geer_debug_set_render_order(self._handle, C.c_void_p(o.ctypes.data), int(o.size),
                                                   _stream(stream)), "geer_debug_set_render_order")

    def device_status(self, stream=None):
        pairs = C.c_int64()
        st = self._L.geer_last_device_status(self._handle, C.byref(pairs), _stream(stream))
        return st, int(pairs.value)

    def debug_preprocess(self, stream=None):
        m = len(self.cams) * self._g.n
        ranges = np.zeros((m, 8), np.uint16)
        counts = np.zeros(m, np.uint32)
        keys = np.zeros(m, np.uint32)
        cull = np.zeros(m, np.uint8)
        P = C.c_void_p
        _check(self._L.geer_debug_preprocess(self._handle, P(ranges.ctypes.data), P(counts.ctypes.data),
                                           P(keys.ctypes.data), P(cull.ctypes.data), _stream(stream)),
               "geer_debug_preprocess")
        return cull, keys, ranges, counts

    def render_counts(self, stream=None):
        """(evaluations executed, contributors applied, entries walked by the backward)
        of the last forward render."""
        e, a, w = C.c_uint64(), C.c_uint64(), C.c_uint64()
        _check(self._L.geer_render_counts(self._handle, C.byref(e), C.byref(a), C.byref(w), _stream(stream)),
               "geer_render_counts")
        return int(e.value), int(a.value), int(w.value)

    def pair_counts(self, stream=None):
        """(tile-Gaussian associations P, super-tile pairs sorted) of the last bin_sort."""
        t, u = C.c_int64(), C.c_int64()
        _check(self._L.geer_pair_counts(self._handle, C.byref(t), C.byref(u), None, None, _stream(stream)),
               "geer_pair_counts")
        return int(t.value), int(u.value)

    def live_items(self, stream=None) -> int:
        """Live (camera, Gaussian) items of the last bin_sort."""
        n = C.c_int64()
        _check(self._L.geer_pair_counts(self._handle, None, None, None, C.byref(n), _stream(stream)), "geer_pair_counts")
        return int(n.value)

    def sort_passes(self, stream=None) -> int:
        """Radix passes of the super-tile sort for the current cameras."""
        p = C.c_int32()
        _check(self._L.geer_pair_counts(self._handle, None, None, C.byref(p), None, _stream(stream)), "geer_pair_counts")
        return int(p.value)

    def tile_counts(self, stream=None) -> np.ndarray:
        """Every tile's list length ((tile, Gaussian) associations) after bin_sort."""
        n = sum(((c.width + 15) // 16) * ((c.height + 15) // 16) for c in self.cams)
        out = np.zeros(n, np.uint32)
        _check(self._L.geer_tile_counts(self._handle, C.c_void_p(out.ctypes.data), _stream(stream)), "geer_tile_counts")
        return out

    def debug_render_state(self, stream=None):
        """Per ray (evaluations, contributors) [n_pixels, 2] and last [n_pixels]; per tile
        the forward's walk record [n_tiles, 2] (super-list position, entries)."""
        npix = sum(c.width * c.height for c in self.cams)
        ntiles = sum(((c.width + 15) // 16) * ((c.height + 15) // 16) for c in self.cams)
        ev = np.zeros((npix, 2), np.uint32)
        last = np.zeros(npix, np.uint32)
        walk = np.zeros((ntiles, 2), np.uint32)
        _check(self._L.geer_debug_render_state(self._handle, C.c_void_p(ev.ctypes.data), C.c_void_p(last.ctypes.data),
                                             C.c_void_p(walk.ctypes.data), _stream(stream)),
               "geer_debug_render_state")
        return ev, last, walk

    def enable_timing(self, on: bool = True, stages=None):
        """Stage timing on (every stage, or the named stages only) or off."""
        if stages is None or not on:
            _check(self._L.geer_enable_timing(self._handle, 1 if on else 0), "geer_enable_timing")
            return
        names = [self._L.geer_stage_name(i).decode() for i in range(N_STAGES)]
        mask = sum(1 << names.index(n) for n in stages)
        _check(self._L.geer_enable_stage_timing(self._handle, mask), "geer_enable_stage_timing")

    def stage_times(self, stream=None) -> dict:
        """Mean ms of the recorded occurrences of each stage (timing must be enabled)."""
        ms = (C.c_float * 16)()
        cnt = (C.c_int32 * 16)()
        _check(self._L.geer_stage_times(self._handle, ms, 16, cnt, _stream(stream)), "geer_stage_times")
        return {self._L.geer_stage_name(i).decode(): (float(ms[i]), int(cnt[i])) for i in range(N_STAGES)}

    def debug_pairs(self, cap: int | None = None, stream=None):
        cap = self.pair_capacity if cap is None else cap
        keys = np.zeros(cap, np.uint64)
        vals = np.zeros(cap, np.uint32)
        count = C.c_int64()
        _check(self._L.geer_debug_pairs(self._handle, C.c_void_p(keys.ctypes.data), C.c_void_p(vals.ctypes.data), cap,
                                      C.byref(count), _stream(stream)), "geer_debug_pairs")
        n = min(int(count.value), cap)
        return keys[:n], vals[:n]


def tile_owners(cams, n_parts: int) -> np.ndarray:
    """Owner part of every tile of the camera set (geer_tile_owners, host only):
    int32 [total tiles] in geer_set_cameras' tile order."""
    arr = cameras_c(cams)
    n = sum(((c.width + 15) // 16) * ((c.height + 15) // 16) for c in cams)
    out = np.zeros(n, np.int32)
    _check(lib().geer_tile_owners(arr, len(cams), int(n_parts), C.c_void_p(out.ctypes.data)), "geer_tile_owners")
    return out


def l1_loss_grad(rgb: torch.Tensor, target: torch.Tensor, grad: torch.Tensor | None = None, stream=None):
    """L1 loss mean|rgb - target| and its gradient, computed by the library kernel.
    Returns (loss tensor [1] on the device, dL/drgb)."""
    if grad is None:
        grad = torch.empty_like(rgb)
    loss = torch.empty(1, dtype=torch.float32, device=rgb.device)
    _check(lib().geer_l1_loss_grad(C.c_void_p(rgb.data_ptr()), C.c_void_p(target.data_ptr()), rgb.numel(),
                                   C.c_void_p(grad.data_ptr()), C.c_void_p(loss.data_ptr()), _stream(stream)),
           "geer_l1_loss_grad")
    return loss, grad


def remap_to_native(beap_img: torch.Tensor, cam, fill=(0.0, 0.0, 0.0), out: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
    """Native camera image [h, w, 3] from the camera's BEAP render [h, w, 3]."""
    if out is None:
        out = torch.empty_like(beap_img)
    cc = camera_c(cam)
    f = (C.c_float * 3)(*[float(x) for x in fill])
    _check(lib().geer_remap_to_native(C.c_void_p(beap_img.data_ptr()), C.byref(cc), f, C.c_void_p(out.data_ptr()),
                                      _stream(stream)), "geer_remap_to_native")
    return out


def native_regions(cam, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """[h, w] uint8 evaluation region of each native pixel: 0 central, 1 peripheral,
    255 without a ray in the BEAP grid."""
    if out is None:
        out = torch.empty((cam.height, cam.width), dtype=torch.uint8, device="cuda")
    cc = camera_c(cam)
    _check(lib().geer_native_regions(C.byref(cc), C.c_void_p(out.data_ptr()), _stream(stream)), "geer_native_regions")
    return out


def image_metrics(pred: torch.Tensor, gt: torch.Tensor, regions: torch.Tensor | None = None, n_regions: int = 1,
                  stream=None) -> list[dict]:
    """Per region: PSNR, mean SSIM and pixel count of pred against gt ([h, w, 3] f32)."""
    h, w = int(pred.shape[0]), int(pred.shape[1])
    acc = torch.empty(3 * n_regions, dtype=torch.float64, device=pred.device)
    out = (C.c_double * (5 * n_regions))()
    reg = C.c_void_p(regions.data_ptr()) if regions is not None else None
    _check(lib().geer_image_metrics(C.c_void_p(pred.data_ptr()), C.c_void_p(gt.data_ptr()), w, h, reg, n_regions,
                                    C.c_void_p(acc.data_ptr()), out, _stream(stream)), "geer_image_metrics")
    return [{"sse": out[5 * r], "ssim_sum": out[5 * r + 1], "count": int(out[5 * r + 2]), "psnr": out[5 * r + 3],
             "ssim": out[5 * r + 4]} for r in range(n_regions)]


def native_to_beap(native_img: torch.Tensor, cam, out: torch.Tensor | None = None,
                   valid: torch.Tensor | None = None, stream=None):
    """(BEAP supervision [h, w, 3], valid [h, w] uint8) of a native camera image [h, w, 3]."""
    if out is None:
        out = torch.empty_like(native_img)
    if valid is None:
        valid = torch.empty((cam.height, cam.width), dtype=torch.uint8, device=native_img.device)
    cc = camera_c(cam)
    _check(lib().geer_native_to_beap(C.c_void_p(native_img.data_ptr()), C.byref(cc), C.c_void_p(out.data_ptr()),
                                     C.c_void_p(valid.data_ptr()), _stream(stream)), "geer_native_to_beap")
    return out, valid


class AdamC(C.Structure):
    _fields_ = [("lr_mean", C.c_float), ("lr_scale", C.c_float), ("lr_quat", C.c_float), ("lr_opacity", C.c_float),
                ("lr_sh_dc", C.c_float), ("lr_sh_rest", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("step", C.c_int32)]


# 3DGS default rates (the mean's is scaled by the scene extent by the caller)
ADAM_DEFAULTS = dict(lr_mean=1.6e-4, lr_scale=5e-3, lr_quat=1e-3, lr_opacity=0.05, lr_sh_dc=2.5e-3,
                     lr_sh_rest=2.5e-3 / 20, beta1=0.9, beta2=0.999, eps=1e-15)


class Adam:
    """Adam over raw Gaussian parameters (mean, log_scale, quat, logit_opacity, sh),
    through geer_adam_step. `gaussians` shares the raw mean / quat / SH tensors and
    holds the activated scale and opacity the step writes: render it directly."""

    def __init__(self, mean, log_scale, quat, logit_opacity, sh, sh_degree: int, **hp):
        def dev(x):
            t = torch.as_tensor(x, dtype=torch.float32)
            return (t.cuda() if t.device.type != "cuda" else t).contiguous().clone()

        self.raw = {"mean": dev(mean), "log_scale": dev(log_scale), "quat": dev(quat),
                    "logit_opacity": dev(logit_opacity), "sh": dev(sh)}
        self.sh_degree = int(sh_degree)
        self.n = int(self.raw["mean"].shape[0])
        self.hp = dict(ADAM_DEFAULTS, **hp)
        per = 11 + 3 * (self.sh_degree + 1) ** 2
        self.m = torch.zeros(self.n * per, dtype=torch.float32, device="cuda")
        self.v = torch.zeros_like(self.m)
        self.t = 0
        self.gaussians = Gaussians(self.raw["mean"], torch.exp(self.raw["log_scale"]), self.raw["quat"],
                                   torch.sigmoid(self.raw["logit_opacity"]), self.raw["sh"], self.sh_degree)

    def step(self, grads: dict, stream=None):
        """One step from the renderer's gradients (dict of mean, scale, quat, opacity, sh)."""
        self.t += 1
        hp = AdamC(**{k: self.hp[k] for k in ("lr_mean", "lr_scale", "lr_quat", "lr_opacity", "lr_sh_dc",
                                              "lr_sh_rest", "beta1", "beta2", "eps")}, step=self.t)
        r, g = self.raw, self.gaussians
        ptr = lambda t: C.c_void_p(t.data_ptr())
        _check(lib().geer_adam_step(C.byref(hp), self.n, self.sh_degree, ptr(r["mean"]), ptr(r["log_scale"]),
                                    ptr(r["quat"]), ptr(r["logit_opacity"]), ptr(r["sh"]), ptr(grads["mean"]),
                                    ptr(grads["scale"]), ptr(grads["quat"]), ptr(grads["opacity"]), ptr(grads["sh"]),
                                    ptr(self.m), ptr(self.v), ptr(g.scale), ptr(g.opacity), _stream(stream)),
               "geer_adam_step")


    def densify(self, accum: torch.Tensor, denom: torch.Tensor, z: torch.Tensor, stream=None, **hp) -> int:
        """Densify and prune (geer_densify_plan / geer_densify_apply) with the
        statistics accum / denom and the split normals z [n, 2, 3]: the raw
        parameters, moments and `gaussians` are replaced by the new set.
        Returns the new count (synchronises)."""
        d = DensifyC(**dict(DENSIFY_DEFAULTS, **hp))
        ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
        L = lib()
        nbytes = L.geer_densify_scratch_bytes(self.n)
        scratch = torch.empty(max(nbytes, 16), dtype=torch.uint8, device="cuda")
        n_out = C.c_int64()
        r = self.raw
        _check(L.geer_densify_plan(C.byref(d), self.n, ptr(r["log_scale"]), ptr(r["logit_opacity"]), ptr(accum),
                                   ptr(denom), ptr(scratch), nbytes, C.byref(n_out), _stream(stream)),
               "geer_densify_plan")
        no = int(n_out.value)
        k = (self.sh_degree + 1) ** 2
        new = {"mean": torch.empty((no, 3), device="cuda"), "log_scale": torch.empty((no, 3), device="cuda"),
               "quat": torch.empty((no, 4), device="cuda"), "logit_opacity": torch.empty(no, device="cuda"),
               "sh": torch.empty((no, k, 3), device="cuda")}
        m = torch.empty(no * (11 + 3 * k), device="cuda")
        v = torch.empty_like(m)
        scale, opacity = torch.empty((no, 3), device="cuda"), torch.empty(no, device="cuda")
        _check(L.geer_densify_apply(self.n, self.sh_degree, ptr(r["mean"]), ptr(r["log_scale"]), ptr(r["quat"]),
                                    ptr(r["logit_opacity"]), ptr(r["sh"]), ptr(self.m), ptr(self.v),
                                    ptr(z.contiguous()), ptr(scratch), nbytes, no, ptr(new["mean"]),
                                    ptr(new["log_scale"]), ptr(new["quat"]), ptr(new["logit_opacity"]),
                                    ptr(new["sh"]), ptr(m), ptr(v), ptr(scale), ptr(opacity), _stream(stream)),
               "geer_densify_apply")
        self.raw, self.m, self.v, self.n = new, m, v, no
        self.gaussians = Gaussians(new["mean"], scale, new["quat"], opacity, new["sh"], self.sh_degree)
        return no

    def opacity_reset(self, value: float = 0.01, stream=None):
        """3DGS opacity reset of the raw logits, their moments and `gaussians`."""
        ptr = lambda t: C.c_void_p(t.data_ptr())
        _check(lib().geer_opacity_reset(self.n, self.sh_degree, value, ptr(self.raw["logit_opacity"]), ptr(self.m),
                                        ptr(self.v), ptr(self.gaussians.opacity), _stream(stream)),
               "geer_opacity_reset")


class DensifyC(C.Structure):
    _fields_ = [("grad_threshold", C.c_float), ("clone_max_scale", C.c_float), ("min_opacity", C.c_float),
                ("max_scale", C.c_float)]


# 3DGS's thresholds (its gradient threshold is for mean2D; ours bounds the
# view-space mean3D gradient norm, a different unit: tune per scene); the clone
# scale is 3DGS's percent_dense (0.01) x the scene extent, here for a 1 m extent
DENSIFY_DEFAULTS = dict(grad_threshold=2e-4, clone_max_scale=0.01, min_opacity=0.005, max_scale=0.0)


def densify_accumulate(ws: "Workspace", d_mean: torch.Tensor, accum: torch.Tensor, denom: torch.Tensor, stream=None):
    """The step's densification statistics (geer_densify_accumulate)."""
    _check(ws._L.geer_densify_accumulate(ws.handle, C.c_void_p(d_mean.data_ptr()), C.c_void_p(accum.data_ptr()),
                                         C.c_void_p(denom.data_ptr()), _stream(stream)), "geer_densify_accumulate")


class Renderer:
    """Forward renders of a camera batch, growing the pair capacity on demand."""

    def __init__(self, cams, n_gauss: int, sh_degree: int, pair_capacity: int | None = None,
                 params: ParamsC | None = None):
        self.cams = list(cams)
        pixels = sum(c.width * c.height for c in self.cams)
        cap = pair_capacity if pair_capacity is not None else max(1 << 16, 4 * n_gauss + pixels // 16)
        self.ws = Workspace(self.cams, n_gauss, sh_degree, cap, params)
        self.n_gauss, self.sh_degree, self.params = n_gauss, sh_degree, params
        self.pixels = pixels

    def _grow(self, need: int):
        cap = int(need * 1.25) + 1024
        self.ws = Workspace(self.cams, self.n_gauss, self.sh_degree, cap, self.params)

    def prepare(self, g: Gaussians) -> int:
        """Preprocess + bin/sort (synchronous pair-count check). Returns P."""
        while True:
            self.ws.preprocess(g)
            try:
                return self.ws.bin_sort(sync=True)
            except GeerError as e:
                if e.status != ERR_CAPACITY:
                    raise
                self._grow(self.ws.last_pairs)

    def forward(self, g: Gaussians, rgb: torch.Tensor | None = None, T: torch.Tensor | None = None):
        self.prepare(g)
        if rgb is None:
            rgb = torch.empty((self.pixels, 3), dtype=torch.float32, device="cuda")
        self.ws.render_fwd(rgb, T)
        return rgb

    def backward(self, g: Gaussians, dL_drgb: torch.Tensor, grads: dict | None = None) -> dict:
        """Gradients of the last forward: accumulated into grads if given, else in
        new tensors (written, not zero-filled first)."""
        accumulate = grads is not None
        if grads is None:
            grads = {k: torch.empty_like(v) for k, v in (("mean", g.mean), ("scale", g.scale), ("quat", g.quat),
                                                         ("opacity", g.opacity), ("sh", g.sh))}
        self.ws.render_bwd(g, dL_drgb.contiguous(), grads, accumulate=accumulate)
        return grads

    def images(self, rgb: torch.Tensor):
        out, off = [], 0
        for c in self.cams:
            n = c.width * c.height
            out.append(rgb[off:off + n].view(c.height, c.width, 3))
            off += n
        return out


class _RenderFn(torch.autograd.Function):
    """rgb = render(mean, scale, quat, opacity, sh); backward through geer_render_bwd."""

    @staticmethod
    def forward(ctx, renderer, sh_degree, mean, scale, quat, opacity, sh):
        g = Gaussians(mean.detach(), scale.detach(), quat.detach(), opacity.detach(), sh.detach(), sh_degree)
        rgb = renderer.forward(g)
        ctx.renderer, ctx.g = renderer, g
        return rgb

    @staticmethod
    def backward(ctx, dL_drgb):
        grads = ctx.renderer.backward(ctx.g, dL_drgb)
        return None, None, grads["mean"], grads["scale"], grads["quat"], grads["opacity"], grads["sh"]


def render(renderer: Renderer, mean, scale, quat, opacity, sh, sh_degree: int) -> torch.Tensor:
    """Differentiable render of all cameras of `renderer`: [sum h*w, 3] f32.

    Gradients flow to mean, scale, quat, opacity (activated) and sh."""
    return _RenderFn.apply(renderer, int(sh_degree), mean, scale, quat, opacity, sh)
