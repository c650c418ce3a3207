"""The C-ABI library builds, loads and exports every entry point include/geer.h
declares; host-side argument checks work without a GPU (no compute calls)."""
import ctypes as C
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "geer.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(geer_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def geer():
    from paper_2505_24053_gb300 import build, geer
    build.build()
    geer.lib()
    return geer


def test_every_declared_symbol_is_exported(geer):
    names = _declared()
    assert len(names) >= 13
    L = geer.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(geer.EXPORTS) <= set(names)


def test_status_strings_and_defaults(geer):
    L = geer.lib()
    assert geer.status_string(geer.OK) == "ok"
    assert "capacity" in geer.status_string(geer.ERR_CAPACITY)
    p = geer.ParamsC()
    assert L.geer_default_params(C.byref(p)) == geer.OK
    assert (p.tile_w, p.tile_h) == (16, 16)
    assert p.alpha_min == pytest.approx(1 / 255) and p.alpha_max == pytest.approx(0.99)
    assert p.T_min == pytest.approx(1e-4) and p.lambda_pad == pytest.approx(1e-3)
    assert (p.assoc, p.snugbox) == (geer.ASSOC_PBF, 0)
    assert L.geer_default_params(None) == geer.ERR_ARG


def test_association_modes_are_validated_on_host(geer):
    """Unknown association methods and SnugBox flags are rejected before any
    device work (the no-allocation entry checks its parameters first)."""
    from paper_2505_24053_gb300 import workloads as wl
    L = geer.lib()
    cam = geer.camera_c(wl.Camera(wl.PINHOLE, 32, 32, math.radians(60)))
    g = geer.GaussiansC()
    g.n, g.sh_degree = 0, 0
    for assoc, snug in ((3, 0), (-1, 0), (1, 2), (2, -1)):
        p = geer.params_c()
        p.assoc, p.snugbox = assoc, snug
        assert L.geer_render_noalloc(C.byref(g), C.byref(cam), C.byref(p), C.c_void_p(256), None, None) == \
            geer.ERR_ARG, (assoc, snug)


def test_workspace_size_checks_arguments_on_host(geer):
    from paper_2505_24053_gb300 import workloads as wl
    L = geer.lib()
    cams = geer.cameras_c([wl.Camera(wl.EQUIDISTANT, 64, 48, math.radians(180))])
    n = C.c_size_t()
    assert L.geer_workspace_size(cams, 1, 1000, 3, 10000, C.byref(n)) == geer.OK
    assert n.value > 1000 * 64
    n2 = C.c_size_t()
    assert L.geer_workspace_size(cams, 1, 2000, 3, 10000, C.byref(n2)) == geer.OK and n2.value > n.value
    bad = [
        wl.Camera(wl.EQUIDISTANT, 0, 48, 1.0),             # empty image
        wl.Camera(wl.PINHOLE, 64, 48, math.radians(190)),  # pinhole beyond 180 deg
        wl.Camera(7, 64, 48, 1.0),                         # unknown model
        wl.Camera(wl.EQUIDISTANT, 64, 48, 7.0),            # FoV >= 2 pi
    ]
    for cam in bad:
        assert L.geer_workspace_size(geer.cameras_c([cam]), 1, 10, 0, 10, C.byref(n)) == geer.ERR_ARG
    assert L.geer_workspace_size(cams, 1, -1, 0, 10, C.byref(n)) == geer.ERR_ARG
    assert L.geer_workspace_size(cams, 1, 10, 4, 10, C.byref(n)) == geer.ERR_ARG
    assert L.geer_workspace_size(cams, 0, 10, 0, 10, C.byref(n)) == geer.ERR_ARG
    assert L.geer_workspace_size(cams, 1, 10, 0, 10, None) == geer.ERR_ARG
    # null handles are rejected before any CUDA call
    assert L.geer_preprocess(None, None, None) == geer.ERR_ARG
    assert L.geer_bin_sort(None, None, None) == geer.ERR_ARG
    assert L.geer_render_fwd(None, None, None, None) == geer.ERR_ARG
    assert L.geer_workspace_destroy(None) == geer.ERR_ARG


def test_densify_arguments_are_checked_on_host(geer):
    """Density control rejects bad thresholds and scratch before any device work."""
    L = geer.lib()
    assert L.geer_densify_scratch_bytes(1000) >= 1000 + 16 and L.geer_densify_scratch_bytes(-1) == 0
    n_out = C.c_int64()
    nb = L.geer_densify_scratch_bytes(10)
    fake = C.c_void_p(1 << 20)  # never dereferenced: every call below fails its checks first
    for bad in (dict(grad_threshold=-1.0), dict(min_opacity=0.0), dict(min_opacity=1.0), dict(clone_max_scale=0.0),
                dict(max_scale=-1.0)):
        d = geer.DensifyC(**dict(geer.DENSIFY_DEFAULTS, **bad))
        assert L.geer_densify_plan(C.byref(d), 10, fake, fake, fake, fake, fake, nb, C.byref(n_out), None) == \
            geer.ERR_ARG, bad
    d = geer.DensifyC(**geer.DENSIFY_DEFAULTS)
    assert L.geer_densify_plan(C.byref(d), 10, fake, fake, fake, fake, C.c_void_p((1 << 20) + 4), nb,
                               C.byref(n_out), None) == geer.ERR_ARG  # misaligned scratch
    assert L.geer_densify_plan(C.byref(d), 10, fake, fake, fake, fake, fake, nb - 1, C.byref(n_out), None) == \
        geer.ERR_ARG  # too small
    assert L.geer_opacity_reset(10, 0, 1.5, fake, fake, fake, None, None) == geer.ERR_ARG
