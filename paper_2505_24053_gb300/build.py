"""In-tree build of the CUDA library libgeer.so for sm_103a (GB300).

Each translation unit under csrc/ is compiled by its own nvcc process in
parallel, then linked into paper_2505_24053_gb300/_build/libgeer.so. Host code is
compiled with -ffp-contract=off so that FP64 camera tables do not depend on
the host compiler's multiply-add contraction.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libgeer.so")
# the checked build: the same sources with GEER_CHECKED=1 (bounds guards record
# their first violation in the device status word)
OUT_CHECKED = os.path.join(OUT, "checked")
LIB_CHECKED = os.path.join(OUT, "libgeer_checked.so")
SOURCES = ["geer_host.cu", "preprocess.cu", "sort.cu", "render.cu", "backward.cu", "remap.cu", "metrics.cu", "train.cu", "densify.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgeer")


def flags(verbose_ptxas: bool = False) -> list[str]:
    f = ["-O3", "-lineinfo", "-std=c++17", *ARCH, "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
         "-I", os.path.join(HERE, "..", "include")]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src, os.path.join(CSRC, "geer_internal.cuh"), os.path.join(HERE, "..", "include", "geer.h"), __file__]
    return any(os.path.getmtime(d) > os.path.getmtime(obj) for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False, checked: bool | None = False) -> str:
    """Compile and link libgeer.so (checked=False), libgeer_checked.so
    (checked=True) or both (checked=None: all translation units of both
    compiled in parallel). Returns the path of the last library linked."""
    variants = [False, True] if checked is None else [bool(checked)]
    cc = nvcc()
    jobs = []  # (variant, source, process)
    objs = {v: [] for v in variants}
    for v in variants:
        out_dir = OUT_CHECKED if v else OUT
        os.makedirs(out_dir, exist_ok=True)
        for src in SOURCES:
            s = os.path.join(CSRC, src)
            o = os.path.join(out_dir, src.replace(".cu", ".o"))
            objs[v].append(o)
            if force or verbose_ptxas or _stale(o, s):
                cmd = [cc, *flags(verbose_ptxas), *(["-DGEER_CHECKED=1"] if v else []), "-c", s, "-o", o]
                jobs.append((v, src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                                                      text=True)))
    failed = []
    for v, src, p in jobs:
        out, _ = p.communicate()
        if out.strip():
            sys.stderr.write(f"--- nvcc {src}{' (checked)' if v else ''}\n{out}")
        if p.returncode != 0:
            failed.append(src + (" (checked)" if v else ""))
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    lib = LIB
    for v in variants:
        lib = LIB_CHECKED if v else LIB
        if any(jv == v for jv, _, _ in jobs) or not os.path.exists(lib):
            tmp = lib + ".tmp"
            subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs[v]], check=True)
            os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, checked=None)
    print(LIB, LIB_CHECKED)
