"""Builds the in-tree shared libraries with nvcc for sm_103a.

``libcog.so`` (the CoG library behind include/cog.h) is compiled from
``csrc/*.cu``: one translation unit per model-state storage type plus the
prior kernel and the host ABI, compiled in parallel, then linked with the
static CUDA runtime so the library loads on a machine without a GPU.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import platform
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build", platform.machine())
LIB = os.path.join(PKG, "libcog.so")
DEBUG_LIB = os.path.join(PKG, "libcog_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# host code: no FP contraction, so the host-side arithmetic (the grouping
# statistics) rounds the same on x86 and Arm
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
                     "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _newer(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, obj: str, headers: list[str], verbose: bool, defs: list[str] | None = None) -> str:
    if not _newer(obj, [src] + headers):
        return ""
    cmd = [nvcc()] + NVCC_FLAGS + (defs or []) + (["-Xptxas", "-v"] if verbose else []) + ["-c", src, "-o",
                                                                                        obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return r.stderr


def build_lib(sources: list[str], headers: list[str], out: str, tag: str, verbose: bool = False,
              defs: list[str] | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    objs = [os.path.join(BUILD, f"{tag}_{os.path.splitext(os.path.basename(s))[0]}.o") for s in sources]
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(sources), os.cpu_count() or 4))) as ex:
        logs = list(ex.map(lambda a: _compile(a[0], a[1], headers, verbose, defs), zip(sources, objs)))
    if verbose:
        for l in logs:
            if l:
                print(l)
    if _newer(out, objs):
        cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "static", "-o", out + ".tmp"] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed for {out}:\n{r.stdout}\n{r.stderr}")
        os.replace(out + ".tmp", out)
    return out


def build(verbose: bool = False, debug: bool = False) -> str:
    """Builds libcog.so, or with debug=True its COG_DEBUG variant
    libcog_debug.so (every data-dependent kernel index bounds-checked)."""
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdrs = sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
                  + glob.glob(os.path.join(ROOT, "include", "*.h")))
    if debug:
        return build_lib(srcs, hdrs, DEBUG_LIB, "cogdbg", verbose, ["-DCOG_DEBUG"])
    return build_lib(srcs, hdrs, LIB, "cog", verbose)


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv))
