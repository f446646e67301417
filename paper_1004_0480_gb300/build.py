"""Build the CUDA library from ``csrc/*.cu`` with nvcc for sm_103a.

Two variants, compiled in parallel and linked with the CUDA runtime linked
statically; each rebuilds only what changed:

  _build/librd.so              the library
  _build_debug/librd_debug.so  the bounds-checked debug variant
                               (RD_DEBUG_BOUNDS, relocatable device code so
                               every kernel shares one error word; loaded
                               when RD_BOUNDS_CHECK=1, see _lib.py)

    python -m paper_1004_0480_gb300.build [--force] [-v]
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "librd.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(BUILD_DEBUG, "librd_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
         f"-I{INCLUDE}", f"-I{CSRC}"]
# (build directory, library, extra compile flags, extra link flags)
VARIANTS = {
    "release": (BUILD, LIB, [], []),
    "debug_bounds": (BUILD_DEBUG, LIB_DEBUG, ["-DRD_DEBUG_BOUNDS", "-rdc=true"], ["-rdc=true"]),
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps_mtime() -> float:
    files = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    files += glob.glob(os.path.join(INCLUDE, "*.h"))
    return max(os.path.getmtime(f) for f in files)


def _compile(src: str, variant: str, force: bool) -> tuple[str, str]:
    bdir, _, cflags, _ = VARIANTS[variant]
    obj = os.path.join(bdir, os.path.basename(src).replace(".cu", ".o"))
    log = obj + ".log"
    if (not force and os.path.exists(obj)
            and os.path.getmtime(obj) >= max(os.path.getmtime(src), _deps_mtime())):
        return obj, ""
    cmd = [nvcc(), *ARCH, *FLAGS, *cflags, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    with open(log, "w") as fh:
        fh.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src} ({variant}):\n{r.stderr[-4000:]}")
    return obj, r.stderr


def _link(variant: str, objs: list[str], force: bool) -> str:
    _, lib, _, lflags = VARIANTS[variant]
    if (force or not os.path.exists(lib)
            or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs)):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, *lflags, "-shared", "-o", tmp, *objs, "-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed ({variant}):\n{r.stderr[-4000:]}")
        os.replace(tmp, lib)
    return lib


def build(force: bool = False, verbose: bool = False,
          variants: tuple[str, ...] = ("release", "debug_bounds")) -> str:
    """Compile and link the requested variants; returns the normal library's
    path (or the only variant's, when one is requested)."""
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    jobs = [(s, v) for v in variants for s in srcs]
    for v in variants:
        os.makedirs(VARIANTS[v][0], exist_ok=True)
    workers = max(1, min(len(jobs), os.cpu_count() or 8))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        results = list(ex.map(lambda j: _compile(j[0], j[1], force), jobs))
    libs = {}
    for v in variants:
        objs = [o for (o, _), (_, vv) in zip(results, jobs) if vv == v]
        libs[v] = _link(v, objs, force)
    if verbose:
        for _, err in results:
            if err:
                print(err, file=sys.stderr)
    return libs.get("release", next(iter(libs.values())))


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
