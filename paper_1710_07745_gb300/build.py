"""Build libcanny.so for sm_103a with nvcc (in-tree, no cmake).

Each ``csrc/*.cu`` compiles to an object in parallel, then one ``nvcc -shared``
link. Output: ``paper_1710_07745_gb300/_build/libcanny.so``; with ``checks=True``
(``--checks``) a checked build (``-DCANNY_CHECKS``: device-side bounds checks
that report instead of faulting) in ``_build_checks/libcanny.so``.

usage: python -m paper_1710_07745_gb300.build [--force] [--checks]
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libcanny.so")
OUT_DIR_CHECKS = os.path.join(PKG, "_build_checks")
LIB_CHECKS = os.path.join(OUT_DIR_CHECKS, "libcanny.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcanny")


def _sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list[str]:
    return _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + \
        sorted(glob.glob(os.path.join(CSRC, "*.h"))) + \
        sorted(glob.glob(os.path.join(INCLUDE, "*.h"))) + [os.path.abspath(__file__)]


def _flags(checks: bool) -> list[str]:
    return NVCC_FLAGS + (["-DCANNY_CHECKS"] if checks else [])


def _stamp(checks: bool = False) -> str:
    h = hashlib.sha256()
    for p in _deps():
        with open(p, "rb") as f:
            h.update(p.encode() + b"\0" + f.read())
    h.update(" ".join(ARCH + _flags(checks)).encode())
    return h.hexdigest()


def up_to_date(checks: bool = False) -> bool:
    lib = LIB_CHECKS if checks else LIB
    stamp_file = lib + ".stamp"
    if not os.path.exists(lib) or not os.path.exists(stamp_file):
        return False
    with open(stamp_file) as f:
        return f.read().strip() == _stamp(checks)


def build(force: bool = False, verbose: bool = False, checks: bool = False) -> str:
    out_dir, lib = (OUT_DIR_CHECKS, LIB_CHECKS) if checks else (OUT_DIR, LIB)
    if not force and up_to_date(checks):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    objs = []

    def compile_one(src: str) -> str:
        obj = os.path.join(out_dir, os.path.splitext(os.path.basename(src))[0] + ".o")
        cmd = [cc, *ARCH, *_flags(checks), "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)
        return obj

    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    with open(lib + ".stamp", "w") as f:
        f.write(_stamp(checks))
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checks="--checks" in sys.argv))
