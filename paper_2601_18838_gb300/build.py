"""Build libkpme.so in-tree with nvcc for sm_103a.

Each CUDA translation unit is compiled in parallel, then linked into
``paper_2601_18838_gb300/libkpme.so`` (git-ignored).  Usage::

    python -m paper_2601_18838_gb300.build [-v] [--force]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libkpme.so")
LIB_DEBUG = os.path.join(PKG, "libkpme_debug.so")   # the checked build (-DKPME_DEBUG)
SOURCES = ["api.cu", "particles.cu", "skp_build.cu", "gemm_simt.cu", "gemm_tc.cu", "gemm_oz.cu", "gemm_ozt.cu", "gemm_ozf.cu", "noalloc.cu", "batch.cu", "tune.cu", "virial_tensor.cu", "lagrange_modes.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _cuda_lib_dir(nvcc: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")


def _flags(debug: bool = False) -> list[str]:
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                "--expt-relaxed-constexpr"]
    if debug:
        f += ["-DKPME_DEBUG"]
    if os.environ.get("KPME_PTXAS_VERBOSE"):
        f += ["-Xptxas", "-v"]
    return f


def _digest(paths, debug: bool = False) -> str:
    h = hashlib.sha256()
    for p in paths:
        with open(p, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(_flags(debug)).encode())
    return h.hexdigest()


def build(verbose: bool = False, force: bool = False, debug: bool = False) -> str:
    """Compile and link libkpme.so (or, debug=True, the checked build libkpme_debug.so, whose
    particle and mesh kernels check their indices; see in_bounds in kpme_internal.cuh)."""
    nvcc = _nvcc()
    bdir = os.path.join(BUILD, "debug") if debug else BUILD
    lib = LIB_DEBUG if debug else LIB
    os.makedirs(bdir, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    headers = sorted(os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".cuh"))
    deps = srcs + headers + [os.path.join(INCLUDE, "kpme.h")]
    stamp = os.path.join(bdir, "libkpme.stamp")
    dig = _digest(deps, debug)
    if not force and os.path.exists(lib) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == dig:
                return lib

    def compile_one(src: str) -> str:
        obj = os.path.join(bdir, os.path.basename(src).replace(".cu", ".o"))
        cmd = [nvcc, "-c", src, "-o", obj] + _flags(debug)
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    libdir = _cuda_lib_dir(nvcc)
    tmp = lib + ".tmp"
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "shared", "-Xlinker", f"-rpath={libdir}"]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    with open(stamp, "w") as fh:
        fh.write(dig)
    return lib


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("-v", "--verbose", action="store_true")
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--debug", action="store_true", help="the checked build, libkpme_debug.so")
    a = ap.parse_args(argv)
    print(build(a.verbose, a.force, a.debug))
    return 0


if __name__ == "__main__":
    sys.exit(main())
