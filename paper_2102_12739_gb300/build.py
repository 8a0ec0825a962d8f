"""Build the CUDA library libdegrid.so in-tree (sm_103a only).

Each translation unit under ``csrc/`` is compiled by nvcc in parallel and the
objects are linked into ``_build/libdegrid.so`` next to this file.  The CUDA
runtime is linked statically, so the library needs only the driver at run
time and loads (without compute) on a machine that has no GPU.

Usage: ``python -m paper_2102_12739_gb300.build [--force] [--verbose]``.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(OUT_DIR, "libdegrid.so")

SOURCES = ["api.cu", "schedule.cu", "degrid.cu", "adjoint.cu", "aux_kernels.cu", "noalloc.cu",
           "host_exec.cu", "peak.cu",
           "gather.cu", "scatter.cu", "predict.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
              "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdegrid.so")


def cuda_lib_dir() -> str:
    """The toolkit's library directory (cuFFT for the subgrid producer)."""
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc())))
    for cand in ("lib64", "lib", os.path.join("targets", "sbsa-linux", "lib"),
                 os.path.join("targets", "x86_64-linux", "lib")):
        d = os.path.join(root, cand)
        if os.path.exists(os.path.join(d, "libcufft.so")):
            return d
    raise RuntimeError(f"libcufft.so not found under {root}")


def link_flags():
    d = cuda_lib_dir()
    return ["-L", d, "-lcufft", "-Xlinker", "-rpath," + d]


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    files += [os.path.join(INCLUDE, "degrid.h"), os.path.abspath(__file__)]
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB_PATH):
        return False
    t = os.path.getmtime(LIB_PATH)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile and link libdegrid.so if it is missing or stale; return its path."""
    if not force and not ptxas_info and up_to_date():
        return LIB_PATH
    os.makedirs(os.path.join(OUT_DIR, "obj"), exist_ok=True)
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, "obj", os.path.splitext(src)[0] + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose or ptxas_info:
        for _, log in results:
            if log.strip():
                sys.stderr.write(log)
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], *link_flags()]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


# Library variants built beside the product library, each in _build/<name>/:
# "bounds" checks every index the coordinate step produces (footprint start,
# GCF rows, 2D weight block, copy-engine box) against the buffers' extents
# and reports a violation through degrid_get_status (DG_ERR_BOUNDS) instead
# of touching memory; the index-safety check the GPU tests run against.
# "timeout" gives the gather kernel's wait for a stage a limit of zero polls
# from a warp's fourth stage on (its copies are then still in flight), so
# that the bounded-wait path runs: the flag that degrid_get_status reports
# as DG_ERR_TIMEOUT, and the full-bound wait for the copies in flight before
# the warp ends; each warp's first three stages are summed normally.
VARIANTS = {"bounds": ("DEGRID_BOUNDS_CHECK",),
            "timeout": ("DG_GATHER_SUM_WAIT_FROM=3", "DG_GATHER_SUM_WAIT_POLLS=0")}


def variant_path(name: str) -> str:
    return os.path.join(OUT_DIR, name, "libdegrid.so")


def build_variant(name: str, force: bool = False) -> str:
    """Compile and link the library variant `name` if it is missing or stale."""
    defines = VARIANTS[name]
    path = variant_path(name)
    if not force and os.path.exists(path) and all(os.path.getmtime(f) <= os.path.getmtime(path)
                                                  for f in _inputs()):
        return path
    out = os.path.dirname(path)
    os.makedirs(out, exist_ok=True)
    cc = nvcc()
    flags = [f"-D{d}" for d in defines]

    def compile_one(src):
        obj = os.path.join(out, os.path.splitext(src)[0] + ".o")
        r = subprocess.run([cc, *ARCH, *NVCC_FLAGS, *flags, "-c", os.path.join(CSRC, src), "-o", obj],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = path + ".tmp%d" % os.getpid()
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs, *link_flags()], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, path)
    return path


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--ptxas-info", action="store_true", help="print -Xptxas -v register usage")
    a = ap.parse_args()
    print(build(force=a.force, verbose=a.verbose, ptxas_info=a.ptxas_info))
