"""Build libsph.so (the CUDA library behind include/sph.h) and libsph_probe.so (the FP32
rate probe behind include/sph_probe.h) in-tree for sm_103a.

Every translation unit is compiled by nvcc for one target, ``-gencode
arch=compute_103a,code=sm_103a``, in parallel, then linked into a shared library with the
CUDA runtime linked statically (the library loads on machines without a GPU, where every
call that needs the device returns SPH_ERR_CUDA).  Objects go to ``_build/`` next to this
file; the library is ``libsph.so`` next to this file.  Both are git-ignored.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(HERE, "libsph.so")
PROBE_PATH = os.path.join(HERE, "libsph_probe.so")

SOURCES = ["sph_scan.cu", "sph_sort.cu", "sph_density.cu", "sph_knn.cu", "sph_solve.cu", "sph_capi.cu",
           "sph_static_eval.cu", "sph_interact.cu"]
PROBE_SOURCES = ["sph_probe.cu"]
HEADERS = [os.path.join(CSRC, h) for h in ("sph_common.cuh", "sph_kernels.cuh", "sph_items.cuh")] + [
    os.path.join(INCLUDE, "sph.h"), os.path.join(INCLUDE, "sph_probe.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
              "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsph.so")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(BUILD_DIR, os.path.splitext(src)[0] + ".o")
    path = os.path.join(CSRC, src)
    if _stale(obj, [path] + HEADERS):
        cmd = [nvcc(), *ARCH, *NVCC_FLAGS, "-c", path, "-o", obj + ".tmp"]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
        if verbose and res.stderr:
            sys.stderr.write(res.stderr)
        os.replace(obj + ".tmp", obj)
    return obj


def _link(path: str, objs, force: bool) -> None:
    if force or _stale(path, objs):
        tmp = path + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"linking {os.path.basename(path)} failed:\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, path)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libsph.so and libsph_probe.so if any source changed; return the
    path of libsph.so."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force:
        for f in os.listdir(BUILD_DIR):
            if f.endswith(".o"):
                os.remove(os.path.join(BUILD_DIR, f))
    srcs = SOURCES + PROBE_SOURCES
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = dict(zip(srcs, ex.map(lambda s: _compile(s, verbose), srcs)))
    _link(LIB_PATH, [objs[s] for s in SOURCES], force)
    _link(PROBE_PATH, [objs[s] for s in PROBE_SOURCES], force)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
