"""Builds the CUDA library libsem_gb300.so in-tree for sm_103a (nvcc + g++, no cmake).

Translation units are compiled in parallel and linked into one shared object next
to this file.  Run ``python -m paper_1512_02548_gb300.build`` or call
:func:`build_library`.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsem_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["kernels_laplace.cu", "kernels_surface.cu", "capi.cu"]
ORDERS = range(2, 13)            # kernels_order.cu is compiled once per GLL order
CXX_SOURCES = ["tables.cpp"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _run(cmd):
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"command failed: {' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
    return res.stdout + res.stderr


def build_library(verbose: bool = False, ptxas_info: bool = False, defines=(), lib_path: str = LIB,
                  build_dir: str = BUILD) -> str:
    """Compile and link the library.  `defines` (e.g. ["SEM_TRACE"]) builds a diagnostic variant,
    normally with its own `lib_path` and `build_dir`."""
    nvcc = _nvcc()
    os.makedirs(build_dir, exist_ok=True)
    inc = ["-I", CSRC, "-I", os.path.join(os.path.dirname(HERE), "include")] + [f"-D{d}" for d in defines]
    jobs = []
    for src in CU_SOURCES:
        obj = os.path.join(build_dir, src + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "--expt-relaxed-constexpr", *inc, "-c", os.path.join(CSRC, src), "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((cmd, obj))
    for P in ORDERS:
        obj = os.path.join(build_dir, f"kernels_order_p{P}.o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "--expt-relaxed-constexpr", f"-DSEM_ORDER={P}", *inc, "-c",
               os.path.join(CSRC, "kernels_order.cu"), "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((cmd, obj))
    for src in CXX_SOURCES:
        obj = os.path.join(build_dir, src + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", *inc, "-c", os.path.join(CSRC, src), "-o", obj]
        jobs.append((cmd, obj))
    with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        outs = list(ex.map(lambda j: _run(j[0]), jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    tmp = lib_path + ".tmp"
    _run([nvcc, *ARCH, "-shared", "-o", tmp, *[o for _, o in jobs], "-lcudart_static", "-lrt", "-ldl", "-lpthread"])
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build_library(verbose=True, ptxas_info="-v" in sys.argv))
