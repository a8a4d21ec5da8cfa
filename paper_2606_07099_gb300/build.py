"""Builds libpf.so in-tree (nvcc for sm_103a, g++ for the host planner).

    python -m paper_2606_07099_gb300.build

The translation units compile in parallel; the library links the CUDA
runtime statically so that it needs nothing but the driver at run time.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def _cuda_home() -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(_nvcc())))


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"command failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stdout + r.stderr


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    cu_flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                       "--expt-relaxed-constexpr"] + inc
    if ptxas_info:
        cu_flags += ["-Xptxas", "-v"]
    cxx = shutil.which("g++") or "g++"
    cxx_flags = ["-O2", "-std=c++17", "-fPIC", "-I", os.path.join(_cuda_home(), "include")] + inc
    jobs = [
        [nvcc, "-c", os.path.join(CSRC, "pf_kernels.cu"), "-o", os.path.join(BUILD, "pf_kernels.o")] + cu_flags,
        [nvcc, "-c", os.path.join(CSRC, "pf_qlim.cu"), "-o", os.path.join(BUILD, "pf_qlim.o")] + cu_flags,
        [nvcc, "-c", os.path.join(CSRC, "pf_bde.cu"), "-o", os.path.join(BUILD, "pf_bde.o")] + cu_flags,
        [nvcc, "-c", os.path.join(CSRC, "pf_noalloc.cu"), "-o", os.path.join(BUILD, "pf_noalloc.o")] + cu_flags,
        [nvcc, "-c", os.path.join(CSRC, "pf_peak.cu"), "-o", os.path.join(BUILD, "pf_peak.o")] + cu_flags,
        [nvcc, "-c", os.path.join(CSRC, "pf_si.cu"), "-o", os.path.join(BUILD, "pf_si.o")] + cu_flags,
        [cxx, "-c", os.path.join(CSRC, "pf_api.cpp"), "-o", os.path.join(BUILD, "pf_api.o")] + cxx_flags,
        [cxx, "-c", os.path.join(CSRC, "pf_plan.cpp"), "-o", os.path.join(BUILD, "pf_plan.o")] + cxx_flags,
    ]
    with ThreadPoolExecutor(len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    tmp = LIB + ".tmp"
    _run([nvcc, "-shared"] + ARCH + ["-o", tmp, os.path.join(BUILD, "pf_kernels.o"),
                                     os.path.join(BUILD, "pf_qlim.o"), os.path.join(BUILD, "pf_bde.o"),
                                     os.path.join(BUILD, "pf_noalloc.o"), os.path.join(BUILD, "pf_peak.o"), os.path.join(BUILD, "pf_si.o"),
                                     os.path.join(BUILD, "pf_api.o"), os.path.join(BUILD, "pf_plan.o"),
                                     "-cudart", "static", "-lpthread", "-ldl", "-lrt"])
    os.replace(tmp, LIB)
    if verbose or ptxas_info:
        for o in outs:
            if o.strip():
                print(o)
    return LIB


if __name__ == "__main__":
    build(verbose=True, ptxas_info="-v" in sys.argv)
    print(LIB)
