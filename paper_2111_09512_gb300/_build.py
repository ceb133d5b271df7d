"""Build libsilu.so in-tree for GB300 (sm_103a) with nvcc and g++.

Translation units compile in parallel; the library links the CUDA runtime
statically, so the package directory is self-contained.  A rebuild happens
only when a source or header is newer than the library.
"""
from __future__ import annotations

import os
import re
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsilu.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["kernels_sweep.cu", "kernels_staged.cu", "kernels_krylov.cu", "kernels_trisolve.cu", "kernels_fused.cu", "api.cu", "batch.cu", "server.cu", "noalloc.cu", "diag.cu", "amg.cu", "schur.cu"]
CXX_SOURCES = ["host_factor.cpp", "amg_setup.cpp"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsilu")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "silu.h"))
    files.append(os.path.abspath(__file__))
    return files


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _inputs())


def _run(cmd):
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + p.stdout + p.stderr)
    return p.stdout + p.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA and C++ unit of libsilu for sm_103a; return the .so path."""
    if not force and not stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-I", INCLUDE, "-I", CSRC]
    jobs = []
    objs = []
    for src in CU_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        jobs.append([nvcc, *ARCH, "-lineinfo", *common, "-Xcompiler", "-fPIC", "-Xptxas", "-v",
                     "-c", os.path.join(CSRC, src), "-o", obj])
    for src in CXX_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        # no FMA contraction on the host: factor values and ILUT drop
        # decisions round exactly as written, on x86 and on Arm alike
        jobs.append(["g++", *common, "-fPIC", "-ffp-contract=off", "-c", os.path.join(CSRC, src), "-o", obj])
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(_run, jobs))
    # ptxas resource reports (registers, spills, shared memory per kernel)
    for src, log in zip(CU_SOURCES, logs):
        with open(os.path.join(BUILD, src + ".ptxas.txt"), "w") as fh:
            fh.write(log)
    if verbose:
        for log in logs:
            print(log)
    tmp = LIB + f".tmp{os.getpid()}"
    _run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


def kernel_resources(src: str) -> dict:
    """{mangled kernel name: (registers, spill store bytes, spill load bytes)} from the
    ptxas report of CUDA unit `src` written by the last build."""
    path = os.path.join(BUILD, src + ".ptxas.txt")
    out, name, spills = {}, None, (0, 0)
    with open(path) as fh:
        for line in fh:
            if "Compiling entry function" in line:
                name = line.split("'")[1]
                spills = (0, 0)
                continue
            m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
            if m and name:
                spills = (int(m.group(1)), int(m.group(2)))
            m = re.search(r"Used (\d+) registers", line)
            if m and name:
                out[name] = (int(m.group(1)), *spills)
                name = None
    return out


if __name__ == "__main__":
    print(build(force=True, verbose=True))
