"""Compile the CUDA library libmrdem.so in-tree for sm_103a.

nvcc for the .cu kernels, g++ (OpenMP) for the host C++, one shared object
linked by nvcc (static CUDA runtime).  Translation units compile in parallel.
"""
from __future__ import annotations

import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmrdem.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")

CU_SOURCES = ["mrdem_detect.cu", "mrdem_forces.cu", "mrdem_closest.cu", "mrdem_merge.cu",
              "mrdem_step.cu", "mrdem_build.cu", "mrdem_frontier.cu"]
CPP_SOURCES = ["mrdem_api.cpp", "mrdem_hierarchy.cpp"]
HEADERS = ["mrdem_geometry.cuh", "mrdem_internal.h", "mrdem_device.cuh", "mrdem_dd.cuh",
           "mrdem_step.cuh"]


def _inputs():
    files = [os.path.join(CSRC, f) for f in CU_SOURCES + CPP_SOURCES + HEADERS]
    files.append(os.path.join(ROOT, "include", "mrdem.h"))
    files.append(os.path.abspath(__file__))
    return files


def _digest(deps, flags):
    """Content hash of the inputs and the compiler flags.  A build is reused
    only when this matches the hash stored beside it: file times are not
    comparable between the machine that edits the sources and the one that
    builds them."""
    h = hashlib.sha256(" ".join(flags).encode())
    for d in deps:
        with open(d, "rb") as f:
            h.update(os.path.basename(d).encode() + b"\0" + f.read())
    return h.hexdigest()


def _stale(target, digest):
    try:
        with open(target + ".inputs") as f:
            return not os.path.exists(target) or f.read().strip() != digest
    except OSError:
        return True


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    deps = _inputs()
    digest = _digest(deps, ARCH + [NVCC, os.uname().machine])
    if not force and not _stale(LIB, digest):
        return LIB
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    jobs = []
    objs = []
    for f in CU_SOURCES:
        o = os.path.join(OUT_DIR, f + ".o")
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "--expt-relaxed-constexpr", *inc, "-c", os.path.join(CSRC, f), "-o", o]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append(cmd)
        objs.append(o)
    for f in CPP_SOURCES:
        o = os.path.join(OUT_DIR, f + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-fopenmp", *inc,
               "-I", os.path.join(CUDA_HOME, "include"), "-c", os.path.join(CSRC, f), "-o", o]
        jobs.append(cmd)
        objs.append(o)
    procs = [(cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
             for cmd in jobs]
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose or ptxas_info:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("compilation failed:\n" + "\n".join(failed))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fopenmp",
                           "-lgomp"])
    os.replace(tmp, LIB)
    with open(LIB + ".inputs", "w") as f:
        f.write(digest + "\n")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
