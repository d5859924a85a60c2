"""Build of the CUDA library `_lib/libtma_smc.so` for sm_103a (in-tree).

Each translation unit is compiled by nvcc in parallel and linked into one
shared library with the CUDA runtime linked statically.  Only stale objects
are rebuilt.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
OBJDIR = os.path.join(LIBDIR, "obj")
LIBPATH = os.path.join(LIBDIR, "libtma_smc.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["wind.cu", "rollout.cu", "rollout_pair.cu", "adjoint.cu", "mala.cu", "resample.cu", "move.cu", "select.cu",
           "batch.cu", "host.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Every CUDA translation unit: single-precision square roots and divisions by
# the hardware approximations (a few ulp), denormals flushed.  All units share
# the flags, so that code compiled in several of them (the step function, the
# Box-Muller transform) gives the same bits everywhere -- the batched path
# reproduces the single-scenario one, the gradient's forward pass decides every
# limit as the rollout does.  Double precision is not affected.
FAST_MATH_SOURCES = {s for s in SOURCES if s.endswith(".cu")}
FAST_MATH_FLAGS = ["-prec-sqrt=false", "-prec-div=false", "-ftz=true"]


def nvcc_path() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(home, "bin", "nvcc")
    if os.path.exists(p):
        return p
    p = shutil.which("nvcc")
    if not p:
        raise RuntimeError("nvcc not found (set CUDA_HOME)")
    return p


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(INCLUDE, "tma_smc.h"))
    return hs


def _flags(ptxas_verbose=False, src=""):
    f = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                "-I", INCLUDE, "-I", CSRC]
    if src in FAST_MATH_SOURCES:
        f += FAST_MATH_FLAGS
    if ptxas_verbose:
        f += ["-Xptxas", "-v"]
    return f


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    os.makedirs(OBJDIR, exist_ok=True)
    nvcc = nvcc_path()
    hdr_mtime = max(os.path.getmtime(h) for h in _headers())
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OBJDIR, src + ".o")
        objs.append(o)
        if force or ptxas_verbose or not os.path.exists(o) or \
                os.path.getmtime(o) < max(os.path.getmtime(s), hdr_mtime):
            jobs.append((s, o))

    def compile_one(job):
        s, o = job
        cmd = [nvcc] + _flags(ptxas_verbose, os.path.basename(s)) + ["-c", s, "-o", o + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {s}:\n{r.stdout}\n{r.stderr}")
        os.replace(o + ".tmp", o)
        return r.stderr

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for log in ex.map(compile_one, jobs):
                if verbose and log:
                    print(log)
    if jobs or force or not os.path.exists(LIBPATH):
        tmp = LIBPATH + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIBPATH)
    return LIBPATH


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_verbose="-v" in sys.argv))
