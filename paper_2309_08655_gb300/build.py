"""In-place build of the CUDA library (sm_103a) with nvcc; no cmake, no torch
extension machinery.  Each translation unit compiles in parallel to an object
file, then nvcc links them into ``librt_axion.so`` next to this file."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librt_axion.so")
SOURCES = ["rt_abi.cu", "rt_sample.cu", "rt_trace.cu", "rt_trace_mixed.cu", "rt_bin.cu",
           "rt_flops.cu", "rt_adjoint.cu", "rt_tail.cu", "rt_trace_rot.cu", "rt_peak.cu",
           "rt_rhs.cu", "rt_trace_df.cu"]
HEADERS = ["rt_device.cuh", "rt_internal.h", "rt_integrator.cuh", "rt_sample_core.cuh",
           "rt_dual.cuh", "rt_backward.cuh", "rt_df.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
           "-Xptxas", "-v"]


def library_path() -> str:
    return LIB


def _nvcc() -> str:
    for cand in [shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]:
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA source for sm_103a and link the shared library."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "rt.h")]
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            cmd = [nvcc, *ARCH, *NVFLAGS, "-I", INCLUDE, "-I", CSRC, "-c", s, "-o", o]
            jobs.append((src, cmd))
    logs = {}
    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        futs = {ex.submit(subprocess.run, cmd, capture_output=True, text=True): src
                for src, cmd in jobs}
        for f in cf.as_completed(futs):
            r = f.result()
            src = futs[f]
            logs[src] = r.stderr
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    if verbose:
        for src, log in logs.items():
            print(f"== {src}\n{log}")
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose=True))
