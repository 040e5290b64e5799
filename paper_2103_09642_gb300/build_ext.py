"""In-tree build of the CUDA library (nvcc, sm_103a only).

Five translation units are compiled in parallel and linked into
``paper_2103_09642_gb300/_build/libedupic_gb300.so``:

* ``kernels_f64.cu``  FP64 particle mode, ``-fmad=false`` (no FMA contraction)
* ``kernels_f32.cu``  FP32 particle mode, fast division and square root; fused
  multiply-adds only where the source writes them (every launch shape rounds alike)
* ``edupic_api.cu``   host orchestration of the C ABI (``include/edupic.h``)
* ``edupic_noalloc.cu``  the entry point that works in a fixed static scratch
* ``edupic_server.cu``  the request server (continuous batching)
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libedupic_gb300.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
          "-Xcompiler", "-fno-fast-math", "-Xcompiler", "-pthread"]
UNITS = {
    "kernels_f64.cu": ["-fmad=false"],
    "kernels_f32.cu": ["-fmad=false", "-prec-div=false", "-prec-sqrt=false", "-ftz=true"],
    "edupic_api.cu": ["-fmad=false"],
    "edupic_noalloc.cu": ["-fmad=false"],
    "edupic_server.cu": ["-fmad=false"],
}
HEADERS = ("edupic_internal.h", "edupic_kernels.cuh", "edupic_launch.cuh", "edupic_host.h")


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the extension")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if stale) and return the path of the shared library."""
    os.makedirs(BUILD, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(HERE, "..", "include", "edupic.h")]
    objs = []
    jobs = []
    for unit, flags in UNITS.items():
        src = os.path.join(CSRC, unit)
        obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [src] + hdrs + [__file__]):
            jobs.append([nvcc(), *ARCH, *COMMON, *flags, "-c", src, "-o", obj])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            futs = [ex.submit(subprocess.run, j, capture_output=True, text=True) for j in jobs]
            for j, f in zip(jobs, futs):
                r = f.result()
                if r.returncode != 0:
                    raise RuntimeError(f"nvcc failed: {' '.join(j)}\n{r.stdout}\n{r.stderr}")
                if verbose and (r.stdout or r.stderr):
                    print(r.stdout, r.stderr)
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        r = subprocess.run([nvcc(), *ARCH, "-shared", "-Xcompiler", "-pthread", "-o", tmp, *objs],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
