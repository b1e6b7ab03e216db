"""In-tree build of the CUDA library libmapgb300.so for sm_103a (nvcc + g++, no cmake).

Translation units compile in parallel into _build/, then link into the package
directory.  The FP64 kernels are compiled without FMA contraction (-fmad=false) so that
each operation rounds separately; the FP32 kernels keep contraction.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmapgb300.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE,
               "-diag-suppress", "177,550"]

UNITS = {
    "kernels_f64.cu": ["-fmad=false"],
    "kernels_f32.cu": ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"],
    "kernels_f64_hllc.cu": ["-fmad=false"],
    "kernels_f32_hllc.cu": ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"],
    "kernels_f64_rfx.cu": ["-fmad=false"],
    "kernels_f32_rfx.cu": ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"],
    "kernels_f64_hllc_rfx.cu": ["-fmad=false"],
    "kernels_f32_hllc_rfx.cu": ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"],
    "kernels_f64_hlld.cu": ["-fmad=false"],
    "kernels_f32_hlld.cu": ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"],
    "kernels_f64_hlld_rfx.cu": ["-fmad=false"],
    "kernels_f32_hlld_rfx.cu": ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"],
    "common.cu": ["-fmad=false"],
    "noalloc.cu": ["-fmad=false"],
}
CPP_UNITS = ["tree.cpp", "capi.cpp"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmapgb300.so")


def _cuda_home(nvcc: str) -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _sources():
    out = []
    for f in os.listdir(CSRC):
        if f.endswith((".cu", ".cuh", ".cpp", ".hpp")):
            out.append(os.path.join(CSRC, f))
    out.append(os.path.join(INCLUDE, "map.h"))
    return out


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources()) or \
        os.path.getmtime(__file__) > t


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    nvcc = _nvcc()
    home = _cuda_home(nvcc)
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    for src, extra in UNITS.items():
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *NVCC_COMMON, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        jobs.append((obj, cmd))
    for src in CPP_UNITS:
        obj = os.path.join(BUILD, src.replace(".cpp", ".o"))
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-I", INCLUDE, "-I", os.path.join(home, "include"),
               "-c", os.path.join(CSRC, src), "-o", obj]
        jobs.append((obj, cmd))

    def run(job):
        obj, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        objs = list(ex.map(run, jobs))
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(link)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
