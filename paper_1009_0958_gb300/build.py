"""Build libvdf.so (the CUDA library) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel into ``_build/`` and
linked into ``paper_1009_0958_gb300/lib/libvdf.so``.  The FP64 unit is built
without floating-point contraction (its recheck kernel must reproduce the
tile kernel's sums bit for bit).  Rebuilds only when a source is newer than
the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libvdf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-strict-aliasing"]
# extra flags per translation unit; every csrc/*.cu is compiled
UNIT_FLAGS = {
    "vdf_fp64.cu": ["-fmad=false"],
    "vdf_fp64_lp.cu": ["-fmad=false"],
    "vdf_acw64.cu": ["-fmad=false"],
    "vdf_win7_64.cu": ["-fmad=false"],
    # FP32 tile kernels: no denormal can occur (integer-valued data; every
    # guarded quantity is 0 or >= 1e-30), so flush-to-zero drops the denormal
    # fix-ups around rsqrtf/__log2f
    "vdf_fp32_s0.cu": ["-ftz=true"],
    "vdf_fp32_s1.cu": ["-ftz=true"],
    "vdf_fp32_s2.cu": ["-ftz=true"],
    "vdf_fp32_s3.cu": ["-ftz=true"],
    "vdf_batch.cu": ["-ftz=true"],
    "vdf_batch_d0.cu": ["-ftz=true"],
    "vdf_batch_d1.cu": ["-ftz=true"],
    "vdf_batch_d2.cu": ["-ftz=true"],
    "vdf_debug.cu": ["-ftz=true"],
    "vdf_fp32f.cu": ["-ftz=true"],
    "vdf_fp32_lp.cu": ["-ftz=true"],
    "vdf_acw32.cu": ["-ftz=true"],
    "vdf_win7_32.cu": ["-ftz=true"],
}


def units() -> dict[str, list[str]]:
    return {os.path.basename(f): UNIT_FLAGS.get(os.path.basename(f), [])
            for f in sorted(glob.glob(os.path.join(CSRC, "*.cu")))}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvdf")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = glob.glob(os.path.join(CSRC, "*")) + [os.path.join(ROOT, "include", "vdf.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps if os.path.isfile(d))


def _compile(unit: str, extra: list[str], verbose: bool) -> str:
    obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
    cmd = [nvcc(), *ARCH, *COMMON, *extra, "-c", os.path.join(CSRC, unit), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {unit}:\n{res.stdout}\n{res.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libvdf.so; returns its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    todo = units()
    with cf.ThreadPoolExecutor(max_workers=min(len(todo), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda kv: _compile(kv[0], kv[1], verbose), todo.items()))
    tmp = LIB + f".tmp{os.getpid()}"
    res = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread",
                          "-Xlinker", "--no-undefined"],
                         capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
