"""Build the CUDA library in-tree for sm_103a (nvcc, no CMake).

Each translation unit under ``csrc/`` is compiled in parallel to an object
under ``_build/`` and linked into ``libmhd_gb300.so`` next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmhd_gb300.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
# Translation units whose arithmetic is FP32 bulk: FP32 divide and square
# root use the hardware approximations (about 2 ulp instead of IEEE
# rounding), well inside the 1e-5 tolerance of these forms.  FP64 divide and
# square root are unaffected by these flags.
FAST_FP32_UNITS = {"stage_mixed.cu", "stage_fp32.cu", "batch_mixed.cu", "batch_fp32.cu"}
FAST_FP32_FLAGS = ["-prec-div=false", "-prec-sqrt=false"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the MHD library needs the CUDA toolkit to build")


def _deps() -> list:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)])


# Build variants: the library, and its bounds-checked build (every kernel
# index checked against its array; a violation sets a status bit instead of
# touching memory), a separate in-tree library for small-case tests.
VARIANTS = {"release": ([], "libmhd_gb300.so", "_build"),
            "bounds": (["-DMHD_BOUNDS_CHECK"], "libmhd_gb300_bounds.so", "_build_bounds")}


def variant_path(variant: str = "release") -> str:
    return os.path.join(HERE, VARIANTS[variant][1])


def needs_build(variant: str = "release") -> bool:
    lib = variant_path(variant)
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra: list | None = None, variant: str = "release") -> str:
    vflags, libname, objdir = VARIANTS[variant]
    lib_path = os.path.join(HERE, libname)
    obj_dir = os.path.join(HERE, objdir)
    if not force and not needs_build(variant):
        return lib_path
    os.makedirs(obj_dir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    cc = nvcc()
    flags = NVCC_FLAGS + vflags + (["-Xptxas", "-v"] if verbose else []) + list(extra or [])

    def one(src):
        obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
        unit = flags + (FAST_FP32_FLAGS if os.path.basename(src) in FAST_FP32_UNITS else [])
        cmd = [cc] + ARCH + unit + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        results = list(ex.map(one, srcs))
    if verbose:
        for _, log in results:
            print(log)
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
