"""Build libpfem.so (the CUDA kernels + C ABI) in-tree for sm_103a with nvcc.

Translation units compile in parallel; the library is linked with the static CUDA runtime
so it only needs the driver.  Objects land in ``_build/`` beside this file.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpfem.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
              "-I" + INCLUDE]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _deps_mtime() -> float:
    files = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    files += glob.glob(os.path.join(INCLUDE, "*.h"))
    return max(os.path.getmtime(f) for f in files)


def build(verbose: bool = False, force: bool = False, ptxas_info: bool = False,
          extra_flags=None, lib_path: str = None, build_dir: str = None) -> str:
    """Compile every translation unit and link libpfem.so.  `extra_flags` (or the
    PFEM_NVCC_FLAGS environment variable, space separated) are appended to the nvcc flags;
    `lib_path`/`build_dir` redirect the outputs (used to build tuning variants side by side)."""
    global BUILD, LIB
    out_lib, out_dir = lib_path or LIB, build_dir or BUILD
    extra_flags = list(extra_flags or []) + os.environ.get("PFEM_NVCC_FLAGS", "").split()
    if extra_flags and build_dir is None:
        out_dir = BUILD + "_" + "_".join(f.strip("-").replace("=", "") for f in extra_flags)
    os.makedirs(out_dir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    dep_t = _deps_mtime()
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + extra_flags

    def compile_one(src: str):
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        if (not force and not ptxas_info and os.path.exists(obj)
                and os.path.getmtime(obj) > max(os.path.getmtime(src), dep_t)):
            return obj, ""
        cmd = [nvcc()] + ARCH + NVCC_FLAGS + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, srcs))
    objs = [o for o, _ in results]
    if verbose or ptxas_info:
        for _, log in results:
            if log:
                print(log)
    if force or not os.path.exists(out_lib) or os.path.getmtime(out_lib) < max(os.path.getmtime(o) for o in objs):
        tmp = out_lib + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, out_lib)
    return out_lib


if __name__ == "__main__":
    import sys
    print(build(verbose=True, force="--force" in sys.argv, ptxas_info="--ptxas" in sys.argv))
