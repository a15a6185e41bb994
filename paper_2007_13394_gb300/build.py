"""Build libpmnu.so in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in its own nvcc process (in parallel), then one
link step produces ``paper_2007_13394_gb300/libpmnu.so``.  Objects go to
``paper_2007_13394_gb300/_build/``.  Nothing here depends on PyTorch.
"""
from __future__ import annotations

import fcntl
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpmnu.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-O3"]
SOURCES = ["cosmo.cpp", "capi.cu", "k_sort.cu", "k_particles.cu", "k_fft.cu", "k_power.cu",
           "k_ic.cu", "k_power_noalloc.cu", "k_fft_tma.cu", "k_adjoint.cu", "k_mlp.cu", "k_mlp_tc.cu"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpmnu")
    return exe


def _compile(src: str, extra) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if r.stderr.strip():
        sys.stderr.write(r.stderr)
    return obj


def _up_to_date() -> bool:
    newest = max(os.path.getmtime(os.path.join(CSRC, f)) for f in os.listdir(CSRC))
    newest = max(newest, os.path.getmtime(os.path.join(HERE, "..", "include", "pm.h")))
    return os.path.exists(LIB) and os.path.getmtime(LIB) > newest


def build(verbose_ptxas: bool = False, force: bool = False) -> str:
    """Compile every source and link libpmnu.so; returns the library path.  Processes
    that build at the same time (the ranks of one job) take turns on a lock file, and
    each re-checks the library once it holds the lock."""
    os.makedirs(BUILD, exist_ok=True)
    if not force and not verbose_ptxas and _up_to_date():
        return LIB
    with open(os.path.join(BUILD, "build.lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        if not force and not verbose_ptxas and _up_to_date():
            return LIB
        extra = ["-Xptxas", "-v"] if verbose_ptxas else []
        with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
            objs = list(ex.map(lambda s: _compile(s, extra), SOURCES))
        tmp = LIB + ".tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose_ptxas="-v" in sys.argv, force="-f" in sys.argv))
