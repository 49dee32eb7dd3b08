"""Build the native library in-tree: nvcc for sm_103a, one object per translation unit, in parallel.

    python -m paper_1210_2258_b300.build [--force]

Produces paper_1210_2258_b300/lib/libsgp_b300.so.  Objects are rebuilt when a source or header
is newer than the object.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
OBJDIR = os.path.join(HERE, "_build")
LIB = os.path.join(LIBDIR, "libsgp_b300.so")
# the slowest units first, so that the pool starts them first
UNITS = ["k_multi_armx_d.cu", "k_multi_armx_f.cu", "k_multi_land_d.cu", "k_multi_land_f.cu", "k_multi_sgp_b.cu",
         "k_mid_b.cu", "k_mid.cu", "k_large.cu", "k_large_b.cu", "k_small.cu", "k_multi_sgp_a.cu", "k_multi_rest.cu",
         "runtime.cu", "warmstart.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-Wno-deprecated-gpu-targets"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _headers_mtime(unit: str) -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    if unit in ("runtime.cu", "warmstart.cu"):
        hs += glob.glob(os.path.join(HERE, "..", "include", "*.h"))
    return max(os.path.getmtime(h) for h in hs)


def _compile(unit: str, force: bool) -> str:
    src = os.path.join(CSRC, unit)
    obj = os.path.join(OBJDIR, unit.replace(".cu", ".o"))
    if not force and os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), _headers_mtime(unit)):
        return obj
    cmd = [nvcc()] + ARCH + FLAGS + ["-c", src, "-o", obj]
    t0 = time.time()
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {unit}:\n{r.stdout}\n{r.stderr}")
    # date the object by the start of its compilation: a source edited while nvcc ran is newer,
    # so the next build recompiles it (objects of one library must agree on the shared structs)
    os.utime(obj, (t0, t0))
    return obj


def build(force: bool = False) -> str:
    os.makedirs(OBJDIR, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(len(UNITS), os.cpu_count() or 8)) as ex:
        objs = list(ex.map(lambda u: _compile(u, force), UNITS))
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) <= max(os.path.getmtime(o) for o in objs):
        cmd = [nvcc()] + ARCH + ["-shared", "-o", LIB] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
