"""Build the sm_103a RK4IP library (``libxsde.so``) in-tree with nvcc.

Each translation unit (and each precision of the kernel files) is compiled by
its own nvcc process in parallel, then linked into a shared library next to
this file.  The result is git-ignored; every machine builds its own copy.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libxsde.so")
# the bounds-checking build (-DXSDE_BOUNDS=1): every kernel checks its global
# indices and copy ranges (csrc/bounds.cuh); a debugging aid, not the product path
BUILD_BOUNDS = os.path.join(HERE, "_build_bounds")
LIB_BOUNDS = os.path.join(HERE, "libxsde_bounds.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]

# (source, XSDE_REAL_BITS or None[, XSDE_PART]), the longest compiles first
UNITS = [
    ("rk4ip_2d.cu", 64, 1),
    ("rk4ip_2d.cu", 32, 1),
    ("rk4ip_adjoint.cu", 32),
    ("rk4ip_adjoint.cu", 64),
    ("rk4ip_2d.cu", 64, 0),
    ("rk4ip_2d.cu", 32, 0),
    ("rk4ip_1d.cu", 32, 6),
    ("rk4ip_1d.cu", 32, 4),
    ("rk4ip_1d.cu", 32, 5),
    ("rk4ip_1d.cu", 32, 7),
    ("rk4ip_1d.cu", 32, 3),
    ("rk4ip_1d.cu", 32, 2),
    ("rk4ip_1d.cu", 32, 1),
    ("rk4ip_1d.cu", 32, 0),
    ("rk4ip_1d.cu", 64, 6),
    ("rk4ip_1d.cu", 64, 7),
    ("rk4ip_1d.cu", 64, 5),
    ("rk4ip_1d.cu", 64, 4),
    ("rk4ip_1d.cu", 64, 3),
    ("rk4ip_1d.cu", 64, 2),
    ("rk4ip_1d.cu", 64, 1),
    ("rk4ip_1d.cu", 64, 0),
    ("rk4ip_2d_warp.cu", None),
    ("rk4ip_2d_tma.cu", None),
    ("ark45_1d.cu", None),
    ("plain.cu", None),
    ("api.cu", None),
    ("rk4ip_0d.cu", None),
    ("noise.cu", None),
    ("peaks.cu", None),
]


def nvcc() -> str:
    exe = shutil.which("nvcc")
    if exe is None and os.path.exists("/usr/local/cuda/bin/nvcc"):
        exe = "/usr/local/cuda/bin/nvcc"
    if exe is None:
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libxsde.so")
    return exe


def _deps() -> list:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "xsde.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def _compile(unit, verbose: bool, bounds: bool = False) -> str:
    src, bits = unit[0], unit[1]
    part = unit[2] if len(unit) > 2 else None
    stem = os.path.splitext(src)[0] + (f"_f{bits}" if bits else "") + (f"_p{part}" if part is not None else "")
    obj = os.path.join(BUILD_BOUNDS if bounds else BUILD, stem + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *(["-DXSDE_BOUNDS=1"] if bounds else []), "-c", os.path.join(CSRC, src), "-o", obj]
    if bits:
        cmd.insert(-4, f"-DXSDE_REAL_BITS={bits}")
    if part is not None:
        cmd.insert(-4, f"-DXSDE_PART={part}")
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, bounds: bool = False) -> str:
    """Compile and link libxsde.so (or, with bounds, libxsde_bounds.so) unless
    it is newer than every source."""
    lib = LIB_BOUNDS if bounds else LIB
    if not force and up_to_date(lib):
        return lib
    os.makedirs(BUILD_BOUNDS if bounds else BUILD, exist_ok=True)
    workers = max(1, min(len(UNITS), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(lambda u: _compile(u, verbose, bounds), UNITS))
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs, "-lcufft"]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, bounds="--bounds" in sys.argv))
