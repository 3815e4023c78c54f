"""Build the CUDA library (libhh_gb300.so) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library with the CUDA runtime linked statically, so the library has
no dependency on torch.  Usage: ``python -m paper_1211_4752_gb300.build``.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
OUT_DIR = PKG / "_lib"
LIB_NAME = "libhh_gb300.so"
SOURCES = ["hh_api.cu", "hh_kernels_common.cu", "hh_kernels_2d.cu",
           "hh_kernels_3d.cu", "hh_cycle2d.cu", "hh_mid2d.cu", "hh_gmres.cu", "hh_noalloc.cu",
           "hh_krylov.cu", "hh_vcycle2d.cu", "hh_coarse2d.cu", "hh_group2d.cu", "hh_tiled3d.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
         "--extended-lambda", "-Xcompiler", "-fPIC", "-I", str(ROOT / "include")]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not Path(cand).exists():
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return cand


def lib_path() -> Path:
    return OUT_DIR / LIB_NAME


def _compile(src: str, extra: list[str]) -> Path:
    obj = OUT_DIR / (Path(src).stem + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", str(CSRC / src), "-o", str(obj)]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    return obj


def build(verbose: bool = False, extra: list[str] | None = None) -> Path:
    OUT_DIR.mkdir(exist_ok=True)
    extra = list(extra or [])
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    tmp = OUT_DIR / (LIB_NAME + ".tmp")
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", str(tmp),
           *map(str, objs)]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib_path())
    if verbose:
        print(f"built {lib_path()}")
    return lib_path()


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
