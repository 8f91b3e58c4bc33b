"""Build the CUDA library libcss.so in-tree (nvcc, sm_103a only).

Each translation unit is compiled in parallel, then linked into
paper_2605_20918_gb300/libcss.so.  Object files go to paper_2605_20918_gb300/_build/.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
SRC = PKG / "csrc"
INC = ROOT / "include"
OUT = PKG / "libcss.so"
BUILD = PKG / "_build"
UNITS = ["css_ctx", "css_color", "css_lanczos", "css_rows", "css_hv_tc", "css_spmm", "css_eigen", "css_density", "css_pbuild",
         "css_noalloc"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the CSS library needs the CUDA toolkit to build")


def _stale() -> bool:
    if not OUT.exists():
        return True
    t = OUT.stat().st_mtime
    deps = list(SRC.glob("*.cu")) + list(SRC.glob("*.cuh")) + [INC / "css.h", Path(__file__)]
    return any(p.stat().st_mtime > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> Path:
    if not force and not _stale():
        return OUT
    BUILD.mkdir(exist_ok=True)
    cc = nvcc()

    def compile_unit(u: str) -> Path:
        obj = BUILD / f"{u}.o"
        cmd = [cc, *ARCH, *FLAGS, f"-I{INC}", "-c", str(SRC / f"{u}.cu"), "-o", str(obj)]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {u}.cu:\n{r.stdout}\n{r.stderr}")
        return obj

    with ThreadPoolExecutor(max_workers=min(len(UNITS), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = OUT.with_suffix(f".{os.getpid()}.tmp.so")
    cmd = [cc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs), "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
