"""Build the CUDA library ``liblbib.so`` in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into a
shared library next to this file.  Only one -gencode (compute_103a /
sm_103a) is emitted.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
OUT = PKG / "_build"
LIB = PKG / "liblbib.so"
SOURCES = ["fluid.cu", "fluid_direct_a.cu", "fluid_direct_b.cu", "fluid_staged.cu", "particles.cu",
           "step_fused.cu", "adjoint.cu", "api.cu", "shapes.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbib.so")


def _flags(extra=()):
    return ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
            "--expt-relaxed-constexpr", *ARCH, *extra]


def _stale(obj: Path, src: Path) -> bool:
    if not obj.exists():
        return True
    deps = [src] + list(CSRC.glob("*.h")) + list(CSRC.glob("*.cuh")) + [PKG.parent / "include" / "lbib.h"]
    return obj.stat().st_mtime < max(d.stat().st_mtime for d in deps)


def build(force: bool = False, verbose: bool = False, extra=()) -> Path:
    OUT.mkdir(exist_ok=True)
    cc = nvcc()
    jobs = []
    for name in SOURCES:
        src = CSRC / name
        obj = OUT / (name + ".o")
        if force or _stale(obj, src):
            jobs.append([cc, *_flags(extra), "-c", str(src), "-o", str(obj)])
    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, jobs))
    objs = [str(OUT / (n + ".o")) for n in SOURCES]
    if jobs or not LIB.exists():
        tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
        run([cc, *ARCH, "-shared", "-o", str(tmp), *objs, "-lcudart"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [])
    print(LIB)
