"""Compile the ib_pf CUDA library for sm_103a (in-tree, no cmake).

Produces ``paper_2104_00350_gb300/_lib/libibpf.so`` from the ``csrc/*.cu`` sources.
Translation units are compiled in parallel, then linked with the static CUDA runtime.
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
CSRC = PKG / "csrc"
OUT_DIR = PKG / "_lib"
LIB = OUT_DIR / "libibpf.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# geometry decisions (subgrid counts, march, averaging cells) want unfused products
PER_FILE = {"geometry.cu": ["-fmad=false"], "geometry3d.cu": ["-fmad=false"]}
SOURCES = ["ib_pf_api.cu", "geometry.cu", "geometry3d.cu", "spectral.cu", "step2d.cu", "step3d.cu",
           "noalloc.cu", "tc_zsolve.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found")


def _compile(src: str, build: Path) -> Path:
    obj = build / (Path(src).stem + ".o")
    cmd = [nvcc(), "-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-O2",
           "-I", str(ROOT / "include"), "-I", str(CSRC), *PER_FILE.get(src, []),
           "-c", str(CSRC / src), "-o", str(obj)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False) -> Path:
    """Build the shared library if any source is newer than it; return its path."""
    srcs = [CSRC / s for s in SOURCES] + list(CSRC.glob("*.h")) + list(CSRC.glob("*.cuh")) + [ROOT / "include" / "ib_pf.h"]
    if LIB.exists() and not force:
        newest = max(p.stat().st_mtime for p in srcs)
        if LIB.stat().st_mtime >= newest:
            return LIB
    build_dir = PKG / "_build"
    build_dir.mkdir(exist_ok=True)
    OUT_DIR.mkdir(exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, build_dir), SOURCES))
    tmp = OUT_DIR / "libibpf.so.tmp"
    cmd = [nvcc(), "-shared", *ARCH, "-cudart", "static", "-o", str(tmp), *map(str, objs)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}", file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
