"""Build the solver's shared library in-tree for sm_103a.

    python -m paper_2101_01776_gb300.build

compiles csrc/*.cu and csrc/*.cpp with nvcc (one process per translation
unit, in parallel) and links paper_2101_01776_gb300/_lib/libirk.so.  Object
files go to paper_2101_01776_gb300/_build/.  Nothing is installed outside the
package directory.

    python -m paper_2101_01776_gb300.build --bounds

builds the bounds-checked debug library _lib/libirk_bounds.so instead
(-DIRK_BOUNDS, objects in _build/bounds/): every checked device index records
a hit instead of reaching memory out of range, and irk_step reports it.  The
binding loads it when IRK_LIBRARY names it.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libirk.so")
BOUNDS_LIB = os.path.join(LIBDIR, "libirk_bounds.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
         "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the solver")
    return cand


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith((".cu", ".cpp")))


def _compile(src: str, bounds: bool = False) -> str:
    obj = os.path.join(BUILD, "bounds" if bounds else "", os.path.basename(src) + ".o")
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    deps.append(os.path.join(ROOT, "include", "irk.h"))
    if os.path.exists(obj) and all(os.path.getmtime(obj) >= os.path.getmtime(d) for d in deps):
        return obj
    cmd = [nvcc()] + ARCH + FLAGS + (["-DIRK_BOUNDS"] if bounds else []) + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def build(verbose: bool = False, bounds: bool = False) -> str:
    """Compile and link the library (the bounds-checked one with bounds=True)."""
    lib = BOUNDS_LIB if bounds else LIB
    os.makedirs(os.path.join(BUILD, "bounds") if bounds else BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    srcs = sources()
    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda f: _compile(f, bounds), srcs))
    if os.path.exists(lib) and all(os.path.getmtime(lib) >= os.path.getmtime(o) for o in objs):
        return lib
    tmp = lib + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print(f"built {lib}")
    return lib


if __name__ == "__main__":
    build(verbose=True, bounds="--bounds" in sys.argv[1:])
    sys.exit(0)
