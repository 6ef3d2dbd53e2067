"""Build libht.so (the CUDA library behind include/ht.h) in-tree for sm_103a.

nvcc compiles every csrc/*.cu in parallel with -gencode arch=compute_103a,code=sm_103a
and links them into paper_2304_12152_gb300/_build/libht.so.  No CMake; a rebuild only
recompiles sources newer than their objects.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libht.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-strict-aliasing",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _deps_mtime() -> float:
    files = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return max((os.path.getmtime(f) for f in files), default=0.0)


def _compile(src: str, extra, build_dir: str = BUILD) -> str:
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), _deps_mtime()):
        return obj
    tmp = obj + f".{os.getpid()}.tmp"
    cmd = [NVCC, *ARCH, *FLAGS, *extra, "-c", src, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if "ptxas" in (r.stderr or "") and extra:
        sys.stderr.write(r.stderr)
    os.replace(tmp, obj)
    return obj


def build(verbose: bool = False, force: bool = False, defines=(), build_dir: str = BUILD) -> str:
    """Compile and link; `defines` (e.g. ["HT_CONV_RIL=4"]) go to every translation
    unit, `build_dir` receives the objects and libht.so."""
    os.makedirs(build_dir, exist_ok=True)
    lib = os.path.join(build_dir, "libht.so")
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    if force:
        for f in glob.glob(os.path.join(build_dir, "*.o")):
            os.remove(f)
    extra = (["-Xptxas", "-v"] if verbose else []) + [f"-D{d}" for d in defines]
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, build_dir), srcs))
    if os.path.exists(lib) and os.path.getmtime(lib) >= max(os.path.getmtime(o) for o in objs):
        return lib
    LIB_ = lib
    tmp = LIB_ + f".{os.getpid()}.tmp"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_)
    return LIB_


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
