"""Build libcht.so in-tree (nvcc, sm_103a, no cmake).

Every ``csrc/*.cu`` file is compiled in parallel to an object file and the
objects are linked into ``paper_2011_11762_gb300/_build/libcht.so`` against
the shared CUDA runtime, so the library shares the runtime (streams, memory
pools) that PyTorch loads.

``build(checked=True)`` builds the bounds-checked debug variant
(``_build/checked/libcht_checked.so``, compiled with -DCHT_BOUNDS_CHECK): its
kernels test every leaf, pair and unit index against its array before using
it and record a bad one in the device status word instead of reading out of
range.  The binding loads it when CHT_BOUNDS_CHECK=1 is set.
"""

from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "libcht.so")
CHECKED_DIR = os.path.join(BUILD_DIR, "checked")
LIB_CHECKED = os.path.join(CHECKED_DIR, "libcht_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-Wall", f"-I{INCLUDE}", f"-I{CSRC}"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (sources() + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(CSRC, "*.cuh"))
            + [os.path.join(INCLUDE, "cht.h"), os.path.abspath(__file__)])


def stale(checked: bool = False) -> bool:
    lib = LIB_CHECKED if checked else LIB
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    """Compile (if stale or forced) and return the library path."""
    lib = LIB_CHECKED if checked else LIB
    out_dir = CHECKED_DIR if checked else BUILD_DIR
    if checked:
        extra = (*extra, "-DCHT_BOUNDS_CHECK=1")
    if not force and not stale(checked):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    srcs = sources()
    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if v else []
    print(build(force=True, verbose=v, extra=extra, checked="--checked" in sys.argv))
