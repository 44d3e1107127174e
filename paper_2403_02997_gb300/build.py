"""Build libtc.so (CUDA, sm_103a) and the generator library in-tree.

nvcc compiles each translation unit in parallel into _build/, then links one
shared library beside this file.  The build is skipped when the library is
newer than every source and header.
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
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtc.so")
# the checked build (-DTC_CHECKED: kernels test the preconditions of their
# data-dependent accesses and report TC_ERR_CUDA instead of touching bad memory)
OBJ_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libtc_checked.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-diag-suppress", "550"]
# extra nvcc flags (e.g. -D defines for kernel variants), from the environment
FLAGS += os.environ.get("TC_NVCC_FLAGS", "").split()


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [
        os.path.join(ROOT, "include", "tc.h"), os.path.abspath(__file__)]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib) or os.environ.get("TC_NVCC_FLAGS"):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def _compile(src: str, obj_dir: str = OBJ, extra=()) -> str:
    obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
    cmd = [NVCC, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """libtc.so, or with checked=True libtc_checked.so (-DTC_CHECKED)."""
    lib, obj_dir = (LIB_CHECKED, OBJ_CHECKED) if checked else (LIB, OBJ)
    extra = ("-DTC_CHECKED",) if checked else ()
    if not force and up_to_date(lib):
        return lib
    os.makedirs(obj_dir, exist_ok=True)
    srcs = sources()
    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(lambda src: _compile(src, obj_dir, extra), srcs))
    tmp = lib + ".tmp"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print(f"built {lib}", file=sys.stderr)
    return lib


def build_all(force: bool = False) -> None:
    """Everything the package needs at run time: libtc.so and libgraphgen.so."""
    from paper_2403_02997_gb300 import gen
    build(force=force)
    gen.build(force=force)


if __name__ == "__main__":
    build_all(force="--force" in sys.argv)
    print(LIB)
