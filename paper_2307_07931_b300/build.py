"""Build libprotox.so in-tree with nvcc for sm_103a (B300), and the checked
variant libprotox_checked.so (-DPX_CHECKED: index bounds checks with a device
fault word in the relaxation and Euler kernels).

Run as `python -m paper_2307_07931_b300.build [--checked]` or through build()
below. Rebuilds when any source under csrc/ or include/ is newer than the
library.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libprotox.so")
LIB_CHECKED = os.path.join(HERE, "libprotox_checked.so")
# translation units whose kernels carry the checked build's bounds checks
CHECKED_SOURCES = ("api.cu", "relax.cu", "euler.cu", "rbsor.cu")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-cudart", "shared"]


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


def deps() -> list[str]:
    # this file too: its flags and source lists shape the libraries
    return (sources() + glob.glob(os.path.join(HERE, "csrc", "*.cuh"))
            + glob.glob(os.path.join(ROOT, "include", "*.h")) + [os.path.abspath(__file__)])


def up_to_date(checked: bool = False) -> bool:
    lib = LIB_CHECKED if checked else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in deps())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          checked: bool = False) -> str:
    """Compile every csrc/*.cu (relocatable device code) and link the shared
    library. checked: the -DPX_CHECKED variant, which recompiles the sources
    that carry the bounds checks and links them with the normal build's
    other objects (built first if needed)."""
    lib = LIB_CHECKED if checked else LIB
    if not force and up_to_date(checked):
        return lib
    if checked and (force or not up_to_date(False)):
        build(force=force, verbose=verbose, extra=extra)
    objdir = os.path.join(ROOT, "_build")
    os.makedirs(os.path.join(objdir, "checked"), exist_ok=True)
    objs = []
    for src in sources():
        name = os.path.basename(src)
        if checked and name not in CHECKED_SOURCES:
            objs.append(os.path.join(objdir, name + ".o"))
            continue
        obj = os.path.join(objdir, "checked" if checked else "", name + ".o")
        flags = FLAGS + (["-DPX_CHECKED"] if checked else [])
        cmd = [NVCC, *ARCH, *flags, *(extra or []), "-dc", "-o", obj, src]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        objs.append(obj)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else None
    print(build(force=True, verbose=v, extra=extra, checked="--checked" in sys.argv))
