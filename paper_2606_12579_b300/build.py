"""Build ``libgmapp.so`` (the C-ABI CUDA library) in-tree for sm_103a.

Each ``csrc/*.cu`` is compiled to an object in ``_build/`` (in parallel),
then linked into ``paper_2606_12579_b300/libgmapp.so``; an object is
recompiled only when its source or a header it includes is newer.  The CUDA runtime is
linked statically, so the library needs only the driver at run time.

``build(bounds_check=True)`` builds the bounds-checked variant
``libgmapp_bc.so`` (objects in ``_build_bc/``, compiled with
-DGMAPP_BOUNDS_CHECK: index checks that set GMAPP_DEVERR_BOUNDS in the
device error word); the package loads it when GMAPP_BOUNDS_CHECK=1.
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import re
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(os.path.dirname(HERE), "_build")
LIB = os.path.join(HERE, "libgmapp.so")
LIB_BC = os.path.join(HERE, "libgmapp_bc.so")
NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [
        os.path.join(os.path.dirname(HERE), "include", "gmapp.h")]


_INCLUDE = re.compile(r'^\s*#\s*include\s+"([^"]+)"', re.M)


def _closure(src: str, seen=None) -> set:
    """The file and every quoted include it reaches (transitively)."""
    seen = set() if seen is None else seen
    src = os.path.normpath(src)
    if src in seen or not os.path.exists(src):
        return seen
    seen.add(src)
    with open(src) as f:
        for inc in _INCLUDE.findall(f.read()):
            _closure(os.path.join(os.path.dirname(src), inc), seen)
    return seen


def _stale(src: str, obj: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in _closure(src))


def _compile(src: str, verbose: bool, bdir: str = BUILD, extra=(), force: bool = True) -> str:
    obj = os.path.join(bdir, os.path.basename(src) + ".o")
    if not force and not verbose and not _stale(src, obj):
        return obj
    cmd = [NVCC, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False, bounds_check: bool = False) -> str:
    lib = LIB_BC if bounds_check else LIB
    bdir = BUILD + "_bc" if bounds_check else BUILD
    extra = ("-DGMAPP_BOUNDS_CHECK",) if bounds_check else ()
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= max(os.path.getmtime(p) for p in _deps())):
        return lib
    os.makedirs(bdir, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, bdir, extra, force), _sources()))
    tmp = lib + ".tmp"
    subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                bounds_check="--bounds-check" in sys.argv))
