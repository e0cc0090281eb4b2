"""Build the CUDA libraries (sm_103a) in-tree under paper_1612_06592_gb300/_build/.

liblp.so: the pipeline (csrc/*.cu) with the plain C ABI of include/lp.h.
libmb.so: the peak microbenchmarks (microbench/*.cu) that measure the roofline
denominators the repository reports against; not part of the pipeline.
Each .cu file is compiled by nvcc in parallel; a library is rebuilt only when
one of its sources or headers is newer than it.
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblp.so")
MB_SRC = os.path.join(HERE, "microbench")
MB_LIB = os.path.join(BUILD, "libmb.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr",
         "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblp.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [
        os.path.join(ROOT, "include", "lp.h"), os.path.abspath(__file__)]


def _mb_sources():
    return sorted(glob.glob(os.path.join(MB_SRC, "*.cu")))


def _fresh(lib, deps) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in deps)


def up_to_date() -> bool:
    return _fresh(LIB, _deps()) and _fresh(MB_LIB, _mb_sources() + [os.path.abspath(__file__)])


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    objs, mb_objs = [], []
    cmds = []
    for src in _sources():
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmds.append([nvcc, *ARCH, *FLAGS, *extra_flags, "-c", src, "-o", obj])
    for src in _mb_sources():
        obj = os.path.join(BUILD, "mb_" + os.path.basename(src)[:-3] + ".o")
        mb_objs.append(obj)
        cmds.append([nvcc, *ARCH, *FLAGS, *extra_flags, "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode != 0:
            print(" ".join(cmd))
            print(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {cmd[-3]}")
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(cmds), os.cpu_count() or 4))) as ex:
        list(ex.map(run, cmds))
    for lib, lib_objs in ((LIB, objs), (MB_LIB, mb_objs)):
        tmp = lib + ".tmp"
        run([nvcc, *ARCH, "-shared", "-o", tmp, *lib_objs])
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
