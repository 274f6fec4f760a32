"""Builds libzkb300.so in-tree with nvcc for sm_103a.

Each .cu file is compiled to an object in parallel, then linked into a
shared library next to this file.  `python paper_2507_07031_b300/build.py`
runs it from the command line (as a script, so that the package binding,
which loads the library, is not imported first).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libzkb300.so")
OBJ = os.path.join(HERE, "_build")
# The checked build (-DZK_CHECK: in-kernel bounds checks that set flags read
# by zk_check_status) goes to its own library and object directory.
LIB_CHECK = os.path.join(HERE, "libzkb300_check.so")
OBJ_CHECK = os.path.join(HERE, "_build_check")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-warn-spills"]


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps_mtime():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(os.path.dirname(HERE), "include", "zk_b300.h"))
    return max(os.path.getmtime(f) for f in files)


def _compile(src: str, extra, objdir: str = OBJ) -> str:
    obj = os.path.join(objdir, src[:-3] + ".o")
    if os.path.exists(obj) and os.path.getmtime(obj) >= _deps_mtime():
        return obj
    cmd = [NVCC, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    if r.stderr.strip():
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False, checked: bool = False) -> str:
    lib, objdir = (LIB_CHECK, OBJ_CHECK) if checked else (LIB, OBJ)
    os.makedirs(objdir, exist_ok=True)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    extra = (["-Xptxas", "-v"] if verbose_ptxas else []) + (["-DZK_CHECK"] if checked else [])
    if force:
        for f in os.listdir(objdir):
            os.remove(os.path.join(objdir, f))
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, objdir), sources()))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, checked="--check" in sys.argv))
