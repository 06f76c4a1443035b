"""Build libcs_b300.so in-tree from csrc/*.cu with nvcc for sm_103a.

    python -m paper_2609_35619_b300.build [--force] [--jobs N] [--debug]

Each translation unit is compiled separately (in parallel) and linked into
one shared library next to this file; a unit is recompiled only when it or a
header changed.  --debug builds the same sources with CS_DEBUG defined (device
index checks that record CS_ERR_BOUNDS instead of accessing out of range) into
libcs_b300_debug.so, for use through CS_B300_LIBRARY.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcs_b300.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libcs_b300_debug.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr"]


def _nvcc():
    n = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(n):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcs_b300.so")
    return n


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, force, extra, bdir=BUILD):
    obj = os.path.join(bdir, os.path.basename(src) + ".o")
    if force or _stale(obj, [src] + _headers()):
        cmd = [_nvcc(), *ARCH, *FLAGS, *extra, "-I", INCLUDE, "-c", src, "-o", obj + ".tmp"]
        subprocess.check_call(cmd)
        os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, jobs: int = 0, extra=(), debug: bool = False) -> str:
    bdir, lib = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    extra = list(extra) + (["-DCS_DEBUG"] if debug else [])
    os.makedirs(bdir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, force, extra, bdir), srcs))
    if force or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call([_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static",
                               "-ldl", "-lrt", "-lpthread"])
        os.replace(tmp, lib)
    return lib


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--jobs", type=int, default=0)
    ap.add_argument("--debug", action="store_true", help="CS_DEBUG build into libcs_b300_debug.so")
    args = ap.parse_args(argv)
    print(build(force=args.force, jobs=args.jobs, debug=args.debug))


if __name__ == "__main__":
    sys.exit(main())
