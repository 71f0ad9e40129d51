"""Build libmickey.so (CUDA, sm_103a) in-tree with nvcc.

Each .cu translation unit is compiled in parallel; the shared library links
the CUDA runtime statically and exports only the C ABI of include/mickey.h.
Run as ``python -m paper_1909_04750_gb300.build`` or call ``build()``.
"""
from __future__ import annotations

import glob
import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libmickey.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden", "-I", INCLUDE] + ARCH


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmickey")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
                  + glob.glob(os.path.join(INCLUDE, "*.h")))


def sources_digest(names=("keystream_kernels.cu", "keystream_device.cuh",
                          "keystream_persistent.cuh", "keystream_persistent8.cu",
                          "keystream_persistent4.cu", "bitslice.cuh", "tables.cuh",
                          "internal.h")) -> str:
    """Short digest of kernel sources without their // comments and blank
    lines (to tie a stored profiler figure to the code it was measured on)."""
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(CSRC, n)) as f:
            for line in f:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def _newest(paths):
    return max((os.path.getmtime(p) for p in paths), default=0.0)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile stale objects and relink; returns the library path."""
    nvcc = _nvcc()
    obj_dir = os.path.join(OUT_DIR, "obj")
    os.makedirs(obj_dir, exist_ok=True)
    hdr_time = _newest(_headers())
    jobs = []
    for src in _sources():
        obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
        if (force or ptxas_info or not os.path.exists(obj)
                or os.path.getmtime(obj) < max(os.path.getmtime(src), hdr_time)):
            jobs.append((src, obj))

    def compile_one(job):
        src, obj = job
        cmd = [nvcc] + NVCC_FLAGS + (["-Xptxas", "-v"] if ptxas_info else []) + \
            ["-c", src, "-o", obj + ".tmp"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, p.stdout, p.stderr))
        os.replace(obj + ".tmp", obj)
        return src, p.stderr

    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for src, err in ex.map(compile_one, jobs):
                if verbose or ptxas_info:
                    print("compiled", os.path.basename(src), file=sys.stderr)
                    if ptxas_info:
                        print(err, file=sys.stderr)
    objs = [os.path.join(obj_dir, os.path.basename(s)[:-3] + ".o") for s in _sources()]
    if force or jobs or not os.path.exists(LIB) or os.path.getmtime(LIB) < _newest(objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (p.stdout, p.stderr))
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                ptxas_info="--ptxas-info" in sys.argv))
