"""Build liblens.so (all CUDA sources for sm_103a) in-tree.

Each translation unit under csrc/ is compiled by nvcc in parallel, then the
objects are linked into ``paper_2211_00354_gb300/_lib/liblens.so``.  The build
is incremental on source/header modification times.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
BUILD = os.path.join(HERE, "_lib", "obj")
LIB = os.path.join(OUT, "liblens.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                     "--expt-relaxed-constexpr", "-I", INCLUDE]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblens")
    return path


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
    hs += glob.glob(os.path.join(INCLUDE, "*.h"))
    return max([os.path.getmtime(h) for h in hs] + [0.0])


def _compile(src: str, obj: str, extra) -> str:
    cmd = [nvcc(), "-c", src, "-o", obj + ".tmp"] + NVCC_FLAGS + list(extra)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    os.replace(obj + ".tmp", obj)
    return r.stderr


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hm = _headers_mtime()
    jobs = []
    objs = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if (force or not os.path.exists(o) or os.path.getmtime(o) < os.path.getmtime(s)
                or os.path.getmtime(o) < hm):
            jobs.append((s, o))
    if jobs:
        workers = min(len(jobs), max(1, os.cpu_count() or 1))
        with cf.ThreadPoolExecutor(workers) as ex:
            futs = {ex.submit(_compile, s, o, extra_flags): s for s, o in jobs}
            for f in cf.as_completed(futs):
                msg = f.result()
                if verbose and msg:
                    print(msg)
    relink = (force or bool(jobs) or not os.path.exists(LIB)
              or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs))
    if relink:
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = [nvcc(), "-shared", "-o", tmp] + ARCH + objs + ["-lcudart_static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, LIB)
    return LIB


PEAKS_SRC = os.path.join(HERE, "pipe_peaks.cu")
PEAKS_BIN = os.path.join(OUT, "pipe_peaks")


def build_peaks(force: bool = False) -> str:
    """The pipe-peak micro-benchmark (pipe_peaks.cu) as a standalone program."""
    os.makedirs(OUT, exist_ok=True)
    if (not force and os.path.exists(PEAKS_BIN)
            and os.path.getmtime(PEAKS_BIN) >= os.path.getmtime(PEAKS_SRC)):
        return PEAKS_BIN
    tmp = PEAKS_BIN + ".tmp%d" % os.getpid()
    cmd = [nvcc(), "-O3", "-std=c++17", "-o", tmp, PEAKS_SRC] + ARCH
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for pipe_peaks.cu:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, PEAKS_BIN)
    return PEAKS_BIN


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
