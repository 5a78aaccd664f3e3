"""Build step of the CUDA library libns.so (sm_103a) from csrc/ with nvcc.

The library is built in-tree (next to this file) so that the process that
loads it is seen to load this repository's native code.  No CPU fallback
exists: callers that cannot load libns.so get an error.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libns.so")
PEAKS_LIB = os.path.join(HERE, "libns_peaks.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _sources():
    out = [os.path.join(INCLUDE, f) for f in sorted(os.listdir(INCLUDE)) if f.endswith(".h")]
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh", ".h")):
            out.append(os.path.join(CSRC, f))
    return out


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library libns.so cannot be built")


def needs_build() -> bool:
    return _stale(LIB) or _stale(PEAKS_LIB)


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/ into libns.so (the stepper's C ABI) and libns_peaks.so
    (the FMA throughput probe of the benchmark) for sm_103a, the translation
    units in parallel; returns the path of libns.so."""
    jobs = []
    parts = [(LIB, ["ns_api.cu", "ns_noalloc.cu", "ns_persist.cu"]),
             (PEAKS_LIB, ["ns_peaks.cu"])]
    for lib, srcs in parts:
        if not force and not _stale(lib):
            continue
        tmp = lib + f".tmp{os.getpid()}"
        objs = []
        for src in srcs:
            obj = os.path.join(HERE, f".{os.path.splitext(src)[0]}.{os.getpid()}.o")
            cmd = [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
            if verbose:
                print(" ".join(cmd))
            jobs.append(subprocess.Popen(cmd))
            objs.append(obj)
        parts_done = (lib, tmp, objs)
        jobs.append(parts_done)
    procs = [j for j in jobs if isinstance(j, subprocess.Popen)]
    rcs = [p.wait() for p in procs]
    links = [j for j in jobs if isinstance(j, tuple)]
    try:
        if any(rcs):
            raise subprocess.CalledProcessError(max(rcs), "nvcc")
        for lib, tmp, objs in links:
            subprocess.run([nvcc(), ARCH, "-shared", *objs, "-o", tmp], check=True)
            os.replace(tmp, lib)
    finally:
        for _, _, objs in links:
            for o in objs:
                if os.path.exists(o):
                    os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
