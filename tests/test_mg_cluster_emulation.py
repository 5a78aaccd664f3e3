"""The cluster multigrid kernel (k_mg_cluster) run on the host: its source and
that of its helpers, taken verbatim from csrc/ns_mg_cluster.cuh and
csrc/ns_mg.cuh, compiled as C++ with one std::thread per CUDA thread of every
CTA of the cluster (tests/emu/cluster_emu.h: per-CTA barriers, a cluster-wide
barrier, cluster-mapped addresses into the other CTAs' shared-memory blocks,
each block poisoned with NaN), under AddressSanitizer and UBSan, and compared
with the numpy V(2,0) cycle of the one-CTA kernel's test -- the same operator
started at the cluster's first level J.

The cases cover walls, periodic and slip axes, clusters of 2, 4 and 8 CTAs,
planes larger than the CTA (several cells per thread and plane), a coarse
level split across the cluster and one held by rank 0, and the plan the
library takes for the 64^3 sweep (4 CTAs) and for one 64^3 state (8 CTAs).
This checks the slab indexing, the halo exchange and the phase order on the
CPU before the kernel runs on a GPU.  No GPU needed."""
from __future__ import annotations

import os
import shutil
import subprocess

import numpy as np
import pytest

from test_mg_block_emulation import (CSRC, EMU, PERIODIC, SLIP, WALL, _kernel_source, _levels,
                                     _vcycle)


def _cluster_source() -> str:
    src = open(os.path.join(CSRC, "ns_mg_cluster.cuh")).read()
    start = src.index("constexpr int MG_CL_THREADS")
    end = src.rindex("}  // namespace nsk")
    body = src[start:end]
    shared = "extern __shared__ __align__(16) unsigned char smem_raw[];"
    assert shared in body
    return body.replace(shared, "unsigned char* smem_raw = emu_smem;")


@pytest.fixture(scope="module")
def emulator(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("cluster_emu")
    cpp = d / "cluster_emu.cpp"
    cpp.write_text('#include "cluster_emu.h"\n\n' + _kernel_source() + "\n\n" +
                   _cluster_source() + "\n\n" +
                   open(os.path.join(EMU, "cluster_emu_main.cpp")).read())
    exe = d / "cluster_emu"
    cmd = [gxx, "-std=c++20", "-O1", "-g", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer", "-pthread",
           "-I", EMU, str(cpp), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "barrier" in r.stderr and "No such file" in r.stderr:
        pytest.skip("the host compiler has no <barrier>")
    assert r.returncode == 0, r.stderr[-3000:]
    return str(exe), d


# (grid, boundaries, CTAs per cluster, threads per CTA, expected J and R in
# FP32: the cluster's first level and the first level of rank 0's one-CTA core)
CASES = [
    ((64, 64, 64), (WALL,) * 3, 4, 128, 1, 5),        # the sweep's plan: 32^3, 16^3 split
    ((64, 64, 64), (WALL,) * 3, 8, 128, 1, 5),        # one state's plan
    ((32, 32, 32), (WALL, WALL, PERIODIC), 2, 128, 1, 4),
    ((32, 32, 32), (WALL, WALL, PERIODIC), 4, 160, 1, 4),
    ((32, 32, 32), (PERIODIC,) * 3, 8, 128, 1, 4),    # slabs of 2 planes, 8^3 to rank 0
    ((24, 20, 32), (PERIODIC, WALL, WALL), 4, 64, 1, 2),
    ((48, 48, 48), (SLIP, WALL, SLIP), 2, 128, 1, 3),  # 6^3 (x not a multiple of 4) to the core
    ((64, 64, 32), (WALL,) * 3, 4, 128, 1, 4),        # planes of 1024 cells, 128 threads
    ((32, 32, 16), (WALL, PERIODIC, WALL), 4, 64, 1, 3),
    ((40, 24, 16), (WALL, WALL, PERIODIC), 2, 64, 1, 2),
    # two split levels across a periodic seam: the prolongation's halo slots
    ((64, 64, 64), (WALL, WALL, PERIODIC), 4, 128, 1, 5),
    ((64, 32, 64), (PERIODIC, WALL, PERIODIC), 8, 128, 1, 4),
]


def _run(exe, args, timeout=300):
    return subprocess.run([exe, *map(str, args)], capture_output=True, text=True,
                          timeout=timeout)


@pytest.mark.parametrize("prec", ["f", "d"])
@pytest.mark.parametrize("n0,bc,C,nt,J,R", CASES)
def test_cluster_kernel_matches_numpy_vcycle(emulator, n0, bc, C, nt, J, R, prec):
    exe, d = emulator
    block_cells = 4096 if prec == "f" else 512
    levs, lc = _levels(n0, block_cells)
    r = _run(exe, [prec, *n0, *bc, C, nt, "-", "-"])
    assert r.returncode == 0, (r.returncode, r.stderr[-3000:])
    plan = list(map(int, r.stdout.split()))
    j_got, r_got, c_got, nl = plan[:4]
    assert c_got == C and nl == len(levs)
    assert [tuple(plan[4 + 3 * i:7 + 3 * i]) for i in range(nl - j_got)] == levs[j_got:]
    assert r_got == R
    if prec == "f":
        assert j_got == J
    else:
        # FP64 slabs take twice the bytes: the cluster may start a level lower
        assert j_got in (J, J + 1) and j_got < R and j_got <= lc
    nj = levs[j_got]
    rng = np.random.default_rng(hash((n0, bc, C, prec)) % 2 ** 32)
    b = rng.normal(size=(nj[2], nj[1], nj[0]))
    dt = np.float32 if prec == "f" else np.float64
    fin, fout = d / f"in_{os.getpid()}.bin", d / f"out_{os.getpid()}.bin"
    b.astype(dt).tofile(fin)
    r = _run(exe, [prec, *n0, *bc, C, nt, fin, fout])
    assert r.returncode == 0, (r.returncode, r.stderr[-3000:])
    got = np.fromfile(fout, dtype=dt).reshape(b.shape).astype(np.float64)
    assert np.isfinite(got).all()
    ih2_0 = [float(n) * n for n in n0]
    want = _vcycle(b.astype(dt).astype(np.float64), levs, j_got, bc, ih2_0)
    scale = np.abs(want).max()
    tol = 2e-5 if prec == "f" else 1e-12
    assert np.abs(got - want).max() <= tol * scale, np.abs(got - want).max() / scale
