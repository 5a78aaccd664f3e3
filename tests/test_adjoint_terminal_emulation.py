"""The adjoint's terminal condition and finishing update run on the host:
k_adj_terminal (lambda = u vol on active faces, 0 on wall-normal boundary
faces, and per-CTA partial sums of J = 1/2 sum of u^2 vol per state, summed in
a fixed order by k_adj_sum) and k_adj_finish (lambda = mu +
dt acc on active faces, 0 elsewhere, acc cleared for reuse), taken verbatim
from csrc/ns_adjoint.cuh and compiled as C++ with every CTA as host threads
(tests/emu/) under AddressSanitizer and UBSan, on grids smaller than the
arrays so that the grid-stride loops take several passes, for two states at
once.  J is compared with the oracle's objective (reading 14: the kinetic
energy at the final time over active faces).  No GPU needed."""
from __future__ import annotations

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1705_06149_gb300 import inputs
from test_mg_block_emulation import CSRC, EMU

BC = {"wall": 0, "periodic": 1, "slip": 2}


def _source() -> str:
    dev = open(os.path.join(CSRC, "ns_device.cuh")).read()
    adj = open(os.path.join(CSRC, "ns_adjoint.cuh")).read()
    a = dev.index("enum { BC_WALL")
    b = dev.index("}  // namespace nsk")
    s = adj.index("// out[s] (+)= sum of part[s][0..n-1] in order")
    start = adj.index("    k_adj_terminal(")
    e = adj.index("\n}\n", start) + 3
    return dev[a:b] + "\n\n" + adj[s:e]


@pytest.fixture(scope="module")
def adjterm_emulator(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("adjterm_emu")
    cpp = d / "adjterm_emu.cpp"
    cpp.write_text('#include "block_emu.h"\n\n' + _source() + "\n\n" +
                   open(os.path.join(EMU, "adjterm_emu_main.cpp")).read())
    exe = d / "adjterm_emu"
    cmd = [gxx, "-std=c++20", "-O1", "-g", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer", "-pthread",
           "-I", EMU, str(cpp), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "barrier" in r.stderr and "No such file" in r.stderr:
        pytest.skip("the host compiler has no <barrier>")
    assert r.returncode == 0, r.stderr[-3000:]
    return str(exe), d


CASES = [
    ((12, 10, 9), ("wall",) * 3),
    ((16, 12, 6), ("periodic", "wall", "slip")),
    ((8, 16, 10), ("wall", "periodic", "periodic")),
]


def _active(shape, c, n, bc):
    act = np.ones(shape, bool)
    if bc[c] != "periodic":
        ax = 2 - c
        idx = np.arange(shape[ax])
        sel = (idx > 0) & (idx < n[c])
        act &= sel.reshape([-1 if a == ax else 1 for a in range(3)])
    return act


@pytest.mark.parametrize("dims,bc", CASES)
def test_adjoint_terminal_and_finish(adjterm_emulator, dims, bc):
    exe, d = adjterm_emulator
    batch, dt = 2, 2e-3
    og = oracle.Grid(*dims, bc=bc)
    hx, hy, hz = og.h
    vol = hx * hy * hz
    rng = np.random.default_rng(sum(dims))
    states = [inputs.random_state(*dims, seed=30 + s, sigma=1.0, bc=bc) for s in range(batch)]
    # the wall faces of u carry values here, to check that they are left out
    u = [np.stack([states[s][c] + (rng.normal(size=og.shape(c)) if s == 1 else 0.0)
                   for s in range(batch)]) for c in range(3)]
    mu = [rng.normal(size=(batch,) + og.shape(c)) for c in range(3)]
    acc = [rng.normal(size=(batch,) + og.shape(c)) for c in range(3)]
    tag = "_".join(map(str, dims))
    fin, fout = d / f"in_{tag}.bin", d / f"out_{tag}.bin"
    with open(fin, "wb") as f:
        for c in range(3):
            for a in (u[c], mu[c], acc[c]):
                a.astype(np.float64).tofile(f)
    r = subprocess.run([exe, *map(str, dims), *(str(BC[x]) for x in bc), str(batch), repr(vol),
                        repr(dt), str(fin), str(fout)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stderr[-3000:])
    out = np.fromfile(fout, dtype=np.float64)
    o = 0
    for c in range(3):
        shp = (batch,) + og.shape(c)
        n = int(np.prod(shp))
        lam, lam2, acc_after = (out[o + q * n:o + (q + 1) * n].reshape(shp) for q in range(3))
        o += 3 * n
        act = _active(og.shape(c), c, dims, bc)[None]
        assert np.array_equal(lam, np.where(act, u[c] * vol, 0.0)), c
        assert np.array_equal(lam2, np.where(act, mu[c] + dt * acc[c], 0.0)), c
        assert np.all(acc_after == 0.0)
    J = out[o:]
    assert J.size == batch
    for s in range(batch):
        want = og.kinetic_objective([u[c][s] for c in range(3)])
        assert abs(J[s] - want) <= 1e-13 * want, (s, J[s], want)
