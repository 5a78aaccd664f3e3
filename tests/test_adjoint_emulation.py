"""The adjoint right side run on the host: k_adj_rhs ((dR/du)^T mu gathered
per stored value, and per-CTA partials of (dR/du_lid)^T mu summed in order by
k_adj_sum, for R = Re^-1 lap u - div(u u) with SMART faces), taken verbatim
from csrc/ns_adjoint.cuh and compiled as C++ with every CTA as host threads
(tests/emu/), under AddressSanitizer and UBSan, against the oracle's
hand-written transpose (a scatter over every stencil term) on walls with the
lid, periodic and slip axes, small and ragged grids: FP64 to 1e-12, FP32 (the
inputs rounded to FP32) to 2e-5 of the largest entry.  The gather visits the
terms in another order than the scatter, so a missed or doubled term (a
ghost mirror, a role of a flux, a transport position) fails the comparison.
No GPU needed."""
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
    s = adj.index("// partial derivatives of smart_face")
    start = adj.index("    k_adj_sum(")
    assert adj.index("    k_adj_rhs(") < start
    e = adj.index("\n}\n", start) + 3
    return dev[a:b] + "\n\n" + adj[s:e]


@pytest.fixture(scope="module")
def adj_emulator(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("adj_emu")
    cpp = d / "adj_emu.cpp"
    cpp.write_text('#include "block_emu.h"\n\n' + _source() + "\n\n" +
                   open(os.path.join(EMU, "adj_emu_main.cpp")).read())
    exe = d / "adj_emu"
    cmd = [gxx, "-std=c++20", "-O1", "-g", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer", "-pthread",
           "-I", EMU, str(cpp), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "barrier" in r.stderr and "No such file" in r.stderr:
        pytest.skip("the host compiler has no <barrier>")
    assert r.returncode == 0, r.stderr[-3000:]
    return str(exe), d


CASES = [
    ((12, 12, 12), ("wall",) * 3),
    ((40, 10, 9), ("wall",) * 3),
    ((16, 12, 6), ("periodic", "wall", "slip")),
    ((8, 16, 10), ("wall", "periodic", "periodic")),
    ((3, 2, 4), ("wall", "slip", "periodic")),
    ((2, 3, 2), ("periodic", "wall", "wall")),
]


@pytest.mark.parametrize("prec", ["d", "f"])
@pytest.mark.parametrize("dims,bc", CASES)
def test_adjoint_rhs_matches_oracle(adj_emulator, dims, bc, prec):
    exe, d = adj_emulator
    re, u_lid = 40.0, 1.0
    st = inputs.random_state(*dims, seed=17, sigma=0.5, bc=bc)
    mu = inputs.random_state(*dims, seed=18, sigma=1.0, bc=bc)[:3]
    og = oracle.Grid(*dims, re=re, u_lid=u_lid, bc=bc)
    want, want_dl = og.rhs_adjoint(*st[:3], mu)
    tol = 1e-12 if prec == "d" else 2e-5
    tag = "_".join(map(str, dims)) + prec
    fin, fout = d / f"in_{tag}.bin", d / f"out_{tag}.bin"
    np.concatenate([np.ravel(a) for a in list(st[:3]) + list(mu)]).astype(np.float64).tofile(fin)
    if prec == "f":  # the FP32 kernel sees the inputs rounded to FP32
        st = [np.asarray(a, dtype=np.float32).astype(np.float64) for a in st]
        mu = [np.asarray(a, dtype=np.float32).astype(np.float64) for a in mu]
        want, want_dl = og.rhs_adjoint(*st[:3], mu)
        np.concatenate([np.ravel(a) for a in list(st[:3]) + list(mu)]).tofile(fin)
    r = subprocess.run([exe, prec, *map(str, dims), *(str(BC[x]) for x in bc), repr(re),
                        repr(u_lid), str(fin), str(fout)], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, (r.returncode, r.stderr[-3000:])
    out = np.fromfile(fout, dtype=np.float64)
    o = 0
    for c in range(3):
        got = out[o:o + want[c].size].reshape(want[c].shape)
        o += want[c].size
        err = np.max(np.abs(got - want[c])) / np.max(np.abs(want[c]))
        assert err <= tol, (c, err)
    assert abs(out[-1] - want_dl) <= tol * max(abs(want_dl), np.max(np.abs(want[0])))
