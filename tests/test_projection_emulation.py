"""The projection kernels run on the host: the divergence of F* with its
per-CTA partial sums (k_divergence) and the velocity correction with the
gauged pressure (k_correct), taken verbatim from csrc/ns_device.cuh and
csrc/ns_kernels.cuh, compiled as C++ with every CTA as host threads
(tests/emu/) under AddressSanitizer and UBSan, in FP64, against the FP64
oracle (Section 2): b = D F* / dt (0 in solid cells), the partial sums add up
to the sum of b, u = F* - dt G p on active faces and 0 on inactive ones, and
the returned pressure is p minus its fluid mean.  No GPU needed."""
from __future__ import annotations

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1705_06149_gb300 import inputs
from test_mg_block_emulation import CSRC, EMU, _extract

BC = {"wall": 0, "periodic": 1, "slip": 2}


def _source() -> str:
    dev = open(os.path.join(CSRC, "ns_device.cuh")).read()
    ker = open(os.path.join(CSRC, "ns_kernels.cuh")).read()
    a = dev.index("enum { BC_WALL")
    b = dev.index("}  // namespace nsk")
    return "\n\n".join([dev[a:b], _extract(ker, r"^enum \{ ST_ITER"),
                        _extract(ker, r"^struct SliceCtl \{"),
                        _extract(ker, r"^    k_divergence\("), _extract(ker, r"^    k_correct\(")])


@pytest.fixture(scope="module")
def proj_emulator(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("proj_emu")
    cpp = d / "proj_emu.cpp"
    cpp.write_text('#include "block_emu.h"\n\n' + _source() + "\n\n" +
                   open(os.path.join(EMU, "proj_emu_main.cpp")).read())
    exe = d / "proj_emu"
    cmd = [gxx, "-std=c++20", "-O1", "-g", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer", "-pthread",
           "-I", EMU, str(cpp), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "barrier" in r.stderr and "No such file" in r.stderr:
        pytest.skip("the host compiler has no <barrier>")
    assert r.returncode == 0, r.stderr[-3000:]
    return str(exe), d


CASES = [
    ((12, 12, 12), ("wall",) * 3, False),
    ((40, 10, 9), ("wall",) * 3, False),
    ((16, 12, 6), ("periodic", "wall", "slip"), False),
    ((24, 16, 8), ("wall", "periodic", "periodic"), False),
    ((20, 18, 16), ("wall",) * 3, True),
    ((16, 16, 12), ("periodic", "wall", "wall"), True),
]


@pytest.mark.parametrize("dims,bc,masked", CASES)
def test_divergence_and_correction_match_oracle(proj_emulator, dims, bc, masked):
    exe, d = proj_emulator
    solid = None
    if masked:
        _, solid = inputs.obstacle_boxes(dims, seed=7, count=3, edge=(0.15, 0.3))
    rs = inputs.random_state(*dims, seed=13, sigma=1.0, bc=bc, solid=solid)
    dt = 2e-3
    og = oracle.Grid(*dims, re=50.0, u_lid=1.0, bc=bc, solid=solid)
    fstar = og.predict(*rs[:3], dt)
    p = np.random.default_rng(3).normal(size=og.shape(3))
    if masked:
        p[solid != 0] = 0.0
    tag = f"{os.getpid()}_{'_'.join(map(str, dims))}_{int(masked)}"
    fin, fsol, fout = d / f"in_{tag}.bin", d / f"solid_{tag}.bin", d / f"out_{tag}.bin"
    np.concatenate([np.ravel(a) for a in fstar] + [np.ravel(p)]).astype(np.float64).tofile(fin)
    if masked:
        np.ascontiguousarray(solid, dtype=np.uint8).tofile(fsol)
    args = [exe, *map(str, dims), *(str(BC[b]) for b in bc), repr(dt), str(fin),
            str(fsol) if masked else "-", str(fout)]
    r = subprocess.run(args, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stderr[-3000:])
    _, sb, bsum, sb32, bsum32 = r.stdout.split()
    out = np.fromfile(fout, dtype=np.float64)
    nb = p.size
    b = out[:nb].reshape(p.shape)
    # the per-CTA partials add up to the sum of b (up to the summation order)
    assert abs(float(sb) - float(bsum)) <= 1e-13 * np.sum(np.abs(b))
    want_b = og.divergence(*fstar) / dt
    assert np.max(np.abs(b - want_b)) <= 1e-12 * np.max(np.abs(want_b))
    grad = og.gradient(p)
    o = nb
    for c in range(3):
        got = out[o:o + fstar[c].size].reshape(fstar[c].shape)
        o += fstar[c].size
        want = fstar[c] - dt * grad[c]
        assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want)), c
    pout = out[o:o + nb].reshape(p.shape)
    o += nb
    # FP32 storage: the FP32 divergence of F* rounded to FP32 (the kernel's
    # operations in its order), times 1/dt as a float-float product (~2^-48)
    b32 = out[o:o + nb].reshape(p.shape)
    f32 = [a.astype(np.float32) for a in fstar]
    ih = [np.float32(n) for n in dims]

    def fdiff(a, c):
        ax = 2 - c
        if bc[c] == "periodic":
            return (np.roll(a, -1, axis=ax) - a).astype(np.float32)
        return np.diff(a, axis=ax).astype(np.float32)

    d32 = (fdiff(f32[0], 0) * ih[0]).astype(np.float32)
    d32 = (d32 + (fdiff(f32[1], 1) * ih[1]).astype(np.float32)).astype(np.float32)
    d32 = (d32 + (fdiff(f32[2], 2) * ih[2]).astype(np.float32)).astype(np.float32)
    want_b32 = d32.astype(np.float64) * (1.0 / dt)
    if masked:
        want_b32[solid != 0] = 0.0
    assert np.max(np.abs(b32 - want_b32)) <= 1e-13 * np.max(np.abs(want_b32))
    assert abs(float(sb32) - float(bsum32)) <= 1e-13 * np.sum(np.abs(b32))
    fluid = np.ones(p.shape, bool) if solid is None else solid == 0
    want_p = np.where(fluid, p - p[fluid].mean(), 0.0)
    assert np.max(np.abs(pout - want_p)) <= 1e-13 * np.max(np.abs(want_p))
