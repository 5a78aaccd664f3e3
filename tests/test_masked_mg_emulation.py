"""The finest multigrid level with solid cells run on the host: the two-sweep
smoothing of a right side (k_mg_src), the restriction of the residual
(k_mg_restrict) and the prolongation (k_mg_prolong), taken verbatim from
csrc/ns_mg.cuh and compiled as C++ with every CTA as host threads
(tests/emu/) under AddressSanitizer and UBSan, in FP64, against the masked
operator written out in numpy: a face joins two fluid cells or drops out of L
(the Neumann condition at solid surfaces and walls), the Jacobi weight of a
cell is -w / (sum of its active faces' weights) and 0 for a cell without any,
y = y0 + c (b - L y0) with y0 = c b, the restriction is the mean of the 8
children's b - L y, and the prolonged correction is added to fluid cells
only.  The face codes are built here from the solid mask by that rule.  No
GPU needed."""
from __future__ import annotations

import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1705_06149_gb300 import inputs
from test_mg_block_emulation import CSRC, EMU, _extract, _prolong

BC = {"wall": 0, "periodic": 1, "slip": 2}
OMEGA = 6.0 / 7.0
FC_FLUID = 64


def _source() -> str:
    dev = open(os.path.join(CSRC, "ns_device.cuh")).read()
    ker = open(os.path.join(CSRC, "ns_kernels.cuh")).read()
    mg = open(os.path.join(CSRC, "ns_mg.cuh")).read()
    a = dev.index("enum { BC_WALL")
    b = dev.index("}  // namespace nsk")
    head = [dev[a:b], _extract(ker, r"^enum \{ ST_ITER"), _extract(ker, r"^struct SliceCtl \{")]
    s = mg.index("constexpr int MG_MAX_LEVELS")
    start = mg.index("    k_mg_prolong_pair(")
    e = mg.index("\n}\n", start) + 3
    return "\n\n".join(head) + "\n\n" + mg[s:e]


@pytest.fixture(scope="module")
def masked_emulator(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("masked_emu")
    cpp = d / "masked_emu.cpp"
    cpp.write_text('#include "block_emu.h"\n\n' + _source() + "\n\n" +
                   open(os.path.join(EMU, "masked_emu_main.cpp")).read())
    exe = d / "masked_emu"
    cmd = [gxx, "-std=c++20", "-O1", "-g", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer", "-pthread",
           "-I", EMU, str(cpp), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "barrier" in r.stderr and "No such file" in r.stderr:
        pytest.skip("the host compiler has no <barrier>")
    assert r.returncode == 0, r.stderr[-3000:]
    return str(exe), d


def _codes(solid, bc):
    """Face codes: bit 2a (2a+1) when the face to the lower (upper) neighbour
    along axis a joins two fluid cells, FC_FLUID for a fluid cell."""
    fluid = solid == 0
    code = np.where(fluid, FC_FLUID, 0).astype(np.int64)
    for a in range(3):
        ax = 2 - a
        n = fluid.shape[ax]
        for dirn, shift in ((0, 1), (1, -1)):  # lower neighbour = roll by +1
            nb = np.roll(fluid, shift, axis=ax)
            ok = fluid & nb
            if bc[a] != "periodic":
                edge = [slice(None)] * 3
                edge[ax] = 0 if dirn == 0 else n - 1
                ok[tuple(edge)] = False
            code |= np.where(ok, 1 << (2 * a + dirn), 0)
    return code.astype(np.uint8)


def _lap_masked(y, code, w):
    s = np.zeros_like(y)
    for a in range(3):
        ax = 2 - a
        lo_ok = (code >> (2 * a)) & 1
        hi_ok = (code >> (2 * a + 1)) & 1
        s += np.where(hi_ok == 1, np.roll(y, -1, axis=ax) - y, 0.0) * w[a]
        s -= np.where(lo_ok == 1, y - np.roll(y, 1, axis=ax), 0.0) * w[a]
    return s


CASES = [
    ((20, 16, 12), ("wall",) * 3),
    ((16, 12, 8), ("periodic", "wall", "slip")),
    ((24, 16, 16), ("wall", "periodic", "wall")),
]


@pytest.mark.parametrize("dims,bc", CASES)
def test_masked_level_matches_numpy(masked_emulator, dims, bc):
    exe, d = masked_emulator
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    _, solid = inputs.obstacle_boxes(dims, seed=11, count=3, edge=(0.15, 0.3))
    assert solid.any()
    code = _codes(solid, bc)
    fluid = solid == 0
    rng = np.random.default_rng(nx * ny)
    b = np.where(fluid, rng.normal(size=shape), 0.0)
    y = np.where(fluid, rng.normal(size=shape), 0.0)
    e = rng.normal(size=(nz // 2, ny // 2, nx // 2))
    yp = np.where(fluid, rng.normal(size=shape), 0.0)
    fin, fout = d / f"in_{nx}_{ny}_{nz}.bin", d / f"out_{nx}_{ny}_{nz}.bin"
    with open(fin, "wb") as f:
        code.tofile(f)
        for a in (b, y, e, yp):
            a.astype(np.float64).tofile(f)
    r = subprocess.run([exe, *map(str, dims), *(str(BC[x]) for x in bc), str(fin), str(fout)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stderr[-3000:])
    out = np.fromfile(fout, dtype=np.float64)
    C, Cc = b.size, e.size
    ys, bcoarse, ypo = out[:C].reshape(shape), out[C:C + Cc].reshape(e.shape), out[C + Cc:].reshape(shape)
    w = [float(n) * n for n in dims]
    dsum = sum(w[a] * ((code >> (2 * a)) & 1) + w[a] * ((code >> (2 * a + 1)) & 1) for a in range(3))
    cw = np.where(dsum > 0, -OMEGA / np.where(dsum > 0, dsum, 1.0), 0.0)
    y0 = cw * b
    want_ys = y0 + cw * (b - _lap_masked(y0, code, w))
    assert np.max(np.abs(ys - want_ys)) <= 1e-13 * np.max(np.abs(want_ys))
    assert np.all(ys[~fluid] == 0.0)
    res = b - _lap_masked(y, code, w)
    want_bc = res.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).mean(axis=(1, 3, 5))
    assert np.max(np.abs(bcoarse - want_bc)) <= 1e-13 * np.max(np.abs(want_bc))
    want_yp = np.where(fluid, yp + _prolong(e, dims, bc_codes(bc)), yp)
    assert np.max(np.abs(ypo - want_yp)) <= 1e-13 * np.max(np.abs(want_yp))


def bc_codes(bc):
    return [BC[x] for x in bc]
