"""The predictor kernels run on the host: k_predict_tile (shared-memory tile
with the ghost values applied while staging, fluxes shared by shuffles and
carried along z) and k_predict_masked (stencil arms that stop at solid
surfaces), taken verbatim from csrc/ns_device.cuh and csrc/ns_kernels.cuh,
compiled as C++ with every CTA as host threads (tests/emu/) under
AddressSanitizer and UBSan, in FP64, against the FP64 oracle's predictor
F* = u + dt (Re^-1 lap u - div(u u)) (Section 2, SMART convection) on grids
with walls, a moving lid, periodic and slip axes, ragged tiles and solid
boxes; the increment form must give F* - u.  No GPU needed."""
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
    ker = open(os.path.join(CSRC, "ns_kernels.cuh")).read()
    a = dev.index("enum { BC_WALL")
    b = dev.index("template <int NV>\n__device__ __forceinline__ void block_sum")
    c = ker.index("constexpr int PT_X")
    start = ker.index("    k_predict_masked(")
    d = ker.index("\n}\n", start) + 3
    body = dev[a:b] + "\n\n" + ker[c:d]
    shared = "extern __shared__ __align__(16) unsigned char psm_raw[];"
    assert shared in body
    return body.replace(shared, "unsigned char* psm_raw = emu_smem;")


@pytest.fixture(scope="module")
def predict_emulator(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("predict_emu")
    cpp = d / "predict_emu.cpp"
    cpp.write_text('#include "block_emu.h"\n\n' + _source() + "\n\n" +
                   open(os.path.join(EMU, "predict_emu_main.cpp")).read())
    exe = d / "predict_emu"
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
    ((40, 10, 9), ("wall",) * 3, False),           # ragged x, y and z tiles
    ((16, 12, 6), ("periodic", "wall", "slip"), False),
    ((24, 16, 8), ("wall", "periodic", "periodic"), False),
    ((2, 2, 2), ("wall",) * 3, False),
    ((20, 18, 16), ("wall",) * 3, True),           # solid boxes
    ((16, 16, 12), ("periodic", "wall", "wall"), True),
]


TILES = [(8, 4), (4, 4), (4, 8), (8, 2), (8, 8), (16, 4)]


@pytest.mark.parametrize("incr", [False, True])
@pytest.mark.parametrize("dims,bc,masked", CASES)
def test_predictor_matches_oracle(predict_emulator, dims, bc, masked, incr):
    _run_predictor(predict_emulator, dims, bc, masked, incr, None)


@pytest.mark.parametrize("tile", TILES[1:])
@pytest.mark.parametrize("dims,bc", [((40, 10, 9), ("wall",) * 3),
                                     ((16, 12, 6), ("periodic", "wall", "slip"))])
def test_predictor_tiles_match_oracle(predict_emulator, dims, bc, tile):
    """Every instantiated tile shape of k_predict_tile (the autotuner's
    choices) against the oracle, on ragged tiles and periodic / slip axes."""
    _run_predictor(predict_emulator, dims, bc, False, True, tile)


def _run_predictor(predict_emulator, dims, bc, masked, incr, tile):
    exe, d = predict_emulator
    solid = None
    if masked:
        _, solid = inputs.obstacle_boxes(dims, seed=5, count=3, edge=(0.15, 0.3))
    rs = inputs.random_state(*dims, seed=9, sigma=1.0, bc=bc, solid=solid)
    re, u_lid, dt = 50.0, 1.0, 2e-3
    og = oracle.Grid(*dims, re=re, u_lid=u_lid, bc=bc, solid=solid)
    want = og.predict(*rs[:3], dt)
    tag = f"{os.getpid()}_{'_'.join(map(str, dims))}_{int(masked)}_{int(incr)}_{tile}"
    fin, fsol, fout = d / f"in_{tag}.bin", d / f"solid_{tag}.bin", d / f"out_{tag}.bin"
    np.concatenate([np.ravel(a) for a in rs[:3]]).astype(np.float64).tofile(fin)
    if masked:
        np.ascontiguousarray(solid, dtype=np.uint8).tofile(fsol)
    args = [exe, *map(str, dims), *(str(BC[b]) for b in bc), repr(re), repr(u_lid), repr(dt),
            "1" if incr else "0", str(fin), str(fsol) if masked else "-", str(fout)]
    if tile is not None:
        args += [str(tile[0]), str(tile[1])]
    r = subprocess.run(args, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stderr[-3000:])
    out = np.fromfile(fout, dtype=np.float64)
    o = 0
    for c in range(3):
        got = out[o:o + want[c].size].reshape(want[c].shape)
        o += want[c].size
        if incr:
            got = got + rs[c]
        err = np.max(np.abs(got - want[c])) / max(np.max(np.abs(want[c])), 1e-300)
        assert err <= 1e-13, (c, err)
