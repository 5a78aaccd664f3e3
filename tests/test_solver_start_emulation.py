"""The kernels that open and close a pressure solve run on the host:
k_sum_cells, the FP64 BiCGStab start from a warm start (k_bicg_init_warm), the
FP64 outer start of the FP32 + refinement solve (k_refine_init), its outer
convergence test and inner start (k_inner_init), the outer correction
(k_refine_update) and the FP64 start of the multigrid-preconditioned solve
with its last-CTA decision (k_mg_init_warm), taken verbatim from
csrc/ns_kernels.cuh and csrc/ns_mg.cuh and compiled as C++ with every CTA as
host threads (tests/emu/) under AddressSanitizer and UBSan, against the FP64
oracle's masked Neumann operator L = D G (Section 2):

  start:       b' = b - fluid mean (0 in solid cells), x = x0, r = b' - L x0,
               r_hat = r, with the sums (r_hat, r), (r, r), sum x, (b', b');
  outer start: p = p_in (0 in solid cells), r32 = fl32(b' - L p);
  inner start: r_hat = r32, e = 0 unless the outer residual has met the
               threshold (done, p_final = m mod 2) or m reached the limit;
  correction:  p = p_old + e, r32 = fl32(b - L p);
  multigrid:   as the start, plus the first restart decision (beta = 0,
               rho = (r, r)).

No GPU needed."""
from __future__ import annotations

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1705_06149_gb300 import inputs
from test_masked_mg_emulation import _codes
from test_mg_block_emulation import CSRC, EMU

BC = {"wall": 0, "periodic": 1, "slip": 2}
ST_ITER, ST_IDLE = 0, 4
OS_REFINE, OS_DONE, OS_FAIL = 0, 1, 2


def _source() -> str:
    dev = open(os.path.join(CSRC, "ns_device.cuh")).read()
    ker = open(os.path.join(CSRC, "ns_kernels.cuh")).read()
    mg = open(os.path.join(CSRC, "ns_mg.cuh")).read()
    a = dev.index("enum { BC_WALL")
    b = dev.index("}  // namespace nsk")
    k0 = ker.index("enum { ST_ITER")
    k1 = ker.index("// predictor  F*")
    k2 = ker.index("// partial sums of a cell field")
    start = ker.index("    k_refine_update(")
    k3 = ker.index("\n}\n", start) + 3
    s = mg.index("constexpr int MG_MAX_LEVELS")
    start = mg.index("    k_mg_init_warm(")
    e = mg.index("\n}\n", start) + 3
    body = mg[s:e]
    shared = "extern __shared__ __align__(16) unsigned char smem_raw[];"
    body = body.replace(shared, "unsigned char* smem_raw = emu_smem;")
    # the line of dashes above the predictor's heading stays out
    head = ker[k0:k1].rstrip().rsplit("\n", 1)[0]
    return "\n\n".join([dev[a:b], head, ker[k2:k3], body])


@pytest.fixture(scope="module")
def start_emulator(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("start_emu")
    cpp = d / "start_emu.cpp"
    cpp.write_text('#include "block_emu.h"\n\n' + _source() + "\n\n" +
                   open(os.path.join(EMU, "start_emu_main.cpp")).read())
    exe = d / "start_emu"
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
    ((20, 18, 16), ("wall",) * 3, True),           # solid boxes
    ((16, 16, 12), ("periodic", "wall", "periodic"), True),
]


def _near(a, b):
    return abs(a - b) <= 1e-14 * abs(b)


def _close(got, want, rel=1e-13):
    scale = max(float(np.max(np.abs(want))), 1e-300)
    return float(np.max(np.abs(got - want))) <= rel * scale


def _inputs(dims, masked):
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    solid = None
    if masked:
        _, solid = inputs.obstacle_boxes(dims, seed=21, count=3, edge=(0.15, 0.3))
        assert solid.any()
    fluid = np.ones(shape, bool) if solid is None else solid == 0
    rng = np.random.default_rng(nx * ny + nz)
    b = np.where(fluid, 1.0 + rng.normal(size=shape), 0.0)  # a nonzero mean to remove
    x0 = np.where(fluid, rng.normal(size=shape), 0.0)
    p = rng.normal(size=shape)                               # solid cells to be zeroed
    pold = np.where(fluid, rng.normal(size=shape), 0.0)
    e = np.where(fluid, 1e-3 * rng.normal(size=shape), 0.0).astype(np.float32)
    return shape, solid, fluid, b, x0, p, pold, e


@pytest.fixture(scope="module")
def start_runs(start_emulator):
    """Every case at once: each run waits mostly on its threads' barriers, so
    they overlap well on the host's cores."""
    exe, d = start_emulator
    procs = {}
    for dims, bc, masked in CASES:
        _, solid, _, b, x0, p, pold, e = _inputs(dims, masked)
        tag = f"{os.getpid()}_{'_'.join(map(str, dims))}_{int(masked)}"
        fin, fsol, fout = d / f"in_{tag}.bin", d / f"solid_{tag}.bin", d / f"out_{tag}.bin"
        with open(fin, "wb") as f:
            for a in (b, x0, p, pold):
                a.astype(np.float64).tofile(f)
            e.tofile(f)
        if masked:
            with open(fsol, "wb") as f:
                np.ascontiguousarray(solid, dtype=np.uint8).tofile(f)
                _codes(solid, bc).tofile(f)
        args = [exe, *map(str, dims), *(str(BC[x]) for x in bc), str(fin),
                str(fsol) if masked else "-", str(fout)]
        procs[(dims, bc, masked)] = (subprocess.Popen(args, stdout=subprocess.PIPE,
                                                      stderr=subprocess.PIPE, text=True), fout)
    out = {}
    for case, (pr, fout) in procs.items():
        so, se = pr.communicate(timeout=300)
        out[case] = (pr.returncode, so, se, fout)
    return out


@pytest.mark.parametrize("dims,bc,masked", CASES)
def test_solver_start_kernels_match_oracle(start_runs, dims, bc, masked):
    shape, solid, fluid, b, x0, p, pold, e = _inputs(dims, masked)
    og = oracle.Grid(*dims, bc=bc, solid=solid)
    rc, stdout, stderr, fout = start_runs[(dims, bc, masked)]
    assert rc == 0, (rc, stderr[-3000:])
    val = {}
    for line in stdout.split("\n"):
        if line.strip():
            k, v = line.split()
            val[k] = float(v)
    raw = open(fout, "rb").read()
    off = 0

    def take(dtype):
        nonlocal off
        a = np.frombuffer(raw, dtype=dtype, count=b.size, offset=off).reshape(shape)
        off += a.nbytes
        return a.astype(np.float64)

    sabs = float(np.sum(np.abs(b)))
    assert abs(val["sum_b"] - b.sum()) <= 1e-13 * sabs
    nfl = int(fluid.sum())
    b1_want = np.where(fluid, b - b.sum() / nfl, 0.0)

    # FP64 BiCGStab start
    b1, x, rr, rh = (take(np.float64) for _ in range(4))
    assert _close(b1, b1_want)
    assert np.array_equal(x, x0)
    r_want = b1_want - og.laplacian(x0)
    assert _close(rr, r_want, 1e-12)
    assert np.array_equal(rh, rr)
    ss = lambda a: float(np.sum(a * a))  # noqa: E731
    assert val["init.part0"] == val["init.part1"]
    assert abs(val["init.part1"] - ss(rr)) <= 1e-12 * ss(rr)
    assert abs(val["init.part2"] - x.sum()) <= 1e-12 * np.sum(np.abs(x))
    assert abs(val["init.part3"] - ss(b1)) <= 1e-12 * ss(b1)
    assert (val["init.status"], val["init.it_cur"], val["init.it_next"]) == (ST_ITER, 0, 0)
    assert (val["init.omega"], val["init.alpha"]) == (1.0, 1.0)

    # FP64 outer start of the refined solve
    b2, p64 = take(np.float64), take(np.float64)
    r32 = take(np.float32)
    assert np.array_equal(b2, b1)
    assert np.array_equal(p64, np.where(fluid, p, 0.0))
    r64_want = b1_want - og.laplacian(np.where(fluid, p, 0.0))
    assert np.all(np.abs(r32 - r64_want) <= 2.0 ** -24 * np.abs(r64_want) + 1e-12 * np.max(np.abs(r64_want)))
    assert np.all(r32[~fluid] == 0.0)
    assert abs(val["rinit.part0"] - ss(r64_want)) <= 1e-12 * ss(r64_want)
    assert abs(val["rinit.part1"] - ss(b1)) <= 1e-12 * ss(b1)
    assert abs(val["rinit.part2"] - p64.sum()) <= 1e-12 * np.sum(np.abs(p64))
    assert (val["rinit.o_status"], val["rinit.o_steps"], val["rinit.p_final"],
            val["rinit.status"]) == (OS_REFINE, 0, 0, ST_IDLE)

    # inner start (m = 0, not converged)
    rhat32, e0 = take(np.float32), take(np.float32)
    assert np.array_equal(rhat32, r32) and np.all(e0 == 0.0)
    s32 = ss(r32)
    for q in (0, 1, 3):
        assert abs(val[f"inner.part{q}"] - s32) <= 1e-12 * s32
    assert val["inner.part2"] == 0.0
    assert (val["inner.status"], val["inner.it_cur"], val["inner.it_next"],
            val["inner.o_steps"]) == (ST_ITER, 0, 0, 0)
    assert (val["inner.omega"], val["inner.alpha"]) == (1.0, 1.0)
    # the kernels reduce the partials in their own order
    assert _near(val["inner.o_bb"], val["rinit.part1"])
    # converged at m = 3: done, result in the buffer of odd steps
    assert val["iconv.untouched"] == 1.0
    assert (val["iconv.o_status"], val["iconv.p_final"], val["iconv.status"]) == (OS_DONE, 1, ST_IDLE)
    assert _near(val["iconv.o_rr"], val["rinit.part0"]) and val["iconv.o_bb"] == 2.0
    assert abs(val["iconv.sx"] - val["rinit.part2"]) <= 1e-14 * np.sum(np.abs(p64))
    # at the outer limit without convergence: failure
    assert val["ifail.untouched"] == 1.0
    assert (val["ifail.o_status"], val["ifail.status"]) == (OS_FAIL, ST_IDLE)
    assert _near(val["ifail.o_rr"], val["rinit.part0"]) and val["ifail.o_bb"] == 2.0

    # outer correction
    pn = take(np.float64)
    ru = take(np.float32)
    pn_want = pold + e.astype(np.float64)
    assert np.array_equal(pn, pn_want)
    ru_want = b - og.laplacian(pn_want)
    assert np.all(np.abs(ru - ru_want) <= 2.0 ** -24 * np.abs(ru_want) + 1e-12 * np.max(np.abs(ru_want)))
    assert abs(val["rupd.part0"] - ss(ru_want)) <= 1e-12 * ss(ru_want)
    assert val["rupd.part1"] == 0.0
    assert abs(val["rupd.part2"] - pn.sum()) <= 1e-12 * np.sum(np.abs(pn))
    assert val["rupd.o_status"] == OS_REFINE

    # FP64 start of the multigrid-preconditioned solve
    b3, x3, r3, rh3 = (take(np.float64) for _ in range(4))
    assert off == len(raw)
    assert np.array_equal(b3, b1)
    assert np.array_equal(x3, x0)
    assert _close(r3, r_want, 1e-12)
    assert np.array_equal(rh3, r3)
    assert val["mginit.counter"] == 0.0
    assert (val["mginit.status"], val["mginit.it_cur"], val["mginit.p_final"]) == (ST_ITER, 0, 0)
    assert (val["mginit.omega"], val["mginit.alpha"]) == (1.0, 1.0)
    assert abs(val["mginit.bb"] - ss(b3)) <= 1e-12 * ss(b3)
    assert abs(val["mginit.rr"] - ss(r3)) <= 1e-12 * ss(r3)
    assert abs(val["mginit.sx"] - x3.sum()) <= 1e-12 * np.sum(np.abs(x3))
    assert (val["mginit.restart"], val["mginit.beta"]) == (1, 0.0)
    assert val["mginit.rho0"] == val["mginit.rr"]
