"""The float-float refinement kernels run on the host: the start of a refined
pressure solve from a warm start (k_mg_refine_init_ff), one outer correction
(k_mg_refine_update_ff) and the velocity correction with the float-float
pressure (k_correct_ff), taken verbatim from csrc/ns_mg.cuh and compiled as
C++ with every CTA as host threads (tests/emu/) under AddressSanitizer and
UBSan, against the same operations in FP64:

  start:      p = w, r = (b - mean b) - L w, r32 = r_hat = hi(r);
  correction: p += e / s, r -= L e / s and the residual's fluid mean,
              r32 = r_hat = hi(r) * s';
  decisions:  each inner solve's tolerance, the looser of itol and what the
              outer target still needs (a factor 2 below it);
  velocity:   u = F* - dt G p on active faces (0 on wall faces), p_out =
              p - mean, q = p - mean, w = 2 (p - mean) - q_old,

with hi + lo within about 2^-45 of the FP64 values (the float-float pairs
carry about 48 bits) and u to FP32 rounding.  No GPU needed."""
from __future__ import annotations

import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1705_06149_gb300 import inputs
from test_mg_block_emulation import CSRC, EMU, _extract, _lap

BC = {"wall": 0, "periodic": 1, "slip": 2}


def _source() -> str:
    dev = open(os.path.join(CSRC, "ns_device.cuh")).read()
    ker = open(os.path.join(CSRC, "ns_kernels.cuh")).read()
    mg = open(os.path.join(CSRC, "ns_mg.cuh")).read()
    a = dev.index("enum { BC_WALL")
    b = dev.index("}  // namespace nsk")
    head = [dev[a:b], _extract(ker, r"^enum \{ ST_ITER"), _extract(ker, r"^enum \{ OS_REFINE"),
            _extract(ker, r"^struct SliceCtl \{")]
    s = mg.index("constexpr int MG_MAX_LEVELS")
    start = mg.index("    k_correct_ff(")
    e = mg.index("\n}\n", start) + 3
    body = mg[s:e]
    shared = "extern __shared__ __align__(16) unsigned char smem_raw[];"
    assert shared in body
    return "\n\n".join(head) + "\n\n" + body.replace(shared, "unsigned char* smem_raw = emu_smem;")


@pytest.fixture(scope="module")
def refine_emulator(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("refine_emu")
    cpp = d / "refine_emu.cpp"
    cpp.write_text('#include "block_emu.h"\n\n' + _source() + "\n\n" +
                   open(os.path.join(EMU, "refine_emu_main.cpp")).read())
    exe = d / "refine_emu"
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
]


def _ff(rng, shape, scale):
    """A float-float field: hi FP32, lo the FP32 rounding of the remainder."""
    x = rng.normal(size=shape) * scale
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


@pytest.mark.parametrize("dims,bc", CASES)
def test_float_float_refinement_matches_fp64(refine_emulator, dims, bc):
    exe, d = refine_emulator
    nx, ny, nz = dims
    cshape = (nz, ny, nx)
    rng = np.random.default_rng(sum(dims))
    b = rng.normal(size=cshape) * 100.0
    wh, wl = _ff(rng, cshape, 1.0)
    e = (rng.normal(size=cshape) * 0.01).astype(np.float32)
    # the pressure as the solver sees it: a large level plus small variations,
    # so that its differences need the low parts
    x = 1000.0 + 1e-2 * rng.normal(size=cshape)
    ph = x.astype(np.float32)
    pl = (x - ph.astype(np.float64)).astype(np.float32)
    rh, rl = _ff(rng, cshape, 1e-3)
    qh, ql = _ff(rng, cshape, 1.0)
    fst = [(1e-2 * f).astype(np.float32)
           for f in inputs.random_state(*dims, seed=3, sigma=1.0, bc=bc)[:3]]
    rmean, mean = 1.25e-4, 0.375
    dt, unscale, fsc, lbox = 2e-3, 0.5, 4.0, 1.3  # h = 1.3 / n: 1/h^2 is not an FP32 number
    fin, fout = d / f"in_{nx}_{ny}_{nz}.bin", d / f"out_{nx}_{ny}_{nz}.bin"
    with open(fin, "wb") as f:
        b.astype(np.float64).tofile(f)
        for a in (wh, wl, e, ph, pl, rh, rl, qh, ql):
            a.tofile(f)
        for a in fst:
            a.tofile(f)
        np.array([rmean, mean], dtype=np.float64).tofile(f)
    args = [exe, *map(str, dims), *(str(BC[x]) for x in bc), repr(lbox), repr(dt), repr(unscale),
            repr(fsc), str(fin), str(fout)]
    r = subprocess.run(args, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stderr[-3000:])
    raw = open(fout, "rb").read()
    off = 0

    def take(dtype, shape):
        nonlocal off
        a = np.frombuffer(raw, dtype=dtype, count=int(np.prod(shape)), offset=off).reshape(shape)
        off += a.nbytes
        return a.astype(np.float64)

    w = [(n / lbox) ** 2 for n in dims]
    f64 = lambda hi, lo: hi.astype(np.float64) + lo.astype(np.float64)  # noqa: E731
    tol = 2.0 ** -45
    # start of the refined solve
    Ph, Pl, Rh, Rl, r32, rhat = (take(np.float32, cshape) for _ in range(6))
    assert np.array_equal(Ph, wh) and np.array_equal(Pl, wl)
    want = (b - b.mean()) - _lap(f64(wh, wl), bc_codes(bc), w)
    scale = np.max(np.abs(b)) + np.max(np.abs(_lap(f64(wh, wl), bc_codes(bc), w))) + 4 * sum(w)
    assert np.max(np.abs((Rh + Rl) - want)) <= tol * scale
    assert np.array_equal(r32, Rh) and np.array_equal(rhat, Rh)
    # one outer correction
    Ph, Pl, Rh, Rl, r32, rhat = (take(np.float32, cshape) for _ in range(6))
    want_p = f64(ph, pl) + e.astype(np.float64) * unscale
    assert np.max(np.abs((Ph + Pl) - want_p)) <= tol * np.max(np.abs(want_p))
    le = _lap(e.astype(np.float64), bc_codes(bc), w)
    want_r = f64(rh, rl) - le * unscale - rmean
    scale = np.max(np.abs(f64(rh, rl))) + np.max(np.abs(le)) * unscale + 4 * sum(w) * 0.01
    assert np.max(np.abs((Rh + Rl) - want_r)) <= tol * scale
    assert np.array_equal(r32, (Rh.astype(np.float32) * np.float32(fsc)).astype(np.float64))
    assert np.array_equal(rhat, r32)
    # velocity correction, gauged pressure and the next warm start
    vel = [take(np.float32, fst[c].shape) for c in range(3)]
    pout = take(np.float64, cshape)
    Wh, Wl, Qh, Ql = (take(np.float32, cshape) for _ in range(4))
    p = f64(ph, pl)
    for c in range(3):
        ax = 2 - c
        want_u = fst[c].astype(np.float64).copy()
        sl = [slice(None)] * 3
        if bc[c] == "periodic":
            grad = (p - np.roll(p, 1, axis=ax)) * (dims[c] / lbox)
            want_u = want_u - dt * grad
        else:
            sl[ax] = slice(1, dims[c])
            inner = (np.take(p, range(1, dims[c]), axis=ax) -
                     np.take(p, range(0, dims[c] - 1), axis=ax)) * (dims[c] / lbox)
            want_u[tuple(sl)] = want_u[tuple(sl)] - dt * inner
            s0 = [slice(None)] * 3
            s0[ax] = 0
            s1 = [slice(None)] * 3
            s1[ax] = -1
            want_u[tuple(s0)] = 0.0
            want_u[tuple(s1)] = 0.0
        err = np.max(np.abs(vel[c] - want_u))
        assert err <= 2e-6 * np.max(np.abs(want_u)), (c, err)
    assert np.max(np.abs(pout - (p - mean))) <= tol * np.max(np.abs(p - mean))
    assert np.max(np.abs((Qh + Ql) - (p - mean))) <= tol * np.max(np.abs(p - mean))
    want_w = 2.0 * (p - mean) - f64(qh, ql)
    assert np.max(np.abs((Wh + Wl) - want_w)) <= tol * np.max(np.abs(want_w))
    # the decisions: each inner solve starts (status 0 = iterate, outer status
    # 0 = refine) with the looser of itol2 and a quarter of the squared
    # reduction the outer target still needs -- at the start (target 1e-4 in
    # squares) that need is the looser one, after the correction (1e-30) itol2
    dec = take(np.float64, (2, 6))
    for (o_bb, o_rr, bb, tol2_in, st, ost), otol2 in zip(dec, (1e-4, 1e-30)):
        assert st == 0 and ost == 0
        assert tol2_in == max(1e-8, 0.25 * otol2 * o_bb / o_rr)
    assert dec[0][3] > 1e-8 and dec[1][3] == 1e-8
    assert dec[0][2] == dec[0][1]  # the start's inner solve: bb = the outer residual
    assert off == len(raw)


def bc_codes(bc):
    return [BC[x] for x in bc]


@pytest.fixture(scope="module")
def decide_emulator(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("decide_emu")
    cpp = d / "decide_emu.cpp"
    cpp.write_text('#include "block_emu.h"\n\n' + _source() + "\n\n" +
                   open(os.path.join(EMU, "decide_emu_main.cpp")).read())
    exe = d / "decide_emu"
    r = subprocess.run([gxx, "-std=c++20", "-O1", "-fsanitize=address,undefined",
                        "-fno-sanitize-recover=undefined", "-pthread", "-I", EMU, str(cpp), "-o",
                        str(exe)], capture_output=True, text=True)
    if r.returncode != 0 and "barrier" in r.stderr and "No such file" in r.stderr:
        pytest.skip("the host compiler has no <barrier>")
    assert r.returncode == 0, r.stderr[-3000:]
    return str(exe)


@pytest.mark.parametrize("ratio,tol2,tol2_in,want", [
    (0.4, 1e-8, 0.5, 1),    # within the state's looser inner tolerance: converged
    (0.4, 1e-8, 0.0, 0),    # no inner tolerance set: the launch's decides, iterate
    (0.6, 1e-8, 0.5, 0),    # outside both
    (1e-9, 1e-8, 0.0, 1),   # within the launch's
    (1e-9, 1e-8, 1e-10, 1),  # a tighter inner tolerance never overrides the launch's
])
def test_convergence_decision_takes_the_looser_tolerance(decide_emulator, ratio, tol2, tol2_in,
                                                         want):
    """bicg_decide stops a state when (r, r) <= max(tol2, tol2_in) (b, b): the
    launch's tolerance, or the looser one an FP32 inner solve was given."""
    out = subprocess.run([decide_emulator, repr(ratio), repr(tol2), repr(tol2_in), "2", "100"],
                         capture_output=True, text=True, check=True).stdout.split()
    assert int(out[0]) == want
    if want == 0:
        # iterating on: beta = (rho_new / rho_old) (alpha / omega), rho_old := rho_new
        assert float(out[1]) == (3.0 / 2.0) * (0.5 / 0.25) and float(out[2]) == 3.0
