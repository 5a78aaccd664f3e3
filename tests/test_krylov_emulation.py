"""Whole plain BiCGStab pressure solves run on the host: the three phases of
an iteration (k_bicg_A, k_bicg_B, k_bicg_C: the convergence test and restart
rule, the parity ping-pong of the search direction, alpha and omega from the
partial sums), the FP64 solve from a warm start with the gauge of the
no-allocation entry point (k_noalloc_gauge), and the FP32 inner solves inside
FP64 iterative refinement (k_refine_init, k_inner_init, k_refine_update),
taken verbatim from csrc/ns_kernels.cuh and csrc/ns_noalloc.cu and compiled as
C++ with every CTA as host threads (tests/emu/) under AddressSanitizer and
UBSan, in the launch sequences of the library's host loops, with the FP64
oracle's L = D G (Section 2: homogeneous Neumann conditions at walls and solid
surfaces) as the operator:

- four iterations (both parities twice, the first a start) of the FP64 solve
  and of an FP32 inner solve agree with BiCGStab as van der Vorst defines it,
  written out below in numpy on the same system;
- a whole FP64 solve takes about the oracle's number of iterations (the two
  sum their dot products in different orders, and BiCGStab's residual
  history is sensitive to rounding), stops at the tolerance, and its gauged
  result matches the oracle's gauged solve; the refinement ends with the
  outer residual at its tolerance after a few outer steps, the result in the
  buffer the outer count selects.

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
ST_CONV, OS_DONE = 1, 1


def _kernel(src: str, marker: str) -> str:
    start = src.index(marker)
    return src[start:src.index("\n}\n", start) + 3]


def _source() -> str:
    dev = open(os.path.join(CSRC, "ns_device.cuh")).read()
    ker = open(os.path.join(CSRC, "ns_kernels.cuh")).read()
    na = open(os.path.join(CSRC, "ns_noalloc.cu")).read()
    a = dev.index("enum { BC_WALL")
    b = dev.index("}  // namespace nsk")
    k0 = ker.index("enum { ST_ITER")
    k1 = ker.index("// predictor  F*")
    k2 = ker.index("// partial sums of a cell field")
    start = ker.index("    k_refine_update(")
    k3 = ker.index("\n}\n", start) + 3
    head = ker[k0:k1].rstrip().rsplit("\n", 1)[0]  # without the dashes above the heading
    return "\n\n".join([dev[a:b], head, ker[k2:k3],
                        _kernel(na, "// p = x - mean(x), the mean taken")])


@pytest.fixture(scope="module")
def krylov_emulator(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("krylov_emu")
    cpp = d / "krylov_emu.cpp"
    cpp.write_text('#include "block_emu.h"\n\n' + _source() + "\n\n" +
                   open(os.path.join(EMU, "krylov_emu_main.cpp")).read())
    exe = d / "krylov_emu"
    cmd = [gxx, "-std=c++20", "-O1", "-g", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer", "-pthread",
           "-I", EMU, str(cpp), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "barrier" in r.stderr and "No such file" in r.stderr:
        pytest.skip("the host compiler has no <barrier>")
    assert r.returncode == 0, r.stderr[-3000:]
    return str(exe), d


CASES = [
    ((8, 8, 8), ("wall",) * 3, False),
    ((12, 6, 5), ("periodic", "wall", "slip"), False),   # ragged y and z tiles
    ((36, 4, 4), ("wall", "periodic", "periodic"), False),  # two x tiles, the second ragged
    ((16, 12, 8), ("wall",) * 3, True),                  # solid boxes
]

KMAX = 4


def _start(exe, d, dims, bc, solid, b, x0, rtol, inner_rtol, refine_rtol, kmax):
    nx, ny, nz = dims
    tag = f"{os.getpid()}_{nx}_{ny}_{nz}_{int(solid is not None)}_{kmax}"
    fin, fsol, fout = d / f"in_{tag}.bin", d / f"solid_{tag}.bin", d / f"out_{tag}.bin"
    np.concatenate([b.ravel(), x0.ravel()]).astype(np.float64).tofile(fin)
    if solid is not None:
        np.ascontiguousarray(solid, dtype=np.uint8).tofile(fsol)
    maxit = 20 * max(dims)
    args = [exe, *map(str, dims), *(str(BC[x]) for x in bc), repr(rtol), str(maxit),
            repr(inner_rtol), repr(refine_rtol), "40", str(kmax), str(fin),
            str(fsol) if solid is not None else "-", str(fout)]
    proc = subprocess.Popen(args, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
    return proc, fout, maxit


def _finish(run):
    proc, fout, maxit = run
    so, se = proc.communicate(timeout=600)
    assert proc.returncode == 0, (proc.returncode, se[-3000:])
    val = {}
    for line in so.split("\n"):
        if line.strip():
            k, v = line.split()
            val[k] = float(v)
    return val, open(fout, "rb").read(), maxit


WHOLE = ((8, 4, 4), ("wall",) * 3)  # one CTA: a solve is hundreds of launches
WHOLE_TOL = (1e-6, 3e-4, 1e-6)      # FP64 rtol, inner rtol, outer rtol


@pytest.fixture(scope="module")
def krylov_runs(krylov_emulator):
    """Every case at once: each run waits mostly on its threads' barriers, so
    they overlap well on the host's cores."""
    exe, d = krylov_emulator
    runs = {}
    for dims, bc, masked in CASES:
        _, solid, _, b, x0 = _inputs(dims, masked)
        runs[(dims, bc, masked)] = _start(exe, d, dims, bc, solid, b, x0, 1e-30, 1e-30, 1e-30,
                                          KMAX)
    _, _, _, b, x0 = _inputs(WHOLE[0], False)
    runs["whole"] = _start(exe, d, WHOLE[0], WHOLE[1], None, b, x0, *WHOLE_TOL, 0)
    return {k: _finish(v) for k, v in runs.items()}


def _inputs(dims, masked):
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    solid = None
    if masked:
        _, solid = inputs.obstacle_boxes(dims, seed=4, count=2, edge=(0.2, 0.35))
        assert solid.any()
    fluid = np.ones(shape, bool) if solid is None else solid == 0
    rng = np.random.default_rng(nx + 7 * ny + 49 * nz)
    b = np.where(fluid, 0.5 + rng.normal(size=shape), 0.0)
    x0 = np.where(fluid, 0.1 * rng.normal(size=shape), 0.0)
    return shape, solid, fluid, b, x0


def _bicgstab(L, b, x, iters):
    """BiCGStab (van der Vorst 1992) from x with the shadow residual r_hat =
    r_0, restarted (p = r, r_hat = r) when (r_hat, r) or omega is 0.
    Returns x, r, alpha, omega after `iters` iterations."""
    r = b - L(x)
    rh = r.copy()
    p = v = None
    rho_old = alpha = omega = 1.0
    for it in range(1, iters + 1):
        rho = float(np.sum(rh * r))
        if it == 1 or rho == 0.0 or omega == 0.0:
            rh = r.copy()
            rho = float(np.sum(r * r))
            p = r.copy()
        else:
            beta = (rho / rho_old) * (alpha / omega)
            p = r + beta * (p - omega * v)
        v = L(p)
        alpha = rho / float(np.sum(rh * v))
        s = r - alpha * v
        t = L(s)
        omega = float(np.sum(t * s)) / float(np.sum(t * t))
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
    return x, r, alpha, omega


@pytest.mark.parametrize("dims,bc,masked", CASES)
def test_bicgstab_iterations_match_definition(krylov_runs, dims, bc, masked):
    shape, solid, fluid, b, x0 = _inputs(dims, masked)
    og = oracle.Grid(*dims, bc=bc, solid=solid)
    val, raw, _ = krylov_runs[(dims, bc, masked)]
    C = b.size
    off = 0

    def take(dtype):
        nonlocal off
        a = np.frombuffer(raw, dtype=dtype, count=C, offset=off).reshape(shape)
        off += a.nbytes
        return a.astype(np.float64)

    x, r = take(np.float64), take(np.float64)
    e = take(np.float32)
    pn = take(np.float64)
    r32 = take(np.float32)
    assert off == len(raw)
    b1 = np.where(fluid, b - b[fluid].mean(), 0.0)
    # FP64: four iterations from x0
    xw, rw, aw, ww = _bicgstab(og.laplacian, b1, x0, KMAX)
    assert val["fp64.status"] == 0 and val["fp64.iters"] == KMAX and val["fp64.restart"] == 0
    assert np.max(np.abs(x - xw)) <= 1e-12 * np.max(np.abs(xw))
    assert np.max(np.abs(r - rw)) <= 1e-10 * np.max(np.abs(rw))
    assert abs(val["fp64.alpha"] - aw) <= 1e-11 * abs(aw)
    assert abs(val["fp64.omega"] - ww) <= 1e-11 * abs(ww)
    assert np.all(x[~fluid] == 0.0) and np.all(r[~fluid] == 0.0)
    # FP32 inner solve of L e = r32 from e = 0, r32 the FP32 outer residual of x0
    r0 = (b1 - og.laplacian(x0)).astype(np.float32).astype(np.float64)
    ew, _, aw, ww = _bicgstab(og.laplacian, r0, np.zeros(shape), KMAX)
    assert np.max(np.abs(e - ew)) <= 1e-4 * np.max(np.abs(ew))
    assert abs(val["ref.alpha"] - aw) <= 1e-4 * abs(aw)
    assert abs(val["ref.omega"] - ww) <= 1e-4 * abs(ww)
    assert np.all(e[~fluid] == 0.0)
    # the outer correction with the kernels' own e
    assert np.array_equal(pn, x0 + e)
    rw = b1 - og.laplacian(pn)
    assert np.all(np.abs(r32 - rw) <= 2.0 ** -24 * np.abs(rw) + 1e-12 * np.max(np.abs(rw)))


def test_whole_solves_match_oracle(krylov_runs):
    dims, bc = WHOLE
    rtol, _, refine_rtol = WHOLE_TOL
    shape, _, _, b, x0 = _inputs(dims, False)
    og = oracle.Grid(*dims, bc=bc)
    val, raw, maxit = krylov_runs["whole"]
    out = np.frombuffer(raw, dtype=np.float64)
    C = b.size
    x, p, pref = (out[q * C:(q + 1) * C].reshape(shape) for q in range(3))
    b1 = b - b.mean()
    nb = np.linalg.norm(b1)
    _, it_o, _, st = og.bicgstab(b1, x0, rtol=rtol, maxit=maxit)
    assert st == 0
    assert val["fp64.status"] == ST_CONV
    assert abs(val["fp64.iters"] - it_o) <= max(1, 0.05 * it_o), (val["fp64.iters"], it_o)
    assert val["fp64.total_iters"] == val["fp64.iters"]
    assert val["fp64.launched"] == val["fp64.iters"] + 1  # the last phase A finds convergence
    assert abs(val["fp64.bb"] - nb * nb) <= 1e-12 * nb * nb
    assert val["fp64.rr"] <= rtol ** 2 * val["fp64.bb"]
    assert np.linalg.norm(b1 - og.laplacian(x)) <= 1.5 * rtol * nb
    assert abs(val["fp64.sx"] - x.sum()) <= 1e-12 * np.sum(np.abs(x))
    # the gauged solution against the oracle's gauged solve
    pg, _ = og.poisson(b, x0=x0, rtol=1e-13, maxit=maxit)
    scale = np.max(np.abs(pg))
    assert np.max(np.abs(p - (x - x.mean()))) <= 1e-14 * scale
    assert np.max(np.abs(p - pg)) <= 1e-4 * scale
    # FP32 inner solves inside FP64 refinement
    assert val["ref.o_status"] == OS_DONE
    # one correction per outer step that found the state refining; the
    # control block's o_steps holds the index of the last inner solve started
    assert 1 <= val["ref.corrections"] <= 10 and val["ref.m"] == val["ref.corrections"]
    assert val["ref.o_steps"] == val["ref.m"] - 1
    assert val["ref.p_final"] == int(val["ref.m"]) % 2
    assert val["ref.o_rr"] <= refine_rtol ** 2 * val["ref.o_bb"]
    assert abs(val["ref.o_bb"] - nb * nb) <= 1e-12 * nb * nb
    assert np.linalg.norm(b1 - og.laplacian(pref)) <= 1.5 * refine_rtol * nb
    assert np.max(np.abs((pref - pref.mean()) - pg)) <= 1e-4 * scale
    assert val["ref.inner_total"] >= val["ref.corrections"]
