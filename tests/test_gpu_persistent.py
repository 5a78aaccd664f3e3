"""Persistent pressure solves: a whole multigrid-preconditioned BiCGStab solve
in one cooperative launch (batch-1 grids, the coarse propagator's path).

Each phase of the persistent solve runs the body of the kernel the launched
path uses, with the same per-CTA partial sums reduced in the same order, so
fine steps, projections and Parareal agree with the launched path (the
default; NS_PERSISTENT=1 at grid creation selects the persistent one) to
rounding level, two persistent runs
agree bit for bit, and both match the FP64 oracle at the parity tolerances.  A barrier wait limit of 1 ns makes
every wait give up: the call reports NS_ERR_TIMEOUT and the GPU stays usable.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from oracle import parareal as opr
from paper_1705_06149_gb300 import Grid, NSError, inputs
from paper_1705_06149_gb300 import _native as N

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32_refine": 1e-5}


def make_grid(persistent: bool, *args, spin_ns=None, **kw):
    saved = {k: os.environ.get(k) for k in ("NS_PERSISTENT", "NS_PERSIST_SPIN_NS")}
    os.environ["NS_PERSISTENT"] = "1" if persistent else "0"
    if spin_ns is not None:
        os.environ["NS_PERSIST_SPIN_NS"] = str(spin_ns)
    try:
        return Grid(*args, **kw)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


CASES = [((64, 64, 64), ("wall",) * 3, None),
         ((32, 32, 32), ("wall",) * 3, None),
         ((40, 24, 16), ("wall", "wall", "periodic"), None),
         ((20, 18, 16), ("wall",) * 3, "boxes")]


def rel_diff(a, b):
    a = a.double()
    b = b.double()
    return float((a - b).norm() / max(float(b.norm()), 1e-300))


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_persistent_steps_agree_with_launched_kernels(prec, case):
    """Two persistent runs agree bit for bit (no race between the phases), and
    agree with the launched kernels to rounding level: the same bodies are
    compiled inside one kernel, where the compiler may contract other products
    into fused multiply-adds."""
    dims, bc, solid_kind = CASES[case]
    solid = None
    if solid_kind:
        _, solid = inputs.obstacle_boxes(dims, seed=3, count=2)
    init = inputs.random_state(*dims, seed=60 + case, sigma=0.2, bc=bc, solid=solid)
    runs = []
    for persistent in (True, True, False):
        g = make_grid(persistent, *dims, re=500.0, bc=bc, precision=prec, batch=1, solid=solid)
        st = g.state_from(init)
        g.reset_stats()
        g.step_fine(st, 1e-3, 3)
        g.project(st)
        runs.append((st, g.stats()))
        g.close()
    (a, sa), (a2, _), (b, sb) = runs
    for c in range(4):
        assert torch.equal(a.fields()[c], a2.fields()[c]), ("repeat", "uvwp"[c], dims, prec)
    tol = 1e-12 if prec == "fp64" else 1e-5
    diffs = [rel_diff(a.fields()[c], b.fields()[c]) for c in range(4)]
    print(f"\npersistent vs launched {prec} {dims}: " + " ".join(f"{x:.2e}" for x in diffs)
          + f"; iterations {sa['krylov_iters']} vs {sb['krylov_iters']}")
    assert max(diffs) <= tol, diffs
    assert sa["steps"] == sb["steps"] and sa["solves"] == sb["solves"], (sa, sb)
    assert abs(sa["krylov_iters"] - sb["krylov_iters"]) <= max(2, sb["krylov_iters"] // 20)
    # one launch per solve instead of several per Krylov iteration
    assert sa["launches"] < sb["launches"]


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_persistent_steps_match_the_oracle(prec):
    dims, bc = (32, 32, 32), ("wall",) * 3
    init = inputs.random_state(*dims, seed=7, sigma=0.2, bc=bc)
    og = oracle.Grid(*dims, re=400.0, bc=bc, rtol=1e-13)
    want = oracle.copy_state(init)
    og.step(want, 1e-3, 4)
    g = make_grid(True, *dims, re=400.0, bc=bc, precision=prec, batch=1, poisson_rtol=1e-13)
    st = g.state_from(init)
    g.step_fine(st, 1e-3, 4)
    got = [a[0] for a in st.numpy()]
    vg = np.concatenate([np.ravel(got[c]) for c in range(3)])
    vw = np.concatenate([np.ravel(want[c]) for c in range(3)])
    assert np.linalg.norm(vg - vw) <= TOL[prec] * np.linalg.norm(vw)
    assert np.linalg.norm(got[3] - want[3]) <= TOL[prec] * np.linalg.norm(want[3])
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_persistent_coarse_chain_matches_launched_chain_and_oracle(prec):
    """Parareal (Eq. 6) whose coarse propagator runs persistent solves against
    the same call whose chain is the CUDA graph of launched kernels, and
    against the oracle's Parareal."""
    n, S, M, K = 16, 20, 2, 2
    og = oracle.Grid(n, n, n, re=100.0, rtol=1e-13)
    y_ref, d_ref = opr.parareal(og.zeros(), 4, opr.fine_propagator(og, 1e-3, S),
                                opr.coarse_propagator(og, 1e-3 * S / M, M), kmax=K)
    out = {}
    for persistent in (True, False):
        g = make_grid(persistent, n, n, n, re=100.0, precision=prec, batch=4, poisson_rtol=1e-13)
        u0 = g.zeros(1)
        slices = g.zeros(5)
        k, d = g.parareal(u0, slices, 4, S, M, 1e-3, kmax=K)
        assert k == K
        out[persistent] = (slices, d)
        g.close()
    (a, da), (b, db) = out[True], out[False]
    tol = 1e-12 if prec == "fp64" else 1e-5
    for c in range(4):
        assert rel_diff(a.fields()[c], b.fields()[c]) <= tol, "uvwp"[c]
    got = a.numpy()
    for s in range(5):
        vg = np.concatenate([np.ravel(got[c][s]) for c in range(3)])
        vw = np.concatenate([np.ravel(y_ref[s][c]) for c in range(3)])
        assert np.linalg.norm(vg - vw) <= TOL[prec] * max(np.linalg.norm(vw), 1e-300)
        assert np.linalg.norm(got[3][s] - y_ref[s][3]) <= TOL[prec] * max(
            np.linalg.norm(y_ref[s][3]), 1e-300)


def test_a_barrier_wait_that_gives_up_is_reported():
    dims = (32, 32, 32)
    g = make_grid(True, *dims, re=400.0, precision="fp32_refine", batch=1, spin_ns=1)
    st = g.state_from(inputs.random_state(*dims, seed=8, sigma=0.2))
    with pytest.raises(NSError) as e:
        g.step_fine(st, 1e-3, 1)
    assert e.value.status == N.NS_ERR_TIMEOUT
    g.close()
    # the context stays usable: a grid with the default limit steps normally
    g2 = make_grid(True, *dims, re=400.0, precision="fp32_refine", batch=1)
    st2 = g2.state_from(inputs.random_state(*dims, seed=8, sigma=0.2))
    g2.step_fine(st2, 1e-3, 2)
    torch.cuda.synchronize()
    assert all(torch.isfinite(t).all() for t in st2.fields())
    g2.close()
