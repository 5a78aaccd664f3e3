"""The V-cycle below the finest level on a thread-block cluster per state.

The cluster kernel computes the V(2,0) cycle of the grid-level and one-CTA
kernels it replaces (the same operator; the order of some operations
differs), so fine steps with it agree with fine steps without it
(NS_MG_CLUSTER=0) to rounding level with about the same iteration counts, on
walls, periodic and slip axes, for the cluster sizes the library picks for a
batch of 32 (4 CTAs), small batches (8 CTAs) and grids whose coarse levels
split only 2 or 4 ways; both match the FP64 oracle.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1705_06149_gb300 import Grid, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32_refine": 1e-5}


def make_grid(cluster: bool, *args, **kw):
    saved = os.environ.get("NS_MG_CLUSTER")
    os.environ["NS_MG_CLUSTER"] = "1" if cluster else "0"
    try:
        return Grid(*args, **kw)
    finally:
        if saved is None:
            os.environ.pop("NS_MG_CLUSTER", None)
        else:
            os.environ["NS_MG_CLUSTER"] = saved


def rel_diff(a, b):
    a = a.double()
    b = b.double()
    return float((a - b).norm() / max(float(b.norm()), 1e-300))


CASES = [((64, 64, 64), ("wall",) * 3, 4),
         ((64, 64, 64), ("wall",) * 3, 32),
         ((64, 64, 64), ("wall", "wall", "periodic"), 2),
         ((48, 48, 48), ("slip", "wall", "slip"), 3),
         ((64, 32, 64), ("periodic", "wall", "periodic"), 1),
         ((32, 32, 16), ("wall", "periodic", "wall"), 2)]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_cluster_vcycle_agrees_with_the_grid_level_kernels(prec, case):
    dims, bc, batch = CASES[case]
    inits = [inputs.random_state(*dims, seed=90 + s, sigma=0.2, bc=bc) for s in range(batch)]
    out = {}
    for cluster in (True, False):
        g = make_grid(cluster, *dims, re=800.0, bc=bc, precision=prec, batch=batch)
        st = g.state_from([np.stack([i[c] for i in inits]) for c in range(4)])
        g.profile(True)
        g.step_fine(st, 1e-3, 3)
        prof = g.profile_read()
        g.profile(False)
        out[cluster] = ([f.clone() for f in st.fields()], prof, g.stats())
        g.close()
    (a, pa, sa), (b, pb, sb) = out[True], out[False]
    assert pa["mg_cluster"]["launches"] > 0 and pa["mg_block"]["launches"] == 0, pa
    assert pb["mg_cluster"]["launches"] == 0 and pb["mg_block"]["launches"] > 0, pb
    tol = 1e-12 if prec == "fp64" else 1e-5
    diffs = [rel_diff(a[c], b[c]) for c in range(4)]
    print(f"\ncluster vs grid-level {prec} {dims} x {batch}: "
          + " ".join(f"{x:.2e}" for x in diffs)
          + f"; Krylov iterations {sa['krylov_iters']} vs {sb['krylov_iters']}")
    assert max(diffs) <= tol, diffs
    assert abs(sa["krylov_iters"] - sb["krylov_iters"]) <= max(2, sb["krylov_iters"] // 10)


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_cluster_steps_match_the_oracle(prec):
    # the setting of the fine-step parity tests (Re 100, 4 steps, solves to
    # 1e-13) on a grid whose 16 x 16 x 8 level splits over 4-CTA clusters: the
    # pressure error of a solve stopped at relative residual rtol is bounded
    # by cond(L) rtol, so the grid stays as small as the parity tests' grids
    dims, bc = (32, 32, 16), ("wall", "periodic", "wall")
    B = 2
    inits = [inputs.random_state(*dims, seed=20 + s, sigma=0.2, bc=bc) for s in range(B)]
    og = oracle.Grid(*dims, re=100.0, bc=bc, rtol=1e-13)
    g = make_grid(True, *dims, re=100.0, bc=bc, precision=prec, batch=B, poisson_rtol=1e-13)
    st = g.state_from([np.stack([i[c] for i in inits]) for c in range(4)])
    g.profile(True)
    g.step_fine(st, 1e-3, 4)
    assert g.profile_read()["mg_cluster"]["launches"] > 0
    got = st.numpy()
    for s in range(B):
        want = oracle.copy_state(inits[s])
        og.step(want, 1e-3, 4)
        vg = np.concatenate([np.ravel(got[c][s]) for c in range(3)])
        vw = np.concatenate([np.ravel(want[c]) for c in range(3)])
        assert np.linalg.norm(vg - vw) <= TOL[prec] * np.linalg.norm(vw)
        assert np.linalg.norm(got[3][s] - want[3]) <= TOL[prec] * np.linalg.norm(want[3])
    g.close()
