"""The headline call at its own size against the FP64 CPU oracle.

ns_parareal_iterate (Section 2.1.2, Eq. 6) on the 64^3 batched-Parareal cavity
(Re 1000, u_lid 1, walls on all faces, 32 time slices), from the workload's
start state (the 16^3 Re 100 cavity at t = 0.2, trilinearly upsampled to 64^3,
N(0, 1e-3^2) face noise with seed 0, projected), with the library's default
coarse propagator (the batch-1 companion grid and its chain graph), compared
slice by slice and field by field with the oracle's Parareal loop
(oracle/parareal.py, the fine sweep over the slices on the host cores).

The run is truncated so that the oracle finishes in minutes: 2 fine steps of
5e-4 per slice, 1 coarse step of 1e-3 per slice (Courant number 0.064, stable),
K = 2 iterations.  Every grid-level kernel of the batched sweep (32 states),
of the batch-1 companion (the chain graph's conditional loops) and the Eq. 6
update over all 32 slices take part.

Tolerances: FP64 relative L2 <= 1e-10 on each of u, v, w and p; FP32 storage
with FP64 refinement <= 1e-5 on the velocity field and on p.  Both sides solve
the pressure to a relative residual of 1e-13 (FP64) so that the solver's own
tolerance stays below the comparison's.  The per-component errors are printed
(`pytest -s` shows them).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import parareal as opr
from paper_1705_06149_gb300 import Grid
from paper_1705_06149_gb300 import inputs

pytestmark = pytest.mark.gpu

N, RE, SLICES = 64, 1000.0, 32
FINE, COARSE, DT = 2, 1, 5e-4
KMAX = 2
RTOL = 1e-13


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def start_state():
    """The workload's start state, computed by the oracle (FP64)."""
    o16 = oracle.Grid(16, 16, 16, re=100.0)
    s16 = o16.zeros()
    o16.step(s16, 1e-3, 200)
    up = inputs.upsample_cavity(s16, 16, N, u_lid=1.0)
    st = inputs.add_face_noise(up, 1e-3, seed=0)
    o64 = oracle.Grid(N, N, N, re=RE, rtol=RTOL)
    u, v, w, _ = o64.project(*st[:3])
    return [u, v, w, np.zeros_like(st[3])]


@pytest.fixture(scope="module")
def headline_oracle():
    u0 = start_state()
    og = oracle.Grid(N, N, N, re=RE, rtol=RTOL)
    F = opr.fine_propagator(og, DT, FINE)
    G = opr.coarse_propagator(og, DT * FINE / COARSE, COARSE)

    def F_batch(states):
        return og.run_batch(states, DT, FINE)

    y, defects = opr.parareal(u0, SLICES, F, G, kmax=KMAX, F_batch=F_batch)
    return u0, y, defects


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_headline_parareal_64cubed_32_slices_matches_oracle(headline_oracle, prec):
    u0_np, y_ref, d_ref = headline_oracle
    g = Grid(N, N, N, re=RE, u_lid=1.0, precision=prec, batch=SLICES, poisson_rtol=RTOL,
             refine_rtol=1e-10)
    u0 = g.state_from([a[None] for a in u0_np])
    slices = g.zeros(SLICES + 1)
    k, defects = g.parareal(u0, slices, SLICES, FINE, COARSE, DT, kmax=KMAX)
    assert k == KMAX
    got = slices.numpy()
    worst = {c: 0.0 for c in "uvwp"}
    worst_vel = 0.0
    for n in range(SLICES + 1):
        g_n = [np.asarray(got[c][n], dtype=np.float64) for c in range(4)]
        w_n = y_ref[n]
        errs = [rel(g_n[c], w_n[c]) for c in range(4)]
        vel = rel(np.concatenate([g_n[c].ravel() for c in range(3)]),
                  np.concatenate([w_n[c].ravel() for c in range(3)]))
        for c, e in zip("uvwp", errs):
            worst[c] = max(worst[c], e)
        worst_vel = max(worst_vel, vel)
        if prec == "fp64":
            for c, e in zip("uvwp", errs):
                assert e <= 1e-10, f"slice {n} field {c}: relative L2 {e:.3e}"
        else:
            assert vel <= 1e-5, f"slice {n} velocity: relative L2 {vel:.3e}"
            assert errs[3] <= 1e-5, f"slice {n} pressure: relative L2 {errs[3]:.3e}"
    print(f"\nheadline Parareal {prec}: worst relative L2 over {SLICES + 1} slices: "
          + ", ".join(f"{c} {worst[c]:.2e}" for c in "uvwp")
          + f", velocity field {worst_vel:.2e}; defects {defects} vs oracle {d_ref}")
    # the defects are max-norm differences of stored values (FP32 storage adds
    # the rounding of O(1) fields)
    rtol_d, dabs = (1e-6, 1e-12) if prec == "fp64" else (1e-3, 5e-7)
    for a, b in zip(defects, d_ref):
        assert abs(a - b) <= rtol_d * b + dabs, (a, b)
    g.close()
