"""Parareal on the quasi-2D driven cavity of the paper's first simulation
(Section 3, Table 1): [0,1] x [0,1] x [0,0.1], 32 x 32 x 5 cells, periodic in
z, Re = 1000, lid speed 1, fine step 0.001, coarse step 0.01.

The horizon is shortened to 8 slices of 50 fine steps (t = 0.4) so that the
oracle's Parareal finishes in seconds; the checks are the ones the paper's
Fig. 3 study makes: the maximum difference to the time-serial solution falls
with every iteration, and K = N gives the serial solution.
"""
import numpy as np
import pytest

import oracle
from oracle import parareal as opr
from paper_1705_06149_gb300 import Grid

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DIMS = (32, 32, 5)
BOX = (1.0, 1.0, 0.1)
BC = ("wall", "wall", "periodic")
RE = 1000.0
N_SLICES, FINE, COARSE = 8, 50, 5
DT_FINE = 1e-3
DT_COARSE = DT_FINE * FINE / COARSE  # 0.01, the paper's coarse step
TOL = {"fp64": 1e-10, "fp32_refine": 1e-5}


def rel(a, b):
    n = np.linalg.norm(np.ravel(b))
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / (n if n > 0 else 1.0)


@pytest.fixture(scope="module")
def sim1_oracle():
    og = oracle.Grid(*DIMS, *BOX, re=RE, u_lid=1.0, bc=BC)
    u0 = og.zeros()
    F = opr.fine_propagator(og, DT_FINE, FINE)
    G = opr.coarse_propagator(og, DT_COARSE, COARSE)
    y, defects = opr.parareal(u0, N_SLICES, F, G, kmax=2,
                              F_batch=lambda ys: og.run_batch(ys, DT_FINE, FINE))
    return y, defects


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_sim1_parareal_matches_oracle(sim1_oracle, prec):
    y_ref, d_ref = sim1_oracle
    g = Grid(*DIMS, *BOX, re=RE, bc=BC, precision=prec, batch=N_SLICES)
    u0 = g.zeros(1)
    slices = g.zeros(N_SLICES + 1)
    k, defects = g.parareal(u0, slices, N_SLICES, FINE, COARSE, DT_FINE, kmax=2)
    assert k == 2
    got = slices.numpy()
    for n in range(N_SLICES + 1):
        vg = np.concatenate([np.ravel(got[c][n]) for c in range(3)])
        vw = np.concatenate([np.ravel(y_ref[n][c]) for c in range(3)])
        assert rel(vg, vw) <= TOL[prec], (n, rel(vg, vw))
        assert rel(got[3][n], y_ref[n][3]) <= TOL[prec], (n, rel(got[3][n], y_ref[n][3]))
    dabs = 0.0 if prec == "fp64" else 5e-7
    for a, b in zip(defects, d_ref):
        assert abs(a - b) <= 1e-3 * b + dabs


def test_sim1_error_to_serial_falls_with_iterations():
    g = Grid(*DIMS, *BOX, re=RE, bc=BC, batch=N_SLICES)
    # one call per slice, as Parareal's fine propagator makes them (each call
    # starts its pressure solves from p, later steps from the extrapolation)
    serial = g.zeros(1)
    for _ in range(N_SLICES):
        g.step_fine(serial, DT_FINE, FINE)
    ref = [f[0] for f in serial.fields()]
    errs = []
    for k in range(0, N_SLICES + 1):
        slices = g.zeros(N_SLICES + 1)
        g.parareal(g.zeros(1), slices, N_SLICES, FINE, COARSE, DT_FINE, kmax=k)
        end = [f[N_SLICES] for f in slices.fields()]
        errs.append(max(float((a - b).abs().max()) for a, b in zip(end, ref)))
    # the coarse sweep alone is far off; every iteration reduces the error
    # (by 40-80x here) until it reaches the level of the pressure solves'
    # stopping tolerance, and K = N is the serial solution exactly
    assert errs[0] > 1e-3
    for k in range(1, N_SLICES):
        if errs[k - 1] > 1e-11:
            assert errs[k] < errs[k - 1] / 10, errs
        else:
            assert errs[k] <= 1e-11, errs
    assert errs[N_SLICES] == 0.0, errs
