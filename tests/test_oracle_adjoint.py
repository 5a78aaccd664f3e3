"""Pins of the oracle's discrete adjoint (no GPU): transpose identities of
each linearised piece and central finite differences of the full objective.

The forward map of one step is u+ = P(u + dt R(u; u_lid)); the SMART fluxes
are piecewise linear in the node values, so central differences with a small
step agree with the adjoint to roundoff unless a branch switch falls inside
the step.
"""
import numpy as np
import pytest

import oracle
from paper_1705_06149_gb300 import inputs


def active_mask(g, c):
    m = np.ones(g.shape(c))
    if g.bc[c] != "periodic":
        ax = 2 - c
        sl0 = [slice(None)] * 3
        sl1 = [slice(None)] * 3
        sl0[ax] = 0
        sl1[ax] = -1
        m[tuple(sl0)] = 0
        m[tuple(sl1)] = 0
    return m


def rhs(g, st):
    conv, diff = g.rhs_terms(*st[:3])
    inv_re = 1.0 / g.re if g.re > 0 else 0.0
    return [inv_re * diff[c] - conv[c] for c in range(3)]


@pytest.mark.parametrize("bc", [("wall",) * 3, ("periodic", "wall", "slip"), ("periodic",) * 3])
def test_rhs_adjoint_is_the_transpose_of_the_linearised_rhs(bc):
    dims = (9, 8, 7)
    rng = np.random.default_rng(7)
    g = oracle.Grid(*dims, re=50.0, u_lid=0.7, bc=bc)
    st = inputs.random_state(*dims, seed=8, sigma=0.5, bc=bc)
    mu = [rng.normal(size=g.shape(c)) * active_mask(g, c) for c in range(3)]
    adj, dlid = g.rhs_adjoint(*st[:3], mu)
    eps = 1e-7
    for trial in range(3):
        d = [rng.normal(size=g.shape(c)) * active_mask(g, c) for c in range(3)]
        plus = [st[c] + eps * d[c] for c in range(3)]
        minus = [st[c] - eps * d[c] for c in range(3)]
        rp, rm = rhs(g, plus), rhs(g, minus)
        lhs = sum(np.sum(mu[c] * (rp[c] - rm[c])) for c in range(3)) / (2 * eps)
        rhs_ = sum(np.sum(d[c] * adj[c]) for c in range(3))
        assert abs(lhs - rhs_) <= 1e-6 * abs(rhs_) + 1e-6, (trial, lhs, rhs_)
    if bc[1] == "wall":
        gp = oracle.Grid(*dims, re=50.0, u_lid=0.7 + eps, bc=bc)
        gm = oracle.Grid(*dims, re=50.0, u_lid=0.7 - eps, bc=bc)
        rp, rm = rhs(gp, st), rhs(gm, st)
        lhs = sum(np.sum(mu[c] * (rp[c] - rm[c])) for c in range(3)) / (2 * eps)
        assert abs(lhs - dlid) <= 1e-6 * abs(dlid) + 1e-6, (lhs, dlid)
        assert abs(dlid) > 1e-3


def test_projection_is_symmetric():
    dims = (8, 9, 7)
    g = oracle.Grid(*dims)
    x = inputs.random_state(*dims, seed=1)
    y = inputs.random_state(*dims, seed=2)
    px = g.project(*x[:3], rtol=1e-14)
    py = g.project(*y[:3], rtol=1e-14)
    a = sum(np.sum(px[c] * y[c]) for c in range(3))
    b = sum(np.sum(x[c] * py[c]) for c in range(3))
    assert abs(a - b) <= 1e-11 * (abs(a) + abs(b))


@pytest.mark.parametrize("start", ["rest", "moving"])
def test_gradient_matches_central_differences(start):
    dims = (8, 8, 8)
    dt, steps = 2e-3, 6
    g = oracle.Grid(*dims, re=40.0, u_lid=1.0, rtol=1e-14)
    if start == "rest":
        st0 = g.zeros()
    else:
        rs = inputs.random_state(*dims, seed=12, sigma=0.3)
        u, v, w, _ = g.project(*rs[:3], rtol=1e-14)
        st0 = [u, v, w, np.zeros(g.shape(3))]
    J, grads, dlid = g.adjoint(st0, dt, steps, rtol=1e-14)

    def objective(state, lid=1.0):
        gg = oracle.Grid(*dims, re=40.0, u_lid=lid, rtol=1e-14)
        s = oracle.copy_state(state)
        gg.step(s, dt, steps)
        return gg.kinetic_objective(s)

    assert abs(objective(st0) - J) <= 1e-14 * abs(J) + 1e-300
    rng = np.random.default_rng(5)
    h = 1e-6
    for trial in range(4):
        d = [rng.normal(size=g.shape(c)) * active_mask(g, c) for c in range(3)]
        nrm = np.sqrt(sum(np.sum(x * x) for x in d))
        d = [x / nrm for x in d]
        plus = [st0[c] + h * d[c] for c in range(3)] + [st0[3]]
        minus = [st0[c] - h * d[c] for c in range(3)] + [st0[3]]
        fd = (objective(plus) - objective(minus)) / (2 * h)
        ad = sum(np.sum(grads[c] * d[c]) for c in range(3))
        assert abs(fd - ad) <= 1e-4 * abs(ad) + 1e-12, (trial, fd, ad)
    fd = (objective(st0, 1.0 + h) - objective(st0, 1.0 - h)) / (2 * h)
    assert abs(fd - dlid) <= 1e-4 * abs(dlid), (fd, dlid)
    for c in range(3):
        assert np.all(grads[c][active_mask(g, c) == 0] == 0.0)
