"""CUDA path with solid cells (obstacles) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from oracle import parareal as opr
from paper_1705_06149_gb300 import Grid, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32_refine": 1e-5}


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def close(got, want, tol, what):
    vg = np.concatenate([np.ravel(got[c]) for c in range(3)])
    vw = np.concatenate([np.ravel(want[c]) for c in range(3)])
    assert rel(vg, vw) <= tol, (what, "velocity", rel(vg, vw))
    assert rel(got[3], want[3]) <= tol, (what, "pressure", rel(got[3], want[3]))


def masked_case(dims, seed, count=3, edge=(0.15, 0.3)):
    _, solid = inputs.obstacle_boxes(dims, seed=seed, count=count, edge=edge)
    return solid


@pytest.mark.parametrize("dims,bc", [((16, 16, 16), ("wall",) * 3),
                                     ((20, 14, 12), ("periodic", "wall", "wall"))])
@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_predictor_with_solids_matches_oracle(dims, bc, prec):
    solid = masked_case(dims, seed=5)
    rs = inputs.random_state(*dims, seed=6, sigma=1.0, bc=bc, solid=solid)
    og = oracle.Grid(*dims, re=50.0, u_lid=1.0, bc=bc, solid=solid)
    want = og.predict(*rs[:3], 2e-3)
    g = Grid(*dims, re=50.0, u_lid=1.0, bc=bc, precision=prec, solid=solid, batch=1)
    got = [t[0].cpu().numpy() for t in g.predict(g.state_from(rs), 2e-3)]
    tol = 1e-13 if prec == "fp64" else 2e-6
    for c in range(3):
        err = np.max(np.abs(got[c] - want[c])) / np.max(np.abs(want[c]))
        assert err <= tol, (c, err)


@pytest.mark.parametrize("pc", ["multigrid", "none"])
@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_steps_with_solids_match_oracle(prec, pc):
    dims = (20, 18, 16)
    solid = masked_case(dims, seed=7)
    og = oracle.Grid(*dims, re=100.0, solid=solid, rtol=1e-13)
    B = 2
    inits = [inputs.random_state(*dims, seed=30 + s, sigma=0.2, solid=solid) for s in range(B)]
    g = Grid(*dims, re=100.0, precision=prec, solid=solid, batch=B, preconditioner=pc,
             poisson_rtol=1e-13)
    st = g.state_from([np.stack([i[c] for i in inits]) for c in range(4)])
    g.step_fine(st, 1e-3, 4)
    got = st.numpy()
    for s in range(B):
        want = oracle.copy_state(inits[s])
        og.step(want, 1e-3, 4)
        close([got[c][s] for c in range(4)], want, TOL[prec], f"slice {s}")
        assert np.all(got[3][s][solid.astype(bool)] == 0.0)


def test_parareal_with_solids_and_a_defect_tolerance():
    dims = (16, 16, 16)
    solid = masked_case(dims, seed=3, count=2)
    og = oracle.Grid(*dims, re=100.0, solid=solid)
    F = opr.fine_propagator(og, 1e-3, 10)
    G = opr.coarse_propagator(og, 5e-3, 2)
    u0 = og.zeros()
    y_ref, d_ref = opr.parareal(u0, 4, F, G, kmax=4)
    g = Grid(*dims, re=100.0, solid=solid, batch=4)
    slices = g.zeros(5)
    k, defects = g.parareal(g.zeros(1), slices, 4, 10, 2, 1e-3, kmax=4)
    got = slices.numpy()
    for n in range(5):
        close([a[n] for a in got], y_ref[n], 1e-10, f"slice {n}")
    for a, b in zip(defects, d_ref):
        # late defects sit at the pressure solves' tolerance (~1e-10): their
        # agreement is absolute, not relative
        assert abs(a - b) <= 1e-3 * b + 1e-11
    # a tolerance between the second and third defects stops after three
    tol = 0.5 * (d_ref[1] + d_ref[2])
    k2, d2 = g.parareal(g.zeros(1), g.zeros(5), 4, 10, 2, 1e-3, kmax=4, tol=tol)
    assert k2 == 3


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_multigrid_with_solids_keeps_the_iteration_count_low(prec):
    """The V-cycle with solid cells on its finest level still preconditions:
    a few iterations per solve on the 32^3 cavity with 8 boxes, where plain
    BiCGStab needs tens; both give the oracle's steps."""
    dims = (32, 32, 32)
    _, solid = inputs.obstacle_boxes(dims, seed=0, count=8)
    init = inputs.random_state(*dims, seed=40, sigma=0.2, solid=solid)
    og = oracle.Grid(*dims, re=1000.0, solid=solid, rtol=1e-13)
    want = oracle.copy_state(init)
    og.step(want, 5e-4, 3)
    iters = {}
    for pc in ("multigrid", "none"):
        g = Grid(*dims, re=1000.0, precision=prec, solid=solid, batch=1, preconditioner=pc,
                 poisson_rtol=1e-13)
        st = g.state_from(init)
        g.step_fine(st, 5e-4, 3)
        close([a[0] for a in st.numpy()], want, TOL[prec], pc)
        s = g.stats()
        iters[pc] = s["krylov_iters"] / s["solves"]
    assert iters["multigrid"] <= 25, iters
    assert iters["none"] >= 3 * iters["multigrid"], iters


def test_obstacle_workload_full_size():
    """The 128^3 cavity with the 8 seeded boxes of the obstacle workload, at its
    full batch of 64 slices in FP32 + FP64 refinement, one fine step of a seeded
    state given to every slice: the masked predictor matches the oracle's at full
    size; every slice ends bit for bit equal to the first (no slice depends on
    its place in the batch); every inactive face (a wall face or a face touching
    a solid cell) holds exactly 0; the divergence is at the FP32 level."""
    n, B, dt = 128, 64, 5e-4
    _, solid = inputs.obstacle_boxes((n, n, n), seed=0, count=8)
    init = inputs.random_state(n, n, n, seed=300, sigma=0.05, solid=solid)
    g = Grid(n, n, n, re=1000.0, precision="fp32_refine", batch=B, solid=solid)
    one = g.state_from(init)
    og = oracle.Grid(n, n, n, re=1000.0, solid=solid)
    want = og.predict(*init[:3], dt)
    got = [t[0].cpu().numpy() for t in g.predict(one, dt)]
    for c in range(3):
        err = np.max(np.abs(got[c] - want[c])) / np.max(np.abs(want[c]))
        assert err <= 2e-6, (c, err)
    st = type(one)(*[t.expand((B,) + tuple(t.shape[1:])).contiguous() for t in one.fields()])
    g.project(st)
    g.step_fine(st, dt, 1)
    torch.cuda.synchronize()
    for t in st.fields():
        assert torch.equal(t, t[:1].expand_as(t)), "slices differ"
    u, v, w, _ = [a[0].astype(np.float64) for a in st.slice(0).numpy()]
    fluid = solid == 0
    # inactive faces of each component (both neighbours along its axis must be fluid)
    act_u = np.zeros((n, n, n + 1), bool)
    act_u[:, :, 1:n] = fluid[:, :, :-1] & fluid[:, :, 1:]
    act_v = np.zeros((n, n + 1, n), bool)
    act_v[:, 1:n, :] = fluid[:, :-1, :] & fluid[:, 1:, :]
    act_w = np.zeros((n + 1, n, n), bool)
    act_w[1:n, :, :] = fluid[:-1, :, :] & fluid[1:, :, :]
    for a, act in ((u, act_u), (v, act_v), (w, act_w)):
        assert np.all(a[~act] == 0.0)
    div = (u[:, :, 1:] - u[:, :, :-1] + v[:, 1:, :] - v[:, :-1, :] + w[1:, :, :] - w[:-1, :, :]) * n
    assert np.max(np.abs(div[fluid])) <= 1e-3, np.max(np.abs(div[fluid]))
    assert np.max(np.abs(u)) > 0.1  # the lid and the seeded state move the fluid
    g.close()
