"""CUDA graphs of fine steps with device-resident solver loops.

A graph launch must reproduce the stream path bit for bit (the same kernels
in the same order, the loops ended by the same device decisions), for
several grids of different shapes and Reynolds numbers captured as
concurrent branches, and report solver failures after the fact.
"""
import numpy as np
import pytest

import oracle
from paper_1705_06149_gb300 import Grid, NSError, StepGraph, inputs
from paper_1705_06149_gb300 import _native as N

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-10, "fp32_refine": 1e-5}

# (dims, bc, Re, batch): one cubic wall cavity, one anisotropic periodic box,
# one with solid boxes
CASES = [((16, 16, 16), ("wall",) * 3, 1000.0, 2),
         ((24, 16, 8), ("periodic", "wall", "wall"), 300.0, 1),
         ((20, 18, 16), ("wall",) * 3, 500.0, 1)]


def make(prec, k, solid=None):
    dims, bc, re, batch = CASES[k]
    g = Grid(*dims, re=re, bc=bc, precision=prec, batch=batch, solid=solid)
    inits = [inputs.random_state(*dims, seed=70 + 10 * k + s, sigma=0.2, bc=bc, solid=solid)
             for s in range(batch)]
    return g, inits


def stack(g, inits):
    return g.state_from([np.stack([i[c] for i in inits]) for c in range(4)])


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_graph_reproduces_the_stream_path_bit_for_bit(prec):
    _, solid = inputs.obstacle_boxes(CASES[2][0], seed=1, count=2, edge=(0.15, 0.3))
    branches, refs = [], []
    dts, nsteps = [1e-3, 2e-3, 1e-3], [3, 2, 4]
    for k in range(3):
        g, inits = make(prec, k, solid if k == 2 else None)
        a = stack(g, inits)
        b = stack(g, inits)
        branches.append((g, a, dts[k], nsteps[k]))
        refs.append((g, b, inits))
    graph = StepGraph(branches)
    for _ in range(2):
        graph.launch()
    graph.check()
    for k, (g, b, inits) in enumerate(refs):
        g.step_fine(b, dts[k], nsteps[k])
        g.step_fine(b, dts[k], nsteps[k])
        for c in range(4):
            assert torch.equal(branches[k][1].fields()[c], b.fields()[c]), (k, c)
    graph.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_graph_counts_steps_solves_and_iterations(prec):
    g, inits = make(prec, 0)
    a, b = stack(g, inits), stack(g, inits)
    graph = StepGraph([(g, a, 1e-3, 3)])
    g.reset_stats()
    graph.launch()
    graph.check()
    s_graph = g.stats()
    g.reset_stats()
    g.step_fine(b, 1e-3, 3)
    s_host = g.stats()
    for key in ("steps", "solves", "krylov_iters", "refine_steps"):
        assert s_graph[key] == s_host[key], (key, s_graph, s_host)
    assert s_graph["launches"] > 0
    graph.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_graph_matches_the_oracle(prec):
    dims, bc, re, _ = CASES[1]
    init = inputs.random_state(*dims, seed=5, sigma=0.2, bc=bc)
    og = oracle.Grid(*dims, re=re, bc=bc, rtol=1e-13)
    want = oracle.copy_state(init)
    og.step(want, 2e-3, 5)
    g = Grid(*dims, re=re, bc=bc, precision=prec, batch=1, poisson_rtol=1e-13)
    st = g.state_from(init)
    graph = StepGraph([(g, st, 2e-3, 5)])
    graph.launch()
    graph.check()
    got = [a[0] for a in st.numpy()]
    vg = np.concatenate([np.ravel(got[c]) for c in range(3)])
    vw = np.concatenate([np.ravel(want[c]) for c in range(3)])
    assert np.linalg.norm(vg - vw) <= TOL[prec] * np.linalg.norm(vw)
    assert np.linalg.norm(got[3] - want[3]) <= TOL[prec] * np.linalg.norm(want[3])
    graph.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_graph_matches_the_oracle_above_the_one_cta_levels(prec):
    """A 32^3 cavity and a 40 x 32 x 24 one (periodic z), two states each, so
    that the finest level (32768 / 30720 cells, far above the 4096-cell one-CTA
    levels) runs in the graph's grid-level kernels: restriction, smoothing,
    prolongation, the BiCGStab phases and the refinement, in the conditional
    while loops."""
    for dims, bc in (((32, 32, 32), ("wall",) * 3), ((40, 32, 24), ("wall", "wall", "periodic"))):
        inits = [inputs.random_state(*dims, seed=40 + s, sigma=0.2, bc=bc) for s in range(2)]
        og = oracle.Grid(*dims, re=400.0, bc=bc, rtol=1e-13)
        wants = []
        for init in inits:
            want = oracle.copy_state(init)
            og.step(want, 1e-3, 4)
            wants.append(want)
        g = Grid(*dims, re=400.0, bc=bc, precision=prec, batch=2, poisson_rtol=1e-13)
        st = g.state_from([np.stack([i[c] for i in inits]) for c in range(4)])
        graph = StepGraph([(g, st, 1e-3, 4)])
        graph.launch()
        graph.check()
        got = st.numpy()
        for s, want in enumerate(wants):
            vg = np.concatenate([np.ravel(got[c][s]) for c in range(3)])
            vw = np.concatenate([np.ravel(want[c]) for c in range(3)])
            ev = np.linalg.norm(vg - vw) / np.linalg.norm(vw)
            ep = np.linalg.norm(got[3][s] - want[3]) / np.linalg.norm(want[3])
            assert ev <= TOL[prec] and ep <= TOL[prec], (dims, s, ev, ep)
        graph.close()
        g.close()


def test_graph_reports_a_solve_that_hits_its_iteration_limit():
    dims = (16, 16, 16)
    g = Grid(*dims, re=100.0, batch=1, poisson_rtol=1e-30, poisson_maxit=3)
    st = g.state_from(inputs.random_state(*dims, seed=9, sigma=0.2))
    graph = StepGraph([(g, st, 1e-3, 2)])
    graph.launch()
    with pytest.raises(NSError) as e:
        graph.check()
    assert e.value.status == N.NS_ERR_NOT_CONVERGED
    # the failure flags are cleared by the check; the graph stays usable
    graph.launch()
    with pytest.raises(NSError):
        graph.check()
    graph.close()


def test_graph_rejects_bad_branches():
    g = Grid(16, 16, 16, batch=1)
    st = g.zeros(1)
    with pytest.raises(NSError) as e:
        StepGraph([(g, st, 1e-3, 1), (g, g.zeros(1), 1e-3, 1)])
    assert e.value.status == N.NS_ERR_ARG
    gp = Grid(16, 16, 16, batch=1, preconditioner="none")
    with pytest.raises(NSError) as e:
        StepGraph([(gp, gp.zeros(1), 1e-3, 1)])
    assert e.value.status == N.NS_ERR_ARG
    with pytest.raises(NSError):
        StepGraph([(g, st, -1.0, 1)])


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_step_fine_many_reproduces_the_stream_path(prec):
    """Several grids of different shapes and Reynolds numbers advanced at once
    (a stream and host thread per grid) give what each grid's own calls give."""
    from paper_1705_06149_gb300 import step_fine_many
    _, solid = inputs.obstacle_boxes(CASES[2][0], seed=1, count=2, edge=(0.15, 0.3))
    branches, refs = [], []
    dts, nsteps = [1e-3, 2e-3, 1e-3], [3, 2, 4]
    for k in range(3):
        g, inits = make(prec, k, solid if k == 2 else None)
        branches.append((g, stack(g, inits), dts[k], nsteps[k]))
        refs.append(stack(g, inits))
    step_fine_many(branches)
    step_fine_many(branches)
    for k, (g, a, dt, n) in enumerate(branches):
        g.step_fine(refs[k], dt, n)
        g.step_fine(refs[k], dt, n)
        for c in range(4):
            assert torch.equal(a.fields()[c], refs[k].fields()[c]), (k, c)


def test_step_fine_many_reports_the_failing_grid():
    from paper_1705_06149_gb300 import step_fine_many
    good = Grid(16, 16, 16, batch=1)
    bad = Grid(16, 16, 16, batch=1, poisson_rtol=1e-30, poisson_maxit=3)
    init = inputs.random_state(16, 16, 16, seed=9, sigma=0.2)
    with pytest.raises(NSError) as e:
        step_fine_many([(good, good.state_from(init), 1e-3, 2),
                        (bad, bad.state_from(init), 1e-3, 2)])
    assert e.value.status == N.NS_ERR_NOT_CONVERGED
    assert "grid 1" in str(e.value)
    with pytest.raises(NSError) as e:
        step_fine_many([(good, good.zeros(1), 1e-3, 1), (good, good.zeros(1), 1e-3, 1)])
    assert e.value.status == N.NS_ERR_ARG


def test_mixed_batch_full_size():
    """The mixed batch at full size (16 states of a 256^3 cavity and 24 cavities
    with sizes from {32, 48, 64, 96}^3 and Re ~ U[100, 2000], seed 0, tiles from
    the autotuner's seed ranking, FP32 + FP64 refinement), two fine steps from
    rest: ns_step_fine_many and one CUDA graph with a branch per grid both give
    grid-by-grid stepping bit for bit; the 16 states of the big grid stay
    identical; the big grid's velocity is divergence-free at the FP32 level."""
    from paper_1705_06149_gb300 import step_fine_many
    from paper_1705_06149_gb300.autotune import seed_order
    dt, steps = 5e-4, 2
    dims, res = inputs.mixed_batch_sizes(24, seed=0)
    specs = [((256, 256, 256), 1000.0, 16)] + [(d, r, 1) for d, r in zip(dims, res)]
    grids = [Grid(*d, re=r, precision="fp32_refine", batch=b, tile_z=seed_order(*d, b)[0][0])
             for d, r, b in specs]
    runs = []
    for how in ("grid by grid", "many", "graph"):
        states = [g.zeros(g_b) for g, (_, _, g_b) in zip(grids, specs)]
        branches = [(g, s, dt, steps) for g, s in zip(grids, states)]
        if how == "grid by grid":
            for g, s in zip(grids, states):
                g.step_fine(s, dt, steps)
        elif how == "many":
            step_fine_many(branches)
        else:
            graph = StepGraph(branches)
            graph.launch()
            graph.check()
            graph.close()
        torch.cuda.synchronize()
        runs.append(states)
    for how, states in zip(("many", "graph"), runs[1:]):
        for k, (a, b) in enumerate(zip(runs[0], states)):
            for c, (ta, tb) in enumerate(zip(a.fields(), b.fields())):
                assert torch.equal(ta, tb), (how, k, c)
    big = runs[0][0]
    for t in big.fields():
        assert torch.equal(t, t[:1].expand_as(t))
    u, v, w = [t[0].double() for t in big.fields()[:3]]
    div = (u[:, :, 1:] - u[:, :, :-1] + v[:, 1:, :] - v[:, :-1, :] + w[1:, :, :] - w[:-1, :, :]) * 256
    assert float(div.abs().max()) <= 1e-3, float(div.abs().max())
    assert float(u.abs().max()) > 0.1  # the lid drives the flow
    for g in grids:
        g.close()
