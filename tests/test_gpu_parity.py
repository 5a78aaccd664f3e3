"""CUDA path (through the C ABI) against the FP64 CPU oracle, element by element.

Tolerances (the targets of the method's two precision modes): relative L2 of
the velocity field (u, v, w taken together) and of the pressure <= 1e-10 in
FP64, where each component is also held to 1e-10 on its own, and <= 1e-5 with
FP32 storage and FP64 refinement.  Stage tests (predictor) use a max-norm
bound relative to the field's maximum.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import parareal as opr
from paper_1705_06149_gb300 import Grid, NSError
from paper_1705_06149_gb300 import _native as N
from paper_1705_06149_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32_refine": 1e-5}


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def assert_state_close(got, want, tol, what=""):
    vel_got = np.concatenate([np.ravel(got[c]) for c in range(3)])
    vel_want = np.concatenate([np.ravel(want[c]) for c in range(3)])
    e = rel(vel_got, vel_want)
    assert e <= tol, f"{what} velocity: relative L2 {e:.3e} > {tol:.1e}"
    e = rel(got[3], want[3])
    assert e <= tol, f"{what} pressure: relative L2 {e:.3e} > {tol:.1e}"
    if tol <= 1e-10:
        for c in range(3):
            e = rel(got[c], want[c])
            assert e <= tol, f"{what} field {'uvw'[c]}: relative L2 {e:.3e} > {tol:.1e}"


def np_divergence(st, h):
    u, v, w = st[:3]
    return (np.diff(u, axis=-1) / h[0] + np.diff(v, axis=-2) / h[1] + np.diff(w, axis=-3) / h[2])


# ---------------------------------------------------------------------------
# stages
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims,bc", [((16, 16, 16), ("wall",) * 3),
                                     ((19, 13, 11), ("wall",) * 3),
                                     ((37, 9, 10), ("periodic", "wall", "slip")),
                                     ((8, 10, 6), ("periodic",) * 3),
                                     ((2, 2, 2), ("wall",) * 3)])
@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_predictor_matches_oracle(dims, bc, prec):
    rs = inputs.random_state(*dims, seed=3, sigma=1.0, bc=bc)
    og = oracle.Grid(*dims, 1.0, 1.3, 0.8, re=50.0, u_lid=1.0, bc=bc)
    want = og.predict(*rs[:3], 2e-3)
    g = Grid(*dims, 1.0, 1.3, 0.8, re=50.0, u_lid=1.0, bc=bc, precision=prec, batch=2)
    st = g.state_from([np.stack([a, a]) for a in rs])
    got = [t.cpu().numpy() for t in g.predict(st, 2e-3)]
    tol = 1e-13 if prec == "fp64" else 2e-6
    for c in range(3):
        scale = max(np.max(np.abs(want[c])), 1e-30)
        for b in range(2):
            err = np.max(np.abs(got[c][b] - want[c])) / scale
            assert err <= tol, (c, b, err)


PCS = ["multigrid", "none"]


@pytest.mark.parametrize("pc", PCS)
@pytest.mark.parametrize("dims", [(24, 20, 18), (32, 16, 8), (19, 13, 11), (64, 64, 64)])
@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_poisson_solve_matches_oracle(prec, dims, pc):
    rng = np.random.default_rng(4)
    og = oracle.Grid(*dims, rtol=1e-13)
    B = 3
    b = rng.normal(size=(B,) + og.shape(3))
    g = Grid(*dims, precision=prec, poisson_rtol=1e-13, refine_rtol=1e-13, batch=B,
             preconditioner=pc)
    bt = torch.tensor(b, device="cuda")
    pt = torch.zeros_like(bt)
    g.poisson_solve(bt, pt)
    got = pt.cpu().numpy()
    for s in range(B):
        want, _ = og.poisson(b[s], rtol=1e-13)
        assert rel(got[s], want) <= 1e-10, (s, rel(got[s], want))
        assert abs(got[s].mean()) <= 1e-12 * np.abs(got[s]).max()


# ---------------------------------------------------------------------------
# one and several fine steps
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims,bc", [((12, 12, 12), ("wall",) * 3),
                                     ((19, 13, 11), ("wall",) * 3),
                                     ((16, 12, 6), ("periodic", "wall", "slip")),
                                     ((40, 24, 8), ("wall", "periodic", "wall")),
                                     ((2, 2, 2), ("wall",) * 3)])
@pytest.mark.parametrize("pc", PCS)
@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_fine_steps_match_oracle(dims, bc, prec, pc):
    steps, dt = 4, 1e-3
    B = 3
    inits = [inputs.random_state(*dims, seed=20 + s, sigma=0.2, bc=bc) for s in range(B)]
    # The pressure error of a solve stopped at relative residual rtol is
    # bounded by cond(L) * rtol (a few hundred on these grids), so both sides
    # solve to 1e-13 for a 1e-10 pressure comparison.  On 2x2x2, cond(L) is 3
    # and the residual's rounding floor (|p| >> |b| h^2) lies above 1e-13.
    rtol = 1e-12 if min(dims) <= 2 else 1e-13
    og = oracle.Grid(*dims, re=100.0, bc=bc, rtol=rtol)
    g = Grid(*dims, re=100.0, bc=bc, precision=prec, batch=B, preconditioner=pc,
             poisson_rtol=rtol)
    st = g.state_from([np.stack([i[c] for i in inits]) for c in range(4)])
    g.step_fine(st, dt, steps)
    got = st.numpy()
    for s in range(B):
        want = oracle.copy_state(inits[s])
        og.step(want, dt, steps)
        assert_state_close([got[c][s] for c in range(4)], want, TOL[prec], f"slice {s}")


def test_taylor_green_matches_oracle():
    n = 16
    L = 2 * np.pi
    bc = ("periodic",) * 3
    og = oracle.Grid(n, n, 4, L, L, L / 4, re=10.0, bc=bc)
    st0 = og.zeros()
    x_f = np.arange(n) * L / n
    x_c = (np.arange(n) + 0.5) * L / n
    st0[0][:] = np.sin(x_f)[None, None, :] * np.cos(x_c)[None, :, None]
    st0[1][:] = -np.cos(x_c)[None, None, :] * np.sin(x_f)[None, :, None]
    want = oracle.copy_state(st0)
    og.step(want, 5e-3, 20)
    g = Grid(n, n, 4, L, L, L / 4, re=10.0, bc=bc, batch=1)
    st = g.state_from(st0)
    g.step_fine(st, 5e-3, 20)
    assert_state_close([a[0] for a in st.numpy()], want, 1e-10, "taylor-green")


# ---------------------------------------------------------------------------
# the 16^3 lid-driven cavity: serial fine run and Parareal
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cavity16_oracle():
    og = oracle.Grid(16, 16, 16, re=100.0, u_lid=1.0)
    u0 = og.zeros()
    F = opr.fine_propagator(og, 1e-3, 50)
    G = opr.coarse_propagator(og, 1e-2, 5)
    serial = opr.serial_fine(u0, 4, F)
    y, defects = opr.parareal(u0, 4, F, G, kmax=4)
    return serial, y, defects


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_cavity16_serial_200_steps(cavity16_oracle, prec):
    serial, _, _ = cavity16_oracle
    g = Grid(16, 16, 16, re=100.0, precision=prec, batch=1)
    st = g.zeros(1)
    g.step_fine(st, 1e-3, 200)
    got = [a[0] for a in st.numpy()]
    assert_state_close(got, serial[4], TOL[prec], "t=0.2")
    div = np_divergence(got, (1 / 16,) * 3)
    assert np.max(np.abs(div)) <= (1e-12 if prec == "fp64" else 1e-4)


@pytest.mark.parametrize("pc", PCS)
@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_cavity16_parareal(cavity16_oracle, prec, pc):
    _, y_ref, d_ref = cavity16_oracle
    g = Grid(16, 16, 16, re=100.0, precision=prec, batch=4, preconditioner=pc)
    u0 = g.zeros(1)
    slices = g.zeros(5)
    k, defects = g.parareal(u0, slices, 4, 50, 5, 1e-3, kmax=4)
    assert k == 4
    got = slices.numpy()
    for n in range(5):
        assert_state_close([a[n] for a in got], y_ref[n], TOL[prec], f"slice {n}")
    # defects are differences of stored values: in FP32 storage they carry the
    # rounding of O(1) fields (unit roundoff 6e-8) on top of the relative term
    dabs = 0.0 if prec == "fp64" else 5e-7
    for a, b in zip(defects[:3], d_ref[:3]):
        assert abs(a - b) <= 1e-3 * b + dabs
    if prec == "fp64":
        # K = N: every slice equals the serial fine solution computed on the GPU
        ser = g.zeros(1)
        for n in range(4):
            g.step_fine(ser, 1e-3, 50)
            for c in range(4):
                assert torch.equal(ser.fields()[c][0], slices.fields()[c][n + 1]), (n, c)


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_lid_speed_change_reaches_the_coarse_propagator(prec):
    """ns_set_lid_speed after a Parareal call: the next call's fine AND coarse
    propagators use the new lid (K < N, so G enters the result), the coarse
    values stored for a resume are dropped, and a graph captured before the
    change refuses to launch."""
    from paper_1705_06149_gb300 import StepGraph
    # both sides solve to 1e-13: w (small in the symmetric cavity) is held to
    # 1e-10 on its own
    og = oracle.Grid(16, 16, 16, re=100.0, u_lid=0.5, rtol=1e-13)
    F = opr.fine_propagator(og, 1e-3, 20)
    G = opr.coarse_propagator(og, 1e-2, 2)
    y_ref, d_ref = opr.parareal(og.zeros(), 4, F, G, kmax=2)
    g = Grid(16, 16, 16, re=100.0, u_lid=1.0, precision=prec, batch=4, poisson_rtol=1e-13)
    u0 = g.zeros(1)
    slices = g.zeros(5)
    g.parareal(u0, slices, 4, 20, 2, 1e-3, kmax=1)  # companion grid and chain graph at lid 1
    other = g.zeros(1)
    graph = StepGraph([(g, other, 1e-3, 1)])
    g.set_lid_speed(0.5)
    with pytest.raises(NSError) as e:
        g.parareal(u0, slices, 4, 20, 2, 1e-3, kmax=1, resume=True)
    assert e.value.status == N.NS_ERR_ARG
    with pytest.raises(NSError) as e:
        graph.launch()
    assert e.value.status == N.NS_ERR_ARG
    graph.close()
    k, defects = g.parareal(u0, slices, 4, 20, 2, 1e-3, kmax=2)
    assert k == 2
    got = slices.numpy()
    for n in range(5):
        assert_state_close([a[n] for a in got], y_ref[n], TOL[prec], f"slice {n}")
    dabs = 0.0 if prec == "fp64" else 5e-7
    for a, b in zip(defects, d_ref):
        assert abs(a - b) <= 1e-3 * b + dabs


def test_parareal_resume_and_tolerance():
    g = Grid(12, 12, 12, re=100.0, batch=3)
    u0 = g.zeros(1)
    a = g.zeros(4)
    k1, d1 = g.parareal(u0, a, 3, 20, 4, 1e-3, kmax=1)
    k2, d2 = g.parareal(u0, a, 3, 20, 4, 1e-3, kmax=1, resume=True)
    b = g.zeros(4)
    k3, d3 = g.parareal(u0, b, 3, 20, 4, 1e-3, kmax=2)
    assert (k1, k2, k3) == (1, 1, 2)
    assert d3 == [d1[0], d2[0]]
    for c in range(4):
        assert torch.equal(a.fields()[c], b.fields()[c])
    c_ = g.zeros(4)
    k4, d4 = g.parareal(u0, c_, 3, 20, 4, 1e-3, kmax=10, tol=d3[1] * 1.0001)
    assert k4 == 2
    with pytest.raises(NSError) as e:
        g.parareal(u0, g.zeros(4), 3, 20, 4, 1e-3, kmax=1, resume=True)
    assert e.value.status == N.NS_ERR_ARG
    # the stored coarse values belong to 3 slices of 20 fine / 4 coarse steps
    # of 1e-3: a resume with other ones is refused, the matching one runs
    for args in ((2, 20, 4, 1e-3), (3, 10, 4, 1e-3), (3, 20, 2, 1e-3), (3, 20, 4, 5e-4)):
        with pytest.raises(NSError) as e:
            g.parareal(u0, c_, *args, kmax=1, resume=True)
        assert e.value.status == N.NS_ERR_ARG, args
    k5, _ = g.parareal(u0, c_, 3, 20, 4, 1e-3, kmax=1, resume=True)
    assert k5 == 1


# ---------------------------------------------------------------------------
# full size of the batched sweep: 64^3, 32 slices, sampled against the oracle
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("pc", PCS)
@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_batched_64cubed_32_slices_sampled(prec, pc):
    n, B, dt = 64, 32, 5e-4
    og = oracle.Grid(n, n, n, re=1000.0)
    g = Grid(n, n, n, re=1000.0, precision=prec, batch=B, preconditioner=pc)
    inits = [inputs.random_state(n, n, n, seed=100 + s, sigma=0.05) for s in range(B)]
    st = g.state_from([np.stack([i[c] for i in inits]) for c in range(4)])
    g.project(st)
    proj = st.numpy()
    g.step_fine(st, dt, 1)
    got = st.numpy()
    for s in (0, B - 1):
        start = [np.array(proj[c][s], dtype=np.float64) for c in range(4)]
        want = oracle.copy_state(start)
        og.step(want, dt, 1)
        assert_state_close([got[c][s] for c in range(4)], want, TOL[prec], f"slice {s}")
    lim = 1e-12 if prec == "fp64" else 1e-3
    for s in range(B):
        div = np_divergence([got[c][s].astype(np.float64) for c in range(3)], (1 / n,) * 3)
        assert np.max(np.abs(div)) <= lim, (s, np.max(np.abs(div)))


# ---------------------------------------------------------------------------
# arguments and failures
# ---------------------------------------------------------------------------

def test_argument_errors():
    g = Grid(8, 8, 8, batch=2)
    st = g.zeros(3)
    with pytest.raises(ValueError):
        g.step_fine(g.state_from([a.cpu().numpy() for a in st.fields()], device="cpu"), 1e-3, 1)
    with pytest.raises(NSError) as e:
        g.step_fine(st, 1e-3, 1)  # batch 3 > capacity 2
    assert e.value.status == N.NS_ERR_ARG
    st = g.zeros(2)
    with pytest.raises(NSError) as e:
        g.step_fine(st, 0.0, 1)
    assert e.value.status == N.NS_ERR_ARG
    before = [t.clone() for t in st.fields()]
    g.step_fine(st, 1e-3, 0)
    assert all(torch.equal(a, b) for a, b in zip(before, st.fields()))
    with pytest.raises(NSError) as e:
        Grid(1, 8, 8)
    assert e.value.status == N.NS_ERR_ARG


def test_nonfinite_input_is_reported():
    g = Grid(8, 8, 8, batch=1)
    st = g.zeros(1)
    st.u[0, 3, 3, 3] = float("nan")
    with pytest.raises(NSError) as e:
        g.step_fine(st, 1e-3, 1)
    assert e.value.status == N.NS_ERR_NONFINITE


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_nonfinite_slice_in_pipelined_parareal_is_reported(prec):
    """A non-finite value in one slice's state stops a pipelined Parareal call
    with NS_ERR_NONFINITE (the solver loops on the device end on the
    non-finite residual; the failure is read from the control blocks after
    the call); the grid then runs a clean call as before.  Calls on other
    slice buffers, unchunked (one iteration) and pipelined, never write the
    first call's slices (the cached graphs are keyed by the buffers)."""
    g = Grid(16, 16, 16, re=400.0, precision=prec, batch=4)
    u0 = g.state_from(inputs.random_state(16, 16, 16, seed=14, sigma=0.2))
    g.project(u0)
    ref = g.zeros(5)
    k, d_ref = g.parareal(u0, ref, 4, 5, 1, 1e-3, kmax=2)
    assert k == 2
    ref_copy = ref.clone()
    bad = g.zeros(5)
    g.parareal(u0, bad, 4, 5, 1, 1e-3, kmax=1)
    bad.u[2, 5, 5, 5] = float("nan")
    with pytest.raises(NSError) as e:
        g.parareal(u0, bad, 4, 5, 1, 1e-3, kmax=3, resume=True)
    assert e.value.status == N.NS_ERR_NONFINITE
    for c in range(4):
        assert torch.equal(ref.fields()[c], ref_copy.fields()[c]), c
    again = g.zeros(5)
    k, d = g.parareal(u0, again, 4, 5, 1, 1e-3, kmax=2)
    assert k == 2 and d == d_ref
    for c in range(4):
        assert torch.equal(again.fields()[c], ref.fields()[c]), c


@pytest.mark.parametrize("pc", PCS)
@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_iteration_limit_is_reported(prec, pc):
    # one Krylov iteration per solve (and, with refinement, one outer
    # correction): no solve reaches its tolerance
    g = Grid(16, 16, 16, precision=prec, poisson_maxit=1, batch=1, preconditioner=pc,
             poisson_rtol=1e-30, refine_rtol=1e-10, refine_maxit=1)
    st = g.zeros(1)
    with pytest.raises(NSError) as e:
        g.step_fine(st, 1e-3, 1)
    assert e.value.status == N.NS_ERR_NOT_CONVERGED
    # the grid stays usable afterwards
    g2 = Grid(16, 16, 16, precision=prec, batch=1)
    g2.step_fine(g2.zeros(1), 1e-3, 1)


@pytest.mark.parametrize("pc", PCS)
@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_chunked_parareal_is_bit_identical(prec, pc):
    """The fine sweep in chunks, each chunk's coarse chain overlapped with the
    sweeps of later chunks (with the multigrid solver: graph launches
    pipelined across the iterations of one call; with plain BiCGStab: a
    second host thread per iteration) computes exactly the unchunked
    iterations: same slices bit for bit, same defects, same work.  Chunks of
    4 and 8 divide the 16 slices, 5 leaves a last chunk of one slice, 0 is the
    library's automatic choice (two chunks for calls of two or more
    iterations); -1 sweeps all slices at once."""
    runs = {}
    for chunk in (-1, 0, 4, 5, 8):
        g = Grid(16, 16, 16, re=400.0, precision=prec, batch=16, parareal_chunk=chunk,
                 preconditioner=pc)
        u0 = g.state_from(inputs.random_state(16, 16, 16, seed=11, sigma=0.2))
        g.project(u0)
        slices = g.zeros(17)
        k1, d1 = g.parareal(u0, slices, 16, 10, 2, 1e-3, kmax=1)
        # two iterations in one call, then one more
        k2, d2 = g.parareal(u0, slices, 16, 10, 2, 1e-3, kmax=2, resume=True)
        k3, d3 = g.parareal(u0, slices, 16, 10, 2, 1e-3, kmax=1, resume=True)
        assert (k1, k2, k3) == (1, 2, 1)
        runs[chunk] = (slices, d1 + d2 + d3, g.stats())
    ref, dref, sref = runs[-1]
    for chunk in (0, 4, 5, 8):
        got, d, s = runs[chunk]
        assert d == dref, (chunk, d, dref)
        for c in range(4):
            assert torch.equal(got.fields()[c], ref.fields()[c]), (chunk, c)
        assert s["steps"] == sref["steps"] and s["solves"] == sref["solves"]
        assert s["krylov_iters"] == sref["krylov_iters"]


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_chunked_parareal_with_cluster_v_cycles_is_bit_identical(prec):
    """On a 32^3 grid the V-cycle's coarse levels run as thread-block
    clusters (4 CTAs per state), launched for 24 slices at once by the
    unchunked sweep and for chunks of 12 by the pipelined schedule; the
    pipelined iterations give the unchunked ones bit for bit."""
    runs = {}
    for chunk in (-1, 0):
        g = Grid(32, 32, 32, re=400.0, precision=prec, batch=24, parareal_chunk=chunk)
        u0 = g.state_from(inputs.random_state(32, 32, 32, seed=13, sigma=0.2))
        g.project(u0)
        slices = g.zeros(25)
        k, d = g.parareal(u0, slices, 24, 4, 1, 1e-3, kmax=2)
        assert k == 2
        runs[chunk] = (slices, d, g.stats())
    (ref, dref, sref), (got, d, s) = runs[-1], runs[0]
    assert d == dref, (d, dref)
    for c in range(4):
        assert torch.equal(got.fields()[c], ref.fields()[c]), c
    assert s["krylov_iters"] == sref["krylov_iters"]


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_pipelined_parareal_stops_at_the_tolerance(prec):
    """With a defect tolerance the pipelined iterations stop after the same
    iteration as the unchunked ones, with the same slices and defects (the
    sweep of the first chunk of the iteration after the last one may have
    run: it writes only the library's F buffers)."""
    runs = {}
    tol = None
    for chunk in (-1, 0, 5):
        g = Grid(16, 16, 16, re=400.0, precision=prec, batch=16, parareal_chunk=chunk)
        u0 = g.state_from(inputs.random_state(16, 16, 16, seed=12, sigma=0.2))
        g.project(u0)
        slices = g.zeros(17)
        if tol is None:
            # a tolerance that the defect first meets at iteration i >= 1
            probe = g.zeros(17)
            _, dp = g.parareal(u0, probe, 16, 10, 2, 1e-3, kmax=5)
            i = max(j for j in range(1, 5) if dp[j] < min(dp[:j]))
            tol = (dp[i] + min(dp[:i])) / 2
            k_want = i + 1
        k, d = g.parareal(u0, slices, 16, 10, 2, 1e-3, kmax=8, tol=tol)
        assert k == k_want and d[-1] <= tol and min(d[:-1]) > tol, (chunk, k, d)
        runs[chunk] = (slices, d)
        # a resume continues from the stored coarse values
        k2, d2 = g.parareal(u0, slices, 16, 10, 2, 1e-3, kmax=1, resume=True)
        runs[chunk] = (slices, d + d2)
    ref, dref = runs[-1]
    for chunk in (0, 5):
        got, d = runs[chunk]
        assert d == dref, (chunk, d, dref)
        for c in range(4):
            assert torch.equal(got.fields()[c], ref.fields()[c]), (chunk, c)
