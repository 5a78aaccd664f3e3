"""Pins of the FP64 oracle against what the mathematics fixes (no GPU).

Each test checks the oracle against a closed form, an identity, a library
routine or a brute-force result -- never against a retyped copy of its own
formulas -- so that a dropped term, a flipped sign or a shifted index in any
part (SMART, diffusion, ghost rules, D, G, L, BiCGStab, gauge, stepper,
Parareal) fails at least one of them.  Paper references are to Croce,
Ruprecht & Krause (arXiv 1705.06149).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import laplacian as graph_laplacian

import oracle
from oracle import parareal as opr
from paper_1705_06149_gb300 import inputs

TWO_PI = 2.0 * math.pi


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def centres(n, L):
    return (np.arange(n) + 0.5) * (L / n)


def nodes(n, L, periodic):
    m = n if periodic else n + 1
    return np.arange(m) * (L / n)


def face_coords(g: oracle.Grid, comp):
    """(X, Y, Z) coordinates of the stored positions of component comp (z,y,x order)."""
    n = (g.nx, g.ny, g.nz)
    L = (g.lx, g.ly, g.lz)
    per = [b == "periodic" for b in g.bc]
    ax = []
    for d in range(3):
        ax.append(nodes(n[d], L[d], per[d]) if d == comp else centres(n[d], L[d]))
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return X, Y, Z


# ---------------------------------------------------------------------------
# SMART (Section 2: "second order TVD SMART upwind scheme ... bounded QUICK")
# ---------------------------------------------------------------------------

def test_smart_normalised_variable_values():
    # hand values of Gaskell & Lau's SMART map (U, C, D -> face)
    assert oracle.smart(0.0, 0.5, 1.0) == pytest.approx(0.75, abs=1e-15)
    assert oracle.smart(0.0, 0.1, 1.0) == pytest.approx(0.3, abs=1e-15)
    assert oracle.smart(0.0, 0.9, 1.0) == pytest.approx(1.0, abs=1e-15)
    assert oracle.smart(0.0, 1.2, 1.0) == pytest.approx(1.2, abs=1e-15)  # upwind branch
    assert oracle.smart(0.0, -0.3, 1.0) == pytest.approx(-0.3, abs=1e-15)  # upwind branch
    # mirrored data: decreasing profile U=1, C=0.5, D=0 -> 0.25
    assert oracle.smart(1.0, 0.5, 0.0) == pytest.approx(0.25, abs=1e-15)
    # flat far field: the face takes the upwind value
    assert oracle.smart(2.0, 5.0, 2.0) == 5.0


def test_smart_reproduces_quick_on_quadratics():
    # QUICK is exact for quadratic profiles; inside the QUICK band SMART is QUICK.
    for a, b, c in [(1.0, 2.0, 1.0), (0.3, -1.0, 4.0), (-2.0, 0.5, 0.0)]:
        f = lambda x: a * x * x + b * x + c  # noqa: E731
        U, C, D = f(-1.0), f(0.0), f(1.0)
        ph = (C - U) / (D - U)
        if 1 / 6 < ph < 5 / 6:
            assert oracle.smart(U, C, D) == pytest.approx(f(0.5), rel=1e-14)


def test_smart_bounded_between_upwind_and_downwind():
    rng = np.random.default_rng(0)
    for _ in range(2000):
        U, C, D = rng.normal(size=3)
        lo, hi = min(U, D), max(U, D)
        f = oracle.smart(U, C, D)
        if lo <= C <= hi:  # monotone data: the face lies between C and D
            assert min(C, D) - 1e-14 <= f <= max(C, D) + 1e-14


# ---------------------------------------------------------------------------
# Laplacian L = D G with homogeneous Neumann faces dropped (Section 2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bc", [("wall",) * 3, ("periodic", "wall", "slip")])
def test_laplacian_cosine_eigenvectors(bc):
    nx, ny, nz = 7, 5, 6
    L = (1.0, 0.7, 1.3)
    g = oracle.Grid(nx, ny, nz, *L, bc=bc)
    h = g.h
    for m in [(1, 0, 0), (0, 2, 0), (1, 1, 3), (2, 3, 1)]:
        parts = []
        lam = 0.0
        for d, n in enumerate((nx, ny, nz)):
            x = centres(n, L[d])
            if bc[d] == "periodic":
                k = TWO_PI * m[d] / L[d]
                parts.append(np.cos(k * x))
                lam -= 4.0 / h[d] ** 2 * math.sin(k * h[d] / 2) ** 2
            else:
                k = math.pi * m[d] / L[d]
                parts.append(np.cos(k * x))
                lam -= 4.0 / h[d] ** 2 * math.sin(k * h[d] / 2) ** 2
        p = np.einsum("k,j,i->kji", parts[2], parts[1], parts[0])
        lp = g.laplacian(p)
        assert np.max(np.abs(lp - lam * p)) <= 1e-11 * max(1.0, abs(lam))


def _graph_laplacian(nx, ny, nz, h, bc, solid):
    """-L from scipy's graph Laplacian of the fluid-cell adjacency graph with
    edge weights 1/h_d^2 (a different construction of the same operator)."""
    n = nx * ny * nz
    idx = np.arange(n).reshape(nz, ny, nx)
    rows, cols, vals = [], [], []
    dims = (nx, ny, nz)
    for d in range(3):
        ax = 2 - d
        a = idx
        b = np.roll(idx, -1, axis=ax)
        sl = [slice(None)] * 3
        if bc[d] != "periodic":
            sl[ax] = slice(0, dims[d] - 1)
        a = a[tuple(sl)].ravel()
        b = b[tuple(sl)].ravel()
        if dims[d] == 1:
            continue
        keep = ~(solid.ravel()[a].astype(bool) | solid.ravel()[b].astype(bool))
        a, b = a[keep], b[keep]
        w = np.full(a.shape, 1.0 / h[d] ** 2)
        rows += [a, b]
        cols += [b, a]
        vals += [w, w]
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    A.sum_duplicates()
    return graph_laplacian(A)


@pytest.mark.parametrize("dims,bc", [((4, 4, 4), ("wall",) * 3),
                                     ((3, 5, 2), ("wall", "periodic", "wall")),
                                     ((5, 4, 3), ("periodic", "slip", "periodic"))])
def test_laplacian_is_graph_laplacian(dims, bc):
    nx, ny, nz = dims
    rng = np.random.default_rng(1)
    solid = (rng.random((nz, ny, nx)) < 0.15).astype(np.uint8)
    for s in (np.zeros_like(solid), solid):
        g = oracle.Grid(nx, ny, nz, 1.0, 0.8, 1.2, bc=bc, solid=s)
        Lg = _graph_laplacian(nx, ny, nz, g.h, bc, s)
        x = rng.normal(size=(nz, ny, nx))
        x[s.astype(bool)] = 0.0
        want = -(Lg @ x.ravel())
        got = g.laplacian(x).ravel()
        assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_poisson_matches_lstsq_on_tiny_grids():
    rng = np.random.default_rng(2)
    for (nx, ny, nz), bc in [((4, 4, 4), ("wall",) * 3), ((3, 5, 2), ("wall", "periodic", "wall"))]:
        solid = np.zeros((nz, ny, nx), dtype=np.uint8)
        g = oracle.Grid(nx, ny, nz, bc=bc, solid=solid)
        A = -_graph_laplacian(nx, ny, nz, g.h, bc, solid).toarray()
        b = rng.normal(size=nx * ny * nz)
        b -= b.mean()
        x_ref = np.linalg.lstsq(A, b, rcond=None)[0]
        x_ref -= x_ref.mean()
        x, _ = g.poisson(b.reshape(nz, ny, nx), rtol=1e-13)
        assert rel(x, x_ref) <= 1e-10


def test_poisson_recovers_manufactured_solution_with_solids():
    rng = np.random.default_rng(3)
    nx, ny, nz = 12, 10, 9
    solid = np.zeros((nz, ny, nx), dtype=np.uint8)
    solid[3:5, 4:7, 2:5] = 1
    g = oracle.Grid(nx, ny, nz, solid=solid)
    p = rng.normal(size=(nz, ny, nx))
    p[solid.astype(bool)] = 0.0
    p[~solid.astype(bool)] -= p[~solid.astype(bool)].mean()
    b = g.laplacian(p)
    x, it = g.poisson(b, rtol=1e-13)
    assert rel(x, p) <= 1e-9
    assert np.all(x[solid.astype(bool)] == 0.0)


def test_poisson_closed_form_second_order():
    # p = cos(pi x) cos(pi y) cos(pi z) satisfies dp/dn = 0 on the unit cube and
    # lap p = -3 pi^2 p: the discrete solution converges at second order.
    errs = []
    for n in (8, 16, 32):
        g = oracle.Grid(n, n, n)
        x = centres(n, 1.0)
        pex = np.einsum("k,j,i->kji", np.cos(math.pi * x), np.cos(math.pi * x), np.cos(math.pi * x))
        ph, _ = g.poisson(-3 * math.pi ** 2 * pex, rtol=1e-13)
        errs.append(np.max(np.abs(ph - (pex - pex.mean()))))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) >= 1.9, (errs, orders)


# ---------------------------------------------------------------------------
# D and G (central differences, Section 2)
# ---------------------------------------------------------------------------

def test_divergence_and_gradient_closed_forms():
    n = (12, 10, 8)
    L = (TWO_PI, TWO_PI, TWO_PI)
    g = oracle.Grid(*n, *L, bc=("periodic",) * 3)
    h = g.h
    X, Y, Z = face_coords(g, 0)
    u = np.sin(X) * np.cos(Z)
    X, Y, Z = face_coords(g, 1)
    v = np.cos(2 * Y)
    X, Y, Z = face_coords(g, 2)
    w = np.sin(Z + X)
    Zc, Yc, Xc = np.meshgrid(centres(n[2], L[2]), centres(n[1], L[1]), centres(n[0], L[0]),
                             indexing="ij")
    # d/dx sin(x) sampled by a centred difference of spacing h: sin(h/2)/(h/2) cos(x)
    sx = math.sin(h[0] / 2) / (h[0] / 2)
    sy = math.sin(h[1]) / (h[1] / 2)
    sz = math.sin(h[2] / 2) / (h[2] / 2)
    want = sx * np.cos(Xc) * np.cos(Zc) - sy * np.sin(2 * Yc) + sz * np.cos(Zc + Xc)
    assert np.max(np.abs(g.divergence(u, v, w) - want)) <= 1e-12
    p = np.sin(Xc) * np.cos(2 * Yc) + np.cos(Zc)
    gu, gv, gw = g.gradient(p)
    X, Y, Z = face_coords(g, 0)
    assert np.max(np.abs(gu - sx * np.cos(X) * np.cos(2 * Y))) <= 1e-12
    X, Y, Z = face_coords(g, 1)
    assert np.max(np.abs(gv - (-sy * np.sin(X) * np.sin(2 * Y)))) <= 1e-12
    X, Y, Z = face_coords(g, 2)
    assert np.max(np.abs(gw - (-sz * np.sin(Z)))) <= 1e-12


@pytest.mark.parametrize("bc", [("wall",) * 3, ("periodic", "wall", "slip")])
def test_divergence_is_minus_gradient_transpose(bc):
    rng = np.random.default_rng(4)
    solid = np.zeros((6, 7, 5), dtype=np.uint8)
    solid[2:4, 3:5, 1:3] = 1
    g = oracle.Grid(5, 7, 6, 1.0, 1.1, 0.9, bc=bc, solid=solid)
    st = inputs.random_state(5, 7, 6, seed=5, bc=bc, solid=solid)
    p = rng.normal(size=g.shape(3))
    p[solid.astype(bool)] = 0
    gu, gv, gw = g.gradient(p)
    lhs = sum(np.sum(a * b) for a, b in zip((gu, gv, gw), st[:3]))
    rhs = -np.sum(p * g.divergence(*st[:3]))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)


# ---------------------------------------------------------------------------
# projection (Chorin-Temam, Section 2)
# ---------------------------------------------------------------------------

def test_projection_is_an_orthogonal_projection():
    solid = np.zeros((9, 8, 10), dtype=np.uint8)
    solid[3:6, 2:4, 4:7] = 1
    for bc, s in [(("wall",) * 3, None), (("periodic", "wall", "wall"), solid)]:
        g = oracle.Grid(10, 8, 9, bc=bc, solid=s)
        st = inputs.random_state(10, 8, 9, seed=6, bc=bc, solid=s)
        pu = g.project(*st[:3], rtol=1e-14)
        div = g.divergence(*pu[:3])
        assert np.max(np.abs(div)) <= 1e-12 * np.max(np.abs(g.divergence(*st[:3])))
        ppu = g.project(*pu[:3], rtol=1e-14)
        assert max(rel(ppu[c], pu[c]) for c in range(3)) <= 1e-12
        inner = sum(np.sum(pu[c] * (st[c] - pu[c])) for c in range(3))
        norm2 = sum(np.sum(st[c] ** 2) for c in range(3))
        assert abs(inner) <= 1e-12 * norm2


def test_step_leaves_discretely_divergence_free_velocity():
    g = oracle.Grid(12, 12, 12, re=100.0)
    st = g.zeros()
    for _ in range(5):
        g.step(st, 1e-3, 1)
        assert np.max(np.abs(g.divergence(*st[:3]))) <= 1e-12
    assert abs(g.fluid_mean(st[3])) <= 1e-14


# ---------------------------------------------------------------------------
# diffusion, convection and the stepper against closed forms
# ---------------------------------------------------------------------------

def test_diffusion_of_a_shear_mode_is_exact_forward_euler():
    # u = sin(y), v = w = 0 on a periodic box: convection vanishes identically,
    # sin is an eigenvector of the 3-point second difference, and forward Euler
    # multiplies it by (1 + dt lam / Re) per step.
    n = (4, 16, 4)
    g = oracle.Grid(*n, TWO_PI, TWO_PI, TWO_PI, re=5.0, bc=("periodic",) * 3)
    h = g.h[1]
    st = g.zeros()
    X, Y, Z = face_coords(g, 0)
    st[0][:] = np.sin(Y)
    conv, diff = g.rhs_terms(*st[:3])
    assert max(np.max(np.abs(c)) for c in conv) == 0.0
    lam = -4.0 / h ** 2 * math.sin(h / 2) ** 2
    dt, steps = 0.01, 40
    g.step(st, dt, steps)
    want = (1.0 + dt * lam / 5.0) ** steps * np.sin(Y)
    assert np.max(np.abs(st[0] - want)) <= 1e-13
    assert np.max(np.abs(st[1])) == 0.0 and np.max(np.abs(st[2])) == 0.0


@pytest.mark.parametrize("c,d", [(0, 1), (0, 2), (1, 0), (1, 2), (2, 0), (2, 1)])
def test_convection_of_an_advected_shear_wave(c, d):
    # component c = sin(x_d), component d = V0 (constant): div(u u) for component
    # c reduces to V0 d/dx_d sin(x_d) = V0 cos(x_d); the component-d term vanishes.
    # A TVD limiter clips to first order near the two extrema (O(h) error on an
    # O(h) fraction of the points), so the RMS error converges at order 1.5;
    # a shifted stencil would give order 1, a flipped sign no convergence.
    V0 = 0.7
    errs = []
    for N in (16, 32, 64):
        n = [4, 4, 4]
        n[d] = N
        g = oracle.Grid(*n, TWO_PI, TWO_PI, TWO_PI, re=0.0, bc=("periodic",) * 3)
        st = g.zeros()
        coords = face_coords(g, c)
        st[c][:] = np.sin(coords[d])
        st[d][:] = V0
        conv, _ = g.rhs_terms(*st[:3])
        assert np.max(np.abs(conv[d])) <= 1e-13
        errs.append(np.sqrt(np.mean((conv[c] - V0 * np.cos(coords[d])) ** 2)))
    order = math.log2(errs[1] / errs[2])
    assert errs[2] < 1e-2 and order >= 1.4, (errs, order)


def test_convection_manufactured_smooth_field():
    sympy = pytest.importorskip("sympy")
    x, y, z = sympy.symbols("x y z")
    U = [sympy.sin(x) * sympy.cos(2 * y) + 0.4 * sympy.cos(z),
         sympy.cos(x + z) * sympy.sin(y) + 0.3,
         sympy.sin(2 * z) * sympy.cos(y) - 0.2 * sympy.sin(x)]
    X3 = (x, y, z)
    conv_exact = [sum(sympy.diff(U[d] * U[c], X3[d]) for d in range(3)) for c in range(3)]
    f_u = [sympy.lambdify(X3, e, "numpy") for e in U]
    f_c = [sympy.lambdify(X3, e, "numpy") for e in conv_exact]
    errs = []
    for N in (16, 32, 64):
        g = oracle.Grid(N, N, N, TWO_PI, TWO_PI, TWO_PI, re=0.0, bc=("periodic",) * 3)
        st = g.zeros()
        for c in range(3):
            Xf, Yf, Zf = face_coords(g, c)
            st[c][:] = f_u[c](Xf, Yf, Zf)
        conv, _ = g.rhs_terms(*st[:3])
        e = 0.0
        for c in range(3):
            Xf, Yf, Zf = face_coords(g, c)
            e = max(e, float(np.sqrt(np.mean((conv[c] - f_c[c](Xf, Yf, Zf)) ** 2))))
        errs.append(e)
    order = math.log2(errs[1] / errs[2])
    assert order >= 1.4, (errs, order)


def test_smart_advection_creates_no_new_extrema():
    # step profile in u(y) carried by v = 1 at Courant number 1/4 (inviscid); the
    # SMART face values satisfy Leonard's universal-limiter bound for explicit
    # Euler at Courant numbers <= 1/3, so the update stays within [0, 1].
    g = oracle.Grid(4, 40, 4, TWO_PI, TWO_PI, TWO_PI, re=0.0, bc=("periodic",) * 3)
    st = g.zeros()
    X, Y, Z = face_coords(g, 0)
    st[0][:] = ((Y > 1.0) & (Y < 3.0)).astype(float)
    st[1][:] = 1.0
    dt = 0.25 * g.h[1]
    for _ in range(60):
        g.step(st, dt, 1)
        assert st[0].min() >= -1e-13 and st[0].max() <= 1.0 + 1e-13
    assert st[0].max() > 0.9  # still transported, not smeared away


def test_couette_profile_is_steady_and_transient_matches_series():
    # lid-driven plane Couette flow between y=0 (at rest) and the lid y=1
    # (speed 1), periodic in x and z: u = y is an exact steady state of the
    # discrete scheme; from rest the profile follows the classical sine series.
    n = (4, 16, 4)
    g = oracle.Grid(*n, re=1.0, u_lid=1.0, bc=("periodic", "wall", "periodic"))
    X, Y, Z = face_coords(g, 0)
    st = g.zeros()
    st[0][:] = Y
    g.step(st, 1e-3, 10)
    assert np.max(np.abs(st[0] - Y)) <= 1e-13
    assert np.max(np.abs(st[1])) <= 1e-14 and np.max(np.abs(st[2])) <= 1e-14

    def series(yy, t):
        s = np.array(yy, copy=True)
        for m in range(1, 400):
            s -= 2.0 * (-1) ** (m + 1) / (m * math.pi) * np.sin(m * math.pi * yy) * math.exp(
                -(m * math.pi) ** 2 * t)
        return s

    errs = []
    T = 0.05
    for ny in (16, 32):
        gg = oracle.Grid(4, ny, 4, re=1.0, bc=("periodic", "wall", "periodic"))
        X, Y, Z = face_coords(gg, 0)
        dt = 0.25 * (1.0 / ny) ** 2
        steps = int(round(T / dt))
        s = gg.zeros()
        gg.step(s, T / steps, steps)
        errs.append(np.max(np.abs(s[0] - series(Y, T))))
    assert errs[1] < 2e-4 and errs[0] / errs[1] > 3.5, errs


def test_taylor_green_vortex_decay():
    # u = sin x cos y F, v = -cos x sin y F, F = exp(-2 t / Re), on [0, 2 pi]^2
    # (periodic), w = 0 (periodic z with no z dependence).
    Re, T = 10.0, 0.4
    errs = []
    for N in (16, 32):
        g = oracle.Grid(N, N, 2, TWO_PI, TWO_PI, TWO_PI * 2 / N, re=Re, bc=("periodic",) * 3)
        st = g.zeros()
        X, Y, Z = face_coords(g, 0)
        st[0][:] = np.sin(X) * np.cos(Y)
        X1, Y1, Z1 = face_coords(g, 1)
        st[1][:] = -np.cos(X1) * np.sin(Y1)
        steps = 400
        g.step(st, T / steps, steps)
        F = math.exp(-2 * T / Re)
        e = max(rel(st[0], np.sin(X) * np.cos(Y) * F), rel(st[1], -np.cos(X1) * np.sin(Y1) * F))
        errs.append(e)
        assert np.max(np.abs(st[2])) <= 1e-13
    order = math.log2(errs[0] / errs[1])
    assert errs[1] < 5e-3 and order >= 1.8, (errs, order)


# ---------------------------------------------------------------------------
# the lid-driven cavity (Section 3): invariants
# ---------------------------------------------------------------------------

def test_cavity_at_rest_stays_at_rest():
    g = oracle.Grid(6, 6, 6, re=100.0, u_lid=0.0)
    st = g.zeros()
    g.step(st, 1e-3, 3)
    assert all(np.max(np.abs(a)) == 0.0 for a in st)


def test_cavity_is_mirror_symmetric_in_z():
    g = oracle.Grid(10, 10, 10, re=100.0, u_lid=1.0)
    st = g.zeros()
    g.step(st, 2e-3, 25)
    u, v, w, p = st
    assert rel(u, u[::-1]) <= 1e-10 and rel(v, v[::-1]) <= 1e-10
    assert rel(w, -w[::-1]) <= 1e-10 and rel(p, p[::-1]) <= 1e-10
    assert np.max(np.abs(u)) > 0.05


def test_kinetic_energy_decays_without_lid():
    g = oracle.Grid(10, 10, 10, re=100.0, u_lid=0.0)
    st0 = inputs.random_state(10, 10, 10, seed=7, sigma=0.2)
    u, v, w, _ = g.project(*st0[:3], rtol=1e-13)
    st = [u, v, w, np.zeros(g.shape(3))]
    e_prev = sum(np.sum(a ** 2) for a in st[:3])
    for _ in range(15):
        g.step(st, 2e-3, 1)
        e = sum(np.sum(a ** 2) for a in st[:3])
        assert e < e_prev
        e_prev = e


def test_temporal_error_is_first_order():
    # the paper's own check of F_dt against F_{dt/10} (Section 3): forward Euler
    # makes the error shrink tenfold per tenfold step reduction.
    T = 0.02
    finals = []
    for steps in (10, 100, 1000):
        g = oracle.Grid(8, 8, 8, re=100.0)
        st = g.zeros()
        g.step(st, T / steps, steps)
        finals.append(st)
    e1 = max(rel(finals[0][c], finals[2][c]) for c in range(3))
    e2 = max(rel(finals[1][c], finals[2][c]) for c in range(3))
    assert 8.0 < e1 / e2 < 14.0, (e1, e2)


# ---------------------------------------------------------------------------
# Parareal (Section 2.1.2, Eq. 6 and its fixed point)
# ---------------------------------------------------------------------------

def _small_parareal_setup():
    g = oracle.Grid(8, 8, 8, re=100.0)
    F = opr.fine_propagator(g, 1e-3, 10)
    G = opr.coarse_propagator(g, 5e-3, 2)
    return g, F, G


def test_parareal_with_as_many_iterations_as_slices_is_the_serial_solution():
    g, F, G = _small_parareal_setup()
    u0 = g.zeros()
    N = 3
    serial = opr.serial_fine(u0, N, F)
    for k in range(N + 1):
        y, defects = opr.parareal(u0, N, F, G, kmax=k)
        for n in range(k + 1):  # slices up to k are exact after k iterations
            for c in range(4):
                assert np.array_equal(y[n][c], serial[n][c]), (k, n, c)
    assert defects[-1] == 0.0 or len(defects) == N
    # K = N reproduces the serial fine solution on every slice bit for bit
    for n in range(N + 1):
        for c in range(4):
            assert np.array_equal(y[n][c], serial[n][c])


def test_parareal_zero_iterations_is_the_coarse_sweep():
    g, F, G = _small_parareal_setup()
    u0 = g.zeros()
    y, defects = opr.parareal(u0, 3, F, G, kmax=0)
    serial_g = opr.serial_fine(u0, 3, G)
    assert defects == []
    for n in range(4):
        for c in range(4):
            assert np.array_equal(y[n][c], serial_g[n][c])


def test_parareal_with_the_fine_propagator_as_coarse_converges_in_one_iteration():
    g, F, _ = _small_parareal_setup()
    u0 = g.zeros()
    y, defects = opr.parareal(u0, 3, F, F, kmax=2)
    serial = opr.serial_fine(u0, 3, F)
    assert defects[0] == 0.0
    for n in range(4):
        for c in range(4):
            assert np.array_equal(y[n][c], serial[n][c])


def test_parareal_defect_decreases():
    g, F, G = _small_parareal_setup()
    u0 = g.zeros()
    _, defects = opr.parareal(u0, 4, F, G, kmax=3)
    assert defects[0] > 0 and defects[1] < defects[0] and defects[2] < defects[1]
