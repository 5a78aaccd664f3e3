"""Hand-value pins of the oracle's ghost rules (Section 2: the 5-point SMART
stencil reads two ghost layers beyond a wall).

The ghost values are read through the oracle's own accessor on a field whose
entries encode their index (1 + i + 10 j + 100 k), so every expected value
below is a number written by hand from the rule: a mirrored index, a dropped
sign or a missing lid term gives another number.  Two SMART fluxes next to
the top wall are then evaluated by hand through the whole convective term:
the tangential first ghost layer at the moving lid, and the wall-normal
component's second ghost layer (the only ghost values beyond the first layer
that reach the result when the wall-normal velocity on the wall is zero).
"""
import numpy as np
import pytest

import oracle


def coded(shape):
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (1.0 + i + 10.0 * j + 100.0 * k).astype(np.float64)


# (component, (i, j, k), value), grid 3 x 4 x 2 cells, walls, u_lid = 1
WALL_CASES = [
    # v, wall-normal along y: odd reflection about the wall face
    (1, (1, -1, 0), -12.0), (1, (1, -2, 0), -22.0),
    (1, (2, 5, 1), -133.0), (1, (2, 6, 1), -123.0),
    # u, tangential along y at the bottom wall: -mirror
    (0, (1, -1, 1), -102.0), (0, (1, -2, 1), -112.0),
    # u, tangential along y at the lid (u_lid = 1): 2 - mirror
    (0, (2, 4, 0), -31.0), (0, (2, 5, 0), -21.0),
    # w, tangential along y at the top wall (the lid moves along x only)
    (2, (0, 4, 2), -231.0), (2, (0, 5, 2), -221.0),
    # w, wall-normal along z
    (2, (1, 1, -1), -112.0), (2, (1, 1, -2), -212.0),
    (2, (1, 1, 3), -112.0), (2, (1, 1, 4), -12.0),
    # u, wall-normal along x (faces 0..3)
    (0, (-1, 2, 1), -122.0), (0, (-2, 2, 1), -123.0),
    (0, (4, 2, 1), -123.0), (0, (5, 2, 1), -122.0),
    # u, tangential along z
    (0, (1, 2, -1), -22.0), (0, (1, 2, -2), -122.0),
    (0, (1, 2, 2), -122.0), (0, (1, 2, 3), -22.0),
    # in range: the stored value itself
    (0, (3, 3, 1), 134.0), (1, (2, 4, 0), 43.0),
]


@pytest.mark.parametrize("c,idx,want", WALL_CASES)
def test_wall_ghosts_by_hand(c, idx, want):
    g = oracle.Grid(3, 4, 2, u_lid=1.0)
    a = coded(g.shape(c))
    assert g.vget(c, a, *idx) == want


# slip along y (u_lid has no effect there), walls elsewhere
SLIP_CASES = [
    (0, (1, 4, 0), 32.0), (0, (1, 5, 0), 22.0),
    (0, (1, -1, 0), 2.0), (0, (1, -2, 0), 12.0),
    (2, (2, -1, 1), 103.0), (2, (2, 4, 1), 133.0),
    (1, (1, -1, 0), -12.0), (1, (1, -2, 0), -22.0),  # normal: as at a wall
    (1, (1, 5, 1), -132.0),
]


@pytest.mark.parametrize("c,idx,want", SLIP_CASES)
def test_slip_ghosts_by_hand(c, idx, want):
    g = oracle.Grid(3, 4, 2, u_lid=1.0, bc=("wall", "slip", "wall"))
    a = coded(g.shape(c))
    assert g.vget(c, a, *idx) == want


# periodic along x: u has 3 faces along x (no duplicate seam face)
PERIODIC_CASES = [
    (0, (-1, 1, 0), 13.0), (0, (-2, 1, 0), 12.0),
    (0, (3, 1, 0), 11.0), (0, (4, 1, 0), 12.0),
    (1, (-1, 1, 0), 13.0), (1, (3, 1, 1), 111.0),
]


@pytest.mark.parametrize("c,idx,want", PERIODIC_CASES)
def test_periodic_ghosts_by_hand(c, idx, want):
    g = oracle.Grid(3, 4, 2, u_lid=1.0, bc=("periodic", "wall", "wall"))
    assert g.shape(0) == (2, 4, 3)
    a = coded(g.shape(c))
    assert g.vget(c, a, *idx) == want


def test_smart_flux_at_the_lid_by_hand():
    """u on the row below the lid (j = 7 of 8), carried downward by v = -0.2
    through its lower edge.  That edge's upwind triple is (far upwind = lid
    ghost 2 u_lid - u_7, upwind u_7, downwind u_6) = (1.4, 0.6, 0.3): the
    normalised value 0.8/1.1 lies in the QUICK band, so the face value is
    1.4 + (0.75 * 8/11 + 0.375)(0.3 - 1.4) = 0.3875.  The lid edge carries no
    flux (v = 0 on the wall), the x fluxes cancel (u constant along x) and
    w = 0, so the convective term is (0 - (-0.2 * 0.3875)) / (1/8) = 0.62.
    One row further down (j = 6) the upper edge is that same 0.3875 and the
    lower edge's triple (u_7, u_6, u_5) = (0.6, 0.3, 0.25) has the normalised
    value 6/7 > 5/6, so its face value is the downwind 0.25:
    (-0.2 * 0.3875 + 0.2 * 0.25) * 8 = -0.22."""
    n = 8
    g = oracle.Grid(4, n, 4, u_lid=1.0)
    f = np.array([0.0, 0.05, 0.1, 0.15, 0.2, 0.25, 0.3, 0.6])
    u = np.zeros(g.shape(0)) + f[None, :, None]
    v = np.zeros(g.shape(1))
    v[:, 1:n, :] = -0.2
    w = np.zeros(g.shape(2))
    conv, _ = g.rhs_terms(u, v, w)
    assert conv[0][1, 7, 2] == pytest.approx(0.62, rel=1e-13)
    assert conv[0][1, 6, 2] == pytest.approx(-0.22, rel=1e-13)


def test_wall_normal_second_ghost_by_hand():
    """v on the last interior y-face below the top wall (j = 7 of faces
    0..8), v_7 = -0.3 (downward), the wall face v_8 = 0.  The cell centre
    above it has U_f = (v_7 + v_8)/2 = -0.15 < 0, so its upwind side is the
    wall: the triple is (far upwind = second ghost layer -v_7 = 0.3, upwind =
    the wall face 0, downwind v_7 = -0.3), normalised value 1/2, QUICK face
    value 0.3 + 0.75 (-0.6) = -0.15 and flux -0.15 * -0.15 = 0.0225.  The
    centre below has U_f = (v_6 + v_7)/2 = -0.2 and the triple (v_8, v_7, v_6)
    = (0, -0.3, -0.1), normalised value 3: first-order upwind -0.3, flux
    0.06.  With u = w = 0 the convective term is (0.0225 - 0.06) * 8 = -0.3."""
    n = 8
    g = oracle.Grid(4, n, 4, u_lid=1.0)
    gj = np.array([0.0, -0.05, -0.05, -0.05, -0.05, -0.05, -0.1, -0.3, 0.0])
    u = np.zeros(g.shape(0))
    v = np.zeros(g.shape(1)) + gj[None, :, None]
    w = np.zeros(g.shape(2))
    conv, _ = g.rhs_terms(u, v, w)
    assert conv[1][1, 7, 1] == pytest.approx(-0.3, rel=1e-13)
