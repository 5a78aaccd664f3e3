"""Pins of the oracle with solid cells (first-order cell decomposition,
Section 2): a solid slab filling the last cells along an axis must act
exactly as a wall there, so the fluid part of the slabbed cavity follows the
smaller cavity; interior boxes keep their faces at rest, the velocity
discretely divergence-free, and the z-mirror symmetry of the cavity."""
import numpy as np
import pytest

import oracle
from paper_1705_06149_gb300 import inputs


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_solid_slab_acts_as_a_wall(axis):
    n_small = [8, 7, 6]
    m = 3  # slab thickness in cells
    n_big = list(n_small)
    n_big[axis] += m
    h = [1.0 / 8, 1.0 / 7, 1.0 / 6]
    L_small = [n_small[d] * h[d] for d in range(3)]
    L_big = [n_big[d] * h[d] for d in range(3)]
    solid = np.zeros((n_big[2], n_big[1], n_big[0]), dtype=np.uint8)
    sl = [slice(None)] * 3
    sl[2 - axis] = slice(n_small[axis], None)
    solid[tuple(sl)] = 1
    # the big grid's lid (y = ly) lies inside the slab when axis == 1, so it
    # must not reach the fluid; the small grid has a resting lid
    gb = oracle.Grid(*n_big, *L_big, re=30.0, u_lid=1.0, solid=solid, rtol=1e-13)
    lid_small = 0.0 if axis == 1 else 1.0
    gs = oracle.Grid(*n_small, *L_small, re=30.0, u_lid=lid_small, rtol=1e-13)
    rs = inputs.random_state(*n_small, seed=4, sigma=0.4)
    u, v, w, _ = gs.project(*rs[:3], rtol=1e-14)
    small = [u, v, w, np.zeros(gs.shape(3))]
    big = gb.zeros()
    for c in range(4):
        idx = tuple(slice(0, s) for s in small[c].shape)
        big[c][idx] = small[c]
    gs.step(small, 2e-3, 6)
    gb.step(big, 2e-3, 6)
    for c in range(4):
        idx = tuple(slice(0, s) for s in small[c].shape)
        got = big[c][idx]
        err = np.max(np.abs(got - small[c])) / max(np.max(np.abs(small[c])), 1e-30)
        assert err <= 1e-9, (axis, c, err)
        rest = big[c].copy()
        rest[idx] = 0.0
        assert np.max(np.abs(rest)) <= 1e-12 * max(np.max(np.abs(small[c])), 1.0), (axis, c)


def test_cavity_with_boxes_keeps_solids_at_rest_and_divergence_free():
    n = 16
    boxes, solid = inputs.obstacle_boxes((n, n, n), seed=2, count=3, edge=(0.15, 0.3))
    g = oracle.Grid(n, n, n, re=100.0, solid=solid)
    st = g.zeros()
    g.step(st, 2e-3, 10)
    assert np.max(np.abs(st[0])) > 0.05
    assert np.max(np.abs(g.divergence(*st[:3]))) <= 1e-12
    assert np.all(st[3][solid.astype(bool)] == 0.0)
    sb = solid.astype(bool)
    # every face touching a solid cell holds zero velocity
    assert np.all(st[0][:, :, 1:][sb] == 0.0) and np.all(st[0][:, :, :-1][sb] == 0.0)
    assert np.all(st[1][:, 1:, :][sb] == 0.0) and np.all(st[1][:, :-1, :][sb] == 0.0)
    assert np.all(st[2][1:, :, :][sb] == 0.0) and np.all(st[2][:-1, :, :][sb] == 0.0)


def test_symmetric_obstacle_keeps_the_cavity_mirror_symmetric():
    n = 12
    solid = np.zeros((n, n, n), dtype=np.uint8)
    solid[4:8, 3:6, 4:7] = 1  # symmetric about z = 1/2 (cells 4..7 of 12)
    g = oracle.Grid(n, n, n, re=100.0, solid=solid, rtol=1e-13)
    st = g.zeros()
    g.step(st, 2e-3, 12)
    u, v, w, p = st
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)  # noqa: E731
    assert rel(u, u[::-1]) <= 1e-9 and rel(v, v[::-1]) <= 1e-9
    assert rel(w, -w[::-1]) <= 1e-9 and rel(p, p[::-1]) <= 1e-9
