"""Seeded synthetic inputs shared by the CUDA path's callers and the oracle's tests.

This module holds input generation only (zeros, seeded noise, box masks,
trilinear resampling): none of the projection method's arithmetic.  Every
generator draws from ``numpy.random.Generator(PCG64(seed))``.

Canonical state layout (x fastest, optional leading batch dimension):
``u[nz][ny][nx+1]``, ``v[nz][ny+1][nx]``, ``w[nz+1][ny][nx]``, ``p[nz][ny][nx]``;
along a periodic axis the normal component has ``n`` faces instead of ``n+1``.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np

WALL, PERIODIC, SLIP = "wall", "periodic", "slip"


def _bcs(bc) -> Tuple[str, str, str]:
    names = {0: WALL, 1: PERIODIC, 2: SLIP}
    return tuple(names.get(b, b) for b in bc)  # type: ignore[return-value]


def shapes(nx: int, ny: int, nz: int, bc: Sequence = (WALL, WALL, WALL)):
    """Array shapes (u, v, w, p) of one state."""
    bc = _bcs(bc)
    n = (nx, ny, nz)
    out = []
    for c in range(3):
        ext = [n[d] + (1 if (d == c and bc[d] != PERIODIC) else 0) for d in range(3)]
        out.append((ext[2], ext[1], ext[0]))
    out.append((nz, ny, nx))
    return out


def zero_state(nx, ny, nz, bc=(WALL, WALL, WALL), batch: Optional[int] = None,
               dtype=np.float64) -> List[np.ndarray]:
    shp = shapes(nx, ny, nz, bc)
    lead = () if batch is None else (batch,)
    return [np.zeros(lead + s, dtype=dtype) for s in shp]


def _zero_boundary_faces(a: np.ndarray, comp: int, bc) -> None:
    """Zero the wall-normal boundary faces of component comp (last 3 dims z,y,x)."""
    bc = _bcs(bc)
    if bc[comp] == PERIODIC:
        return
    axis = a.ndim - 1 - comp
    idx0 = [slice(None)] * a.ndim
    idx1 = [slice(None)] * a.ndim
    idx0[axis] = 0
    idx1[axis] = -1
    a[tuple(idx0)] = 0.0
    a[tuple(idx1)] = 0.0


def random_state(nx, ny, nz, seed: int, sigma: float = 1.0, bc=(WALL, WALL, WALL),
                 batch: Optional[int] = None, p_sigma: float = 0.0,
                 solid: Optional[np.ndarray] = None) -> List[np.ndarray]:
    """Gaussian N(0, sigma^2) velocity on every face that is not a wall-normal
    boundary face (and not next to a solid cell); pressure N(0, p_sigma^2) in
    fluid cells.  Not divergence-free: the first projection makes it so."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shp = shapes(nx, ny, nz, bc)
    lead = () if batch is None else (batch,)
    st = [rng.standard_normal(lead + s) * sigma for s in shp[:3]]
    for c in range(3):
        _zero_boundary_faces(st[c], c, bc)
    p = rng.standard_normal(lead + shp[3]) * p_sigma if p_sigma > 0 else np.zeros(lead + shp[3])
    st.append(p)
    if solid is not None:
        zero_solid_faces(st, solid, bc)
    return st


def zero_solid_faces(st: List[np.ndarray], solid: np.ndarray, bc=(WALL, WALL, WALL)) -> None:
    """Zero velocity faces touching a solid cell, and the pressure inside solids."""
    bc = _bcs(bc)
    s = solid.astype(bool)
    nz, ny, nx = s.shape
    for c in range(3):
        a = st[c]
        n = (nx, ny, nz)[c]
        axis_s = 2 - c
        # cell on the low and high side of every stored face along axis c
        nf = a.shape[-1 - c]
        lo = np.arange(nf) - 1
        hi = np.arange(nf)
        if bc[c] == PERIODIC:
            lo %= n
            hi %= n
        lo_c = np.clip(lo, 0, n - 1)
        hi_c = np.clip(hi, 0, n - 1)
        s_lo = np.take(s, lo_c, axis=axis_s) & (lo >= 0).reshape(
            [-1 if ax == axis_s else 1 for ax in range(3)])
        s_hi = np.take(s, hi_c, axis=axis_s) & (hi <= n - 1).reshape(
            [-1 if ax == axis_s else 1 for ax in range(3)])
        mask = s_lo | s_hi
        a[..., mask] = 0.0
    st[3][..., s] = 0.0


def obstacle_boxes(n: Tuple[int, int, int], seed: int = 0, count: int = 8,
                   edge: Tuple[float, float] = (0.05, 0.2), y_max: float = 0.8,
                   gap_cells: int = 2, max_tries: int = 100000):
    """Seeded axis-aligned boxes in the unit cube and their cell mask.

    Box edges ~ U[edge] per axis; each box lies inside [2h, 1-2h]^3, below
    y = y_max (away from the lid), and at least gap_cells cells away from every
    other box (rejection sampling).  A cell is solid iff its centre lies inside
    a box.  Returns (boxes [count][2][3] as (lo, hi) xyz, mask [nz][ny][nx] uint8).
    """
    nx, ny, nz = n
    h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    rng = np.random.Generator(np.random.PCG64(seed))
    boxes = []
    tries = 0
    while len(boxes) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place the boxes")
        size = rng.uniform(edge[0], edge[1], size=3)
        lo_min = 2 * h
        hi_max = 1.0 - 2 * h
        hi_max = np.array([hi_max[0], min(hi_max[1], y_max), hi_max[2]])
        span = hi_max - lo_min - size
        if np.any(span <= 0):
            continue
        lo = lo_min + rng.uniform(0.0, 1.0, size=3) * span
        hi = lo + size
        ok = True
        for (blo, bhi) in boxes:
            gap = np.maximum(blo - hi, lo - bhi)  # per-axis separation
            if np.max(gap / h) < gap_cells:
                ok = False
                break
        if ok:
            boxes.append((lo, hi))
    xc = (np.arange(nx) + 0.5) * h[0]
    yc = (np.arange(ny) + 0.5) * h[1]
    zc = (np.arange(nz) + 0.5) * h[2]
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    mask = np.zeros((nz, ny, nx), dtype=np.uint8)
    for lo, hi in boxes:
        inside = ((X > lo[0]) & (X < hi[0]) & (Y > lo[1]) & (Y < hi[1]) &
                  (Z > lo[2]) & (Z < hi[2]))
        mask[inside] = 1
    return np.array([[lo, hi] for lo, hi in boxes]), mask


def _face_positions(n: int, staggered: bool) -> np.ndarray:
    """Coordinates (in cell units of the unit interval) of stored positions."""
    if staggered:
        return np.arange(n + 1) / n
    return (np.arange(n) + 0.5) / n


def upsample_cavity(state: List[np.ndarray], n_from: int, n_to: int,
                    u_lid: float = 1.0) -> List[np.ndarray]:
    """Trilinear resampling of a wall-bounded cavity state (all six faces walls,
    lid on y = 1 moving along +x) from n_from^3 to n_to^3 cells.

    Each staggered component is interpolated at its own fine positions.  Beyond
    the outermost coarse nodes the tangential components take the wall-reflected
    ghost value (2 u_wall - mirror), which pins the interpolant to the wall
    speed at the wall; the normal components are zero on their wall faces.  The
    pressure is reset to zero.
    """
    out = []
    for c in range(3):
        a = np.asarray(state[c], dtype=np.float64)
        # pad tangential axes with one ghost layer on each side
        pads = []
        coords_from = []
        coords_to = []
        for d in range(3):  # x, y, z
            ax = 2 - d
            if d == c:
                pads.append((0, 0))
                coords_from.append(_face_positions(n_from, True))
                coords_to.append(_face_positions(n_to, True))
            else:
                pads.append((1, 1))
                cf = _face_positions(n_from, False)
                coords_from.append(np.concatenate([[cf[0] - 1.0 / n_from], cf,
                                                   [cf[-1] + 1.0 / n_from]]))
                coords_to.append(_face_positions(n_to, False))
        pad_width = [pads[2], pads[1], pads[0]]
        ap = np.pad(a, pad_width)
        for d in range(3):
            if d == c:
                continue
            ax = 2 - d
            lo = [slice(None)] * 3
            lo_src = [slice(None)] * 3
            hi = [slice(None)] * 3
            hi_src = [slice(None)] * 3
            lo[ax] = 0
            lo_src[ax] = 1
            hi[ax] = -1
            hi_src[ax] = -2
            wall_hi = u_lid if (c == 0 and d == 1) else 0.0
            ap[tuple(lo)] = -ap[tuple(lo_src)]
            ap[tuple(hi)] = 2.0 * wall_hi - ap[tuple(hi_src)]
        # separable linear interpolation along x, y, z
        res = ap
        for d in range(3):
            ax = 2 - d
            xf = coords_from[d]
            xt = coords_to[d]
            idx = np.clip(np.searchsorted(xf, xt) - 1, 0, len(xf) - 2)
            t = (xt - xf[idx]) / (xf[idx + 1] - xf[idx])
            shp = [1, 1, 1]
            shp[ax] = -1
            t = t.reshape(shp)
            res = np.take(res, idx, axis=ax) * (1 - t) + np.take(res, idx + 1, axis=ax) * t
        res = np.ascontiguousarray(res)
        _zero_boundary_faces(res, c, (WALL, WALL, WALL))
        out.append(res)
    out.append(np.zeros((n_to, n_to, n_to)))
    return out


def add_face_noise(state: List[np.ndarray], sigma: float, seed: int,
                   bc=(WALL, WALL, WALL)) -> List[np.ndarray]:
    """state + N(0, sigma^2) on every face that is not a wall-normal boundary face."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for c in range(3):
        noise = rng.standard_normal(state[c].shape) * sigma
        _zero_boundary_faces(noise, c, bc)
        out.append(np.asarray(state[c], dtype=np.float64) + noise)
    out.append(np.array(state[3], dtype=np.float64, copy=True))
    return out


def mixed_batch_sizes(count: int = 24, seed: int = 0,
                      sizes: Sequence[int] = (32, 48, 64, 96),
                      re_range: Tuple[float, float] = (100.0, 2000.0)):
    """Independent cavities for a mixed-size batch: (nx, ny, nz) drawn
    independently from `sizes`, Re ~ U[re_range]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = rng.choice(np.asarray(sizes), size=(count, 3))
    res = rng.uniform(re_range[0], re_range[1], size=count)
    return [(int(a), int(b), int(c)) for a, b, c in dims], [float(r) for r in res]
