"""Tile autotuner: cells per thread along z (`tile_z`) for a grid and batch.

The paper splits the domain over processors by minimising the subdomains'
surface (Eq. 2), because the halo a subdomain exchanges grows with it.  On
the GPU the analogue is the CTA tile: 32 x 4 threads, each marching `tile_z`
cells along z.  A taller tile re-reads fewer halo cells per cell (its surface
per volume falls), but leaves fewer CTAs per launch, and once a launch has
too few CTAs to fill the SMs (152 on a GB300) the tile stops paying.  The
seed ranks the candidates by that model; the tuner then times a few fine
steps of each of the best ones through the C ABI and keeps the fastest.
"""
from __future__ import annotations

import math
import time
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

TX, TY = 32, 4          # threads per CTA in x and y (the kernels' tiling)
CTA_SLOTS = 152 * 8     # SMs x CTAs of 128 threads resident per SM (register-bound)


def surface_per_cell(tz: int) -> float:
    """Halo cells a 32 x 4 x tz tile reads per interior cell (one-cell halo)."""
    vol = TX * TY * tz
    halo = (TX + 2) * (TY + 2) * (tz + 2) - vol
    return halo / vol


def seed_cost(nx: int, ny: int, nz: int, batch: int, tz: int) -> float:
    """Relative cost per cell of `tile_z = tz`: the halo surface per cell
    (Eq. 2's quantity for one tile), times the waves a launch takes over the
    waves it would take if its CTAs filled every slot."""
    ctas = math.ceil(nx / TX) * math.ceil(ny / TY) * math.ceil(nz / tz) * batch
    waves = math.ceil(ctas / CTA_SLOTS)
    fill = ctas / (waves * CTA_SLOTS)
    return (1.0 + surface_per_cell(tz)) / fill


def seed_order(nx: int, ny: int, nz: int, batch: int,
               candidates: Iterable[int] = (2, 4, 8, 16)) -> List[Tuple[int, float]]:
    """Candidates (even, at most nz) ranked by the seed cost, best first."""
    cands = sorted({min(max(2, c & ~1), max(2, nz & ~1)) for c in candidates})
    return sorted(((c, seed_cost(nx, ny, nz, batch, c)) for c in cands), key=lambda x: x[1])


def autotune_tile_z(nx: int, ny: int, nz: int, batch: int = 1, top: int = 3, steps: int = 3,
                    dt: float = 5e-4, candidates: Iterable[int] = (2, 4, 8, 16),
                    grid_kwargs: Optional[dict] = None, seed: int = 0) -> Dict:
    """Time `steps` fine steps (after one warm step) of a seeded state for the
    `top` seed-ranked candidates; returns {"tile_z": best, "seed": [...],
    "ms_per_step": {tz: ms}}.  grid_kwargs go to Grid (re, precision, bc...)."""
    import torch

    from . import inputs
    from .api import Grid
    kw = dict(grid_kwargs or {})
    bc = kw.get("bc", ("wall", "wall", "wall"))
    order = seed_order(nx, ny, nz, batch, candidates)
    init = inputs.random_state(nx, ny, nz, seed=seed, sigma=0.1, bc=bc,
                               solid=kw.get("solid"))
    times: Dict[int, float] = {}
    for tz, _ in order[:max(1, top)]:
        g = Grid(nx, ny, nz, batch=batch, tile_z=tz, **kw)
        st = g.state_from([_stack(init[c], batch) for c in range(4)])
        g.project(st)
        g.step_fine(st, dt, 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step_fine(st, dt, steps)
        torch.cuda.synchronize()
        times[tz] = 1e3 * (time.perf_counter() - t0) / steps
        g.close()
    best = min(times, key=times.get)
    return {"tile_z": best, "seed": order, "ms_per_step": times}


def _stack(a, batch: int):
    import numpy as np
    return np.stack([a] * batch)
