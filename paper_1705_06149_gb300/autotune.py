"""Tile autotuner: the 3D tiles of the stencil and solver kernels for a grid.

The paper splits the domain over processors by minimising the subdomains'
surface (Eq. 2), because the halo a subdomain exchanges grows with it.  On the
GPU the analogue is the CTA tile, and two of them are tunable per grid:

- the predictor's tile, 32 x py x pz cells (one thread per (x, y) column
  marching z, the tile plus a two-cell halo staged in shared memory), with
  (py, pz) among the instantiated shapes;
- the solver kernels' tile, 32 x 4 threads each marching `tile_z` cells along
  z (the multigrid solver's finest level; its x-pair kernels cover 64 x 4).

A taller or deeper tile re-reads fewer halo cells per cell (Eq. 2's surface
per volume falls) but gives each thread more cells and leaves fewer CTAs per
launch, and once a launch has too few CTAs to fill the SMs (the device's SM
count times the CTAs that fit on an SM) its time is the per-CTA latency and
the tile stops paying.  The seed ranks the candidates by that model with
the SM count and residency queried from the device; the tuner then times the
best seeded candidates through the C ABI and keeps the fastest.  Timed choices
are cached per (grid, boundary conditions, precision, batch, device) in a JSON
file (NS_AUTOTUNE_CACHE, else ~/.cache/paper_1705_06149_gb300/autotune.json).

Neither choice changes the method's arithmetic: every face of the predictor
is evaluated from the same operands whatever its tile, and `tile_z` fixes the
order of the solver's per-state reductions, so results move at rounding
level only.
"""
from __future__ import annotations

import json
import math
import os
import time
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

TX, TY = 32, 4                       # threads per CTA of the cell kernels
PT_X = 32                            # predictor tile width
PREDICT_TILES = ((8, 4), (4, 4), (4, 8), (8, 2), (8, 8), (16, 4))
TILE_Z = (2, 4, 8, 16)
SMEM_PER_SM = 228 * 1024             # bytes of shared memory an SM offers CTAs
THREADS_PER_SM = 2048
REGS_PER_SM = 65536
SOLVER_REGS = 64                     # registers per thread of the solver kernels
PREDICT_REGS = 32                    # registers per thread of the predictor


def device_sms(default: int = 152) -> int:
    """The SM count of the current CUDA device (default without one)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.get_device_properties(torch.cuda.current_device())
                       .multi_processor_count)
    except Exception:
        pass
    return default


def resident_ctas(threads: int, regs: int, smem: int) -> int:
    """CTAs of `threads` threads using `regs` registers each and `smem` bytes
    of shared memory that fit on one SM."""
    by_threads = THREADS_PER_SM // threads
    by_regs = REGS_PER_SM // (threads * regs)
    by_smem = SMEM_PER_SM // smem if smem > 0 else 32
    return max(1, min(32, by_threads, by_regs, by_smem))


def surface_per_cell(tx: int, ty: int, tz: int, halo: int = 1) -> float:
    """Halo cells a tx x ty x tz tile reads per interior cell (Eq. 2's surface
    per volume of one subdomain)."""
    vol = tx * ty * tz
    return ((tx + 2 * halo) * (ty + 2 * halo) * (tz + 2 * halo) - vol) / vol


def tile_time_per_cell(cells: int, tile_cells: int, threads: int, surface: float,
                       slots: int, sms: int) -> float:
    """Model time per cell of a launch of `cells` cells in tiles of
    `tile_cells` cells, `threads` threads a CTA, `surface` halo cells read per
    cell and `slots` CTAs resident at once: a CTA's time is the elements each
    of its threads stages, tile_cells (1 + surface) / threads; the launch takes
    the longer of its waves of CTAs (latency-bound, few CTAs) and of its total
    work spread over every thread slot of the GPU (throughput-bound)."""
    ctas = max(1, math.ceil(cells / tile_cells))
    t_cta = tile_cells * (1.0 + surface) / threads
    waves = math.ceil(ctas / slots)
    total = max(waves * t_cta, ctas * t_cta * threads / (sms * THREADS_PER_SM))
    return total / cells


def seed_cost(nx: int, ny: int, nz: int, batch: int, tz: int, sms: int = 152) -> float:
    """Model time per cell of the solver tile 32 x 4 x tz (one-cell halo)."""
    cells = (math.ceil(nx / TX) * TX) * (math.ceil(ny / TY) * TY) * (math.ceil(nz / tz) * tz)
    slots = sms * resident_ctas(TX * TY, SOLVER_REGS, 0)
    return tile_time_per_cell(cells * batch, TX * TY * tz, TX * TY,
                              surface_per_cell(TX, TY, tz), slots, sms)


def predict_seed_cost(nx: int, ny: int, nz: int, batch: int, py: int, pz: int,
                      elem_bytes: int = 4, sms: int = 152) -> float:
    """Model time per cell of the predictor tile 32 x py x pz (two-cell halo,
    three staged components)."""
    threads = PT_X * py
    smem = 3 * (PT_X + 4) * (py + 4) * (pz + 4) * elem_bytes
    cells = (math.ceil(nx / PT_X) * PT_X) * (math.ceil(ny / py) * py) * (math.ceil(nz / pz) * pz)
    slots = sms * resident_ctas(threads, PREDICT_REGS, smem)
    return tile_time_per_cell(cells * batch, PT_X * py * pz, threads,
                              surface_per_cell(PT_X, py, pz, halo=2), slots, sms)


def seed_order(nx: int, ny: int, nz: int, batch: int,
               candidates: Iterable[int] = TILE_Z, sms: Optional[int] = None
               ) -> List[Tuple[int, float]]:
    """tile_z candidates (even, at most nz) ranked by the seed cost, best first."""
    sms = device_sms() if sms is None else sms
    cands = sorted({min(max(2, c & ~1), max(2, nz & ~1)) for c in candidates})
    return sorted(((c, seed_cost(nx, ny, nz, batch, c, sms)) for c in cands),
                  key=lambda x: x[1])


def predict_seed_order(nx: int, ny: int, nz: int, batch: int, elem_bytes: int = 4,
                       sms: Optional[int] = None) -> List[Tuple[Tuple[int, int], float]]:
    """Predictor tiles ranked by the seed cost, best first."""
    sms = device_sms() if sms is None else sms
    return sorted(((t, predict_seed_cost(nx, ny, nz, batch, t[0], t[1], elem_bytes, sms))
                   for t in PREDICT_TILES), key=lambda x: x[1])


# ---------------------------------------------------------------------------
# timed choice and its cache
# ---------------------------------------------------------------------------

def cache_path() -> str:
    p = os.environ.get("NS_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_1705_06149_gb300",
                        "autotune.json")


def cache_key(nx: int, ny: int, nz: int, batch: int, precision: str,
              bc: Sequence[str], device: str) -> str:
    return f"{nx}x{ny}x{nz}|b{batch}|{precision}|{','.join(bc)}|{device}"


def _load_cache() -> Dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store_cache(key: str, value: Dict) -> None:
    path = cache_path()
    data = _load_cache()
    data[key] = value
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = f"{path}.{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home: the choice is still returned


def _stack(a, batch: int):
    import numpy as np
    return np.stack([a] * batch)


def autotune(nx: int, ny: int, nz: int, batch: int = 1, precision: str = "fp32_refine",
             top: int = 3, steps: int = 2, dt: float = 5e-4, grid_kwargs: Optional[dict] = None,
             seed: int = 0, use_cache: bool = True) -> Dict:
    """Chooses the predictor tile and tile_z for a grid by timing the best
    seeded candidates: `top` predictor tiles (their predictor launches alone)
    and `top` tile_z values (`steps` fine steps
    after a warm one).  Returns {"predict_tile": (py, pz), "tile_z": tz,
    "seed": {...}, "ms": {...}, "cached": bool}; timed results are cached."""
    import torch

    from . import inputs
    from .api import Grid
    kw = dict(grid_kwargs or {})
    bc = tuple(kw.get("bc", ("wall", "wall", "wall")))
    dev = torch.cuda.get_device_name(torch.cuda.current_device())
    key = cache_key(nx, ny, nz, batch, precision, bc, dev)
    if use_cache and kw.get("solid") is None:
        hit = _load_cache().get(key)
        if hit:
            return {"predict_tile": tuple(hit["predict_tile"]), "tile_z": hit["tile_z"],
                    "seed": hit.get("seed"), "ms": hit.get("ms"), "cached": True}
    sms = device_sms()
    esz = 4 if precision == "fp32_refine" else 8
    porder = predict_seed_order(nx, ny, nz, batch, esz, sms)
    zorder = seed_order(nx, ny, nz, batch, sms=sms)
    init = inputs.random_state(nx, ny, nz, seed=seed, sigma=0.1, bc=bc, solid=kw.get("solid"))
    ms_pred: Dict[str, float] = {}
    ms_step: Dict[str, float] = {}
    # predictor tiles: time the predictor launches on one grid object each
    best_tz = zorder[0][0]
    for tile, _ in porder[:max(1, top)]:
        g = Grid(nx, ny, nz, batch=batch, precision=precision, tile_z=best_tz,
                 predict_tile=tile, **kw)
        st = g.state_from([_stack(init[c], batch) for c in range(4)])
        g.predict(st, dt)
        torch.cuda.synchronize()
        reps = 5
        t0 = time.perf_counter()
        for _ in range(reps):
            g.predict(st, dt)
        torch.cuda.synchronize()
        ms_pred[f"{tile[0]}x{tile[1]}"] = 1e3 * (time.perf_counter() - t0) / reps
        g.close()
    best_tile = min(porder[:max(1, top)], key=lambda t: ms_pred[f"{t[0][0]}x{t[0][1]}"])[0]
    # tile_z: whole fine steps with the chosen predictor tile
    for tz, _ in zorder[:max(1, top)]:
        g = Grid(nx, ny, nz, batch=batch, precision=precision, tile_z=tz,
                 predict_tile=best_tile, **kw)
        st = g.state_from([_stack(init[c], batch) for c in range(4)])
        g.project(st)
        g.step_fine(st, dt, 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step_fine(st, dt, steps)
        torch.cuda.synchronize()
        ms_step[str(tz)] = 1e3 * (time.perf_counter() - t0) / steps
        g.close()
    best_tz = int(min(ms_step, key=ms_step.get))
    out = {"predict_tile": tuple(best_tile), "tile_z": best_tz,
           "seed": {"predict": [[list(t), c] for t, c in porder],
                    "tile_z": [[t, c] for t, c in zorder], "sms": sms},
           "ms": {"predict": ms_pred, "step": ms_step}, "cached": False}
    if use_cache and kw.get("solid") is None:
        _store_cache(key, {k: v for k, v in out.items() if k != "cached"})
    return out


def autotune_tile_z(nx: int, ny: int, nz: int, batch: int = 1, top: int = 3, steps: int = 3,
                    dt: float = 5e-4, candidates: Iterable[int] = TILE_Z,
                    grid_kwargs: Optional[dict] = None, seed: int = 0) -> Dict:
    """tile_z alone (the predictor tile left at its default): times `steps`
    fine steps (after one warm step) of a seeded state for the `top`
    seed-ranked candidates; returns {"tile_z": best, "seed": [...],
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


COARSE_TILE_Z = (4, 8)


def parareal_candidates(nx: int, ny: int, nz: int, slices: int, top: int = 2,
                        coarse_candidates: Iterable[int] = COARSE_TILE_Z,
                        sms: Optional[int] = None) -> List[Tuple[int, int]]:
    """The (tile_z, coarse_tile_z) pairs autotune_parareal times: the `top`
    seeded tile_z values for a batch of half the slices (the pipelined
    schedule's chunks), each with every coarse candidate."""
    order = seed_order(nx, ny, nz, (slices + 1) // 2, sms=sms)
    return [(tz, ctz) for tz, _ in order[:max(1, top)] for ctz in coarse_candidates]


def autotune_parareal(nx: int, ny: int, nz: int, slices: int, fine_steps: int,
                      coarse_steps: int, dt: float, precision: str = "fp32_refine",
                      coarse_candidates: Iterable[int] = COARSE_TILE_Z, top: int = 2,
                      iterations: int = 3, init=None, grid_kwargs: Optional[dict] = None,
                      seed: int = 0, use_cache: bool = True) -> Dict:
    """Chooses the fine sweep's tile_z and the coarse propagator's
    coarse_tile_z for ns_parareal_iterate by timing Parareal iterations.

    A call of two or more iterations sweeps the slices in two chunks pipelined
    with the coarse chain, so the sweep's candidates are the `top` seeded
    tile_z values for a batch of half the slices; the chain shares the GPU
    with the sweeps, and which march suits it then is measured rather than
    modelled (the seed model assumes a launch has the SMs to itself), over
    `coarse_candidates`.  Each pair is timed over `iterations` iterations of
    one call after the coarse sweep and a warm call of two iterations, from
    `init` (u, v, w, p of one state; default a seeded random state).  Returns
    {"tile_z", "coarse_tile_z", "ms_per_iteration": {"tz/ctz": ms}, "seed",
    "cached"}; timed results are cached."""
    import torch

    from . import inputs
    from .api import Grid
    kw = dict(grid_kwargs or {})
    bc = tuple(kw.get("bc", ("wall", "wall", "wall")))
    dev = torch.cuda.get_device_name(torch.cuda.current_device())
    key = (cache_key(nx, ny, nz, slices, precision, bc, dev) +
           f"|parareal|S{fine_steps}|M{coarse_steps}|dt{dt:g}")
    if use_cache and kw.get("solid") is None:
        hit = _load_cache().get(key)
        if hit:
            return {"tile_z": hit["tile_z"], "coarse_tile_z": hit["coarse_tile_z"],
                    "ms_per_iteration": hit.get("ms_per_iteration"), "seed": hit.get("seed"),
                    "cached": True}
    order = seed_order(nx, ny, nz, (slices + 1) // 2)
    if init is None:
        init = inputs.random_state(nx, ny, nz, seed=seed, sigma=0.1, bc=bc,
                                   solid=kw.get("solid"))
    times: Dict[str, float] = {}
    for tz, ctz in parareal_candidates(nx, ny, nz, slices, top, coarse_candidates):
        g = Grid(nx, ny, nz, batch=slices, precision=precision, tile_z=tz, coarse_tile_z=ctz,
                 **kw)
        u0 = g.state_from(init)
        g.project(u0)
        ys = g.zeros(slices + 1)
        g.parareal(u0, ys, slices, fine_steps, coarse_steps, dt, kmax=0)
        g.parareal(u0, ys, slices, fine_steps, coarse_steps, dt, kmax=2, resume=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.parareal(u0, ys, slices, fine_steps, coarse_steps, dt, kmax=iterations, resume=True)
        torch.cuda.synchronize()
        times[f"{tz}/{ctz}"] = 1e3 * (time.perf_counter() - t0) / iterations
        g.close()
    best = min(times, key=times.get)
    tz, ctz = (int(x) for x in best.split("/"))
    out = {"tile_z": tz, "coarse_tile_z": ctz, "ms_per_iteration": times,
           "seed": [[t, c] for t, c in order], "cached": False}
    if use_cache and kw.get("solid") is None:
        _store_cache(key, {k: v for k, v in out.items() if k != "cached"})
    return out
