"""Serial Parareal loop of the oracle (paper Section 2.1.2, Eq. 6).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Notation follows the paper: y^k_n is the approximation at t_n after iteration k,
F the fine propagator (forward Euler with step delta t), G the coarse propagator
(forward Euler with step Delta t = N_r delta t), and Eq. 6 the update

    y^{k+1}_{n+1} = G(y^{k+1}_n) + F(y^k_n) - G(y^k_n).

The update is evaluated as F(y^k_n) + (G(y^{k+1}_n) - G(y^k_n)), so that when
the two coarse values are bit-identical the new value is F(y^k_n) exactly; the
fixed point of the iteration is the serial fine solution y_{n+1} = F(y_n).
The state y is the full (u, v, w, p) tuple: p is the warm start of the next
pressure solve and its defect is reported alongside the velocity's.
"""
from __future__ import annotations

from typing import Callable, List

import numpy as np

from . import Grid, copy_state

State = List[np.ndarray]


def fine_propagator(grid: Grid, dt_fine: float, steps: int) -> Callable[[State], State]:
    return lambda y: grid.step(copy_state(y), dt_fine, steps)


def coarse_propagator(grid: Grid, dt_coarse: float, steps: int) -> Callable[[State], State]:
    return lambda y: grid.step(copy_state(y), dt_coarse, steps)


def parareal(u0: State, n_slices: int, F: Callable[[State], State],
             G: Callable[[State], State], kmax: int, tol: float = 0.0,
             F_batch: Callable[[List[State]], List[State]] | None = None):
    """Run Parareal from u0 over n_slices slices.

    Returns (y, defects): y is the list y_0..y_N after the last iteration, and
    defects[k] = max over slices n >= 1 and all four fields of
    |y^{k+1}_n - y^k_n|.  The loop stops after kmax iterations, or earlier when
    a defect is <= tol (tol > 0).  kmax = 0 returns the serial coarse sweep.
    """
    # iteration 0: serial coarse sweep y^0_{n+1} = G(y^0_n)
    y = [copy_state(u0)]
    g_old = []
    for n in range(n_slices):
        g = G(y[n])
        g_old.append(g)
        y.append(copy_state(g))
    defects = []
    for _k in range(kmax):
        # fine propagator on every slice, independent of each other
        if F_batch is not None:
            Fy = F_batch([copy_state(y[n]) for n in range(n_slices)])
        else:
            Fy = [F(y[n]) for n in range(n_slices)]
        y_new = [copy_state(u0)]
        d = 0.0
        for n in range(n_slices):
            g = G(y_new[n])
            nxt = [Fy[n][c] + (g[c] - g_old[n][c]) for c in range(4)]
            d = max(d, max(float(np.max(np.abs(nxt[c] - y[n + 1][c]))) for c in range(4)))
            g_old[n] = g
            y_new.append(nxt)
        y = y_new
        defects.append(d)
        if tol > 0.0 and d <= tol:
            break
    return y, defects


def serial_fine(u0: State, n_slices: int, F: Callable[[State], State]):
    """The serial fine solution y_{n+1} = F(y_n) at every slice boundary."""
    y = [copy_state(u0)]
    for n in range(n_slices):
        y.append(F(y[n]))
    return y
