"""torch.autograd bridge for the discrete adjoint (ns_adjoint).

KineticEnergy.apply(u, v, w, u_lid, grid, dt, nsteps, ckpt_every) returns the
kinetic-energy objective J = 1/2 sum over active faces of component^2 hx hy hz
after nsteps fine steps from (u, v, w) with lid speed u_lid (a 0-d tensor),
one value per state.  Its backward gives dJ/du0 (every active face) and
dJ/du_lid from the hand-written adjoint kernels.  When a gradient is wanted,
the forward pass runs the adjoint (with checkpointed recomputation) and keeps
the gradients, so backward only scales them by the incoming gradient; when
none is, it runs the fine steps and the objective alone.  The velocity
tensors carry the grid's precision (float64, or float32 on fp32_refine grids).
"""
from __future__ import annotations

import torch

from .api import Grid, State


class KineticEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, v, w, u_lid, grid: Grid, dt: float, nsteps: int, ckpt_every: int = 25):
        grid.set_lid_speed(float(u_lid))
        p = torch.zeros((u.shape[0],) + grid.shapes()[3], dtype=torch.float64, device=u.device)
        st = State(u.detach().contiguous(), v.detach().contiguous(), w.detach().contiguous(), p)
        if not any(ctx.needs_input_grad[:4]):
            fin = st.clone()
            grid.step_fine(fin, dt, nsteps)
            return torch.tensor(grid.kinetic_energy(fin), dtype=torch.float64, device=u.device)
        J, grad, dlid = grid.adjoint(st, dt, nsteps, ckpt_every)
        ctx.save_for_backward(grad.u, grad.v, grad.w,
                              torch.tensor(dlid, dtype=torch.float64, device=u.device))
        return torch.tensor(J, dtype=torch.float64, device=u.device)

    @staticmethod
    def backward(ctx, gJ):
        gu, gv, gw, dlid = ctx.saved_tensors
        scale = gJ.reshape(-1, 1, 1, 1)
        return (gu * scale, gv * scale, gw * scale, (dlid * gJ).sum(), None, None, None, None)


def kinetic_energy(u, v, w, u_lid, grid: Grid, dt: float, nsteps: int, ckpt_every: int = 25):
    return KineticEnergy.apply(u, v, w, u_lid, grid, dt, nsteps, ckpt_every)
