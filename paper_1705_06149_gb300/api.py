"""Python binding of the C ABI: torch tensors in, the same calls out.

Only argument marshalling lives here: shapes and dtypes are checked, device
pointers and the current CUDA stream are handed to libns.so, and host (CPU)
tensors are staged through device memory for the end-to-end calls.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch

from . import _native as N
from .inputs import shapes as _shapes

_BC = {"wall": N.NS_BC_WALL, "periodic": N.NS_BC_PERIODIC, "slip": N.NS_BC_SLIP}
_PREC = {"fp64": N.NS_FP64, "fp32_refine": N.NS_FP32_REFINE}


@dataclass
class State:
    """A batch of states (u, v, w, p) in the canonical layout."""
    u: torch.Tensor
    v: torch.Tensor
    w: torch.Tensor
    p: torch.Tensor

    @property
    def batch(self) -> int:
        return int(self.u.shape[0])

    def fields(self) -> List[torch.Tensor]:
        return [self.u, self.v, self.w, self.p]

    def clone(self) -> "State":
        return State(*[t.clone() for t in self.fields()])

    def to(self, device, non_blocking: bool = False) -> "State":
        return State(*[t.to(device, non_blocking=non_blocking) for t in self.fields()])

    def numpy(self) -> List[np.ndarray]:
        return [t.detach().cpu().numpy() for t in self.fields()]

    def slice(self, i: int, n: int = 1) -> "State":
        return State(*[t[i:i + n] for t in self.fields()])

    def _c(self) -> N.StateC:
        return N.StateC(self.u.data_ptr(), self.v.data_ptr(), self.w.data_ptr(),
                        self.p.data_ptr(), self.batch)


class Grid:
    """One MAC grid with its workspace on the current CUDA device.

    precision: "fp64" (all FP64) or "fp32_refine" (FP32 velocity, stencils and
    inner Krylov iterations; FP64 pressure, refinement residual/correction,
    means and defects).  batch is the largest number of states one call
    advances (the number of Parareal slices).  preconditioner: "multigrid"
    (BiCGStab with one V-cycle as right preconditioner) or "none" (plain
    BiCGStab).
    """

    def __init__(self, nx: int, ny: int, nz: int, lx: float = 1.0, ly: float = 1.0,
                 lz: float = 1.0, re: float = 100.0, u_lid: float = 1.0,
                 bc: Sequence[str] = ("wall", "wall", "wall"), precision: str = "fp64",
                 poisson_rtol: float = 1e-12, poisson_maxit: int = 0,
                 refine_rtol: float = 1e-10, inner_rtol: float = 3e-4, batch: int = 1,
                 preconditioner: str = "multigrid", solid: Optional[np.ndarray] = None,
                 tile_z: int = 0, parareal_chunk: int = 0, refine_maxit: int = 0,
                 predict_tile: Tuple[int, int] = (0, 0), coarse_tile_z: int = 0,
                 device: Optional[torch.device] = None):
        self.lib = N.load()
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.nx, self.ny, self.nz = nx, ny, nz
        self.bc = tuple(bc)
        self.precision = precision
        self.capacity = batch
        self.vel_dtype = torch.float32 if precision == "fp32_refine" else torch.float64
        desc = N.GridDesc()
        desc.nx, desc.ny, desc.nz = nx, ny, nz
        desc.lx, desc.ly, desc.lz = lx, ly, lz
        desc.re, desc.u_lid = re, u_lid
        for a in range(3):
            desc.bc[a] = _BC[bc[a]] if isinstance(bc[a], str) else int(bc[a])
        self._solid = None
        if solid is not None:
            self._solid = np.ascontiguousarray(np.asarray(solid, dtype=np.uint8).reshape(nz, ny, nx))
            desc.solid_mask = self._solid.ctypes.data
        else:
            desc.solid_mask = None
        desc.precision = _PREC[precision]
        desc.poisson_rtol = poisson_rtol
        desc.poisson_maxit = poisson_maxit
        desc.refine_rtol = refine_rtol
        desc.inner_rtol = inner_rtol
        desc.batch = batch
        desc.preconditioner = {"none": N.NS_PC_NONE, "multigrid": N.NS_PC_MULTIGRID}[preconditioner]
        desc.refine_maxit = refine_maxit
        desc.tile_z = tile_z
        desc.parareal_chunk = parareal_chunk
        desc.predict_tile_y, desc.predict_tile_z = int(predict_tile[0]), int(predict_tile[1])
        desc.coarse_tile_z = int(coarse_tile_z)
        self.preconditioner = preconditioner
        self._desc = desc
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream(self.device).cuda_stream
            h = ctypes.c_void_p()
            N.check(self.lib.ns_create_grid(ctypes.byref(desc), ctypes.c_void_p(stream),
                                            ctypes.byref(h)), "ns_create_grid")
        self._h = h
        self._stream = stream

    # --- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.ns_destroy_grid(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _sync_stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        if s != self._stream:
            N.check(self.lib.ns_set_stream(self._h, ctypes.c_void_p(s)), "ns_set_stream")
            self._stream = s

    # --- states -----------------------------------------------------------
    def shapes(self):
        return _shapes(self.nx, self.ny, self.nz, self.bc)

    def zeros(self, batch: int = 1, device=None) -> State:
        dev = self.device if device is None else device
        shp = self.shapes()
        return State(*[torch.zeros((batch,) + s, dtype=self.vel_dtype, device=dev)
                       for s in shp[:3]],
                     torch.zeros((batch,) + shp[3], dtype=torch.float64, device=dev))

    def state_from(self, arrays: Sequence, device=None) -> State:
        """State from per-field arrays shaped [batch][...] or [...] (batch 1)."""
        dev = self.device if device is None else device
        shp = self.shapes()
        out = []
        for c, a in enumerate(arrays):
            t = torch.as_tensor(np.asarray(a))
            if t.dim() == 3:
                t = t.unsqueeze(0)
            assert tuple(t.shape[1:]) == shp[c], (t.shape, shp[c])
            dt = torch.float64 if c == 3 else self.vel_dtype
            out.append(t.to(device=dev, dtype=dt).contiguous())
        return State(*out)

    def _check(self, st: State, what: str):
        shp = self.shapes()
        for c, t in enumerate(st.fields()):
            want = torch.float64 if c == 3 else self.vel_dtype
            if t.dtype != want or not t.is_contiguous() or t.device != self.device:
                raise ValueError(f"{what}: field {c} must be a contiguous {want} tensor on "
                                 f"{self.device}")
            if tuple(t.shape[1:]) != shp[c] or t.shape[0] != st.batch:
                raise ValueError(f"{what}: field {c} has shape {tuple(t.shape)}, expected "
                                 f"[batch]{shp[c]}")

    # --- the C ABI calls ------------------------------------------------------
    def step_fine(self, st: State, dt: float, nsteps: int) -> State:
        self._check(st, "step_fine")
        self._sync_stream()
        N.check(self.lib.ns_step_fine(self._h, st._c(), dt, nsteps), "ns_step_fine")
        return st

    def step_coarse(self, st: State, dt: float, nsteps: int) -> State:
        self._check(st, "step_coarse")
        self._sync_stream()
        N.check(self.lib.ns_step_coarse(self._h, st._c(), dt, nsteps), "ns_step_coarse")
        return st

    def project(self, st: State) -> State:
        self._check(st, "project")
        self._sync_stream()
        N.check(self.lib.ns_project(self._h, st._c()), "ns_project")
        return st

    def predict(self, st: State, dt: float) -> Tuple[torch.Tensor, torch.Tensor, torch.Tensor]:
        self._check(st, "predict")
        self._sync_stream()
        out = [torch.empty_like(t) for t in (st.u, st.v, st.w)]
        N.check(self.lib.ns_predict(self._h, st._c(), dt, *[o.data_ptr() for o in out]),
                "ns_predict")
        return tuple(out)

    def poisson_solve(self, b: torch.Tensor, p: torch.Tensor) -> int:
        """Gauged solve of L p = b for a batch; p is the warm start and the output."""
        for t in (b, p):
            if t.dtype != torch.float64 or not t.is_contiguous() or t.device != self.device:
                raise ValueError("poisson_solve: b and p must be contiguous float64 on device")
        if b.dim() == 3:
            b, p = b.unsqueeze(0), p.unsqueeze(0)
        self._sync_stream()
        it = ctypes.c_int(0)
        N.check(self.lib.ns_poisson_solve(self._h, b.data_ptr(), p.data_ptr(), int(b.shape[0]),
                                          ctypes.byref(it)), "ns_poisson_solve")
        return it.value

    def parareal(self, u0: State, slices: State, n_slices: int, fine_steps: int,
                 coarse_steps: int, dt_fine: float, kmax: int, tol: float = 0.0,
                 resume: bool = False):
        """Parareal (Eq. 6).  Returns (iterations done, list of defects)."""
        self._check(u0, "parareal(u0)")
        self._check(slices, "parareal(slices)")
        self._sync_stream()
        k = ctypes.c_int(0)
        d = (ctypes.c_double * max(kmax, 1))()
        N.check(self.lib.ns_parareal_iterate(self._h, u0._c(), slices._c(), n_slices, fine_steps,
                                             coarse_steps, dt_fine, kmax, tol, int(resume),
                                             ctypes.byref(k), d), "ns_parareal_iterate")
        return k.value, [d[i] for i in range(k.value)]

    def parareal_host(self, u0: State, slices_host: State, n_slices: int, fine_steps: int,
                      coarse_steps: int, dt_fine: float, kmax: int, tol: float = 0.0,
                      resume: bool = False, slices_dev: Optional[State] = None):
        """End-to-end Parareal with the slices in host memory: copies them to
        the device (from pinned memory when they are pinned), runs, copies
        them back.  Returns (iterations, defects, bytes H2D, bytes D2H)."""
        dev = slices_dev if slices_dev is not None else self.zeros(slices_host.batch)
        h2d = 0
        for src, dst in zip(slices_host.fields(), dev.fields()):
            dst.copy_(src, non_blocking=True)
            h2d += src.numel() * src.element_size()
        k, d = self.parareal(u0, dev, n_slices, fine_steps, coarse_steps, dt_fine, kmax, tol,
                             resume)
        d2h = 0
        for src, dst in zip(dev.fields(), slices_host.fields()):
            dst.copy_(src, non_blocking=True)
            d2h += src.numel() * src.element_size()
        torch.cuda.current_stream(self.device).synchronize()
        return k, d, h2d, d2h

    def kinetic_energy(self, st: State) -> List[float]:
        """J = 1/2 sum over active faces of component^2 * hx*hy*hz per state."""
        self._check(st, "kinetic_energy")
        self._sync_stream()
        J = (ctypes.c_double * st.batch)()
        N.check(self.lib.ns_kinetic_energy(self._h, st._c(), J), "ns_kinetic_energy")
        return [J[i] for i in range(st.batch)]

    def adjoint(self, u0: State, dt: float, nsteps: int, ckpt_every: int = 25):
        """Discrete adjoint of nsteps fine steps (FP64, or FP32 storage with
        FP64-accurate refinement on fp32_refine grids).  Returns
        (J per state, gradient State (u, v, w; p zero), dJ/du_lid per state)
        for J = 1/2 sum over active faces of component^2 * hx*hy*hz."""
        self._check(u0, "adjoint(u0)")
        self._sync_stream()
        B = u0.batch
        J = (ctypes.c_double * B)()
        dl = (ctypes.c_double * B)()
        grad = self.zeros(B)
        N.check(self.lib.ns_adjoint(self._h, u0._c(), dt, nsteps, ckpt_every, J, grad._c(), dl),
                "ns_adjoint")
        return [J[i] for i in range(B)], grad, [dl[i] for i in range(B)]

    def set_lid_speed(self, u_lid: float):
        N.check(self.lib.ns_set_lid_speed(self._h, float(u_lid)), "ns_set_lid_speed")

    def stats(self) -> dict:
        s = N.Stats()
        N.check(self.lib.ns_get_stats(self._h, ctypes.byref(s)), "ns_get_stats")
        return {f: getattr(s, f) for f, _ in N.Stats._fields_}

    def reset_stats(self):
        N.check(self.lib.ns_reset_stats(self._h), "ns_reset_stats")

    def profile(self, on: bool, min_batch: int = 1):
        """Per-launch CUDA-event timing of calls with batch >= min_batch."""
        N.check(self.lib.ns_profile_enable(self._h, int(on), int(min_batch)),
                "ns_profile_enable")

    def profile_read(self) -> dict:
        arr = (N.KernelTime * len(N.KERNEL_KINDS))()
        N.check(self.lib.ns_profile_read(self._h, arr, len(N.KERNEL_KINDS)), "ns_profile_read")
        return {k: {"ms": arr[i].ms, "launches": arr[i].launches,
                    "cell_units": arr[i].cell_units}
                for i, k in enumerate(N.KERNEL_KINDS)}


def step_fine_many(branches):
    """Advance several grids at once: for each (grid, state, dt, nsteps), what
    grid.step_fine(state, dt, nsteps) computes, every grid on a stream and host
    thread of its own so their kernels overlap."""
    lib = N.load()
    grids = [b[0] for b in branches]
    for g, b in zip(grids, branches):
        g._sync_stream()
        g._check(b[1], "step_fine_many")
    n = len(branches)
    N.check(lib.ns_step_fine_many((ctypes.c_void_p * n)(*[g._h.value for g in grids]),
                                  (N.StateC * n)(*[b[1]._c() for b in branches]),
                                  (ctypes.c_double * n)(*[float(b[2]) for b in branches]),
                                  (ctypes.c_int * n)(*[int(b[3]) for b in branches]), n),
            "ns_step_fine_many")


class StepGraph:
    """A CUDA graph of fine steps of several grids, one concurrent branch per
    (grid, state, dt, nsteps): each launch advances every state exactly as
    grid.step_fine(state, dt, nsteps) would, with every solver loop resident
    on the device (conditional while nodes).  The states' buffers are captured:
    keep them alive, and do not reallocate them, while the graph exists."""

    def __init__(self, branches):
        self.lib = N.load()
        self._grids = [b[0] for b in branches]
        self._states = [b[1] for b in branches]  # keeps the captured buffers alive
        n = len(branches)
        for g, st in zip(self._grids, self._states):
            g._sync_stream()
            g._check(st, "StepGraph")
        grids = (ctypes.c_void_p * n)(*[g._h.value for g in self._grids])
        states = (N.StateC * n)(*[st._c() for st in self._states])
        dts = (ctypes.c_double * n)(*[float(b[2]) for b in branches])
        steps = (ctypes.c_int * n)(*[int(b[3]) for b in branches])
        h = ctypes.c_void_p()
        N.check(self.lib.ns_graph_create(grids, states, dts, steps, n, ctypes.byref(h)),
                "ns_graph_create")
        self._h = h

    def launch(self, stream=None):
        s = stream if stream is not None else torch.cuda.current_stream()
        N.check(self.lib.ns_graph_launch(self._h, ctypes.c_void_p(s.cuda_stream)),
                "ns_graph_launch")

    def check(self, stream=None):
        s = stream if stream is not None else torch.cuda.current_stream()
        N.check(self.lib.ns_graph_check(self._h, ctypes.c_void_p(s.cuda_stream)),
                "ns_graph_check")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            torch.cuda.synchronize()
            self.lib.ns_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
