"""FP64 CPU oracle for the projection time-stepper and Parareal (paper Section 2).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It shares
no code with the CUDA library: the stepper is plain C (``ns_oracle.c``), the
Parareal loop is plain Python (``parareal.py``).

State arrays follow the canonical layout (x fastest):
``u[nz][ny][nx+1]``, ``v[nz][ny+1][nx]``, ``w[nz+1][ny][nx]``, ``p[nz][ny][nx]``
(``n`` faces instead of ``n+1`` along a periodic axis), all float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ns_oracle.c")
_LIB = os.path.join(_HERE, "libns_oracle.so")
_lock = threading.Lock()
_lib = None

WALL, PERIODIC, SLIP = 0, 1, 2
_BC_NAMES = {"wall": WALL, "periodic": PERIODIC, "slip": SLIP}

OK, ERR_ARG, ERR_NOT_CONVERGED, ERR_NONFINITE = 0, 1, 4, 5


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile ns_oracle.c into libns_oracle.so (gcc, OpenMP across slices)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        # -O3 without -march=native: the same results on the x86 build host and
        # the Arm GPU host; -ffp-contract=off keeps every product rounded
        cmd = ["gcc", "-O3", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
               "-fopenmp", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("re", ctypes.c_double), ("u_lid", ctypes.c_double),
                ("bc", ctypes.c_int * 3), ("solid", ctypes.c_void_p)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            gp = ctypes.POINTER(_Grid)
            ip = ctypes.POINTER(ctypes.c_int)
            lib.og_vget.restype = ctypes.c_double
            lib.og_vget.argtypes = [gp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int]
            lib.og_smart.restype = ctypes.c_double
            lib.og_smart.argtypes = [ctypes.c_double] * 3
            lib.og_count.restype = ctypes.c_int
            lib.og_count.argtypes = [gp, ctypes.c_int]
            lib.og_predict.argtypes = [gp, dp, dp, dp, ctypes.c_double, dp, dp, dp]
            lib.og_rhs.argtypes = [gp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
            lib.og_divergence.argtypes = [gp, dp, dp, dp, dp]
            lib.og_laplacian.argtypes = [gp, dp, dp]
            lib.og_gradient.argtypes = [gp, dp, dp, dp, dp]
            lib.og_fluid_mean.restype = ctypes.c_double
            lib.og_fluid_mean.argtypes = [gp, dp]
            lib.og_bicgstab.argtypes = [gp, dp, dp, ctypes.c_double, ctypes.c_int, ip, dp]
            lib.og_poisson.argtypes = [gp, dp, dp, ctypes.c_double, ctypes.c_int, ip, dp]
            lib.og_step.argtypes = [gp, dp, dp, dp, dp, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, ip]
            lib.og_run.argtypes = [gp, dp, dp, dp, dp, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_int, ip]
            ppd = ctypes.POINTER(dp)
            lib.og_run_batch.argtypes = [gp, ctypes.c_int, ppd, ppd, ppd, ppd,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_int]
            lib.og_threads.restype = ctypes.c_int
            lib.og_project.argtypes = [gp, dp, dp, dp, dp, ctypes.c_double, ctypes.c_int, ip]
            lib.og_rhs_adjoint.argtypes = [gp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
            lib.og_adjoint.argtypes = [gp, dp, dp, dp, dp, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_int, dp, dp, dp, dp, dp]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle arrays: C-contiguous float64"
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(st: int, what: str):
    if st != OK:
        raise OracleError(f"{what} failed with status {st}")


def smart(U: float, C: float, D: float) -> float:
    """SMART face value from far-upwind U, upwind C and downwind D values."""
    return _load().og_smart(U, C, D)


@dataclass
class Grid:
    """A MAC grid on the box [0,lx]x[0,ly]x[0,lz] with nx x ny x nz cells."""
    nx: int
    ny: int
    nz: int
    lx: float = 1.0
    ly: float = 1.0
    lz: float = 1.0
    re: float = 100.0
    u_lid: float = 1.0
    bc: Sequence[str] = ("wall", "wall", "wall")
    solid: Optional[np.ndarray] = None
    rtol: float = 1e-12
    maxit: int = 0  # 0: 20 * max(n) per solve
    _c: _Grid = field(init=False, repr=False)

    def __post_init__(self):
        self._solid_keep = None
        solid_ptr = None
        if self.solid is not None:
            self._solid_keep = np.ascontiguousarray(self.solid, dtype=np.uint8).reshape(
                self.nz, self.ny, self.nx)
            solid_ptr = self._solid_keep.ctypes.data
        bc = (ctypes.c_int * 3)(*[_BC_NAMES[b] if isinstance(b, str) else int(b) for b in self.bc])
        self._c = _Grid(self.nx, self.ny, self.nz, self.lx, self.ly, self.lz, self.re,
                        self.u_lid, bc, solid_ptr)
        if self.maxit <= 0:
            self.maxit = 20 * max(self.nx, self.ny, self.nz)

    # --- shapes -----------------------------------------------------------
    def shape(self, comp: int):
        """Array shape of component comp (0 u, 1 v, 2 w, 3 p)."""
        n = [self.nx, self.ny, self.nz]
        if comp == 3:
            return (self.nz, self.ny, self.nx)
        ext = [n[d] + (1 if (d == comp and self._c.bc[d] != PERIODIC) else 0) for d in range(3)]
        return (ext[2], ext[1], ext[0])

    def zeros(self):
        return [np.zeros(self.shape(c)) for c in range(4)]

    @property
    def h(self):
        return (self.lx / self.nx, self.ly / self.ny, self.lz / self.nz)

    def _g(self):
        return ctypes.byref(self._c)

    # --- operators --------------------------------------------------------
    def vget(self, c, a, i, j, k):
        """Value of velocity component c of field a at (i, j, k), which may lie
        up to two positions outside the stored range along one axis (the ghost
        rules of the convective stencil)."""
        return _load().og_vget(self._g(), c, _ptr(np.ascontiguousarray(a, dtype=np.float64)),
                               i, j, k)

    def predict(self, u, v, w, dt):
        """F* = u + dt (Re^-1 lap u - div(u u)) on active faces (Section 2)."""
        out = [np.empty(self.shape(c)) for c in range(3)]
        _check(_load().og_predict(self._g(), _ptr(u), _ptr(v), _ptr(w), dt,
                                  *[_ptr(o) for o in out]), "predict")
        return out

    def rhs_terms(self, u, v, w):
        """(conv, diff) per component: div(u u) with SMART faces, and lap u."""
        conv = [np.empty(self.shape(c)) for c in range(3)]
        diff = [np.empty(self.shape(c)) for c in range(3)]
        _check(_load().og_rhs(self._g(), _ptr(u), _ptr(v), _ptr(w),
                              *[_ptr(o) for o in conv], *[_ptr(o) for o in diff]), "rhs")
        return conv, diff

    def divergence(self, u, v, w):
        out = np.empty(self.shape(3))
        _load().og_divergence(self._g(), _ptr(u), _ptr(v), _ptr(w), _ptr(out))
        return out

    def laplacian(self, p):
        out = np.empty(self.shape(3))
        _load().og_laplacian(self._g(), _ptr(p), _ptr(out))
        return out

    def gradient(self, p):
        out = [np.empty(self.shape(c)) for c in range(3)]
        _load().og_gradient(self._g(), _ptr(p), *[_ptr(o) for o in out])
        return out

    def fluid_mean(self, x):
        return _load().og_fluid_mean(self._g(), _ptr(x))

    def bicgstab(self, b, x0, rtol=None, maxit=None):
        """Raw BiCGStab on L x = b from x0; returns (x, iterations, rel. residual)."""
        x = np.array(x0, dtype=np.float64, copy=True)
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0)
        st = _load().og_bicgstab(self._g(), _ptr(np.ascontiguousarray(b)), _ptr(x),
                                 self.rtol if rtol is None else rtol,
                                 self.maxit if maxit is None else maxit,
                                 ctypes.byref(it), ctypes.byref(rr))
        return x, it.value, rr.value, st

    def poisson(self, b, x0=None, rtol=None, maxit=None):
        """Gauged Neumann solve: mean(b) removed first, mean(p) removed after."""
        x = np.zeros(self.shape(3)) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0)
        st = _load().og_poisson(self._g(), _ptr(np.ascontiguousarray(b, dtype=np.float64)),
                                _ptr(x), self.rtol if rtol is None else rtol,
                                self.maxit if maxit is None else maxit,
                                ctypes.byref(it), ctypes.byref(rr))
        _check(st, "poisson")
        return x, it.value

    def project(self, u, v, w, rtol=None):
        """Returns (Pu, Pv, Pw, phi): the discrete Helmholtz projection."""
        u, v, w = (np.array(a, dtype=np.float64, copy=True) for a in (u, v, w))
        phi = np.zeros(self.shape(3))
        it = ctypes.c_int(0)
        _check(_load().og_project(self._g(), _ptr(u), _ptr(v), _ptr(w), _ptr(phi),
                                  self.rtol if rtol is None else rtol, self.maxit,
                                  ctypes.byref(it)), "project")
        return u, v, w, phi

    def rhs_adjoint(self, u, v, w, mu):
        """((dR/du)^T mu per component, (dR/du_lid)^T mu) for R = Re^-1 lap u - div(u u)."""
        out = [np.empty(self.shape(c)) for c in range(3)]
        dl = ctypes.c_double(0)
        _check(_load().og_rhs_adjoint(self._g(), _ptr(u), _ptr(v), _ptr(w),
                                      *[_ptr(np.ascontiguousarray(m)) for m in mu],
                                      *[_ptr(o) for o in out], ctypes.byref(dl)), "rhs_adjoint")
        return out, dl.value

    def adjoint(self, state0, dt, nsteps, rtol=None):
        """(J, dJ/du0 per component, dJ/du_lid) for J = 1/2 sum over active
        faces of component^2 * hx*hy*hz after nsteps fine steps from state0."""
        st = [np.ascontiguousarray(a, dtype=np.float64) for a in state0]
        grads = [np.empty(self.shape(c)) for c in range(3)]
        J = ctypes.c_double(0)
        dl = ctypes.c_double(0)
        _check(_load().og_adjoint(self._g(), *[_ptr(a) for a in st], dt, nsteps,
                                  self.rtol if rtol is None else rtol, self.maxit,
                                  ctypes.byref(J), *[_ptr(o) for o in grads], ctypes.byref(dl)),
               "adjoint")
        return J.value, grads, dl.value

    def kinetic_objective(self, state):
        """J = 1/2 sum over active faces of component^2 * hx*hy*hz."""
        hx, hy, hz = self.h
        vol = hx * hy * hz
        total = 0.0
        for c in range(3):
            a = np.array(state[c], copy=True)
            ax = 2 - c
            if self._c.bc[c] != PERIODIC:
                sl0 = [slice(None)] * 3
                sl1 = [slice(None)] * 3
                sl0[ax] = 0
                sl1[ax] = -1
                a[tuple(sl0)] = 0.0
                a[tuple(sl1)] = 0.0
            total += 0.5 * vol * float(np.sum(a * a))
        return total

    # --- time stepping ----------------------------------------------------
    def step(self, state, dt, nsteps=1, iters=None):
        """Advance state=[u,v,w,p] in place by nsteps forward-Euler projection steps."""
        u, v, w, p = state
        buf = (ctypes.c_int * max(nsteps, 1))()
        st = _load().og_run(self._g(), _ptr(u), _ptr(v), _ptr(w), _ptr(p), dt, nsteps,
                            self.rtol, self.maxit, buf)
        if iters is not None:
            iters.extend(buf[i] for i in range(nsteps))
        _check(st, "step")
        return state

    def run_batch(self, states, dt, nsteps):
        """Advance a list of independent states (OpenMP across states)."""
        lib = _load()
        nb = len(states)
        dp = ctypes.POINTER(ctypes.c_double)
        arrs = [(dp * nb)(*[_ptr(s[c]) for s in states]) for c in range(4)]
        _check(lib.og_run_batch(self._g(), nb, *arrs, dt, nsteps, self.rtol, self.maxit),
               "run_batch")
        return states


def threads() -> int:
    """OpenMP threads the batched oracle runs on."""
    return _load().og_threads()


def copy_state(s):
    return [np.array(a, copy=True) for a in s]
