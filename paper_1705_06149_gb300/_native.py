"""ctypes view of the C ABI in include/ns.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

NS_OK, NS_ERR_ARG, NS_ERR_CUDA, NS_ERR_OOM, NS_ERR_NOT_CONVERGED, NS_ERR_NONFINITE, \
    NS_ERR_TIMEOUT = range(7)
NS_FP64, NS_FP32_REFINE = 0, 1
NS_BC_WALL, NS_BC_PERIODIC, NS_BC_SLIP = 0, 1, 2
NS_PC_NONE, NS_PC_MULTIGRID = 0, 1

STATUS_NAMES = {0: "NS_OK", 1: "NS_ERR_ARG", 2: "NS_ERR_CUDA", 3: "NS_ERR_OOM",
                4: "NS_ERR_NOT_CONVERGED", 5: "NS_ERR_NONFINITE", 6: "NS_ERR_TIMEOUT"}

# every entry point declared in include/ns.h
EXPORTS = ("ns_create_grid", "ns_destroy_grid", "ns_set_stream", "ns_step_fine",
           "ns_step_coarse", "ns_project", "ns_predict", "ns_poisson_solve",
           "ns_parareal_iterate", "ns_adjoint", "ns_get_stats", "ns_reset_stats",
           "ns_profile_enable", "ns_profile_read", "ns_poisson_solve_noalloc",
           "ns_set_lid_speed", "ns_kinetic_energy", "ns_step_fine_many", "ns_graph_create", "ns_graph_launch", "ns_graph_check",
           "ns_graph_destroy", "ns_last_error")

KERNEL_KINDS = ("predict", "divergence", "solve_init", "krylov_A", "krylov_B", "krylov_C",
                "inner_init", "refine", "correct", "parareal", "mg_lap_v", "mg_lap_t",
                "mg_restrict0", "mg_prolong0", "mg_coarse", "adjoint", "mg_block",
                "persist", "mg_cluster")


class NSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("re", ctypes.c_double), ("u_lid", ctypes.c_double),
                ("bc", ctypes.c_int * 3), ("solid_mask", ctypes.c_void_p),
                ("precision", ctypes.c_int), ("poisson_rtol", ctypes.c_double),
                ("poisson_maxit", ctypes.c_int), ("refine_rtol", ctypes.c_double),
                ("inner_rtol", ctypes.c_double), ("refine_maxit", ctypes.c_int),
                ("batch", ctypes.c_int),
                ("preconditioner", ctypes.c_int), ("tile_z", ctypes.c_int),
                ("parareal_chunk", ctypes.c_int),
                ("predict_tile_y", ctypes.c_int), ("predict_tile_z", ctypes.c_int),
                ("coarse_tile_z", ctypes.c_int)]


class StateC(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("p", ctypes.c_void_p), ("batch", ctypes.c_int)]


class KernelTime(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("launches", ctypes.c_longlong),
                ("cell_units", ctypes.c_longlong)]


class Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("steps", ctypes.c_longlong), ("solves", ctypes.c_longlong),
                ("krylov_iters", ctypes.c_longlong), ("refine_steps", ctypes.c_longlong),
                ("last_max_iters", ctypes.c_int), ("last_rel_residual", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libns.so; raises if it is missing (there is no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if build_if_missing:
                _build.build()
            else:
                raise RuntimeError(
                    f"CUDA library {path} is missing: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'` "
                    "(there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
        gpp = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "ns_create_grid": [ctypes.POINTER(GridDesc), vp, gpp],
            "ns_destroy_grid": [vp],
            "ns_set_stream": [vp, vp],
            "ns_step_fine": [vp, StateC, ctypes.c_double, ctypes.c_int],
            "ns_step_coarse": [vp, StateC, ctypes.c_double, ctypes.c_int],
            "ns_project": [vp, StateC],
            "ns_predict": [vp, StateC, ctypes.c_double, vp, vp, vp],
            "ns_poisson_solve": [vp, vp, vp, ctypes.c_int, ip],
            "ns_parareal_iterate": [vp, StateC, StateC, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                    ip, dp],
            "ns_adjoint": [vp, StateC, ctypes.c_double, ctypes.c_int, ctypes.c_int, vp, StateC,
                           vp],
            "ns_get_stats": [vp, ctypes.POINTER(Stats)],
            "ns_set_lid_speed": [vp, ctypes.c_double],
            "ns_kinetic_energy": [vp, StateC, dp],
            "ns_reset_stats": [vp],
            "ns_profile_enable": [vp, ctypes.c_int, ctypes.c_int],
            "ns_profile_read": [vp, ctypes.POINTER(KernelTime), ctypes.c_int],
            "ns_step_fine_many": [vp, vp, dp, ip, ctypes.c_int],
            "ns_graph_create": [vp, vp, dp, ip, ctypes.c_int, gpp],
            "ns_graph_launch": [vp, vp],
            "ns_graph_check": [vp, vp],
            "ns_graph_destroy": [vp],
            "ns_poisson_solve_noalloc": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ip, ctypes.c_double,
                                         ctypes.c_int, vp, vp, vp, ip],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        lib.ns_last_error.argtypes = []
        lib.ns_last_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


def check(status: int, what: str = ""):
    if status != NS_OK:
        msg = _lib.ns_last_error().decode() if _lib is not None else ""
        raise NSError(status, f"{what}: {msg}" if what else msg)
