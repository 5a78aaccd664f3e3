"""GB300-native batched projection stepper and Parareal driver for the 3D
incompressible Navier-Stokes equations (Croce, Ruprecht & Krause, arXiv
1705.06149).

Every step of the computation runs in the hand-written sm_103a kernels of
``libns.so`` (C ABI in ``include/ns.h``); this package only marshals torch
tensors (device memory, the current CUDA stream) into those calls.
"""
from .api import Grid, State, StepGraph, step_fine_many  # noqa: F401
from ._native import NSError, load  # noqa: F401
