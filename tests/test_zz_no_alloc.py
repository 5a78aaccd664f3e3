"""The allocation-free pressure solve (ns_poisson_solve_noalloc) against the
grid-object solve (ns_poisson_solve), through the C ABI.

This entry point exists for callers that cannot allocate GPU memory when they
need a solve; it keeps its scratch in one fixed device array.  The test calls
it twice in a row (the array keeps the first call's contents) and checks both
results against the regular solve at the FP64 parity tolerance (relative L2
1e-10), and that an oversized grid is rejected.  The file is named so that
pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1705_06149_gb300 import Grid
from paper_1705_06149_gb300 import _native as N

pytestmark = pytest.mark.gpu

MAX_CELLS = 65536  # NS_NOALLOC_MAX_CELLS in include/ns.h


def _noalloc(lib, dims, L, bc, b, p, rtol=1e-12):
    bcs = (ctypes.c_int * 3)(*bc)
    it = ctypes.c_int(0)
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.ns_poisson_solve_noalloc(dims[0], dims[1], dims[2], L[0], L[1], L[2], bcs, rtol, 0,
                                      ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(p.data_ptr()),
                                      ctypes.c_void_p(stream), ctypes.byref(it))
    return st, it.value


def test_noalloc_solve_matches_grid_solve_on_consecutive_calls():
    lib = N.load()
    torch.cuda.set_device(0)
    rng = np.random.default_rng(31)
    cases = [((24, 20, 16), (1.0, 1.0, 1.0), (0, 0, 0)),
             ((30, 17, 12), (1.0, 0.8, 1.3), (1, 0, 2))]
    for dims, L, bc in cases:
        names = {0: "wall", 1: "periodic", 2: "slip"}
        g = Grid(*dims, *L, bc=tuple(names[x] for x in bc), batch=1)
        for call in range(2):
            b = torch.tensor(rng.normal(size=(dims[2], dims[1], dims[0])), device="cuda")
            b_keep = b.clone()
            p0 = torch.tensor(rng.normal(size=b.shape) * 0.1, device="cuda")
            p_ref = p0.clone().unsqueeze(0)
            g.poisson_solve(b.unsqueeze(0).contiguous(), p_ref)
            p = p0.clone()
            st, it = _noalloc(lib, dims, L, bc, b, p)
            assert st == N.NS_OK, (dims, call, st)
            assert it > 0
            assert torch.equal(b, b_keep)  # b is read only
            ref = p_ref[0].cpu().numpy()
            got = p.cpu().numpy()
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert err <= 1e-10, (dims, call, err)
        g.close()


def test_noalloc_rejects_grids_beyond_its_maximum():
    lib = N.load()
    dims = (64, 32, 33)  # 67584 cells > 65536
    assert dims[0] * dims[1] * dims[2] > MAX_CELLS
    b = torch.zeros((dims[2], dims[1], dims[0]), dtype=torch.float64, device="cuda")
    p = torch.zeros_like(b)
    st, _ = _noalloc(lib, dims, (1.0, 1.0, 1.0), (0, 0, 0), b, p)
    assert st == N.NS_ERR_ARG
