"""The one-CTA multigrid kernel (k_mg_block) run on the host: its source and
that of its helpers, taken verbatim from csrc/ns_mg.cuh, compiled as C++ with
1024 std::threads for the CTA (tests/emu/), under AddressSanitizer and UBSan,
and compared with a plain numpy V(2,0) cycle of the same definition:

  down, per level: y = w b / d, one damped-Jacobi sweep y += w (b - L y) / d,
  residual r = b - L y, coarse right side = mean of the 8 children of r;
  coarsest level: y = 0, then min(32, 8 ceil(nmax / 2)) sweeps;
  up: y += trilinear prolongation (weights 3/4, 1/4 per axis; the cell itself
  beyond a wall, wrapped across a periodic seam),

L the cell-centred Neumann Laplacian (wall faces dropped), d its diagonal,
w = 6/7.  This checks the kernel's index arithmetic and phase order on the CPU
(every shared-memory access inside the block the library allocates) before it
runs on a GPU.  No GPU needed."""
from __future__ import annotations

import os
import re
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1705_06149_gb300", "csrc")
EMU = os.path.join(ROOT, "tests", "emu")

OMEGA = 6.0 / 7.0
WALL, PERIODIC, SLIP = 0, 1, 2


def _extract(src: str, pattern: str) -> str:
    """A top-level definition starting at the line matching `pattern` (with
    a preceding bare `template <...>` line), up to its closing brace."""
    lines = src.split("\n")
    for i, line in enumerate(lines):
        if re.search(pattern, line):
            s = i - 1 if i > 0 and re.match(r"^template <[^>]*>\s*$", lines[i - 1]) else i
            if i > 1 and re.match(r"^__global__", lines[i - 1]) and \
                    re.match(r"^template <[^>]*>\s*$", lines[i - 2]):
                s = i - 2
            depth, seen = 0, False
            for j in range(i, len(lines)):
                depth += lines[j].count("{") - lines[j].count("}")
                seen = seen or "{" in lines[j]
                if seen and depth == 0:
                    return "\n".join(lines[s:j + 1])
                if not seen and lines[j].rstrip().endswith(";"):
                    return "\n".join(lines[s:j + 1])
    raise AssertionError(f"not found in the kernel source: {pattern}")


def _kernel_source() -> str:
    dev = open(os.path.join(CSRC, "ns_device.cuh")).read()
    ker = open(os.path.join(CSRC, "ns_kernels.cuh")).read()
    mg = open(os.path.join(CSRC, "ns_mg.cuh")).read()
    parts = [
        _extract(dev, r"^enum \{ BC_WALL"),
        _extract(ker, r"^enum \{ ST_ITER"),
        _extract(ker, r"^struct SliceCtl \{"),
        _extract(mg, r"^constexpr int MG_MAX_LEVELS"),
        _extract(mg, r"^constexpr double MG_OMEGA"),
        _extract(mg, r"^constexpr int MG_BLOCK_THREADS"),
        _extract(mg, r"^constexpr int MG_COARSEST_SWEEPS"),
        _extract(mg, r"^struct Lev \{"),
        _extract(mg, r"^template <typename T> __device__ __forceinline__ T lw\("),
        _extract(mg, r"^template <> __device__ __forceinline__ float lw<float>"),
        _extract(mg, r"^template <> __device__ __forceinline__ double lw<double>"),
        _extract(mg, r"^struct MgPlan \{"),
        _extract(mg, r"^__device__ __forceinline__ int lindex\("),
        _extract(mg, r"^template <typename T> __device__ __forceinline__ T neg_over\("),
        _extract(mg, r"^template <> __device__ __forceinline__ float neg_over<float>"),
        _extract(mg, r"^template <> __device__ __forceinline__ double neg_over<double>"),
        _extract(mg, r"^__device__ __forceinline__ T diag_at\("),
        _extract(mg, r"^__device__ __forceinline__ int iter_parity\("),
        _extract(mg, r"^__device__ __forceinline__ void tri_axis\("),
        _extract(mg, r"^__device__ __forceinline__ T prolong_off\("),
        _extract(mg, r"^constexpr int MG_BLOCK_PER_THREAD"),
        _extract(mg, r"^constexpr int MG_BLOCK_MAX_CELLS"),
        _extract(mg, r"^struct LevRcp \{"),
        _extract(mg, r"^__device__ __forceinline__ LevRcp lev_rcp\("),
        _extract(mg, r"^__device__ __forceinline__ void lev_ijk\("),
        _extract(mg, r"^__device__ __forceinline__ int blk_pack\("),
        _extract(mg, r"^__device__ __forceinline__ T blk_wd\("),
        _extract(mg, r"^__device__ __forceinline__ T blk_lap\("),
        _extract(mg, r"^__device__ __forceinline__ int mg_coarsest_sweeps\("),
        _extract(mg, r"^__device__ __forceinline__ void mg_coarsest_warp\("),
        _extract(mg, r"^__device__ __forceinline__ void mg_block_core\("),
        _extract(mg, r"^__device__ __forceinline__ void mg_block_levels\("),
        _extract(mg, r"^    k_mg_block\("),
    ]
    src = "\n\n".join(parts)
    shared = "extern __shared__ __align__(16) unsigned char smem_raw[];"
    assert shared in src
    return src.replace(shared, "unsigned char* smem_raw = emu_smem;")


@pytest.fixture(scope="module")
def emulator(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("block_emu")
    cpp = d / "block_emu.cpp"
    cpp.write_text('#include "block_emu.h"\n\n' + _kernel_source() + "\n\n" +
                   open(os.path.join(EMU, "block_emu_main.cpp")).read())
    exe = d / "block_emu"
    cmd = [gxx, "-std=c++20", "-O1", "-g", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer", "-pthread",
           "-I", EMU, str(cpp), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "barrier" in r.stderr and "No such file" in r.stderr:
        pytest.skip("the host compiler has no <barrier>")
    assert r.returncode == 0, r.stderr[-3000:]
    return str(exe), d


# ---------------------------------------------------------------------------
# numpy V(2,0) cycle (float64), arrays indexed [z][y][x]
# ---------------------------------------------------------------------------

def _levels(n0, block_cells):
    levs = [tuple(n0)]
    while all(n % 2 == 0 and n >= 4 for n in levs[-1]):
        levs.append(tuple(n // 2 for n in levs[-1]))
    lc = len(levs) - 1
    for m, n in enumerate(levs):
        if n[0] * n[1] * n[2] <= block_cells:
            lc = m
            break
    return levs, lc


def _lap(y, bc, w):
    s = np.zeros_like(y)
    for d in range(3):
        ax = 2 - d
        hi = np.roll(y, -1, axis=ax)
        lo = np.roll(y, 1, axis=ax)
        if bc[d] != PERIODIC:
            sl_hi = [slice(None)] * 3
            sl_hi[ax] = -1
            hi[tuple(sl_hi)] = y[tuple(sl_hi)]
            sl_lo = [slice(None)] * 3
            sl_lo[ax] = 0
            lo[tuple(sl_lo)] = y[tuple(sl_lo)]
        s += (hi - y) * w[d] - (y - lo) * w[d]
    return s


def _diag(n, bc, w):
    d = np.zeros((n[2], n[1], n[0]))
    for a in range(3):
        idx = np.arange(n[a])
        act = np.full(n[a], 2.0) if bc[a] == PERIODIC else \
            (idx > 0).astype(float) + (idx + 1 < n[a]).astype(float)
        shape = [1, 1, 1]
        shape[2 - a] = n[a]
        d -= w[a] * act.reshape(shape)
    return d


def _prolong(e, nf, bc):
    out = e
    for a in range(3):
        ax = 2 - a
        nc = e.shape[ax]
        f = np.arange(nf[a])
        c0 = f >> 1
        nb = np.where(f & 1, c0 + 1, c0 - 1)
        if bc[a] == PERIODIC:
            c1 = nb % nc
        else:
            c1 = np.where((nb < 0) | (nb >= nc), c0, nb)
        out = 0.75 * np.take(out, c0, axis=ax) + 0.25 * np.take(out, c1, axis=ax)
    return out


def _vcycle(b, levs, lc, bc, ih2_0):
    ys, bs = {}, {lc: b}
    nl = len(levs)
    w = lambda m: [ih2_0[a] * 0.25 ** m for a in range(3)]  # noqa: E731
    for m in range(lc, nl - 1):
        n = levs[m]
        wd = OMEGA / _diag(n, bc, w(m))
        y = wd * bs[m]
        y = y + wd * (bs[m] - _lap(y, bc, w(m)))
        r = bs[m] - _lap(y, bc, w(m))
        bs[m + 1] = r.reshape(n[2] // 2, 2, n[1] // 2, 2, n[0] // 2, 2).mean(axis=(1, 3, 5))
        ys[m] = y
    m = nl - 1
    n = levs[m]
    wd = OMEGA / _diag(n, bc, w(m))
    y = np.zeros((n[2], n[1], n[0]))
    for _ in range(min(32, 4 * ((max(n) + 1) // 2) * 2)):
        y = y + wd * (bs[m] - _lap(y, bc, w(m)))
    ys[m] = y
    for m in range(nl - 2, lc - 1, -1):
        ys[m] = ys[m] + _prolong(ys[m + 1], levs[m], bc)
    return ys[lc]


CASES = [
    ((12, 12, 12), (WALL,) * 3, 4096),       # the smoke grid: 12^3 > 6^3 > 3^3 (27 cells)
    ((12, 12, 12), (WALL,) * 3, 512),        # one-CTA levels from 6^3 (FP64 setting)
    ((64, 64, 64), (WALL,) * 3, 4096),       # the bench grid's 16^3 > 8^3 > 4^3 > 2^3
    ((16, 12, 8), (PERIODIC, WALL, WALL), 4096),
    ((24, 20, 18), (WALL, PERIODIC, WALL), 4096),
    ((8, 8, 8), (PERIODIC,) * 3, 4096),
    ((16, 16, 16), (SLIP, WALL, SLIP), 4096),
    ((4, 4, 2), (WALL,) * 3, 4096),          # a single level of 32 cells (warp path)
    ((40, 24, 8), (WALL,) * 3, 4096),        # coarsest 10 x 6 x 2 (120 cells, CTA path)
    ((1024, 2, 2), (WALL,) * 3, 4096),       # longest extent a one-CTA level may have
]


@pytest.mark.parametrize("prec", ["f", "d"])
@pytest.mark.parametrize("n0,bc,block_cells", CASES)
def test_block_kernel_matches_numpy_vcycle(emulator, n0, bc, block_cells, prec):
    exe, d = emulator
    levs, lc = _levels(n0, block_cells)
    nlc = levs[lc]
    rng = np.random.default_rng(hash((n0, bc, block_cells)) % 2 ** 32)
    b = rng.normal(size=(nlc[2], nlc[1], nlc[0]))
    dt = np.float32 if prec == "f" else np.float64
    fin, fout = d / f"in_{os.getpid()}.bin", d / f"out_{os.getpid()}.bin"
    b.astype(dt).tofile(fin)
    r = subprocess.run([exe, prec, *map(str, n0), *map(str, bc), str(block_cells),
                        str(fin), str(fout)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr[-3000:])
    got_levels = list(map(int, r.stdout.split()))
    assert got_levels[:2] == [lc, len(levs)]
    assert [tuple(got_levels[2 + 3 * i:5 + 3 * i]) for i in range(len(levs) - lc)] == levs[lc:]
    got = np.fromfile(fout, dtype=dt).reshape(b.shape).astype(np.float64)
    ih2_0 = [float(n) * n for n in n0]
    want = _vcycle(b.astype(dt).astype(np.float64), levs, lc, bc, ih2_0)
    scale = np.abs(want).max()
    tol = 2e-5 if prec == "f" else 1e-12
    assert np.abs(got - want).max() <= tol * scale, np.abs(got - want).max() / scale
