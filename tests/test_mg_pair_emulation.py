"""The finest-level multigrid kernels that give each thread an x pair of cells
(k_mg_src_pair, k_mg_lapdot_pair, k_mg_update_pair, k_mg_prolong_pair and
the restriction) run on the host: the source of csrc/ns_mg.cuh from its
constants to the last BiCGStab kernel is compiled as C++ (tests/emu/: every
CTA of a grid as 128 std::threads with real barriers, warp shuffles through
per-warp buffers) under AddressSanitizer and UBSan, and each x-pair kernel is
compared with the one-cell-per-thread kernel it replaces on the same seeded
inputs (two states, both iteration parities, restart and zero-start cases):

- the stored vectors (y, p, s, r_hat, v, t, x, r, the prolonged y) must agree
  bit for bit, since every cell's arithmetic is the same;
- the scalars from dot products (alpha, omega, the decision sums) must agree to
  FP32 rounding, since the pair kernels sum in a different order;
- the restriction must agree with a plain loop over the 8 children.

This checks the x-pair index arithmetic (neighbours, walls, periodic seams,
ragged tiles, the state offset) on the CPU.  No GPU needed."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

from test_mg_block_emulation import CSRC, EMU, _extract

WALL, PERIODIC, SLIP = 0, 1, 2


def _source() -> str:
    dev = open(os.path.join(CSRC, "ns_device.cuh")).read()
    ker = open(os.path.join(CSRC, "ns_kernels.cuh")).read()
    mg = open(os.path.join(CSRC, "ns_mg.cuh")).read()
    head = [
        _extract(dev, r"^enum \{ BC_WALL"),
        _extract(dev, r"^constexpr int TX ="),
        _extract(dev, r"^constexpr int TY ="),
        _extract(dev, r"^constexpr int NTHREADS ="),
        _extract(dev, r"^constexpr int NWARPS ="),
        _extract(dev, r"^constexpr int NSUB ="),
        _extract(dev, r"^__device__ __forceinline__ int sub_id\("),
        _extract(dev, r"^__device__ __forceinline__ void sub_sync\("),
        _extract(dev, r"^__device__ __forceinline__ int tid_flat\("),
        _extract(dev, r"^__device__ __forceinline__ void block_sum\("),
        _extract(ker, r"^enum \{ ST_ITER"),
        _extract(ker, r"^struct SliceCtl \{"),
    ]
    a = mg.index("constexpr int MG_MAX_LEVELS")
    start = mg.index("    k_mg_update_pair(")
    end = mg.index("\n}\n", start) + 3
    body = mg[a:end]
    shared = "extern __shared__ __align__(16) unsigned char smem_raw[];"
    assert shared in body
    body = body.replace(shared, "unsigned char* smem_raw = emu_smem;")
    return "\n\n".join(head) + "\n\n" + body


@pytest.fixture(scope="module")
def pair_emulator(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("pair_emu")
    cpp = d / "pair_emu.cpp"
    cpp.write_text('#include "block_emu.h"\n\n' + _source() + "\n\n" +
                   open(os.path.join(EMU, "pair_emu_main.cpp")).read())
    exe = d / "pair_emu"
    cmd = [gxx, "-std=c++20", "-O1", "-g", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer", "-pthread",
           "-I", EMU, str(cpp), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "barrier" in r.stderr and "No such file" in r.stderr:
        pytest.skip("the host compiler has no <barrier>")
    assert r.returncode == 0, r.stderr[-3000:]
    return str(exe)


CASES = [
    ((64, 8, 8), (WALL,) * 3, 8),               # a full 64-wide x tile of pairs
    ((32, 6, 6), (PERIODIC, WALL, SLIP), 4),    # periodic seam in x, ragged y and z tiles
    ((80, 4, 6), (WALL, PERIODIC, PERIODIC), 4),  # ragged x tile (80 = 64 + 16)
    ((16, 10, 4), (PERIODIC, PERIODIC, WALL), 2),  # ragged y tile (10 = 4 + 4 + 2)
]

EXACT = ("src0_y", "src0_p", "src0_p1", "src0_s", "src0_rhat", "src1_y", "src1_p", "src1_p1",
         "src1_rhat", "src2_y", "src2_s", "src3_y", "lapv_v0", "lapv_v1", "lapt_t", "upd_x",
         "upd_r", "upd0_x", "upd0_r", "prolong_y")


@pytest.fixture(scope="module")
def pair_runs(pair_emulator):
    """All cases at once: each run waits mostly on its threads' barriers, so
    they overlap well on the host's cores."""
    procs = {case: subprocess.Popen([pair_emulator, *map(str, case[0]), *map(str, case[1]),
                                     str(case[2])], stdout=subprocess.PIPE,
                                    stderr=subprocess.PIPE, text=True)
             for case in CASES}
    out = {}
    for case, pr in procs.items():
        so, se = pr.communicate(timeout=600)
        out[case] = (pr.returncode, so, se)
    return out


@pytest.mark.parametrize("n,bc,tz", CASES)
def test_pair_kernels_match_cell_kernels(pair_runs, n, bc, tz):
    rc, stdout, stderr = pair_runs[(n, bc, tz)]
    assert rc == 0, (rc, stderr[-3000:])
    res = {}
    for line in stdout.split("\n"):
        if line.strip():
            name, diff, scale = line.split()
            res.setdefault(name, []).append((float(diff), float(scale)))
    for name in EXACT:
        assert name in res, name
        for diff, scale in res[name]:
            assert diff == 0.0, (name, diff, scale)
    for name in ("lapv_alpha", "lapt_omega", "upd_rr", "upd_sx", "upd_rho"):
        for diff, scale in res[name]:
            assert diff <= 1e-5 * max(scale, 1e-30), (name, diff, scale)
    for diff, scale in res["restrict_b"]:
        assert diff <= 2e-5 * scale, ("restrict_b", diff, scale)
