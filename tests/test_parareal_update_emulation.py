"""The Parareal update kernel run on the host: k_parareal_update, taken
verbatim from csrc/ns_kernels.cuh and compiled as C++ with every CTA as host
threads (tests/emu/) under AddressSanitizer and UBSan, against Eq. 6 written
out: y_{n+1} = F(y_n) + (G(y^{k+1}_n) - G(y^k_n)) evaluated in that order
(bit for bit), G_old replaced by G_new, and the defect the largest |change of
y| over all values (bit for bit; a NaN anywhere makes it NaN).  Ragged sizes
and grid-stride loops over fewer threads than values.  No GPU needed."""
from __future__ import annotations

import os
import shutil
import subprocess

import numpy as np
import pytest

from test_mg_block_emulation import CSRC, EMU, _extract


@pytest.fixture(scope="module")
def update_emulator(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    ker = open(os.path.join(CSRC, "ns_kernels.cuh")).read()
    d = tmp_path_factory.mktemp("update_emu")
    cpp = d / "update_emu.cpp"
    cpp.write_text('#include "block_emu.h"\n\n' + _extract(ker, r"^    k_parareal_update\(") +
                   "\n\n" + open(os.path.join(EMU, "update_emu_main.cpp")).read())
    exe = d / "update_emu"
    cmd = [gxx, "-std=c++20", "-O1", "-g", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer", "-pthread",
           "-I", EMU, str(cpp), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "barrier" in r.stderr and "No such file" in r.stderr:
        pytest.skip("the host compiler has no <barrier>")
    assert r.returncode == 0, r.stderr[-3000:]
    return str(exe), d


@pytest.mark.parametrize("n,blocks,nan", [(10007, 3, False), (256, 1, False), (1, 2, False),
                                          (5000, 4, True)])
def test_parareal_update_is_eq6(update_emulator, n, blocks, nan):
    exe, d = update_emulator
    rng = np.random.default_rng(n)
    fy, gnew, gold, y = (rng.normal(size=n) for _ in range(4))
    if nan:
        fy[n // 3] = np.nan
    fin, fout = d / f"in_{n}_{blocks}.bin", d / f"out_{n}_{blocks}.bin"
    np.concatenate([fy, gnew, gold, y]).tofile(fin)
    r = subprocess.run([exe, str(n), str(blocks), str(fin), str(fout)], capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
    out = np.fromfile(fout, dtype=np.float64)
    want_y = fy + (gnew - gold)
    np.testing.assert_array_equal(out[:n], want_y)
    np.testing.assert_array_equal(out[n:2 * n], gnew)
    want_d = np.max(np.abs(want_y - y))  # NaN if any value is NaN
    if nan:
        assert np.isnan(out[-1])
    else:
        assert out[-1] == want_d
