"""The loop-condition kernel of the graph-resident pressure solves
(k_loop_cond) run on the host: one warp of host threads, taken verbatim from
csrc/ns_mg.cuh and compiled as C++ (tests/emu/) under AddressSanitizer and
UBSan, with the graph's conditional handle replaced by a variable.  Checked
on batches below and above one warp (the grid-stride over states) against the
rule the solver's while loops need:

- a start mode resets the body count, an iteration mode adds one to it and
  to the running total;
- the loop runs again while any state is iterating (FP64) or still refining
  (FP32 + refinement) and the body count is below the cap;
- when the loop ends, a state that did not converge gets the sticky bit 1, a
  non-finite one the bit 2, the refinement steps are added to its total and
  its solve is counted.

No GPU needed."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

from test_mg_block_emulation import CSRC, EMU, _extract

ST_ITER, ST_CONV, ST_MAXIT, ST_NONFINITE, ST_IDLE = 0, 1, 2, 3, 4
OS_REFINE, OS_DONE, OS_FAIL, OS_NONFINITE = 0, 1, 2, 3
LC_FP64_START, LC_FP64_ITER, LC_REFINE_START, LC_REFINE_ITER = 0, 1, 2, 3

PRELUDE = """
using cudaGraphConditionalHandle = unsigned long long;
unsigned emu_cond = 99;
// the kernel must pass on the handle it was given (7 below)
inline void cudaGraphSetConditional(cudaGraphConditionalHandle h, unsigned v) {
    emu_cond = h == 7ull ? v : 98u;
}
"""


def _source() -> str:
    ker = open(os.path.join(CSRC, "ns_kernels.cuh")).read()
    mg = open(os.path.join(CSRC, "ns_mg.cuh")).read()
    head = [_extract(ker, r"^enum \{ ST_ITER"), _extract(ker, r"^enum \{ OS_REFINE"),
            _extract(ker, r"^struct SliceCtl \{")]
    a = mg.index("struct LoopCount {")
    start = mg.index("    k_loop_cond(")
    e = mg.index("\n}\n", start) + 3
    return PRELUDE + "\n\n".join(head) + "\n\n" + mg[a:e]


@pytest.fixture(scope="module")
def loop_emulator(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("loop_emu")
    cpp = d / "loop_emu.cpp"
    cpp.write_text('#include "block_emu.h"\n\n' + _source() + "\n\n" +
                   open(os.path.join(EMU, "loop_emu_main.cpp")).read())
    exe = d / "loop_emu"
    cmd = [gxx, "-std=c++20", "-O1", "-g", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer", "-pthread",
           "-I", EMU, str(cpp), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "barrier" in r.stderr and "No such file" in r.stderr:
        pytest.skip("the host compiler has no <barrier>")
    assert r.returncode == 0, r.stderr[-3000:]
    return str(exe), d


def _expected(mode, cap, inner, inner_total, states):
    """The rule, state by state (status, o_status, o_steps, fail, total_outer,
    total_solves)."""
    if mode in (LC_FP64_START, LC_REFINE_START):
        inner = 0
    else:
        inner += 1
        inner_total += 1
    outer = mode in (LC_REFINE_START, LC_REFINE_ITER)
    if outer:
        active = any(s[1] == OS_REFINE for s in states)
    else:
        active = any(s[0] == ST_ITER for s in states)
    go = active and inner < cap
    out = []
    for st, ost, osteps, fail, tot_o, tot_s in states:
        if not go:
            if outer:
                fail |= 2 if ost == OS_NONFINITE else (1 if ost != OS_DONE else 0)
                tot_o += osteps
            else:
                fail |= 2 if st == ST_NONFINITE else (1 if st != ST_CONV else 0)
            tot_s += 1
        out.append((fail, tot_o, tot_s))
    return int(go), inner, inner_total, out


def _state(status=ST_CONV, o_status=OS_DONE, o_steps=0, fail=0, tot_o=5, tot_s=9):
    return (status, o_status, o_steps, fail, tot_o, tot_s)


SCENARIOS = {
    "fp64_start_one_iterating": (LC_FP64_START, 100, 17, 40,
                                 [_state(), _state(ST_ITER), _state(ST_IDLE)]),
    "fp64_iter_all_ended": (LC_FP64_ITER, 100, 3, 40,
                            [_state(ST_CONV), _state(ST_MAXIT), _state(ST_NONFINITE, fail=1),
                             _state(ST_IDLE)]),
    "fp64_iter_cap_reached": (LC_FP64_ITER, 4, 3, 40, [_state(ST_ITER), _state(ST_CONV)]),
    "fp64_iter_below_cap": (LC_FP64_ITER, 5, 3, 40, [_state(ST_ITER), _state(ST_CONV)]),
    "refine_iter_refining": (LC_REFINE_ITER, 100, 8, 40,
                             [_state(ST_CONV, OS_REFINE, 2), _state(ST_CONV, OS_DONE, 3)]),
    "refine_iter_all_ended": (LC_REFINE_ITER, 100, 8, 40,
                              [_state(ST_CONV, OS_DONE, 3), _state(ST_MAXIT, OS_FAIL, 7),
                               _state(ST_NONFINITE, OS_NONFINITE, 1, fail=2)]),
    "refine_start_none_refining": (LC_REFINE_START, 100, 8, 40,
                                   [_state(ST_IDLE, OS_DONE, 0), _state(ST_IDLE, OS_DONE, 0)]),
    # more states than lanes: only a state a lane reaches on its second pass
    "fp64_iter_70_states_one_late": (LC_FP64_ITER, 1000, 10, 40,
                                     [_state(ST_CONV)] * 65 + [_state(ST_ITER)] +
                                     [_state(ST_MAXIT)] * 4),
    "refine_start_70_states_one_late": (LC_REFINE_START, 1000, 10, 40,
                                        [_state(ST_IDLE, OS_DONE, 2)] * 40 +
                                        [_state(ST_IDLE, OS_REFINE, 0)] +
                                        [_state(ST_IDLE, OS_FAIL, 1)] * 29),
    "refine_iter_70_states_ended": (LC_REFINE_ITER, 1000, 10, 40,
                                    [_state(ST_CONV, OS_DONE, q % 4) for q in range(60)] +
                                    [_state(ST_MAXIT, OS_FAIL, 9)] * 10),
}


@pytest.mark.parametrize("name", sorted(SCENARIOS))
def test_loop_condition_follows_rule(loop_emulator, name):
    exe, d = loop_emulator
    mode, cap, inner, inner_total, states = SCENARIOS[name]
    fin = d / f"{name}.txt"
    lines = [f"{mode} {cap} {inner} {inner_total} {len(states)}"]
    lines += [" ".join(map(str, s)) for s in states]
    fin.write_text("\n".join(lines) + "\n")
    r = subprocess.run([exe, str(fin)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr[-3000:])
    rows = [list(map(int, ln.split())) for ln in r.stdout.strip().split("\n")]
    go, inner_w, total_w, per_state = _expected(mode, cap, inner, inner_total, states)
    assert rows[0] == [go, inner_w, total_w], (rows[0], (go, inner_w, total_w))
    assert [tuple(x) for x in rows[1:]] == per_state
