"""The issue order of Parareal iterations pipelined across iterations
(csrc/ns_pipeline.h, the host logic the library runs with CUDA streams and
events) replayed on the CPU: the stream operations it issues for C chunks and
K iterations, with and without an early stop at a defect tolerance, are
turned into a happens-before graph (stream order, and each event wait bound
to the event's latest record issued before it, as CUDA binds it), and every
pair of operations that touch the same data with at least one write must be
ordered by it the way the unpipelined iteration orders them: per iteration
the copy of y into the F buffers and the fine sweep of every chunk, then the
chain of every chunk (which reads F and y of the chunk's first slice and
writes y of its other slices and of the next chunk's first slice, the coarse
state, and the defect).  No GPU needed."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1705_06149_gb300", "csrc")
EMU = os.path.join(ROOT, "tests", "emu")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path_factory.mktemp("pipeline") / "pipeline_emu"
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC,
                        os.path.join(EMU, "pipeline_emu_main.cpp"), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return str(exe)


def issue(exe, C, K, check, stop):
    out = subprocess.run([exe, str(C), str(K), str(int(check)), str(stop)], capture_output=True,
                         text=True, check=True).stdout.split("\n")
    ops = [line.split() for line in out if line]
    assert ops[-1][0] == "issued"
    return ops[:-1], int(ops[-1][1])


def accesses(kind, c, C):
    """(item, write?) of one operation on chunk c."""
    if kind == "copy":
        return [(("yfirst", c), False), (("yrest", c), False), (("F", c), True)]
    if kind == "sweep":
        return [(("F", c), False), (("F", c), True), ("workspace", True)]
    if kind == "chain":
        nxt = ("yfirst", c + 1) if c + 1 < C else ("ylast",)
        return [(("F", c), False), (("yfirst", c), False), (("yrest", c), True), (nxt, True),
                ("coarse", True), (("gold", c), True), ("defect", True)]
    if kind == "reset":
        return [("defect", True)]
    if kind == "out":
        return [("defect", False)]
    return []


def check_order(ops, C, iterations):
    # label the work operations with their iteration (per chunk, in issue order)
    count = {"copy": [0] * C, "sweep": [0] * C, "chain": [0] * C}
    nodes = []        # (label, stream, deps)
    last = {}         # stream -> last node
    records = {}      # (kind, chunk) -> node of its latest record
    pending = {"S": [], "C": []}
    resets = outs = 0
    for op in ops:
        if op[0] == "conv":
            continue
        if op[0] == "wait":
            r = records.get((int(op[2]), int(op[3])))
            if r is not None:
                pending[op[1]].append(r)
            continue
        if op[0] == "record":
            st = op[1]
            label = ("record", int(op[2]), int(op[3]))
        elif op[0] in count:
            c = int(op[1])
            st = "C" if op[0] == "chain" else "S"
            label = (op[0], count[op[0]][c], c)
            count[op[0]][c] += 1
        elif op[0] == "reset":
            st, label = "C", ("reset", resets, 0)
            resets += 1
        else:
            st, label = "C", ("out", int(op[1]), 0)
            outs += 1
        deps = set(pending[st])
        pending[st] = []
        if st in last:
            deps.add(last[st])
        n = len(nodes)
        nodes.append((label, st, deps))
        last[st] = n
        if label[0] == "record":
            records[(label[1], label[2])] = n
    # transitive happens-before
    before = []
    for _, _, deps in nodes:
        s = set()
        for d in deps:
            s.add(d)
            s |= before[d]
        before.append(s)
    index = {lab: i for i, (lab, _, _) in enumerate(nodes) if lab[0] != "record"}
    # the unpipelined order of the same work (a speculative sweep of the
    # iteration after the last one at the end)
    ref = []
    for k in range(iterations):
        for c in range(C):
            ref += [("copy", k, c), ("sweep", k, c)]
        ref.append(("reset", k, 0))
        ref += [("chain", k, c) for c in range(C)]
        ref.append(("out", k, 0))
    for c in range(C):
        if count["sweep"][c] > iterations:
            ref += [("copy", iterations, c), ("sweep", iterations, c)]
    assert sorted(ref) == sorted(index), "the pipelined run issues other work"
    assert resets == outs == iterations
    for i, a in enumerate(ref):
        for b in ref[i + 1:]:
            acc_a = accesses(a[0], a[2], C)
            acc_b = accesses(b[0], b[2], C)
            conflict = any(x == y and (wx or wy) for x, wx in acc_a for y, wy in acc_b)
            if conflict:
                assert index[a] in before[index[b]], f"{a} not ordered before {b}"


CASES = [(2, 1), (2, 2), (2, 5), (3, 3), (4, 4), (5, 2)]


@pytest.mark.parametrize("C,K", CASES)
def test_pipelined_order_matches_the_unpipelined_dependencies(driver, C, K):
    ops, k = issue(driver, C, K, False, 0)
    assert k == K
    check_order(ops, C, K)
    # the sweeps run one after another (they share the grid's workspace) and
    # at most one sweep runs ahead of the last iteration
    assert sum(1 for o in ops if o[0] == "sweep") == C * K


@pytest.mark.parametrize("C,K,stop", [(2, 5, 2), (2, 5, 1), (3, 4, 3), (4, 6, 2), (2, 3, 3)])
def test_pipelined_order_stops_at_the_tolerance(driver, C, K, stop):
    ops, k = issue(driver, C, K, True, stop)
    assert k == min(stop, K)
    check_order(ops, C, k)
    # the defect of iteration n is read (conv n) before any chain of iteration
    # n + 1 is issued, and iterations stop at the first one that meets it
    conv_at = {int(o[1]): i for i, o in enumerate(ops) if o[0] == "conv"}
    assert sorted(conv_at) == list(range(min(stop, K - 1)))
    chains = [i for i, o in enumerate(ops) if o[0] == "chain"]
    for n, i in conv_at.items():
        later = chains[(n + 1) * C:(n + 2) * C]
        assert all(i < j for j in later)
    # beyond the last iteration at most chunk 0's sweep was issued
    extra = sum(1 for o in ops if o[0] == "sweep") - C * k
    assert extra in (0, 1)
