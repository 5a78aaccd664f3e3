"""The C ABI library builds, loads and exports every declared entry point
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "ns.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ns_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = declared_entry_points()
    for want in ("ns_create_grid", "ns_step_fine", "ns_step_coarse", "ns_parareal_iterate",
                 "ns_adjoint", "ns_last_error"):
        assert want in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    from paper_1705_06149_gb300 import build as nb
    from paper_1705_06149_gb300 import _native
    path = nb.build()
    lib = ctypes.CDLL(path)
    for name in declared_entry_points():
        assert hasattr(lib, name), name
    assert set(declared_entry_points()) == set(_native.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True)
    if out.returncode == 0:
        exported = set(re.findall(r"\bT (ns_[a-z_]+)\b", out.stdout))
        assert set(declared_entry_points()) <= exported


def test_peaks_library_exports_its_declared_probe():
    from paper_1705_06149_gb300 import build as nb
    nb.build()
    src = open(os.path.join(ROOT, "include", "ns_peaks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = sorted(set(re.findall(r"\b(nsp_[a-z_]+)\s*\(", src)))
    assert names == ["nsp_fma_probe"]
    lib = ctypes.CDLL(nb.PEAKS_LIB)
    for name in names:
        assert hasattr(lib, name), name


def test_last_error_is_empty_string_initially():
    from paper_1705_06149_gb300 import _native
    lib = _native.load(build_if_missing=True)
    assert isinstance(lib.ns_last_error(), bytes)


def test_create_grid_rejects_bad_descriptions_without_a_gpu():
    # argument validation happens before any CUDA call
    from paper_1705_06149_gb300 import _native as N
    lib = N.load(build_if_missing=True)
    d = N.GridDesc()
    d.nx, d.ny, d.nz = 1, 8, 8
    d.lx = d.ly = d.lz = 1.0
    d.re = 100.0
    d.batch = 1
    d.poisson_rtol = 1e-12
    h = ctypes.c_void_p()
    assert lib.ns_create_grid(ctypes.byref(d), None, ctypes.byref(h)) == N.NS_ERR_ARG
    assert b"at least 2 cells" in lib.ns_last_error()
    d.nx = 8
    d.re = -1.0
    assert lib.ns_create_grid(ctypes.byref(d), None, ctypes.byref(h)) == N.NS_ERR_ARG
    d.re = 100.0
    d.batch = 0
    assert lib.ns_create_grid(ctypes.byref(d), None, ctypes.byref(h)) == N.NS_ERR_ARG
    assert not h.value


def test_input_generators_are_seeded_and_shaped():
    import numpy as np
    from paper_1705_06149_gb300 import inputs
    a = inputs.random_state(5, 4, 3, seed=9)
    b = inputs.random_state(5, 4, 3, seed=9)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert [x.shape for x in a] == [(3, 4, 6), (3, 5, 5), (4, 4, 5), (3, 4, 5)]
    assert np.all(a[0][..., 0] == 0) and np.all(a[0][..., -1] == 0)
    boxes, mask = inputs.obstacle_boxes((32, 32, 32), seed=0, count=4)
    assert boxes.shape == (4, 2, 3) and mask.any()
    assert np.all(boxes[:, 1, 1] <= 0.8 + 1e-12)


def test_binding_structs_have_the_header_layout(tmp_path):
    """The ctypes mirrors of ns_grid_desc, ns_state and ns_stats have the
    size and field offsets the C compiler gives the header's structs."""
    import shutil
    from paper_1705_06149_gb300 import _native as N
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"ns_grid_desc": N.GridDesc, "ns_state": N.StateC, "ns_stats": N.Stats}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "ns.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(line.rsplit(" ", 1) for line in
               subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for cname, py in mirrors.items():
        assert int(got[f"{cname} size"]) == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert int(got[f"{cname} {f[0]}"]) == getattr(py, f[0]).offset, (cname, f[0])
