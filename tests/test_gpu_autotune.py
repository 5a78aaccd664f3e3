"""The tile autotuner on the GPU, and tile_z changing results only at
rounding level (it fixes the reduction order, not the arithmetic)."""
import numpy as np
import pytest

from paper_1705_06149_gb300 import Grid, inputs
from paper_1705_06149_gb300.autotune import autotune_tile_z

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_autotune_times_the_seeded_candidates():
    r = autotune_tile_z(32, 32, 32, batch=2, top=2, steps=1,
                        grid_kwargs={"re": 500.0, "precision": "fp32_refine"})
    seeded = [c for c, _ in r["seed"][:2]]
    assert set(r["ms_per_step"]) == set(seeded)
    assert r["tile_z"] in seeded
    assert all(t > 0 for t in r["ms_per_step"].values())


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32_refine", 1e-5)])
def test_tile_z_changes_results_only_at_rounding_level(prec, tol):
    init = inputs.random_state(24, 20, 16, seed=3, sigma=0.2)
    out = []
    for tz in (2, 8):
        g = Grid(24, 20, 16, re=300.0, precision=prec, tile_z=tz)
        st = g.state_from(init)
        g.step_fine(st, 1e-3, 3)
        out.append(st.numpy())
    for c in range(4):
        a, b = np.ravel(out[0][c][0]), np.ravel(out[1][c][0])
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b), c


@pytest.mark.parametrize("prec", ["fp64", "fp32_refine"])
def test_predictor_tiles_agree_to_rounding(prec):
    """Every face is evaluated from the same operands whatever the tile, so
    every predictor tile the autotuner may choose gives the same predictor
    and steps up to rounding (the compiler may fuse products into
    multiply-adds differently per instantiated shape)."""
    from paper_1705_06149_gb300.autotune import PREDICT_TILES
    dims = (40, 24, 20)  # ragged against every tile
    init = inputs.random_state(*dims, seed=5, sigma=0.3)
    ref = None
    for tile in PREDICT_TILES:
        g = Grid(*dims, re=300.0, precision=prec, batch=2, predict_tile=tile)
        st = g.state_from([np.stack([a, a]) for a in init])
        f = g.predict(st, 1e-3)
        g.step_fine(st, 1e-3, 2)
        torch.cuda.synchronize()
        got = [t.clone() for t in f] + [t.clone() for t in st.fields()]
        if ref is None:
            ref = got
        else:
            # the predictor alone agrees to a few ulps; two steps carry those
            # through the pressure solves (conditioning ~1e3)
            tol = 1e-11 if prec == "fp64" else 1e-5
            for a, b in zip(got, ref):
                a, b = a.double(), b.double()
                assert float((a - b).norm()) <= tol * float(b.norm()), tile
        g.close()


def test_predictor_tile_outside_the_instantiated_set_is_rejected():
    from paper_1705_06149_gb300 import NSError
    from paper_1705_06149_gb300 import _native as N
    with pytest.raises(NSError) as e:
        Grid(16, 16, 16, predict_tile=(2, 2))
    assert e.value.status == N.NS_ERR_ARG


def test_autotune_3d_times_seeded_tiles_and_caches(tmp_path, monkeypatch):
    from paper_1705_06149_gb300 import autotune as at
    monkeypatch.setenv("NS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    r = at.autotune(48, 32, 32, batch=2, precision="fp32_refine", top=2, steps=1,
                    grid_kwargs={"re": 500.0})
    assert not r["cached"]
    seeded_tiles = [tuple(t) for t, _ in r["seed"]["predict"][:2]]
    seeded_z = [t for t, _ in r["seed"]["tile_z"][:2]]
    assert tuple(r["predict_tile"]) in seeded_tiles
    assert r["tile_z"] in seeded_z
    assert len(r["ms"]["predict"]) == 2 and len(r["ms"]["step"]) == 2
    assert r["seed"]["sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    again = at.autotune(48, 32, 32, batch=2, precision="fp32_refine", top=2, steps=1,
                        grid_kwargs={"re": 500.0})
    assert again["cached"]
    assert tuple(again["predict_tile"]) == tuple(r["predict_tile"])
    assert again["tile_z"] == r["tile_z"]


def test_parareal_autotuner_times_seeded_pairs_and_caches(tmp_path, monkeypatch):
    from paper_1705_06149_gb300 import autotune as at
    monkeypatch.setenv("NS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    args = (16, 16, 16, 8, 10, 2, 1e-3)
    kw = dict(precision="fp32_refine", coarse_candidates=(2, 8), iterations=2,
              grid_kwargs={"re": 400.0})
    r = at.autotune_parareal(*args, **kw)
    assert not r["cached"]
    seeded = [t for t, _ in r["seed"][:2]]
    assert set(r["ms_per_iteration"]) == {f"{t}/{c}" for t in seeded for c in (2, 8)}
    assert r["tile_z"] in seeded and r["coarse_tile_z"] in (2, 8)
    assert all(t > 0 for t in r["ms_per_iteration"].values())
    again = at.autotune_parareal(*args, **kw)
    assert again["cached"]
    assert (again["tile_z"], again["coarse_tile_z"]) == (r["tile_z"], r["coarse_tile_z"])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32_refine", 1e-5)])
def test_coarse_tile_z_changes_parareal_only_at_rounding_level(prec, tol):
    """The coarse propagator's march fixes the order of its reductions only:
    Parareal iterates with coarse_tile_z 2 and 8 agree to rounding after two
    iterations, and after K = N = 4 every slice is the serial fine solution
    on both, bit for bit (the same fine kernels on the same inputs)."""
    init = inputs.random_state(16, 16, 16, seed=5, sigma=0.2)
    half, full = [], []
    for ctz in (2, 8):
        g = Grid(16, 16, 16, re=300.0, precision=prec, batch=4, coarse_tile_z=ctz)
        u0 = g.state_from(init)
        g.project(u0)
        ys = g.zeros(5)
        k, _ = g.parareal(u0, ys, 4, 10, 2, 1e-3, kmax=2)
        assert k == 2
        half.append(ys.clone())
        k, _ = g.parareal(u0, ys, 4, 10, 2, 1e-3, kmax=2, resume=True)
        assert k == 2
        full.append(ys)
        g.close()
    for c in range(4):
        a, b = half[0].fields()[c].double(), half[1].fields()[c].double()
        assert float((a - b).norm()) <= tol * float(b.norm()), c
        assert torch.equal(full[0].fields()[c], full[1].fields()[c]), c
