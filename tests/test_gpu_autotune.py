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
