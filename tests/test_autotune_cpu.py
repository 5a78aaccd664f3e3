"""The tile autotuner's seed model (host logic, no GPU)."""
from paper_1705_06149_gb300 import autotune as at


def test_surface_per_cell_falls_with_the_tile_height():
    s = [at.surface_per_cell(tz) for tz in (2, 4, 8, 16, 32)]
    assert all(a > b for a, b in zip(s, s[1:]))
    # 32 x 4 x 8 tile with a one-cell halo: 34*6*10 cells read for 1024
    assert abs(at.surface_per_cell(8) - (34 * 6 * 10 - 1024) / 1024) < 1e-15


def test_seed_prefers_tall_tiles_for_a_full_batch_and_short_ones_for_one_state():
    # 64^3 x 32 states: thousands of CTAs either way, so the surface decides
    assert at.seed_order(64, 64, 64, 32)[0][0] == 8
    # one 64^3 state: 256 CTAs at tz = 8 leave most SMs idle
    assert at.seed_order(64, 64, 64, 1)[0][0] == 2


def test_seed_candidates_are_even_and_fit_the_grid():
    order = at.seed_order(32, 32, 5, 1, candidates=(2, 3, 8, 16))
    assert {c for c, _ in order} <= {2, 4}
    assert all(c % 2 == 0 for c, _ in order)
