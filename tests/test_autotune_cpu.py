"""The tile autotuner's seed model and cache (host logic, no GPU)."""
import json

from paper_1705_06149_gb300 import autotune as at


def test_surface_per_cell_falls_with_the_tile_extents():
    s = [at.surface_per_cell(32, 4, tz) for tz in (2, 4, 8, 16, 32)]
    assert all(a > b for a, b in zip(s, s[1:]))
    # 32 x 4 x 8 tile with a one-cell halo: 34*6*10 cells read for 1024
    assert abs(at.surface_per_cell(32, 4, 8) - (34 * 6 * 10 - 1024) / 1024) < 1e-15
    # the predictor's two-cell halo around 32 x 8 x 4: 36*12*8 staged for 1024
    assert abs(at.surface_per_cell(32, 8, 4, halo=2) - (36 * 12 * 8 - 1024) / 1024) < 1e-15


def test_residency_follows_threads_registers_and_shared_memory():
    assert at.resident_ctas(128, 64, 0) == 8            # register-bound
    assert at.resident_ctas(256, 32, 0) == 8            # thread-bound
    assert at.resident_ctas(256, 32, 100 * 1024) == 2   # shared-memory-bound


def test_seed_prefers_tall_tiles_for_a_full_batch_and_short_ones_for_one_state():
    # 64^3 x 32 states: thousands of CTAs either way, so the surface decides
    assert at.seed_order(64, 64, 64, 32, sms=152)[0][0] == 8
    # one 64^3 state: 256 CTAs at tz = 8 leave most SMs idle
    assert at.seed_order(64, 64, 64, 1, sms=152)[0][0] == 2
    # fewer SMs fill sooner: the taller tile wins for one state on 16 SMs
    assert at.seed_order(64, 64, 64, 1, sms=16)[0][0] > 2


def test_seed_candidates_are_even_and_fit_the_grid():
    order = at.seed_order(32, 32, 5, 1, candidates=(2, 3, 8, 16), sms=152)
    assert {c for c, _ in order} <= {2, 4}
    assert all(c % 2 == 0 for c, _ in order)


def test_predictor_seed_ranks_every_instantiated_tile():
    big = at.predict_seed_order(64, 64, 64, 32, 4, sms=152)
    assert {t for t, _ in big} == set(at.PREDICT_TILES)
    # a full batch fills the GPU with most tiles: a small surface per cell
    # with every SM's slots filled wins (32 x 8 x 8 fits 3 CTAs an SM by
    # shared memory, and its waves leave slots idle)
    assert big[0][0] == (16, 4)
    one = at.predict_seed_order(32, 32, 32, 1, 4, sms=152)
    # one small state leaves SMs idle with any tile: the shortest march per
    # thread (the fewest staged elements per thread) wins
    assert one[0][0] == (8, 2)


def test_cache_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("NS_AUTOTUNE_CACHE", str(path))
    key = at.cache_key(64, 48, 32, 1, "fp32_refine", ("wall",) * 3, "GPU")
    assert key == "64x48x32|b1|fp32_refine|wall,wall,wall|GPU"
    at._store_cache(key, {"predict_tile": [4, 8], "tile_z": 2})
    at._store_cache("other", {"predict_tile": [8, 4], "tile_z": 8})
    data = json.loads(path.read_text())
    assert data[key] == {"predict_tile": [4, 8], "tile_z": 2}
    assert at._load_cache()["other"]["tile_z"] == 8


def test_parareal_candidates_pair_seeded_sweep_marches_with_the_chain_candidates():
    # the pipelined schedule sweeps half the slices per launch: the sweep's
    # candidates are the seed's best marches for that batch, not the full one
    pairs = at.parareal_candidates(64, 64, 64, 32, top=2, coarse_candidates=(4, 8), sms=152)
    half = [t for t, _ in at.seed_order(64, 64, 64, 16, sms=152)[:2]]
    assert pairs == [(tz, ctz) for tz in half for ctz in (4, 8)]
    assert len(set(pairs)) == 4
    # an odd slice count rounds the chunk up
    assert at.parareal_candidates(32, 32, 32, 7, top=1, coarse_candidates=(8,), sms=152) == \
        [(at.seed_order(32, 32, 32, 4, sms=152)[0][0], 8)]
