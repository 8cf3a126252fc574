"""The seeded input module: its stream matches the published SplitMix64 check
values, and each workload recipe has the sizes and ranges it promises."""
import numpy as np

import ka_inputs as ki
import oracle_pins as pins


def test_stream_matches_published_values():
    seed, vals = pins._golden_splitmix()
    got = ki.splitmix64(seed, np.arange(len(vals), dtype=np.uint64))
    assert [int(v) for v in got] == vals
    assert [int(v) for v in ki.uniform_u32(seed, len(vals))] == [v >> 32 for v in vals]


def test_offset_start_is_a_window_of_the_same_stream():
    a = ki.uniform_u32(9, 100)
    b = ki.uniform_u32(9, 40, start=60)
    assert np.array_equal(a[60:], b)


def test_thresholds():
    assert ki.threshold_for(0.0) == 0
    assert ki.threshold_for(0.5) == 1 << 31
    assert ki.threshold_for(1.0) == 0xFFFFFFFF
    assert ki.threshold_for(0.01) == int(0.01 * 2**32)


def test_batch_recipe():
    b = ki.config_batch()
    assert b.n.size == 4096
    assert b.n.min() >= 256 and b.n.max() <= 1 << 20
    assert 0.01 <= b.selectivity.min() and b.selectivity.max() < 0.99
    assert np.unique(b.seeds).size == 4096
    # mean of floor(2^U), U ~ U[8, 20): (2^20 - 2^8) / (12 ln 2) ~ 1.26e5
    assert 0.8e5 < b.n.mean() < 1.7e5


def test_serve_recipe():
    tr = ki.config_serve(rate_hz=20000.0, duration_s=1.0)
    r = tr.arrival_s.size
    assert 19000 * 0.9 < r < 21000 * 1.1
    assert np.all(np.diff(tr.arrival_s) >= 0)
    assert tr.n.min() >= 1 << 10 and tr.n.max() <= 1 << 24
    assert set(np.unique(tr.n_stages)) <= {1, 2, 3, 4}
    assert tr.stage_kind.shape == (r, 4) and tr.stage_kind.max() <= 3


def test_index_pairs_zero_fraction():
    a, b = ki.index_pairs(100000, 0.25)
    frac = ((a == 0).sum() + (b == 0).sum()) / 200000
    assert abs(frac - 0.25) < 0.01
