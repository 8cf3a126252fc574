"""Randomised properties of the oracle (CPU only): on arbitrary arrays with
edge values mixed in, for every predicate, the compaction equals numpy's
boolean-mask selection by the oracle's own flag map, its length is the
number of set flags, the exclusive scan equals numpy's cumulative sum
shifted by one (mod 2^32), the move phase over (flags, offsets) rebuilds
the compaction, and the three-phase composition agrees. Each property pits
one oracle function against another or against a numpy primitive."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402

EDGES = [0, 1, 2, 3, 4, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFE, 0xFFFFFFFF]
PREDS = [("and_mask_eq0", 3), ("and_mask_eq0", 0), ("lt", 0), ("lt", 1 << 31), ("lt", 0xFFFFFFFF),
         ("topbits_lt", 8), ("topbits_lt", 0), ("popc_odd", 0), ("mod_ne0", 3), ("mod_ne0", 1), ("ne", 0),
         ("ne", 0xFFFFFFFF), ("all", 0)]

arrays = st.lists(st.one_of(st.integers(0, 0xFFFFFFFF), st.sampled_from(EDGES)), max_size=300).map(
    lambda v: np.array(v, dtype=np.uint32))


@settings(max_examples=60, deadline=None)
@given(x=arrays, which=st.integers(0, len(PREDS) - 1))
def test_compaction_is_the_masked_selection(x, which):
    pred, param = PREDS[which]
    f = oracle.predicate_map(x, pred, param)
    assert set(np.unique(f)) <= {0, 1}
    y, k = oracle.compact(x, pred, param)
    assert k == int(f.sum())
    assert np.array_equal(y, x[f.astype(bool)])


@settings(max_examples=60, deadline=None)
@given(x=arrays, which=st.integers(0, len(PREDS) - 1))
def test_scan_and_move_rebuild_the_compaction(x, which):
    pred, param = PREDS[which]
    f = oracle.predicate_map(x, pred, param)
    o, total = oracle.exclusive_scan(f)
    expect = (np.cumsum(f.astype(np.uint64)) - f).astype(np.uint32)
    assert np.array_equal(o, expect) and total == int(f.sum())
    y, k = oracle.compact(x, pred, param)
    assert np.array_equal(oracle.scatter(x, f, o, k), y)
    _, _, tot3, y3 = oracle.three_phase(x, pred, param)
    assert tot3 == k and np.array_equal(y3[:k], y)


@settings(max_examples=40, deadline=None)
@given(v=st.lists(st.integers(0, 0xFFFFFFFF), max_size=200).map(lambda a: np.array(a, dtype=np.uint32)))
def test_scan_of_arbitrary_words_wraps_mod_2_32(v):
    o, total = oracle.exclusive_scan(v)
    s = np.concatenate([[0], np.cumsum(v.astype(np.uint64))]) % (1 << 32)
    assert np.array_equal(o, s[:-1].astype(np.uint32)) and total == int(s[-1])
