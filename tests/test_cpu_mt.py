"""The benchmark's multi-threaded CPU compaction (oracle/cpu_mt.c, a context
baseline, not the oracle) gives the oracle's result for any thread count,
including more threads than entries and chunks that keep nothing."""
import numpy as np
import pytest

import ka_inputs as ki
import oracle
from oracle import cpu_mt


@pytest.mark.parametrize("n", [0, 1, 7, 1000, 100003])
@pytest.mark.parametrize("threads", [1, 3, 16])
@pytest.mark.parametrize("t", [0, 1 << 31, 2**32 - 1])
def test_matches_oracle(n, threads, t):
    x = ki.uniform_u32(41, n) if n else np.zeros(0, dtype=np.uint32)
    y, k = cpu_mt.compact_lt(x, t, threads)
    ey, ek = oracle.compact(x, "lt", t)
    assert k == ek and np.array_equal(y, ey)


def test_kept_only_in_one_chunk():
    x = np.full(1000, 100, dtype=np.uint32)
    x[640:660] = np.arange(20, dtype=np.uint32)
    y, k = cpu_mt.compact_lt(x, 20, 8)
    assert k == 20 and np.array_equal(y, np.arange(20, dtype=np.uint32))
