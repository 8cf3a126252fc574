"""Streamed compaction of host memory (ka_compact_host) against the oracle,
bit for bit: several predicates over one upload, many chunks with a ragged
last chunk, pinned and pageable host buffers, the hash transform, inputs
shorter than a chunk, empty input, the full N = 2^28 workload with the
default chunk, and argument errors."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import ka_inputs as ki  # noqa: E402
import oracle  # noqa: E402


@pytest.fixture(scope="module")
def ka(cuda_ok):
    import paper_1709_07781_gb300 as m
    return m


def scratch(ka, chunk, n_pred):
    s, nbytes = ka.ka_compact_host_scratch_size(chunk, n_pred)
    assert s == 0
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    base = (buf.data_ptr() + 255) // 256 * 256
    return buf, base, nbytes


def host_u32(n, pinned):
    if pinned:
        return torch.empty(max(n, 1), dtype=torch.int32, pin_memory=True)
    return np.empty(max(n, 1), dtype=np.uint32)


def as_np(t, k):
    if isinstance(t, np.ndarray):
        return t[:k]
    return t[:k].numpy().view(np.uint32)


def run(ka, x, preds, chunk, pinned=True):
    """preds: list of (pred name, param, xform); returns per predicate (kept, count)."""
    n = x.size
    h_in = host_u32(n, pinned)
    as_np(h_in, n)[:] = x
    outs = [host_u32(n, pinned) for _ in preds]
    buf, base, nbytes = scratch(ka, chunk, len(preds))
    s, counts = ka.ka_compact_host(h_in, n, [ka.PRED[p] for p, _, _ in preds], [q for _, q, _ in preds],
                                   [xf for _, _, xf in preds], outs, chunk, base, nbytes)
    assert s == 0, ka.ka_strerror(s)
    del buf
    return [(as_np(o, k).copy(), k) for o, k in zip(outs, counts)]


def expect(x, pred, param, xform):
    src = oracle.map_hash(x) if xform else x
    return oracle.compact(src, pred, param)


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("n", [1, 4095, 65536, 5 * 65536 + 12345])
def test_several_predicates_many_chunks(ka, n, pinned):
    x = ki.uniform_u32(31, n)
    preds = [("lt", 1 << 31, 0), ("popc_odd", 0, ka.KA_XFORM_HASH), ("and_mask_eq0", 3, 0),
             ("mod_ne0", 3, ka.KA_XFORM_HASH)]
    got = run(ka, x, preds, 65536, pinned)
    for (p, q, xf), (y, k) in zip(preds, got):
        ey, ek = expect(x, p, q, xf)
        assert k == ek and np.array_equal(y, ey), p


@pytest.mark.parametrize("chunk", [4, 1000, 4097, 1 << 20])
def test_chunk_sizes(ka, chunk):
    n = 3 * 4097 + 11
    x = ki.uniform_u32(32, n)
    (y, k), = run(ka, x, [("lt", 3 << 30, 0)], chunk)
    ey, ek = oracle.compact(x, "lt", 3 << 30)
    assert k == ek and np.array_equal(y, ey)


def test_nothing_kept_and_everything_kept(ka):
    x = ki.uniform_u32(33, 200001)
    (y0, k0), (y1, k1) = run(ka, x, [("lt", 0, 0), ("all", 0, 0)], 65536)
    assert k0 == 0
    assert k1 == x.size and np.array_equal(y1, x)


def test_empty_input(ka):
    buf, base, nbytes = scratch(ka, 0, 2)
    out = [np.zeros(1, dtype=np.uint32), np.zeros(1, dtype=np.uint32)]
    s, counts = ka.ka_compact_host(np.zeros(1, dtype=np.uint32), 0, [ka.PRED["all"]] * 2, [0, 0], [0, 0], out, 0,
                                   base, nbytes)
    assert s == 0 and counts == [0, 0]


def test_full_size_default_chunk(ka):
    n = (1 << 28) + 5
    x = ki.uniform_u32(2, n)
    (y, k), = run(ka, x, [("lt", 1 << 31, 0)], 0)
    ey, ek = oracle.compact(x, "lt", 1 << 31)
    assert k == ek and np.array_equal(y, ey)


def test_invalid_arguments(ka):
    buf, base, nbytes = scratch(ka, 1024, 1)
    x = np.zeros(16, dtype=np.uint32)
    out = [np.zeros(16, dtype=np.uint32)]
    lt = ka.PRED["lt"]
    assert ka.ka_compact_host_scratch_size(1024, 0)[0] == ka.KA_E_ARG
    assert ka.ka_compact_host_scratch_size(1024, ka.KA_HOST_MAX_PRED + 1)[0] == ka.KA_E_ARG
    assert ka.ka_compact_host_scratch_size(1 << 33, 1)[0] == ka.KA_E_ARG
    assert ka.ka_compact_host(x, 16, [lt], [5], [0], out, 1024, base, nbytes - 1)[0] == ka.KA_E_WORKSPACE
    assert ka.ka_compact_host(x, 16, [lt], [5], [0], out, 1024, base + 4, nbytes)[0] == ka.KA_E_ARG
    assert ka.ka_compact_host(x, 16, [lt], [5], [7], out, 1024, base, nbytes)[0] == ka.KA_E_ARG
    assert ka.ka_compact_host(x, 16, [99], [5], [0], out, 1024, base, nbytes)[0] != 0
    assert ka.ka_compact_host(None, 16, [lt], [5], [0], out, 1024, base, nbytes)[0] == ka.KA_E_ARG
    assert ka.ka_compact_host(x, 16, [lt], [5], [0], [None], 1024, base, nbytes)[0] == ka.KA_E_ARG
    # the scratch works after the refusals
    s, counts = ka.ka_compact_host(np.arange(16, dtype=np.uint32), 16, [lt], [5], [0], out, 1024, base, nbytes)
    assert s == 0 and counts == [5] and np.array_equal(out[0][:5], np.arange(5, dtype=np.uint32))
