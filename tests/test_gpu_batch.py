"""Batched compaction (one persistent launch over many instances) and batched
generation, through the C ABI, bit for bit against the CPU oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import ka_inputs as ki  # noqa: E402
import oracle  # noqa: E402
from gpu_util import SENTINEL, Workspace, dev, empty, stream, to_dev, to_host  # noqa: E402

ITEM = np.dtype([("in", "<u8"), ("out", "<u8"), ("n_ptr", "<u8"), ("count", "<u8"), ("n", "<u4"),
                 ("pred", "<i4"), ("param", "<u4"), ("xform", "<u4")])
GEN = np.dtype([("out", "<u8"), ("seed", "<u8"), ("n", "<u4"), ("pad", "<u4")])
assert ITEM.itemsize == 48 and GEN.itemsize == 24


@pytest.fixture(scope="module")
def ka(cuda_ok):
    import paper_1709_07781_gb300 as m
    return m


def table_to_dev(arr: np.ndarray) -> torch.Tensor:
    raw = np.frombuffer(arr.tobytes(), dtype=np.uint8)
    t = torch.empty(raw.size, dtype=torch.uint8, device=dev())
    t.copy_(torch.from_numpy(raw.copy()))
    return t


class Arena:
    """One device buffer carved into per-instance regions (16-byte aligned
    unless an element offset is asked for)."""

    def __init__(self, sizes, extra=16, offsets=None):
        self.offs = []
        pos = 0
        for i, n in enumerate(sizes):
            pos = (pos + 3) // 4 * 4 + (offsets[i] if offsets else 0)
            self.offs.append(pos)
            pos += int(n) + extra
        self.buf = empty(pos + 16)

    def ptr(self, i):
        return self.buf.data_ptr() + 4 * self.offs[i]

    def host(self):
        return to_host(self.buf)


def run_batch(ka, xs, preds, xforms=None, tile=None, offsets=None, ws=None, grid=0):
    m = len(xs)
    sizes = [x.size for x in xs]
    src = Arena(sizes, offsets=offsets)
    host_in = src.host().copy()
    for i, x in enumerate(xs):
        host_in[src.offs[i]: src.offs[i] + x.size] = x
    src.buf.copy_(torch.from_numpy(host_in.view(np.int32)))
    dst = Arena(sizes, offsets=offsets)
    counts = empty(m)
    items = np.zeros(m, dtype=ITEM)
    for i in range(m):
        items[i] = (src.ptr(i), dst.ptr(i), 0, counts.data_ptr() + 4 * i, sizes[i], ka.PRED[preds[i][0]],
                    preds[i][1], xforms[i] if xforms else 0)
    d_items = table_to_dev(items)
    ws = ws or Workspace(ka, sum(sizes) + 1, tile, batch_items=m)
    s = ka.ka_compact_batch(d_items, m, m, ws.ptr, ws.nbytes, tile, grid, stream())
    assert s == 0, ka.ka_strerror(s)
    torch.cuda.synchronize()
    return dst, to_host(counts, m), ws


def check(xs, preds, xforms, dst, counts):
    out = dst.host()
    for i, x in enumerate(xs):
        src = oracle.map_hash(x) if xforms and xforms[i] else x
        y, k = oracle.compact(src, preds[i][0], preds[i][1])
        assert counts[i] == k, (i, x.size, counts[i], k)
        o = dst.offs[i]
        assert np.array_equal(out[o: o + k], y), i
        assert np.all(out[o + k: o + x.size + 16] == SENTINEL), i


SIZES = [0, 1, 3, 511, 512, 513, 2047, 4096, 4097, 10000, 65536 + 5, 300001, 2, 0, 77]
PREDS = [("lt", ki.threshold_for(0.3)), ("and_mask_eq0", 3), ("popc_odd", 0), ("mod_ne0", 3), ("topbits_lt", 8),
         ("ne", 0), ("all", 0)]


TMA_SHAPES = [(768, 16), (704, 16), (512, 16), (256, 16)]


@pytest.mark.parametrize("shape", [(128, 4), (256, 8), (512, 8), (128, 16)] + TMA_SHAPES)
def test_batch_mixed_sizes_and_predicates(ka, shape):
    xs = [ki.uniform_u32(100 + i, n) for i, n in enumerate(SIZES)]
    preds = [PREDS[i % len(PREDS)] for i in range(len(xs))]
    xforms = [i % 3 == 0 for i in range(len(xs))]
    dst, counts, ws = run_batch(ka, xs, preds, xforms=xforms, tile=shape)
    check(xs, preds, xforms, dst, counts)
    assert ws.status(ka) == 0


@pytest.mark.parametrize("shape", [None, (256, 8)] + TMA_SHAPES)
def test_batch_unaligned_inputs_and_small_grid(ka, shape):
    xs = [ki.uniform_u32(7 + i, n) for i, n in enumerate([1000, 4097, 123, 70000, 5, 12288, 12287, 3 * 12288 + 1])]
    preds = [("lt", ki.threshold_for(0.5))] * len(xs)
    for grid in (3, 0):
        dst, counts, _ = run_batch(ka, xs, preds, offsets=[1, 2, 3, 0, 1, 2, 3, 1], grid=grid, tile=shape)
        check(xs, preds, None, dst, counts)


@pytest.mark.parametrize("shape", TMA_SHAPES)
def test_batch_in_place(ka, shape):
    """out_i == in_i for every item, inputs at every 4-byte offset."""
    xs = [ki.uniform_u32(300 + i, n) for i, n in enumerate([70000, 3, 12289, 0, 40001, 9000])]
    offsets = [1, 2, 3, 0, 2, 1]
    src = Arena([x.size for x in xs], offsets=offsets)
    host_in = src.host().copy()
    for i, x in enumerate(xs):
        host_in[src.offs[i]: src.offs[i] + x.size] = x
    src.buf.copy_(torch.from_numpy(host_in.view(np.int32)))
    counts = empty(len(xs))
    items = np.zeros(len(xs), dtype=ITEM)
    for i, x in enumerate(xs):
        items[i] = (src.ptr(i), src.ptr(i), 0, counts.data_ptr() + 4 * i, x.size, ka.KA_PRED_POPC_ODD, 0, 1)
    ws = Workspace(ka, sum(x.size for x in xs) + 1, shape, batch_items=len(xs))
    assert ka.ka_compact_batch(table_to_dev(items), len(xs), len(xs), ws.ptr, ws.nbytes, shape, 0, stream()) == 0
    torch.cuda.synchronize()
    out, c = src.host(), to_host(counts, len(xs))
    for i, x in enumerate(xs):
        y, k = oracle.compact(oracle.map_hash(x), "popc_odd", 0)
        assert c[i] == k and np.array_equal(out[src.offs[i]: src.offs[i] + k], y), i
        assert np.array_equal(out[src.offs[i] + k: src.offs[i] + x.size], x[k:]), i


@pytest.mark.parametrize("shape", [(128, 4)] + TMA_SHAPES)
def test_batch_mostly_empty_items(ka, shape):
    """Four empty items to each tiny one: G consecutive tiles then span far
    more items than the producer's 128-item search window, so the item of a
    tile is found by the full search, and empty items lie between the items
    of consecutive tiles."""
    sizes = [0 if i % 5 else 1 + (37 * i) % 900 for i in range(3000)] + [5000, 0, 0, 1]
    xs = [ki.uniform_u32(4000 + i, n) for i, n in enumerate(sizes)]
    preds = [PREDS[i % len(PREDS)] for i in range(len(xs))]
    dst, counts, ws = run_batch(ka, xs, preds, tile=shape)
    check(xs, preds, None, dst, counts)
    assert ws.status(ka) == 0


@pytest.mark.parametrize("shape", TMA_SHAPES)
def test_batch_map_hints_are_checked(ka, shape):
    """Every tile's map word carries the tag of the coming launch but names a
    wrong item, as a word left by another use of the workspace might: the
    plan rewrites the words of small items' tiles, and the producer checks
    every other hint against the item's tiles and finds the item by search."""
    sizes = [70000, 3, 12289, 0, 40001, 9000, 300001, 1, 513, 200000]
    xs = [ki.uniform_u32(700 + i, n) for i, n in enumerate(sizes)]
    preds = [PREDS[i % len(PREDS)] for i in range(len(xs))]
    m = len(xs)
    ws = Workspace(ka, sum(sizes) + 1, shape, batch_items=m)
    ticket = int(ws.header_words()[0].item())
    tag = ((ticket >> 32) + 1) & 0xFFFFFFFF  # the plan draws epoch E, the compaction kernel E + 1
    r256 = lambda b: (b + 255) // 256 * 256  # noqa: E731
    off = 256 + r256((m + 1) * 4) + r256(m * 32)  # header, tile offsets, plan records: then 32-byte entries
    base = ws.ptr - ws.buf.data_ptr() + off
    n_entries = (ws.nbytes - off) // 32
    rng = np.random.default_rng(3)
    hints = (np.uint64(tag) << np.uint64(32)) | rng.integers(0, m, n_entries).astype(np.uint64)
    words = ws.buf[base: base + 32 * n_entries].view(torch.int64).view(n_entries, 4)
    words[:, 1] = torch.from_numpy(hints.view(np.int64)).to(words.device)
    dst, counts, _ = run_batch(ka, xs, preds, tile=shape, ws=ws)
    check(xs, preds, None, dst, counts)
    assert ws.status(ka) == 0


@pytest.mark.parametrize("shape", [(128, 4), (768, 16)])
def test_batch_many_tiny_instances(ka, shape):
    """Thousands of one-tile items: the item search jumps far between tiles."""
    rng_sizes = ki.log_uniform_sizes(5, 3000, 0, 9)
    xs = [ki.uniform_u32(1000 + i, int(n)) for i, n in enumerate(rng_sizes)]
    preds = [("and_mask_eq0", 1)] * len(xs)
    dst, counts, _ = run_batch(ka, xs, preds, tile=shape)
    check(xs, preds, None, dst, counts)


def test_batch_workspace_reuse(ka):
    xs = [ki.uniform_u32(i, 5000 + 77 * i) for i in range(20)]
    preds = [("popc_odd", 0)] * 20
    ws = Workspace(ka, sum(x.size for x in xs) + 1, None, batch_items=20)
    for rep in range(25):
        sub = xs[rep % 5: rep % 5 + 15]
        dst, counts, _ = run_batch(ka, sub, preds[:len(sub)], ws=ws)
        check(sub, preds[:len(sub)], None, dst, counts)


@pytest.mark.parametrize("shape", [None, (768, 16)])
def test_batch_chained_lengths_and_in_out_count(ka, shape):
    """Second batch reads each item's live length from the first batch's count
    words and writes its result count back into the same word."""
    xs = [ki.uniform_u32(50 + i, n) for i, n in enumerate([5000, 1, 0, 40000, 4096])]
    preds1 = [("and_mask_eq0", 1)] * 5
    dst1, counts1, _ = run_batch(ka, xs, preds1, tile=shape)
    counts_dev = to_dev(counts1.astype(np.uint32))
    dst2 = Arena([x.size for x in xs])
    items = np.zeros(5, dtype=ITEM)
    for i, x in enumerate(xs):
        c = counts_dev.data_ptr() + 4 * i
        items[i] = (dst1.ptr(i), dst2.ptr(i), c, c, x.size, ka.KA_PRED_MOD_NE0, 3, 0)
    ws = Workspace(ka, sum(x.size for x in xs) + 1, shape, batch_items=5)
    assert ka.ka_compact_batch(table_to_dev(items), 5, 5, ws.ptr, ws.nbytes, shape, 0, stream()) == 0
    torch.cuda.synchronize()
    out = dst2.host()
    got = to_host(counts_dev, 5)
    for i, x in enumerate(xs):
        y1, _ = oracle.compact(x, "and_mask_eq0", 1)
        y2, k2 = oracle.compact(y1, "mod_ne0", 3)
        assert got[i] == k2
        assert np.array_equal(out[dst2.offs[i]: dst2.offs[i] + k2], y2)


@pytest.mark.parametrize("shape", [None, (768, 16)])
def test_batch_invalid_item_reports_arg_error(ka, shape):
    xs = [ki.uniform_u32(1, 1000), ki.uniform_u32(2, 1000)]
    src = Arena([1000, 1000])
    dst = Arena([1000, 1000])
    counts = empty(2)
    items = np.zeros(2, dtype=ITEM)
    items[0] = (src.ptr(0), dst.ptr(0), 0, counts.data_ptr(), 1000, ka.KA_PRED_MOD_NE0, 0, 0)  # zero modulus
    items[1] = (src.ptr(1), dst.ptr(1), 0, counts.data_ptr() + 4, 1000, ka.KA_PRED_ALL, 0, 0)
    ws = Workspace(ka, 2001, shape, batch_items=2)
    assert ka.ka_compact_batch(table_to_dev(items), 2, 2, ws.ptr, ws.nbytes, shape, 0, stream()) == 0
    torch.cuda.synchronize()
    assert ws.status(ka) == ka.KA_E_ARG
    c = to_host(counts, 2)
    assert c[0] == 0 and c[1] == 1000


def test_generate_batch(ka):
    sizes = [0, 1, 5, 4096, 4097, 100000, 3]
    arena = Arena(sizes, offsets=[0, 1, 2, 3, 0, 1, 2])
    items = np.zeros(len(sizes), dtype=GEN)
    seeds = [11, 0, 2**63 + 5, 7, 8, 9, 10]
    for i, n in enumerate(sizes):
        items[i] = (arena.ptr(i), seeds[i], n, 0)
    ws = Workspace(ka, sum(sizes) + 1, None, batch_items=len(sizes))
    assert ka.ka_generate_batch(table_to_dev(items), len(sizes), len(sizes), ws.ptr, ws.nbytes, stream()) == 0
    torch.cuda.synchronize()
    out = arena.host()
    for i, n in enumerate(sizes):
        o = arena.offs[i]
        assert np.array_equal(out[o: o + n], oracle.generate(seeds[i], n)), i
        assert np.all(out[o + n: o + n + 16] == SENTINEL)


@pytest.mark.parametrize("shape", [None, (128, 16), (768, 16)])
def test_batch_4096_instances_full_size(ka, shape):
    """The 4096-instance workload (sizes log-uniform 2^8..2^20, per-instance
    thresholds), data generated on the device, every instance checked."""
    spec = ki.config_batch()
    m = spec.n.size
    sizes = [int(v) for v in spec.n]
    src = Arena(sizes, extra=0)
    dst = Arena(sizes, extra=4)
    gen = np.zeros(m, dtype=GEN)
    items = np.zeros(m, dtype=ITEM)
    counts = empty(m)
    for i in range(m):
        gen[i] = (src.ptr(i), int(spec.seeds[i]), sizes[i], 0)
        items[i] = (src.ptr(i), dst.ptr(i), 0, counts.data_ptr() + 4 * i, sizes[i], ka.KA_PRED_LT, int(spec.t[i]), 0)
    total = sum(sizes)
    ws = Workspace(ka, total + 1, shape, batch_items=m)
    assert ka.ka_generate_batch(table_to_dev(gen), m, m, ws.ptr, ws.nbytes, stream()) == 0
    assert ka.ka_compact_batch(table_to_dev(items), m, m, ws.ptr, ws.nbytes, shape, 0, stream()) == 0
    torch.cuda.synchronize()
    assert ws.status(ka) == 0
    got = to_host(counts, m)
    out = dst.host()
    for i in range(m):
        x = oracle.generate(int(spec.seeds[i]), sizes[i])
        y, k = oracle.compact(x, "lt", int(spec.t[i]))
        assert got[i] == k, i
        o = dst.offs[i]
        assert np.array_equal(out[o: o + k], y), i
