"""The warp-specialised TMA compaction (tile shapes (256, 16), (512, 16) and
(768, 16)) against the oracle, bit for bit: ragged tails, inputs and outputs
at every 4-byte offset, live lengths from a device word, in place, hash
transform, empty input, repeated launches on one workspace, and the full
N = 2^28 workload at 1 %, 50 %, 99 %."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import ka_inputs as ki  # noqa: E402
import oracle  # noqa: E402
from gpu_util import SENTINEL, Workspace, empty, stream, to_dev, to_host, word  # noqa: E402

TMA_SHAPES = [(768, 16), (512, 16), (256, 16)]
# entries per tile of each shape's compaction (26 compute warps for (768, 16))
TILE = {(768, 16): 13312, (512, 16): 8192, (256, 16): 4096}


@pytest.fixture(scope="module")
def ka(cuda_ok):
    import paper_1709_07781_gb300 as m
    return m


def compact(ka, d_x, n, pred, param, shape, xform=0, d_n=None, out=None, cap=None, ws=None):
    cap = n if cap is None else cap
    out = empty(cap + 16) if out is None else out
    count = empty(1)
    ws = ws or Workspace(ka, cap, shape)
    s = ka.ka_compact(d_x, cap if d_n is not None else n, d_n, ka.PRED[pred], param, xform, out, count, ws.ptr,
                      ws.nbytes, shape, stream())
    assert s == 0, ka.ka_strerror(s)
    torch.cuda.synchronize()
    assert ws.status(ka) == 0
    return out, word(count)


@pytest.mark.parametrize("shape", TMA_SHAPES)
@pytest.mark.parametrize("n", [1, 4095, 4096, 8191, 8192, 8193, 3 * 8192 + 5, 12287, 12288, 12289, 3 * 12288 + 5,
                               13311, 13312, 13313, 3 * 13312 + 5,
                               1 << 20, (1 << 22) + 12345, (1 << 23) + 1])
def test_tma_sizes(ka, shape, n):
    x = ki.uniform_u32(n + 7, n)
    out, k = compact(ka, to_dev(x), n, "lt", ki.threshold_for(0.37), shape)
    y, ek = oracle.compact(x, "lt", ki.threshold_for(0.37))
    assert k == ek
    assert np.array_equal(to_host(out, k), y)
    assert np.all(to_host(out)[k:n + 16] == SENTINEL)


@pytest.mark.parametrize("shape", TMA_SHAPES)
@pytest.mark.parametrize("pred,param", [("and_mask_eq0", 3), ("popc_odd", 0), ("mod_ne0", 3), ("ne", 0),
                                        ("topbits_lt", 8), ("all", 0), ("lt", 0)])
def test_tma_predicates_and_hash(ka, shape, pred, param):
    n = (1 << 21) + 333
    x = ki.uniform_u32(99, n)
    x[::997] = 0
    for xform in (0, 1):
        out, k = compact(ka, to_dev(x), n, pred, param, shape, xform=xform)
        y, ek = oracle.compact(oracle.map_hash(x) if xform else x, pred, param)
        assert k == ek and np.array_equal(to_host(out, k), y)


@pytest.mark.parametrize("shape", TMA_SHAPES)
def test_tma_live_length_in_place_and_empty(ka, shape):
    n = (1 << 22) + 17
    x = ki.uniform_u32(5, n)
    # live length from a device word (a previous stage's count)
    live = 3_000_001
    d_n = to_dev(np.array([live], dtype=np.uint32))
    out, k = compact(ka, to_dev(x), n, "popc_odd", 0, shape, d_n=d_n, cap=n)
    y, ek = oracle.compact(x[:live], "popc_odd", 0)
    assert k == ek and np.array_equal(to_host(out, k), y)
    assert np.all(to_host(out)[k:n] == SENTINEL)
    # in place
    d = to_dev(x)
    out, k = compact(ka, d, n, "and_mask_eq0", 1, shape, out=d)
    y, ek = oracle.compact(x, "and_mask_eq0", 1)
    assert k == ek and np.array_equal(to_host(d, k), y) and np.array_equal(to_host(d)[k:], x[k:])
    # empty (host length 0, and device length 0)
    out, k = compact(ka, empty(16), 0, "all", 0, shape)
    assert k == 0 and np.all(to_host(out) == SENTINEL)
    out, k = compact(ka, empty(1 << 16), 1 << 16, "all", 0, shape, d_n=to_dev(np.array([0], dtype=np.uint32)))
    assert k == 0


@pytest.mark.parametrize("shape", TMA_SHAPES)
@pytest.mark.parametrize("out_off", [1, 2, 3])
def test_tma_unaligned_output(ka, shape, out_off):
    """Aligned input (the TMA path) with an output view at every 4-byte offset."""
    n = (1 << 20) + 77
    x = ki.uniform_u32(31 + out_off, n)
    base = empty(n + 32)
    out, k = compact(ka, to_dev(x), n, "mod_ne0", 5, shape, out=base[out_off:])
    y, ek = oracle.compact(x, "mod_ne0", 5)
    assert k == ek and np.array_equal(to_host(base[out_off:], k), y)
    assert np.all(to_host(base)[:out_off] == SENTINEL) and np.all(to_host(base)[out_off + k:] == SENTINEL)


@pytest.mark.parametrize("shape", TMA_SHAPES)
@pytest.mark.parametrize("in_off", [1, 2, 3])
def test_tma_unaligned_input(ka, shape, in_off):
    """Input views starting 4, 8 or 12 bytes past a 16-byte boundary: the tiles
    are shifted back to the boundary and the lead entries belong to no tile."""
    T = TILE[shape]
    for n in [1, 2, 3, 5, T - in_off, T - in_off + 1, T, 3 * T + 7, (1 << 21) + 3]:
        x = ki.uniform_u32(70 + in_off, n + in_off)
        buf = to_dev(x, pad=16)
        out, k = compact(ka, buf[in_off:], n, "lt", ki.threshold_for(0.55), shape)
        y, ek = oracle.compact(x[in_off:], "lt", ki.threshold_for(0.55))
        assert k == ek and np.array_equal(to_host(out, k), y), (n, in_off)
        assert np.all(to_host(out)[k:n + 16] == SENTINEL)
    # live length from a device word, hash transform, and in place, all unaligned
    n = (1 << 21) + 99
    x = ki.uniform_u32(80 + in_off, n + in_off)
    live = n - 1000
    d_n = to_dev(np.array([live], dtype=np.uint32))
    out, k = compact(ka, to_dev(x)[in_off:], n, "popc_odd", 0, shape, xform=1, d_n=d_n)
    y, ek = oracle.compact(oracle.map_hash(x[in_off:in_off + live]), "popc_odd", 0)
    assert k == ek and np.array_equal(to_host(out, k), y)
    d = to_dev(x)
    out, k = compact(ka, d[in_off:], n, "ne", 0, shape, out=d[in_off:])
    y, ek = oracle.compact(x[in_off:], "ne", 0)
    assert k == ek and np.array_equal(to_host(d)[in_off:in_off + k], y)
    assert np.array_equal(to_host(d)[:in_off], x[:in_off])


def varied_segments(seed, n, seg=512):
    """Uniform entries rewritten so that `x < 2^31` keeps them with a
    selectivity that changes every `seg` entries (0, 1, 3, 4.5, 50 or 100 %):
    the kept counts of one tile's 512-entry segments then fall on both sides
    of the 16 entries a segment may keep and still be spilled, and each tile
    mixes spilled and held segments."""
    u = ki.uniform_u32(seed, n)
    rng = np.random.default_rng(seed)
    frac = np.array([0.0, 0.01, 0.03, 0.045, 0.5, 1.0])[rng.integers(0, 6, size=(n + seg - 1) // seg)]
    keep = (u.astype(np.float64) / 2.0**32) < np.repeat(frac, seg)[:n]
    return np.where(keep, u >> np.uint32(1), u | np.uint32(0x80000000)).astype(np.uint32)


def patterned_segments(seed, n, seg=512):
    """Entries rewritten so that `x < 2^31` keeps, in each `seg`-entry
    segment, one of these sets (entry r * 128 + 4 l + c of a segment is row r,
    lane l, column c of its warp's registers): none; the 16 entries of one
    lane (lane 0 or lane 31: the most entries one lane of a spilled segment
    can store, 16 trips); those 16 and one more (17: held); 16 entries spread
    over random rows, lanes and columns; 15 consecutive entries across a row
    boundary; 17 to 30 random entries; all of them."""
    rng = np.random.default_rng(seed)
    u = ki.uniform_u32(seed, n)
    keep = np.zeros(n, dtype=bool)
    lane_set = lambda l: np.array([r * 128 + 4 * l + c for r in range(4) for c in range(4)])
    for b in range(0, n, seg):
        m = min(seg, n - b)
        kind = int(rng.integers(0, 8))
        if kind == 0:
            idx = np.array([], dtype=np.int64)
        elif kind in (1, 2):
            idx = lane_set(0 if kind == 1 else 31)
        elif kind == 3:
            idx = np.append(lane_set(int(rng.integers(0, 32))), int(rng.integers(0, seg)))
        elif kind == 4:
            idx = rng.choice(seg, size=16, replace=False)
        elif kind == 5:
            start = int(rng.choice([120, 250, 380, int(rng.integers(0, seg - 15))]))
            idx = np.arange(start, start + 15)
        elif kind == 6:
            idx = rng.choice(seg, size=int(rng.integers(17, 31)), replace=False)
        else:
            idx = np.arange(seg)
        idx = np.unique(idx)
        keep[b + idx[idx < m]] = True
    return np.where(keep, u >> np.uint32(1), u | np.uint32(0x80000000)).astype(np.uint32)


@pytest.mark.parametrize("shape", TMA_SHAPES)
@pytest.mark.parametrize("in_off", [0, 3])
def test_tma_spill_patterns(ka, shape, in_off):
    """The spilled segments' stores by set bit at their extremes: one lane
    holding every kept entry, exactly 16 (spilled) against 17 (held), kept
    runs across row boundaries, and spread entries, mixed with held and empty
    segments in every tile; aligned and offset input."""
    n = (1 << 22) + 777
    x = patterned_segments(500 + in_off, n + in_off)
    d = to_dev(x, pad=16)
    y, ek = oracle.compact(x[in_off:], "lt", 1 << 31)
    out, k = compact(ka, d[in_off:], n, "lt", 1 << 31, shape)
    assert k == ek and np.array_equal(to_host(out, k), y)
    assert np.all(to_host(out)[k:n + 16] == SENTINEL)


@pytest.mark.parametrize("shape", TMA_SHAPES)
@pytest.mark.parametrize("s", [0.001, 0.01, 0.02, 0.03, 0.04, 0.0625])
def test_tma_low_selectivity(ka, shape, s):
    """Selectivities whose segments keep at most 16 entries (compacted into
    the warps' spill rings and written out by their warps 7 tiles later),
    around 16 (both kinds in one tile) and above it."""
    T = TILE[shape]
    for n in [5, T - 1, 3 * T + 5, (1 << 22) + 12345]:
        x = ki.uniform_u32(int(s * 1e4) + n, n)
        out, k = compact(ka, to_dev(x), n, "lt", ki.threshold_for(s), shape)
        y, ek = oracle.compact(x, "lt", ki.threshold_for(s))
        assert k == ek and np.array_equal(to_host(out, k), y), (n, s)
        assert np.all(to_host(out)[k:n + 16] == SENTINEL)


@pytest.mark.parametrize("shape", TMA_SHAPES)
@pytest.mark.parametrize("s", [0.005, 0.03, 0.3])
def test_tma_hash_transform_spilled_and_held(ka, shape, s):
    """The hash transform on both write-out paths: the spilled and the held
    segments must both store the hashed values that passed the test."""
    n = (1 << 22) + 1001
    x = ki.uniform_u32(900 + int(1000 * s), n)
    t = ki.threshold_for(s)
    out, k = compact(ka, to_dev(x), n, "lt", t, shape, xform=1)
    y, ek = oracle.compact(oracle.map_hash(x), "lt", t)
    assert k == ek and np.array_equal(to_host(out, k), y)
    assert np.all(to_host(out)[k:n + 16] == SENTINEL)


@pytest.mark.parametrize("shape", TMA_SHAPES)
@pytest.mark.parametrize("in_off", [0, 1, 2, 3])
def test_tma_mixed_segments(ka, shape, in_off):
    """Tiles whose segments keep anywhere from none to all of their entries,
    at every input offset, with an unaligned output, in place, and with a live
    length from a device word."""
    n = (1 << 22) + 777
    x = varied_segments(400 + in_off, n + in_off)
    d = to_dev(x, pad=16)
    y, ek = oracle.compact(x[in_off:], "lt", 1 << 31)
    base = empty(n + 32)
    out, k = compact(ka, d[in_off:], n, "lt", 1 << 31, shape, out=base[1 + in_off:])
    assert k == ek and np.array_equal(to_host(base[1 + in_off:], k), y)
    assert np.all(to_host(base)[:1 + in_off] == SENTINEL) and np.all(to_host(base)[1 + in_off + k:] == SENTINEL)
    live = n - 4321
    out, k = compact(ka, d[in_off:], n, "lt", 1 << 31, shape, d_n=to_dev(np.array([live], dtype=np.uint32)))
    yl, el = oracle.compact(x[in_off:in_off + live], "lt", 1 << 31)
    assert k == el and np.array_equal(to_host(out, k), yl)
    out, k = compact(ka, d[in_off:], n, "lt", 1 << 31, shape, out=d[in_off:])
    assert k == ek and np.array_equal(to_host(d)[in_off:in_off + k], y)
    assert np.array_equal(to_host(d)[:in_off], x[:in_off]) and np.array_equal(to_host(d)[in_off + k:n + in_off],
                                                                             x[in_off + k:])


@pytest.mark.parametrize("shape", TMA_SHAPES)
def test_tma_workspace_reuse_and_shape_mix(ka, shape):
    ws = Workspace(ka, 1 << 22, (128, 4))  # sized for the smallest tile: fits every shape
    for i in range(30):
        n = [1 << 22, 12345, (1 << 21) + 1, 8192, 77][i % 5]
        x = ki.uniform_u32(1000 + i, n)
        sh = shape if i % 3 else (256, 4)  # alternate with the register kernel on one workspace
        out, k = compact(ka, to_dev(x), n, "lt", ki.threshold_for(0.6), sh, ws=ws)
        y, ek = oracle.compact(x, "lt", ki.threshold_for(0.6))
        assert k == ek and np.array_equal(to_host(out, k), y), (i, n, sh)


@pytest.mark.parametrize("shape", [(768, 16), (512, 16)])
@pytest.mark.parametrize("s", [0.01, 0.5, 0.99])
def test_full_size_2_28(ka, s, shape):
    """The benchmark workload itself: N = 2^28 generated on the device (seed 2),
    keep x < floor(s 2^32), the large-input shapes; every output checked."""
    n = 1 << 28
    x_dev = torch.empty(n, dtype=torch.int32, device="cuda")
    assert ka.ka_generate(x_dev, n, 2, stream()) == 0
    t = ki.threshold_for(s)
    out, k = compact(ka, x_dev, n, "lt", t, shape)
    del x_dev
    x = oracle.generate(2, n)
    y, ek = oracle.compact(x, "lt", t)
    assert k == ek
    assert np.array_equal(to_host(out, k), y)


@pytest.mark.parametrize("what", ["compact", "scan", "batch"])
def test_tma_lookback_timeout_reports_status(ka, what):
    """A look-back whose predecessors never publish gives up after the spin
    limit and reports KA_E_DEVICE_TIMEOUT; the launch ends and the context
    stays usable. The missing publications are made on the host: the
    workspace's ticket count is set one short of the grid, so the first block
    to arrive draws the launch's last ticket and resets the count to the next
    epoch. Blocks whose tickets land after that reset run in the next epoch,
    and neither side accepts the other's status words (every access stays in
    bounds and every wait is bounded). Whether a block lands before or after
    the reset depends on the order in which the tickets reach memory, so the
    launch is repeated, the workspace re-initialised each time, until one
    splits; a launch that does not split must give the right result."""
    n = (1 << 22) + 5
    shape = (768, 16) if what != "scan" else (512, 16)
    # the persistent grid: one block per SM for (768, 16), two for (512, 16)
    per_sm = {768: 1, 512: 2}[shape[0]]
    tiles = (n + shape[0] * shape[1] - 1) // (shape[0] * shape[1])
    G = min(tiles, torch.cuda.get_device_properties(0).multi_processor_count * per_sm)
    assert G > 1
    x = ki.uniform_u32(8, n)
    d_x = to_dev(x)
    out, count = empty(n + 16), empty(1)
    if what == "batch":
        items = np.zeros(1, dtype=[("in_", "<u8"), ("out", "<u8"), ("n_ptr", "<u8"), ("count", "<u8"), ("n", "<u4"),
                                   ("pred", "<i4"), ("param", "<u4"), ("xform", "<u4")])
        items[0] = (d_x.data_ptr(), out.data_ptr(), 0, count.data_ptr(), n, ka.KA_PRED_LT, 1 << 31, 0)
        raw = np.frombuffer(items.tobytes(), dtype=np.uint8)
        d_items = torch.from_numpy(raw.copy()).cuda()
        ws = Workspace(ka, n, shape, batch_items=1)
    else:
        ws = Workspace(ka, n, shape)
    if what == "scan":
        want_out, want_count = oracle.exclusive_scan(x)
    else:
        want_out, want_count = oracle.compact(x, "lt", 1 << 31)

    def launch():
        if what == "compact":
            return ka.ka_compact(d_x, n, None, ka.KA_PRED_LT, 1 << 31, 0, out, count, ws.ptr, ws.nbytes, shape,
                                 stream())
        if what == "scan":
            return ka.ka_exclusive_scan(d_x, n, None, out, count, ws.ptr, ws.nbytes, shape, stream())
        return ka.ka_compact_batch(d_items, 1, 1, ws.ptr, ws.nbytes, shape, 0, stream())

    def check_result():
        k = word(count)
        assert k == want_count
        assert np.array_equal(to_host(out, n if what == "scan" else k), want_out)

    hdr = ws.header_words()
    timed_out = False
    for _ in range(32):
        assert ka.ka_workspace_init(ws.ptr, ws.nbytes, stream()) == 0
        assert ka.ka_workspace_set_spin_limit(ws.ptr, 64, stream()) == 0
        torch.cuda.synchronize()
        epoch = int(hdr[0].item()) >> 32
        hdr[0] = (epoch << 32) | (G - 1)  # G - 1 tickets of this epoch already taken
        assert launch() == 0
        torch.cuda.synchronize()
        st = ws.status(ka)
        if st == ka.KA_E_DEVICE_TIMEOUT:
            timed_out = True
            break
        assert st == 0
        check_result()  # every block landed before the reset: one epoch, a normal launch
    assert timed_out
    # re-initialised, the same workspace works again
    assert ka.ka_workspace_init(ws.ptr, ws.nbytes, stream()) == 0
    out.fill_(int(np.uint32(SENTINEL).view(np.int32)))
    assert launch() == 0
    torch.cuda.synchronize()
    assert ws.status(ka) == 0
    check_result()
