"""Stage kernels through the C ABI against the CPU oracle, bit for bit.

Integer work: every comparison is exact (no tolerance). Sizes span several
tiles of every shape plus ragged tails; inputs include non-16-byte-aligned
views, 0 % and 100 % selectivity, in-place runs, live lengths read from a
device word, and sentinel-filled outputs (nothing may be written past the
result's length)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import ka_inputs as ki  # noqa: E402
import oracle  # noqa: E402
from gpu_util import SENTINEL, Workspace, empty, stream, to_dev, to_host, word  # noqa: E402

SHAPES = [(128, 4), (128, 8), (128, 16), (256, 4), (256, 8), (256, 16), (512, 4), (512, 8)]
SIZES = [0, 1, 3, 4, 5, 127, 511, 512, 513, 1023, 1025, 2047, 2048, 2049, 4095, 4096, 4097, 3 * 4096 + 17,
         12287, 12288, 12289, 13311, 13312, 13313, 65537, (1 << 20) + 3]
TMA_SHAPES = [(768, 16), (512, 16)]  # (256, 16) is in SHAPES
PREDS = [("and_mask_eq0", 3), ("lt", ki.threshold_for(0.5)), ("topbits_lt", 8), ("popc_odd", 0),
         ("mod_ne0", 3), ("ne", 0), ("mod_ne0", 12), ("topbits_lt", 0), ("lt", 0), ("lt", 0xFFFFFFFF)]


@pytest.fixture(scope="module")
def ka(cuda_ok):
    import paper_1709_07781_gb300 as m
    return m


def run_compact(ka, x_dev, n, pred, param, xform=0, tile=None, d_n=None, out=None, cap=None, ws=None):
    cap = n if cap is None else cap
    out = empty(cap + 16) if out is None else out
    count = empty(1)
    ws = ws or Workspace(ka, cap, tile)
    s = ka.ka_compact(x_dev, cap if d_n is not None else n, d_n, ka.PRED[pred], param, xform, out, count,
                      ws.ptr, ws.nbytes, tile, stream())
    assert s == 0, ka.ka_strerror(s)
    torch.cuda.synchronize()
    assert ws.status(ka) == 0
    return out, word(count), ws


# ---------------------------------------------------------------------------
def test_generate_matches_oracle_generator(ka):
    for seed in (0, 1, 0xDEADBEEFCAFEF00D):
        n = 1_000_000
        d = empty(n + 3)
        assert ka.ka_generate(d, n, seed, stream()) == 0
        assert np.array_equal(to_host(d, n), oracle.generate(seed, n))
        # unaligned destination and ragged length
        assert ka.ka_generate(d[1:], 1001, seed, stream()) == 0
        assert np.array_equal(to_host(d[1:], 1001), oracle.generate(seed, 1001))


@pytest.mark.parametrize("n", [0, 1, 5, 1000, (1 << 20) + 3])
def test_map_hash(ka, n):
    x = ki.uniform_u32(40 + n, n)
    d_x = to_dev(x, pad=4)
    out = empty(n + 4)
    n_out = empty(1)
    assert ka.ka_map_hash(d_x, n, None, out, n_out, stream()) == 0
    torch.cuda.synchronize()
    assert np.array_equal(to_host(out, n), oracle.map_hash(x))
    assert word(n_out) == n
    assert np.all(to_host(out)[n:n + 4] == SENTINEL)


def test_map_hash_live_length_from_device(ka):
    n, live = 10000, 6001
    x = ki.uniform_u32(3, n)
    d_n = to_dev(np.array([live], dtype=np.uint32))
    out = empty(n)
    n_out = empty(1)
    assert ka.ka_map_hash(to_dev(x), n, d_n, out, n_out, stream()) == 0
    torch.cuda.synchronize()
    assert np.array_equal(to_host(out, live), oracle.map_hash(x[:live]))
    assert np.all(to_host(out)[live:] == SENTINEL) and word(n_out) == live


@pytest.mark.parametrize("pred,param", PREDS)
def test_predicate_flags(ka, pred, param):
    n = (1 << 16) + 7
    x = ki.uniform_u32(7, n)
    x[:8] = [0, 1, 2, 3, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFF, 12]
    f = empty(n)
    assert ka.ka_predicate(to_dev(x), n, None, ka.PRED[pred], param, f, stream()) == 0
    torch.cuda.synchronize()
    assert np.array_equal(to_host(f, n), oracle.predicate_map(x, pred, param))


def test_predicate_rejects_zero_modulus(ka):
    d = empty(16)
    assert ka.ka_predicate(d, 16, None, ka.KA_PRED_MOD_NE0, 0, d, stream()) == ka.KA_E_ARG
    assert ka.ka_predicate(d, 16, None, 99, 0, d, stream()) == ka.KA_E_ARG


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", SHAPES + TMA_SHAPES)
def test_exclusive_scan_shapes_and_sizes(ka, shape):
    ws = Workspace(ka, (1 << 20) + 64, shape)
    for n in SIZES:
        for kind in ("flags", "values"):
            v = ki.uniform_u32(n + 17, n)
            if kind == "flags":
                v = (v & 1).astype(np.uint32)
            d_v = to_dev(v)
            out = empty(n + 4)
            total = empty(1)
            s = ka.ka_exclusive_scan(d_v, n, None, out, total, ws.ptr, ws.nbytes, shape, stream())
            assert s == 0
            torch.cuda.synchronize()
            o, tot = oracle.exclusive_scan(v)
            assert np.array_equal(to_host(out, n), o), (shape, n, kind)
            assert word(total) == tot
            assert np.all(to_host(out)[n:n + 4] == SENTINEL)
    assert ws.status(ka) == 0


@pytest.mark.parametrize("shape", [None, (768, 16), (512, 16), (256, 16)])
def test_exclusive_scan_in_place_and_unaligned(ka, shape):
    n = 100003
    v = ki.uniform_u32(5, n)
    o, tot = oracle.exclusive_scan(v)
    ws = Workspace(ka, n + 8)
    d = to_dev(v)
    total = empty(1)
    assert ka.ka_exclusive_scan(d, n, None, d, total, ws.ptr, ws.nbytes, shape, stream()) == 0
    torch.cuda.synchronize()
    assert np.array_equal(to_host(d, n), o) and word(total) == tot
    # input and output views at every 4-byte offset, matching and not
    for off_in, off_out in ((1, 1), (2, 2), (3, 3), (1, 0), (0, 3), (2, 1)):
        d = to_dev(np.concatenate([np.zeros(off_in, np.uint32), v]))
        out = empty(n + off_out + 4)
        assert ka.ka_exclusive_scan(d[off_in:], n, None, out[off_out:], total, ws.ptr, ws.nbytes, shape,
                                    stream()) == 0
        torch.cuda.synchronize()
        got = to_host(out)
        assert np.array_equal(got[off_out:off_out + n], o) and word(total) == tot, (off_in, off_out)
        assert np.all(got[:off_out] == SENTINEL) and np.all(got[off_out + n:] == SENTINEL)


@pytest.mark.parametrize("shape", TMA_SHAPES)
def test_exclusive_scan_live_length_and_full_size(ka, shape):
    """Live length from a device word; the N = 2^28 flags of the three-launch
    comparison (keep x < 2^31), every output checked."""
    n = (1 << 22) + 9
    v = (ki.uniform_u32(6, n) & 1).astype(np.uint32)
    live = n - 12345
    d_n = to_dev(np.array([live], dtype=np.uint32))
    ws = Workspace(ka, n, shape)
    out, total = empty(n), empty(1)
    assert ka.ka_exclusive_scan(to_dev(v), n, d_n, out, total, ws.ptr, ws.nbytes, shape, stream()) == 0
    torch.cuda.synchronize()
    o, tot = oracle.exclusive_scan(v[:live])
    got = to_host(out)
    assert np.array_equal(got[:live], o) and word(total) == tot and np.all(got[live:] == SENTINEL)
    N = 1 << 28
    x = torch.empty(N, dtype=torch.int32, device="cuda")
    assert ka.ka_generate(x, N, 2, stream()) == 0
    f = torch.empty_like(x)
    assert ka.ka_predicate(x, N, None, ka.KA_PRED_LT, 1 << 31, f, stream()) == 0
    del x
    ws = Workspace(ka, N, shape)
    o_dev, total = torch.empty_like(f), empty(1)
    assert ka.ka_exclusive_scan(f, N, None, o_dev, total, ws.ptr, ws.nbytes, shape, stream()) == 0
    torch.cuda.synchronize()
    flags = to_host(f)
    del f
    o, tot = oracle.exclusive_scan(flags)
    assert word(total) == tot and np.array_equal(to_host(o_dev), o)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [0, 1, 7, 2048, 2049, 100000, (1 << 20) + 5])
def test_three_phase_pipeline(ka, n):
    x = ki.uniform_u32(n + 3, n)
    d_x = to_dev(x)
    f, o, y = empty(n), empty(n), empty(n + 8)
    total = empty(1)
    ws = Workspace(ka, n)
    assert ka.ka_predicate(d_x, n, None, ka.KA_PRED_AND_MASK_EQ0, 3, f, stream()) == 0
    assert ka.ka_exclusive_scan(f, n, None, o, total, ws.ptr, ws.nbytes, None, stream()) == 0
    assert ka.ka_scatter(d_x, f, o, n, None, y, stream()) == 0
    torch.cuda.synchronize()
    ef, eo, etot, ey = oracle.three_phase(x, "and_mask_eq0", 3)
    assert np.array_equal(to_host(f, n), ef)
    assert np.array_equal(to_host(o, n), eo)
    assert word(total) == etot
    assert np.array_equal(to_host(y, etot), ey)
    assert np.all(to_host(y)[etot:] == SENTINEL)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", SHAPES)
def test_compact_shapes_and_sizes(ka, shape):
    ws = Workspace(ka, (1 << 20) + 64, shape)
    for n in SIZES:
        x = ki.uniform_u32(n + 101, n)
        out, k, _ = run_compact(ka, to_dev(x), n, "and_mask_eq0", 3, tile=shape, ws=ws)
        y, ek = oracle.compact(x, "and_mask_eq0", 3)
        assert k == ek, (shape, n)
        assert np.array_equal(to_host(out, k), y), (shape, n)
        assert np.all(to_host(out)[k:n + 16] == SENTINEL), (shape, n)


@pytest.mark.parametrize("pred,param", PREDS)
def test_compact_predicates(ka, pred, param):
    n = 300007
    x = ki.uniform_u32(77, n)
    x[::1000] = 0
    for xform in (0, 1):
        out, k, _ = run_compact(ka, to_dev(x), n, pred, param, xform=xform)
        src = oracle.map_hash(x) if xform else x
        y, ek = oracle.compact(src, pred, param)
        assert k == ek and np.array_equal(to_host(out, k), y)
        assert np.all(to_host(out)[k:n + 16] == SENTINEL)


@pytest.mark.parametrize("s", [0.0, 0.01, 0.5, 0.99, 1.0])
def test_compact_selectivities(ka, s):
    n = (1 << 21) + 9
    x = ki.uniform_u32(2, n)
    t = ki.threshold_for(s) if s < 1.0 else 0xFFFFFFFF
    if s == 1.0:
        x[x == 0xFFFFFFFF] = 0
    out, k, _ = run_compact(ka, to_dev(x), n, "lt", t)
    y, ek = oracle.compact(x, "lt", t)
    assert k == ek and np.array_equal(to_host(out, k), y)
    if s == 0.0:
        assert k == 0
    if s == 1.0:
        assert k == n


def test_compact_unaligned_views(ka):
    n = 123457
    x = ki.uniform_u32(9, n)
    y, ek = oracle.compact(x, "popc_odd", 0)
    for off in (1, 2, 3):
        d = to_dev(np.concatenate([np.zeros(off, np.uint32), x]), pad=16)
        out = empty(n + 32)
        out_k = empty(1)
        ws = Workspace(ka, n)
        assert ka.ka_compact(d[off:], n, None, ka.KA_PRED_POPC_ODD, 0, 0, out[off:], out_k, ws.ptr, ws.nbytes,
                             None, stream()) == 0
        torch.cuda.synchronize()
        assert word(out_k) == ek and np.array_equal(to_host(out[off:], ek), y)


def test_compact_in_place(ka):
    n = (1 << 20) + 333
    x = ki.uniform_u32(12, n)
    d = to_dev(x)
    count = empty(1)
    ws = Workspace(ka, n)
    assert ka.ka_compact(d, n, None, ka.KA_PRED_LT, ki.threshold_for(0.3), 0, d, count, ws.ptr, ws.nbytes,
                         None, stream()) == 0
    torch.cuda.synchronize()
    y, ek = oracle.compact(x, "lt", ki.threshold_for(0.3))
    assert word(count) == ek and np.array_equal(to_host(d, ek), y)
    # entries past the result keep their old values (nothing written there)
    assert np.array_equal(to_host(d)[ek:], x[ek:]) or ek == n


def test_compact_live_length_and_chaining(ka):
    """Stage k+1 reads stage k's length from the device count word."""
    n = 500000
    x = ki.uniform_u32(44, n)
    ws1, ws2 = Workspace(ka, n), Workspace(ka, n)
    d_x = to_dev(x)
    y1, c1 = empty(n), empty(1)
    y2, c2 = empty(n + 8), empty(1)
    assert ka.ka_compact(d_x, n, None, ka.KA_PRED_AND_MASK_EQ0, 1, 0, y1, c1, ws1.ptr, ws1.nbytes, None,
                         stream()) == 0
    assert ka.ka_compact(y1, n, c1, ka.KA_PRED_POPC_ODD, 0, 0, y2, c2, ws2.ptr, ws2.nbytes, None, stream()) == 0
    torch.cuda.synchronize()
    e1, k1 = oracle.compact(x, "and_mask_eq0", 1)
    e2, k2 = oracle.compact(e1, "popc_odd", 0)
    assert word(c1) == k1 and word(c2) == k2
    assert np.array_equal(to_host(y2, k2), e2)
    assert np.all(to_host(y2)[k2:] == SENTINEL)
    # aliasing the output count with the live-length word is refused
    assert ka.ka_compact(y1, n, c1, ka.KA_PRED_ALL, 0, 0, y2, c1, ws2.ptr, ws2.nbytes, None, stream()) == ka.KA_E_ARG


def test_compact_empty_input_writes_zero_count(ka):
    ws = Workspace(ka, 4096)
    count = empty(1)
    out = empty(8)
    assert ka.ka_compact(out, 0, None, ka.KA_PRED_ALL, 0, 0, out, count, ws.ptr, ws.nbytes, None, stream()) == 0
    torch.cuda.synchronize()
    assert word(count) == 0 and np.all(to_host(out) == SENTINEL)
    # live length 0 from the device
    d_n = to_dev(np.array([0], dtype=np.uint32))
    count2 = empty(1)
    assert ka.ka_compact(out, 8, d_n, ka.KA_PRED_ALL, 0, 0, out, count2, ws.ptr, ws.nbytes, None, stream()) == 0
    torch.cuda.synchronize()
    assert word(count2) == 0


def test_workspace_reuse_many_launches(ka):
    """The epoch/ticket scheme leaves the workspace ready for the next launch."""
    ws = Workspace(ka, 1 << 18, (256, 4))
    for i in range(60):
        n = [1, 1000, 1 << 18, 5000, 4097][i % 5]
        x = ki.uniform_u32(i, n)
        out, k, _ = run_compact(ka, to_dev(x), n, "lt", ki.threshold_for(0.4), tile=(256, 4), ws=ws)
        y, ek = oracle.compact(x, "lt", ki.threshold_for(0.4))
        assert k == ek and np.array_equal(to_host(out, k), y)


def test_workspace_too_small_is_refused(ka):
    ws = Workspace(ka, 1024, (128, 4))
    d = empty(1 << 16)
    c = empty(1)
    assert ka.ka_compact(d, 1 << 16, None, ka.KA_PRED_ALL, 0, 0, d, c, ws.ptr, ws.nbytes, (128, 4),
                         stream()) == ka.KA_E_WORKSPACE
    assert ka.ka_compact(d, 16, None, ka.KA_PRED_ALL, 0, 0, d, c, ws.ptr + 8, ws.nbytes, None,
                         stream()) == ka.KA_E_ARG


def test_lookback_timeout_reports_status(ka):
    """A look-back whose predecessor never publishes gives up after the spin
    limit and reports KA_E_DEVICE_TIMEOUT; the context stays usable. The
    missing predecessor is made on the host: the workspace's ticket word is
    advanced by one, so tile 0 is never handed out (every access stays in
    bounds and every wait is bounded)."""
    n = 64 * 1024
    shape = (256, 4)
    ws = Workspace(ka, n, shape)
    assert ka.ka_workspace_set_spin_limit(ws.ptr, 64, stream()) == 0
    hdr = ws.header_words()
    torch.cuda.synchronize()
    hdr[0] = hdr[0] + 1  # same epoch, one ticket already taken
    x = ki.uniform_u32(1, n)
    out, count = empty(n), empty(1)
    assert ka.ka_compact(to_dev(x), n, None, ka.KA_PRED_ALL, 0, 0, out, count, ws.ptr, ws.nbytes, shape,
                         stream()) == 0
    torch.cuda.synchronize()
    assert ws.status(ka) == ka.KA_E_DEVICE_TIMEOUT
    # re-initialised, the same workspace works again
    assert ka.ka_workspace_init(ws.ptr, ws.nbytes, stream()) == 0
    out, k, _ = run_compact(ka, to_dev(x), n, "all", 0, tile=shape, ws=ws)
    assert k == n and np.array_equal(to_host(out, n), x)


def test_fuse_fills_literals_direct(ka):
    """prepare_index then remove zeros (Sec. 4.1, Listing 5), chained on device."""
    k = 250001
    a, b = ki.index_pairs(k, 0.3)
    index = empty(2 * k)
    n_idx = empty(1)
    assert ka.ka_prepare_index(to_dev(a), to_dev(b), k, None, index, n_idx, stream()) == 0
    out, count = empty(2 * k + 8), empty(1)
    ws = Workspace(ka, 2 * k)
    assert ka.ka_compact(index, 2 * k, n_idx, ka.KA_PRED_NE, 0, 0, out, count, ws.ptr, ws.nbytes, None,
                         stream()) == 0
    torch.cuda.synchronize()
    assert np.array_equal(to_host(index, 2 * k), oracle.prepare_index(a, b))
    y, ek = oracle.fuse_fills_literals(a, b)
    assert word(count) == ek and np.array_equal(to_host(out, ek), y)


@pytest.mark.parametrize("fused", [False, True])
def test_pipeline4_direct(ka, fused):
    """Hash map, then three chained compactions; lengths stay on the device."""
    n = (1 << 22) + 11
    x = ki.uniform_u32(3, n)
    expect = oracle.pipeline(x, ki.PIPELINE4)
    d_x = to_dev(x)
    bufs = [empty(n + 8) for _ in range(4)]
    cnts = [empty(1) for _ in range(4)]
    wss = [Workspace(ka, n) for _ in range(3)]
    st = stream()
    if fused:
        assert ka.ka_compact(d_x, n, None, ka.KA_PRED_TOPBITS_LT, 8, ka.KA_XFORM_HASH, bufs[1], cnts[1],
                             wss[0].ptr, wss[0].nbytes, None, st) == 0
    else:
        assert ka.ka_map_hash(d_x, n, None, bufs[0], cnts[0], st) == 0
        assert ka.ka_compact(bufs[0], n, cnts[0], ka.KA_PRED_TOPBITS_LT, 8, 0, bufs[1], cnts[1], wss[0].ptr,
                             wss[0].nbytes, None, st) == 0
    assert ka.ka_compact(bufs[1], n, cnts[1], ka.KA_PRED_POPC_ODD, 0, 0, bufs[2], cnts[2], wss[1].ptr,
                         wss[1].nbytes, None, st) == 0
    assert ka.ka_compact(bufs[2], n, cnts[2], ka.KA_PRED_MOD_NE0, 3, 0, bufs[3], cnts[3], wss[2].ptr,
                         wss[2].nbytes, None, st) == 0
    torch.cuda.synchronize()
    for i in (1, 2, 3):
        k = word(cnts[i])
        assert k == expect[i].size
        assert np.array_equal(to_host(bufs[i], k), expect[i])
        assert np.all(to_host(bufs[i])[k:n + 8] == SENTINEL)


# ---------------------------------------------------------------------------
def three_phase(ka, d_x, n, pred, param, xform=0, d_n=None, ws=None, cap=None):
    cap = n if cap is None else cap
    if ws is None:
        s, nb = ka.ka_three_phase_workspace_size(cap)
        assert s == 0
        buf = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
        ptr = (buf.data_ptr() + 255) // 256 * 256
        assert ka.ka_workspace_init(ptr, nb, stream()) == 0
        ws = (buf, ptr, nb)
    out, count = empty(cap + 16), empty(1)
    s = ka.ka_compact_three_phase(d_x, cap if d_n is not None else n, d_n, ka.PRED[pred], param, xform, out, count,
                                  ws[1], ws[2], stream())
    assert s == 0, ka.ka_strerror(s)
    torch.cuda.synchronize()
    assert ka.ka_workspace_status(ws[1], stream()) == (0, 0)
    return out, word(count), ws


@pytest.mark.parametrize("pred,param", PREDS[:6])
def test_three_phase_billeter(ka, pred, param):
    """Count per tile, scan of the counts, move: the same result as the oracle
    (sizes across tile boundaries, hash transform, unaligned input)."""
    for n in [0, 1, 4095, 4096, 4097, 3 * 4096 + 5, 100003, (1 << 20) + 7]:
        x = ki.uniform_u32(n + 3, n + 3)
        for xform in (0, 1):
            for off in (0, 1):
                out, k, _ = three_phase(ka, to_dev(x)[off:], n, pred, param, xform)
                src = x[off:off + n]
                y, ek = oracle.compact(oracle.map_hash(src) if xform else src, pred, param)
                assert k == ek and np.array_equal(to_host(out, k), y), (n, xform, off)
                assert np.all(to_host(out)[k:n + 16] == SENTINEL)


def test_three_phase_live_length_and_reuse(ka):
    n = (1 << 21) + 11
    x = ki.uniform_u32(42, n)
    ws = None
    for rep, live in enumerate([n, 5, 0, 12345, n - 1, 4096]):
        d_n = to_dev(np.array([live], dtype=np.uint32))
        out, k, ws = three_phase(ka, to_dev(x), n, "lt", ki.threshold_for(0.3), d_n=d_n, ws=ws)
        y, ek = oracle.compact(x[:live], "lt", ki.threshold_for(0.3))
        assert k == ek and np.array_equal(to_host(out, k), y), rep
