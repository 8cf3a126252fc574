"""Arrays at the largest lengths the C ABI takes: 2^32 - 1 entries (every
element count lives in a 32-bit device word), and 2^32 - 4 for the TMA kernels
(their tiles start on a 16-byte boundary). At these lengths a 32-bit entry
index plus a grid stride, or the last tile's later segments, pass 2^32; the
kernels keep such positions in 64 bits.

The inputs are closed forms (x_j = j, all ones) whose results are closed forms
too (the multiples of 4, an iota), checked over the whole array on the device;
the generator and the element-wise maps are also checked against the oracle
at sampled positions (the head, the last 64 Ki entries, and spread samples).
Each test holds at most about 32 GiB of device memory."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from gpu_util import SENTINEL, Workspace, dev, empty, stream, word  # noqa: E402

N_MAX = (1 << 32) - 1  # the largest array the API takes
N_TMA = (1 << 32) - 4  # the largest the TMA kernels take
CH = 1 << 28           # entries per chunk of a device-side check


ITEM = np.dtype([("in", "<u8"), ("out", "<u8"), ("n_ptr", "<u8"), ("count", "<u8"), ("n", "<u4"),
                 ("pred", "<i4"), ("param", "<u4"), ("xform", "<u4")])
GEN = np.dtype([("out", "<u8"), ("seed", "<u8"), ("n", "<u4"), ("pad", "<u4")])


@pytest.fixture(scope="module")
def ka(cuda_ok):
    import paper_1709_07781_gb300 as m
    return m


@pytest.fixture(autouse=True)
def release_memory():
    yield
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def table_to_dev(arr: np.ndarray) -> torch.Tensor:
    raw = np.frombuffer(arr.tobytes(), dtype=np.uint8).copy()
    return torch.from_numpy(raw).to(dev())


def as_i32(v: torch.Tensor) -> torch.Tensor:
    """int64 values in [0, 2^32) -> the int32 tensor with the same bits."""
    return torch.where(v >= 2**31, v - 2**32, v).to(torch.int32)


def affine(start: int, count: int, a: int, b: int) -> torch.Tensor:
    """(a + b k) mod 2^32 for k in [start, start + count), as int32 bits
    (b k stays below 2^63 for the b used here)."""
    k = torch.arange(start, start + count, dtype=torch.int64, device=dev())
    return as_i32((a + b * k) % 2**32)


def fill_affine(t: torch.Tensor, n: int, a: int = 0, b: int = 1):
    for c in range(0, n, CH):
        m = min(CH, n - c)
        t[c:c + m] = affine(c, m, a, b)


def equals_affine(t: torch.Tensor, n: int, a: int, b: int) -> bool:
    for c in range(0, n, CH):
        m = min(CH, n - c)
        if not torch.equal(t[c:c + m], affine(c, m, a, b)):
            return False
    return True


def samples(n: int, seed: int = 5) -> np.ndarray:
    """The head, the last 64 Ki positions and 4096 spread positions below n."""
    rng = np.random.default_rng(seed)
    s = np.concatenate([np.arange(4096), np.arange(n - 65536, n), rng.integers(0, n, 4096)])
    return np.unique(s).astype(np.int64)


def read(t: torch.Tensor, idx: np.ndarray) -> np.ndarray:
    return t[torch.from_numpy(idx).to(dev())].cpu().numpy().view(np.uint32)


def sentinel_after(t: torch.Tensor, k: int, span: int = 4096) -> bool:
    w = t[k:k + span]
    return bool((w == int(np.uint32(SENTINEL).view(np.int32))).all())


@pytest.mark.parametrize("offset", [0, 1])
def test_generate_max_length(ka, offset):
    """Vector path (16-byte aligned start) and scalar path (one entry past it)."""
    seed = 11
    buf = empty(N_MAX + 8)
    x = buf[offset:]
    assert ka.ka_generate(x, N_MAX, seed, stream()) == 0
    torch.cuda.synchronize()
    idx = samples(N_MAX)
    expect = np.array([oracle.splitmix64(seed, int(i)) >> 32 for i in idx], dtype=np.uint32)
    assert np.array_equal(read(x, idx), expect)
    assert sentinel_after(x, N_MAX, 4)


def test_predicate_and_hash_max_length(ka):
    """x_j = j: keep x < t flags exactly the first t entries."""
    x = empty(N_MAX + 4)
    fill_affine(x, N_MAX)
    y = empty(N_MAX + 4)
    t = 3_000_000_000
    assert ka.ka_predicate(x, N_MAX, None, ka.PRED["lt"], t, y, stream()) == 0
    torch.cuda.synchronize()
    ones = sum(int(y[c:c + min(CH, N_MAX - c)].sum(dtype=torch.int64)) for c in range(0, N_MAX, CH))
    assert ones == t and sentinel_after(y, N_MAX, 4)
    idx = samples(N_MAX)
    assert np.array_equal(read(y, idx), oracle.predicate_map(idx.astype(np.uint32), "lt", t))
    assert ka.ka_map_hash(x, N_MAX, None, y, None, stream()) == 0
    torch.cuda.synchronize()
    assert np.array_equal(read(y, idx), oracle.map_hash(idx.astype(np.uint32)))
    assert sentinel_after(y, N_MAX, 4)


@pytest.mark.parametrize("lead", [0, 1])
def test_compact_tma_max_length(ka, lead):
    """Tile (768, 16): 13312 entries per tile, which does not divide 2^32, so
    the last tile's later segments lie past 2^32. Input x_j = j + lead (the
    view starts `lead` entries past a 16-byte boundary); keep x & 3 == 0:
    the multiples of 4 in [lead, lead + n)."""
    n = N_TMA
    buf = empty(n + 8)
    fill_affine(buf, n + 8)
    x = buf[lead:]
    k_exp = (lead + n - 1) // 4 - (lead + 3) // 4 + 1
    first = (lead + 3) // 4 * 4
    out = empty(k_exp + 4096)
    cnt = empty(1)
    ws = Workspace(ka, n, (768, 16))
    assert ka.ka_compact(x, n, None, ka.PRED["and_mask_eq0"], 3, 0, out, cnt, ws.ptr, ws.nbytes, (768, 16),
                         stream()) == 0
    torch.cuda.synchronize()
    assert ws.status(ka) == 0
    assert word(cnt) == k_exp
    assert equals_affine(out, k_exp, first, 4)
    assert sentinel_after(out, k_exp)


def test_compact_tma_max_length_keep_all(ka):
    n = N_TMA
    x = empty(n)
    fill_affine(x, n, 12345, 40503)
    out = empty(n + 4)
    cnt = empty(1)
    ws = Workspace(ka, n, (768, 16))
    assert ka.ka_compact(x, n, None, ka.PRED["all"], 0, 0, out, cnt, ws.ptr, ws.nbytes, (768, 16), stream()) == 0
    torch.cuda.synchronize()
    assert ws.status(ka) == 0 and word(cnt) == n
    assert all(torch.equal(out[c:c + min(CH, n - c)], x[c:c + min(CH, n - c)]) for c in range(0, n, CH))
    assert sentinel_after(out, n, 4)


def test_compact_autotuned_above_tma_limit(ka):
    """n = 2^32 - 1 with no shape given: the library picks a shape whose
    kernel takes that length (the TMA kernels stop at 2^32 - 4)."""
    x = empty(N_MAX)
    fill_affine(x, N_MAX)
    k_exp = 1 << 30  # multiples of 4 below 2^32 - 1
    out = empty(k_exp + 4096)
    cnt = empty(1)
    ws = Workspace(ka, N_MAX)
    assert ka.ka_compact(x, N_MAX, None, ka.PRED["and_mask_eq0"], 3, 0, out, cnt, ws.ptr, ws.nbytes, None,
                         stream()) == 0
    torch.cuda.synchronize()
    assert ws.status(ka) == 0 and word(cnt) == k_exp
    assert equals_affine(out, k_exp, 0, 4) and sentinel_after(out, k_exp)


@pytest.mark.parametrize("n,tile", [(N_TMA, (768, 16)), (N_MAX, None)])
def test_scan_max_length(ka, n, tile):
    """Exclusive scan of all ones is the iota; the total is n."""
    f = torch.ones(n, dtype=torch.int32, device=dev())
    o = empty(n + 4)
    total = empty(1)
    ws = Workspace(ka, n, tile)
    assert ka.ka_exclusive_scan(f, n, None, o, total, ws.ptr, ws.nbytes, tile, stream()) == 0
    torch.cuda.synchronize()
    assert ws.status(ka) == 0 and word(total) == n
    assert equals_affine(o, n, 0, 1) and sentinel_after(o, n, 4)


def test_three_phase_max_length(ka):
    x = empty(N_MAX)
    fill_affine(x, N_MAX)
    k_exp = 1 << 30
    out = empty(k_exp + 4096)
    cnt = empty(1)
    s, nbytes = ka.ka_three_phase_workspace_size(N_MAX)
    assert s == 0
    wsb = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev())
    wp = (wsb.data_ptr() + 255) // 256 * 256
    assert ka.ka_workspace_init(wp, nbytes, stream()) == 0
    assert ka.ka_compact_three_phase(x, N_MAX, None, ka.PRED["and_mask_eq0"], 3, 0, out, cnt, wp, nbytes,
                                     stream()) == 0
    torch.cuda.synchronize()
    s, dev_status = ka.ka_workspace_status(wp, stream())
    assert s == 0 and dev_status == 0
    assert word(cnt) == k_exp
    assert equals_affine(out, k_exp, 0, 4) and sentinel_after(out, k_exp)


def test_batch_with_a_max_length_item(ka):
    """One item of 2^32 - 1 entries starting one entry past a 16-byte
    boundary (its tiles then cover 2^32 + 1 positions), beside small items;
    then batched generation into the same unaligned item."""
    n = N_MAX
    buf = empty(n + 8)
    fill_affine(buf, n + 8)
    x = buf[1:]                 # x_j = j + 1
    k_exp = n // 4              # multiples of 4 in [1, n]
    out = empty(k_exp + 4096)
    small = [oracle.generate(7 + i, m) for i, m in enumerate((1000, 5, 70001))]
    s_in = [torch.from_numpy(v.view(np.int32)).to(dev()) for v in small]
    s_out = [empty(v.size + 16) for v in small]
    counts = empty(4)
    items = np.zeros(4, dtype=ITEM)
    items[0] = (x.data_ptr(), out.data_ptr(), 0, counts.data_ptr(), n, ka.PRED["and_mask_eq0"], 3, 0)
    t = 2_000_000_000
    for i in range(3):
        items[1 + i] = (s_in[i].data_ptr(), s_out[i].data_ptr(), 0, counts.data_ptr() + 4 * (1 + i), small[i].size,
                        ka.PRED["lt"], t, 0)
    ws = Workspace(ka, n + sum(v.size for v in small) + 64, None, batch_items=4)
    assert ka.ka_compact_batch(table_to_dev(items), 4, 4, ws.ptr, ws.nbytes, None, 0, stream()) == 0
    torch.cuda.synchronize()
    assert ws.status(ka) == 0
    assert word(counts, 0) == k_exp
    assert equals_affine(out, k_exp, 4, 4) and sentinel_after(out, k_exp)
    for i, v in enumerate(small):
        y, k = oracle.compact(v, "lt", t)
        assert word(counts, 1 + i) == k
        assert np.array_equal(s_out[i][:k].cpu().numpy().view(np.uint32), y)
    del out
    gen = np.zeros(1, dtype=GEN)
    gen[0] = (x.data_ptr(), 23, n, 0)
    assert ka.ka_generate_batch(table_to_dev(gen), 1, 4, ws.ptr, ws.nbytes, stream()) == 0
    torch.cuda.synchronize()
    idx = samples(n)
    expect = np.array([oracle.splitmix64(23, int(i)) >> 32 for i in idx], dtype=np.uint32)
    assert np.array_equal(read(x, idx), expect)
    # the entries on either side of the item are untouched
    assert word(buf, 0) == 0 and word(buf, n + 1) == 0 and word(buf, n + 2) == 1
