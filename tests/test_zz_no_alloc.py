"""ka_compact_static (compaction whose workspace is the library's own fixed
device array) against the CPU oracle and against ka_compact with a
caller-allocated workspace, bit for bit, over calls made one after another on
one stream; and its device-side failure report, read through the array's
address. Collected last, so it runs both after every other GPU test (the array
then keeps whatever earlier calls left) and alone in a fresh process (its first
call does the set-up)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import ka_inputs as ki  # noqa: E402
import oracle  # noqa: E402
from gpu_util import SENTINEL, Workspace, empty, stream, to_dev, to_host, word  # noqa: E402


@pytest.fixture(scope="module")
def ka(cuda_ok):
    import paper_1709_07781_gb300 as m
    return m


def run_both(ka, d_x, n, pred, param, xform=0, d_n=None, live=None, x=None):
    """The same compaction through both entry points, both checked against the
    oracle on the host copy x of the live input."""
    live = n if live is None else live
    out_ref, cnt_ref = empty(n + 16), empty(1)
    ws = Workspace(ka, n)
    s = ka.ka_compact(d_x, n, d_n, ka.PRED[pred], param, xform, out_ref, cnt_ref, ws.ptr, ws.nbytes, None,
                      stream())
    assert s == 0, ka.ka_strerror(s)
    out, cnt = empty(n + 16), empty(1)
    s = ka.ka_compact_static(d_x, n, d_n, ka.PRED[pred], param, xform, out, cnt, None, stream())
    assert s == 0, ka.ka_strerror(s)
    torch.cuda.synchronize()
    assert ws.status(ka) == 0
    k_ref, k = word(cnt_ref), word(cnt)
    assert k == k_ref
    assert 0 < k < live
    assert np.array_equal(to_host(out, k), to_host(out_ref, k))
    assert np.all(to_host(out)[k:n + 16] == SENTINEL)
    want, ek = oracle.compact(oracle.map_hash(x) if xform else x, pred, param)
    assert k == ek and np.array_equal(to_host(out, k), want)
    s, ws_ptr, _ = ka.ka_compact_static_workspace(stream())
    assert s == 0 and ka.ka_workspace_status(ws_ptr, stream()) == (0, 0)
    return k


def test_static_matches_workspace_entry_point_two_calls(ka):
    # call 1: mid-size, plain threshold, 16-byte-aligned input
    n1 = (1 << 20) + 37
    x1 = ki.uniform_u32(501, n1)
    run_both(ka, to_dev(x1), n1, "lt", ki.threshold_for(0.37), x=x1)
    # call 2, right after: the largest size allowed, hash transform, modulus test
    n2 = ka.KA_STATIC_MAX_N
    x2 = ki.uniform_u32(502, n2)
    run_both(ka, to_dev(x2), n2, "mod_ne0", 3, xform=1, x=x2)


def test_static_live_length_and_unaligned_input(ka):
    # input starts 4 bytes past a 16-byte boundary (the register kernel), and
    # the live length comes from a device word below the capacity
    cap = (1 << 22) + 5
    live = (1 << 21) + 77
    x = ki.uniform_u32(503, cap + 1)
    buf = to_dev(x)
    d_n = to_dev(np.array([live], dtype=np.uint32))
    run_both(ka, buf[1:], cap, "popc_odd", 0, d_n=d_n, live=live, x=x[1:1 + live])
    run_both(ka, buf[1:], cap, "and_mask_eq0", 3, d_n=d_n, live=live, x=x[1:1 + live])


def test_static_allocates_nothing_per_call(ka):
    n = (1 << 23) + 3
    d_x = to_dev(ki.uniform_u32(504, n))
    outs = [empty(n + 16) for _ in range(2)]
    cnts = [empty(1) for _ in range(2)]
    assert ka.ka_compact_static(d_x, n, None, ka.PRED["lt"], ki.threshold_for(0.5), 0, outs[0], cnts[0], None,
                                stream()) == 0
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for i in range(4):
        assert ka.ka_compact_static(d_x, n, None, ka.PRED["lt"], ki.threshold_for(0.5), 0, outs[i & 1],
                                    cnts[i & 1], None, stream()) == 0
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    assert word(cnts[0]) == word(cnts[1])
    k = word(cnts[0])
    assert np.array_equal(to_host(outs[0], k), to_host(outs[1], k))


def test_static_rejects_sizes_above_the_limit(ka):
    d_x, out, cnt = empty(16), empty(16), empty(1)
    s = ka.ka_compact_static(d_x, ka.KA_STATIC_MAX_N + 1, None, ka.PRED["lt"], 5, 0, out, cnt, None, stream())
    assert s == ka.KA_E_TOO_LARGE
    assert "KA_STATIC_MAX_N" in ka.ka_strerror(s)
    torch.cuda.synchronize()
    assert word(cnt) == SENTINEL  # nothing launched


class _DeviceWords:
    """A view of n 64-bit words at a raw device address, for torch."""

    def __init__(self, addr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i8", "data": (addr, False),
                                         "strides": None, "version": 3}


def test_static_device_timeout_is_reported_and_cleared(ka):
    """A look-back of a ka_compact_static call that gives up is reported by
    ka_workspace_status on the array's address, and ka_workspace_init clears
    it. The failure is made on the host: one ticket of the array's current
    launch epoch is taken before the call, so tile 0 of the register kernel is
    never handed out and tile 1's look-back waits for it until a spin limit of
    64 polls runs out (every access stays in bounds, every wait is bounded)."""
    s, ws_ptr, nbytes = ka.ka_compact_static_workspace(stream())
    assert s == 0 and ws_ptr % 256 == 0 and nbytes > 256
    n = 64 * 1024
    x = ki.uniform_u32(505, n)
    d_x, out, cnt = to_dev(x), empty(n), empty(1)
    shape = (256, 4)
    assert ka.ka_workspace_set_spin_limit(ws_ptr, 64, stream()) == 0
    torch.cuda.synchronize()
    hdr = torch.as_tensor(_DeviceWords(ws_ptr, 32), device="cuda")
    hdr[0] = hdr[0] + 1  # same epoch, one ticket already taken
    torch.cuda.synchronize()
    assert ka.ka_compact_static(d_x, n, None, ka.PRED["all"], 0, 0, out, cnt, shape, stream()) == 0
    assert ka.ka_workspace_status(ws_ptr, stream()) == (0, ka.KA_E_DEVICE_TIMEOUT)
    # cleared on the caller's stream, the array works again, for both kernels
    assert ka.ka_workspace_init(ws_ptr, nbytes, stream()) == 0
    assert ka.ka_workspace_status(ws_ptr, stream()) == (0, 0)
    for sh in (shape, None):
        out, cnt = empty(n + 16), empty(1)
        assert ka.ka_compact_static(d_x, n, None, ka.PRED["lt"], ki.threshold_for(0.3), 0, out, cnt, sh,
                                    stream()) == 0
        assert ka.ka_workspace_status(ws_ptr, stream()) == (0, 0)
        want, k = oracle.compact(x, "lt", ki.threshold_for(0.3))
        assert word(cnt) == k and np.array_equal(to_host(out, k), want)
