"""Kernel actors through the C ABI: spawn, compose, request/receive with device
references and with host buffers (value mode), results bit-identical to the
oracle and to direct launches; reference lifetime, budget, type errors and
host-side fault injection."""
import ctypes
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import ka_inputs as ki  # noqa: E402
import oracle  # noqa: E402
from gpu_util import empty, stream, to_dev  # noqa: E402


@pytest.fixture(scope="module")
def ka(cuda_ok):
    import paper_1709_07781_gb300 as m
    return m


@pytest.fixture()
def system(ka):
    s, h = ka.ka_system_create(0)
    assert s == 0, ka.ka_strerror(s)
    yield h
    assert ka.ka_system_destroy(h, 1) == 0


def spawn(ka, sys_h, kind, pred=0, param=0, xform=0, tile=(0, 0)):
    s, a = ka.ka_spawn_stage(sys_h, kind, pred, param, xform, tile)
    assert s == 0, ka.ka_strerror(s)
    return a


def compose(ka, *actors):
    """compose(C, B, A) = C . B . A (A runs first)."""
    cur = actors[-1]
    for nxt in reversed(actors[:-1]):
        s, cur = ka.ka_compose(nxt, cur)
        assert s == 0, ka.ka_strerror(s)
    return cur


_cudart = None


def d2h(ptr: int, k: int) -> np.ndarray:
    """Copy k uint32 from a raw device pointer (test plumbing: cudaMemcpy)."""
    global _cudart
    if _cudart is None:
        _cudart = ctypes.CDLL("libcudart.so.13")
    out = np.empty(k, dtype=np.uint32)
    if k:
        torch.cuda.synchronize()
        assert _cudart.cudaMemcpy(ctypes.c_void_p(out.ctypes.data), ctypes.c_void_p(ptr), ctypes.c_size_t(4 * k),
                                  2) == 0  # cudaMemcpyDeviceToHost
    return out


def result_data(ka, ref_h, k):
    s, p, cap, dt, acc = ka.ka_ref_info(ref_h)
    assert s == 0 and cap >= k
    return d2h(p, k)


def test_three_actor_pipeline_device_refs(ka, system):
    """Cfg 1: predicate -> exclusive scan -> scatter, N = 2^20, keep (x & 3) == 0."""
    n = 1 << 20
    x = ki.uniform_u32(1, n)
    d_x = to_dev(x)
    pred = spawn(ka, system, ka.KA_STAGE_PREDICATE, ka.KA_PRED_AND_MASK_EQ0, 3)
    scan = spawn(ka, system, ka.KA_STAGE_EXSCAN)
    move = spawn(ka, system, ka.KA_STAGE_SCATTER)
    pipe = compose(ka, move, scan, pred)
    assert ka.ka_actor_arity(pipe) == (0, 1, 1)
    s, rx = ka.ka_ref_wrap(system, d_x, n, n)
    assert s == 0
    torch.cuda.synchronize()
    s, req = ka.ka_request(pipe, ka.make_msg([rx]))
    assert s == 0
    s, msg = ka.ka_receive(req)
    assert s == 0, ka.ka_strerror(s)
    y, k = oracle.compact(x, "and_mask_eq0", 3)
    assert msg.count == k and msg.n_refs == 1
    assert np.array_equal(result_data(ka, msg.refs[0], k), y)
    assert ka.ka_ref_count(msg.refs[0]) == (0, k)
    assert ka.ka_ref_release(msg.refs[0]) == 0
    assert ka.ka_ref_release(msg.refs[0]) == ka.KA_E_STALE
    assert ka.ka_ref_release(rx) == 0
    for a in (pipe, pred, scan, move):
        assert ka.ka_actor_release(a) == 0
    assert ka.ka_actor_release(pipe) == ka.KA_E_STALE
    assert ka.ka_system_pool_bytes(system)[1] == 0


def test_value_mode_upload_and_read_back(ka, system):
    """First stage uploads host data, last stage reads the result back (Sec. 3.5)."""
    n = 300001
    x = ki.uniform_u32(5, n)
    comp = spawn(ka, system, ka.KA_STAGE_COMPACT, ka.KA_PRED_LT, ki.threshold_for(0.37))
    out = np.zeros(n, dtype=np.uint32)
    s, req = ka.ka_request(comp, ka.make_msg(h_in=x, h_out=out))
    assert s == 0
    s, msg = ka.ka_receive(req)
    assert s == 0
    y, k = oracle.compact(x, "lt", ki.threshold_for(0.37))
    assert msg.count == k and np.array_equal(out[:k], y) and not out[k:].any()
    for i in range(msg.n_refs):
        ka.ka_ref_release(msg.refs[i])
    ka.ka_actor_release(comp)


@pytest.mark.parametrize("fused_map", [False, True])
def test_four_stage_pipeline_matches_oracle_and_direct(ka, system, fused_map):
    """Cfg 3 (smaller N): hash map, keep top-bits < 8, keep popc odd, keep % 3 != 0."""
    n = (1 << 22) + 5
    x = ki.uniform_u32(3, n)
    stages = []
    if fused_map:
        stages.append(spawn(ka, system, ka.KA_STAGE_COMPACT, ka.KA_PRED_TOPBITS_LT, 8, ka.KA_XFORM_HASH))
    else:
        stages.append(spawn(ka, system, ka.KA_STAGE_MAP_HASH))
        stages.append(spawn(ka, system, ka.KA_STAGE_COMPACT, ka.KA_PRED_TOPBITS_LT, 8))
    stages.append(spawn(ka, system, ka.KA_STAGE_COMPACT, ka.KA_PRED_POPC_ODD, 0))
    stages.append(spawn(ka, system, ka.KA_STAGE_COMPACT, ka.KA_PRED_MOD_NE0, 3))
    pipe = compose(ka, *reversed(stages))
    out = np.zeros(n, dtype=np.uint32)
    s, req = ka.ka_request(pipe, ka.make_msg(h_in=x, h_out=out))
    assert s == 0
    s, msg = ka.ka_receive(req)
    assert s == 0, ka.ka_strerror(s)
    expect = oracle.pipeline(x, ki.PIPELINE4)[-1]
    assert msg.count == expect.size and np.array_equal(out[:msg.count], expect)
    for i in range(msg.n_refs):
        ka.ka_ref_release(msg.refs[i])
    for a in [pipe] + stages:
        ka.ka_actor_release(a)


@pytest.mark.parametrize("fused_map", [False, True])
def test_four_stage_pipeline_full_size(ka, system, fused_map):
    """The 4-stage workload at its full size (N = 2^26, seed 3), device
    references as the overhead comparison runs it: the last stage's data and
    count equal the oracle's."""
    w = ki.config_pipeline4()
    x = torch.empty(w.n, dtype=torch.int32, device="cuda")
    assert ka.ka_generate(x, w.n, w.seed, stream()) == 0
    torch.cuda.synchronize()
    stages = []
    if fused_map:
        stages.append(spawn(ka, system, ka.KA_STAGE_COMPACT, ka.KA_PRED_TOPBITS_LT, 8, ka.KA_XFORM_HASH))
    else:
        stages.append(spawn(ka, system, ka.KA_STAGE_MAP_HASH))
        stages.append(spawn(ka, system, ka.KA_STAGE_COMPACT, ka.KA_PRED_TOPBITS_LT, 8))
    stages.append(spawn(ka, system, ka.KA_STAGE_COMPACT, ka.KA_PRED_POPC_ODD, 0))
    stages.append(spawn(ka, system, ka.KA_STAGE_COMPACT, ka.KA_PRED_MOD_NE0, 3))
    pipe = compose(ka, *reversed(stages))
    s, rx = ka.ka_ref_wrap(system, x, w.n, w.n)
    assert s == 0
    s, req = ka.ka_request(pipe, ka.make_msg([rx]))
    assert s == 0
    s, msg = ka.ka_receive(req)
    assert s == 0, ka.ka_strerror(s)
    expect = oracle.pipeline(oracle.generate(w.seed, w.n), w.stages)[-1]
    assert msg.count == expect.size and msg.n_refs == 1
    assert np.array_equal(result_data(ka, msg.refs[0], msg.count), expect)
    ka.ka_ref_release(msg.refs[0])
    ka.ka_ref_release(rx)
    for a in [pipe] + stages:
        ka.ka_actor_release(a)


def test_generate_stage_and_empty_stage(ka, system):
    gen = spawn(ka, system, ka.KA_STAGE_GENERATE)
    nop = spawn(ka, system, ka.KA_STAGE_EMPTY)
    comp = spawn(ka, system, ka.KA_STAGE_COMPACT, ka.KA_PRED_POPC_ODD, 0)
    pipe = compose(ka, comp, nop, gen)
    out = np.zeros(70000, dtype=np.uint32)
    s, req = ka.ka_request(pipe, ka.make_msg(seed=99, gen_n=70000, h_out=out))
    assert s == 0
    s, msg = ka.ka_receive(req)
    assert s == 0
    y, k = oracle.compact(oracle.generate(99, 70000), "popc_odd", 0)
    assert msg.count == k and np.array_equal(out[:k], y)
    for i in range(msg.n_refs):
        ka.ka_ref_release(msg.refs[i])
    for a in (pipe, gen, nop, comp):
        ka.ka_actor_release(a)


def test_result_that_is_the_input_keeps_one_handle(ka, system):
    """An empty stage passes its input on, so each receive returns the
    wrapped reference itself: every such result comes back as the wrapping
    handle, each receive's hold is released through it, and the wrapping
    hold goes last, after which the handle is stale (and the system's
    teardown frees the reference once)."""
    n = 4096
    x = torch.zeros(n, dtype=torch.int32, device="cuda")
    s, rx = ka.ka_ref_wrap(system, x, n, n)
    assert s == 0
    nop = spawn(ka, system, ka.KA_STAGE_EMPTY)
    assert ka.ka_ref_retain(rx) == 0  # an extra external hold, shared by the handle
    for _ in range(5):
        s, req = ka.ka_request(nop, ka.make_msg([rx]))
        assert s == 0
        s, msg = ka.ka_receive(req)
        assert s == 0 and msg.n_refs == 1
        assert msg.refs[0] == rx
        assert ka.ka_ref_release(msg.refs[0]) == 0
    assert ka.ka_ref_release(rx) == 0  # the retained hold
    assert ka.ka_ref_count(rx) == (0, n)
    assert ka.ka_ref_release(rx) == 0  # the wrapping hold: the handle ends
    assert ka.ka_ref_release(rx) == ka.KA_E_STALE
    assert ka.ka_ref_count(rx)[0] == ka.KA_E_STALE
    ka.ka_actor_release(nop)


def test_new_systems_do_not_see_old_completion_tags(ka):
    """Systems made and destroyed in turn, one request each: every first
    request waits for completion tag 1 in its slot, which a destroyed
    system's slot (pinned memory is handed back uncleared) would already
    hold. Each result must still be the real one."""
    n = (1 << 20) + 7
    x = ki.uniform_u32(31, n)
    d_x = to_dev(x)
    _, k = oracle.compact(x, "lt", ki.threshold_for(0.3))
    for _ in range(12):
        s, sys_h = ka.ka_system_create(0)
        assert s == 0
        comp = spawn(ka, sys_h, ka.KA_STAGE_COMPACT, ka.KA_PRED_LT, ki.threshold_for(0.3))
        s, rx = ka.ka_ref_wrap(sys_h, d_x, n, n)
        assert s == 0
        s, req = ka.ka_request(comp, ka.make_msg([rx]))
        assert s == 0
        s, msg = ka.ka_receive(req)
        assert s == 0 and msg.count == k
        for i in range(msg.n_refs):
            ka.ka_ref_release(msg.refs[i])
        ka.ka_ref_release(rx)
        ka.ka_actor_release(comp)
        assert ka.ka_system_destroy(sys_h, 1) == 0


@pytest.mark.parametrize("fused", [True, False])
def test_fuse_fills_literals_composite(ka, system, fused):
    """fuse = move . count . prepare (Sec. 4.1, Listing 5), refs only between stages."""
    k = 100003
    a, b = ki.index_pairs(k, 0.4)
    prep = spawn(ka, system, ka.KA_STAGE_PREPARE)
    if fused:
        rest = [spawn(ka, system, ka.KA_STAGE_COMPACT, ka.KA_PRED_NE, 0)]
    else:
        rest = [spawn(ka, system, ka.KA_STAGE_PREDICATE, ka.KA_PRED_NE, 0), spawn(ka, system, ka.KA_STAGE_EXSCAN),
                spawn(ka, system, ka.KA_STAGE_SCATTER)]
    pipe = compose(ka, *reversed([prep] + rest))
    d_a, d_b = to_dev(a), to_dev(b)  # borrowed by the refs: keep alive until received
    s, ra = ka.ka_ref_wrap(system, d_a, k, k)
    s, rb = ka.ka_ref_wrap(system, d_b, k, k)
    torch.cuda.synchronize()
    out = np.zeros(2 * k, dtype=np.uint32)
    s, req = ka.ka_request(pipe, ka.make_msg([ra, rb], h_out=out))
    assert s == 0
    s, msg = ka.ka_receive(req)
    assert s == 0
    y, kk = oracle.fuse_fills_literals(a, b)
    assert msg.count == kk and np.array_equal(out[:kk], y)
    for i in range(msg.n_refs):
        ka.ka_ref_release(msg.refs[i])
    for r in (ra, rb):
        ka.ka_ref_release(r)
    for x in [pipe, prep] + rest:
        ka.ka_actor_release(x)


def test_compose_type_mismatch(ka, system):
    pred = spawn(ka, system, ka.KA_STAGE_PREDICATE, ka.KA_PRED_LT, 5)   # (x) -> (x, f)
    comp = spawn(ka, system, ka.KA_STAGE_COMPACT, ka.KA_PRED_LT, 5)     # (x) -> (y)
    s, _ = ka.ka_compose(comp, pred)
    assert s == ka.KA_E_TYPE
    # message arity checked at the first stage
    d1, d2 = empty(16), empty(16)
    s, r1 = ka.ka_ref_wrap(system, d1, 16, 16)
    s, r2 = ka.ka_ref_wrap(system, d2, 16, 16)
    s, req = ka.ka_request(comp, ka.make_msg([r1, r2]))
    assert s == 0
    s, msg = ka.ka_receive(req)
    assert s == ka.KA_E_TYPE
    assert ka.ka_spawn_stage(system, 99)[0] == ka.KA_E_ARG
    assert ka.ka_spawn_stage(system, ka.KA_STAGE_COMPACT, ka.KA_PRED_MOD_NE0, 0)[0] == ka.KA_E_ARG
    for r in (r1, r2):
        ka.ka_ref_release(r)
    ka.ka_actor_release(pred)
    ka.ka_actor_release(comp)


def test_refs_not_serializable(ka, system):
    s, r = ka.ka_ref_alloc(system, 1000)
    assert s == 0
    assert ka.ka_ref_serialize(r)[0] == ka.KA_E_NOT_SERIALIZABLE
    s, used, budget = ka.ka_system_pool_bytes(system)
    assert used >= 4000 and budget == 64 << 30
    assert ka.ka_ref_retain(r) == 0
    assert ka.ka_ref_release(r) == 0
    assert ka.ka_ref_info(r)[0] == 0      # still held once
    assert ka.ka_ref_release(r) == 0
    assert ka.ka_ref_info(r)[0] == ka.KA_E_STALE
    assert ka.ka_system_pool_bytes(system)[1] == 0


def test_pool_returns_to_zero_after_many_requests(ka, system):
    comp = spawn(ka, system, ka.KA_STAGE_COMPACT, ka.KA_PRED_AND_MASK_EQ0, 1)
    x = ki.uniform_u32(8, 50000)
    d_x = to_dev(x)
    s, rx = ka.ka_ref_wrap(system, d_x, x.size, x.size)
    torch.cuda.synchronize()
    y, k = oracle.compact(x, "and_mask_eq0", 1)
    reqs = []
    for _ in range(50):
        s, q = ka.ka_request(comp, ka.make_msg([rx]))
        assert s == 0
        reqs.append(q)
    for q in reqs:
        s, msg = ka.ka_receive(q)
        assert s == 0 and msg.count == k
        ka.ka_ref_release(msg.refs[0])
    assert ka.ka_system_pool_bytes(system)[1] == 0
    ka.ka_ref_release(rx)
    ka.ka_actor_release(comp)


def test_budget_rejects_oversized_request(ka):
    s, sys_h = ka.ka_system_create(0, budget_bytes=1 << 20)
    assert s == 0
    comp = spawn(ka, sys_h, ka.KA_STAGE_COMPACT, ka.KA_PRED_ALL, 0)
    x = ki.uniform_u32(1, 1 << 20)  # 4 MiB output > 1 MiB budget
    d_x = to_dev(x)
    s, rx = ka.ka_ref_wrap(sys_h, d_x, x.size, x.size)
    torch.cuda.synchronize()
    s, q = ka.ka_request(comp, ka.make_msg([rx]))
    assert s == 0
    s, msg = ka.ka_receive(q)
    assert s == ka.KA_E_BUDGET
    assert ka.ka_system_pool_bytes(sys_h)[1] == 0
    ka.ka_ref_release(rx)
    ka.ka_actor_release(comp)
    assert ka.ka_system_destroy(sys_h, 0) == 0


def test_injected_stage_failure_propagates_and_releases(ka, system):
    gen = spawn(ka, system, ka.KA_STAGE_GENERATE)
    comp = spawn(ka, system, ka.KA_STAGE_COMPACT, ka.KA_PRED_LT, 1 << 31)
    pipe = compose(ka, comp, gen)
    assert ka.ka_debug_fail_stage(comp, 1) == 0  # first message passes, later ones fail
    s, q1 = ka.ka_request(pipe, ka.make_msg(seed=1, gen_n=4096))
    s, m1 = ka.ka_receive(q1)
    assert s == 0
    ka.ka_ref_release(m1.refs[0])
    s, q2 = ka.ka_request(pipe, ka.make_msg(seed=2, gen_n=4096))
    s, m2 = ka.ka_receive(q2)
    assert s == ka.KA_E_INJECTED and m2.n_refs == 0
    assert ka.ka_system_pool_bytes(system)[1] == 0   # generated buffer released
    assert ka.ka_debug_fail_stage(comp, -1) == 0
    s, q3 = ka.ka_request(pipe, ka.make_msg(seed=3, gen_n=4096))
    s, m3 = ka.ka_receive(q3)
    assert s == 0
    ka.ka_ref_release(m3.refs[0])
    for a in (pipe, gen, comp):
        ka.ka_actor_release(a)


def test_dispatcher_death_notifies_monitor(ka):
    s, sys_h = ka.ka_system_create(0)
    seen = []
    cb = ka.MONITOR_FN(lambda user, reason: seen.append(reason))
    assert ka.ka_system_monitor(sys_h, cb, None) == 0
    comp = spawn(ka, sys_h, ka.KA_STAGE_EMPTY)
    assert ka.ka_debug_kill_dispatcher(sys_h) == 0
    assert seen == [ka.KA_E_CLOSED]
    s, rx = ka.ka_ref_alloc(sys_h, 16)
    assert ka.ka_request(comp, ka.make_msg([rx]))[0] == ka.KA_E_CLOSED
    ka.ka_ref_release(rx)
    ka.ka_actor_release(comp)
    assert ka.ka_system_destroy(sys_h, 1) == 0


def test_receive_timeout_then_result(ka, system):
    comp = spawn(ka, system, ka.KA_STAGE_COMPACT, ka.KA_PRED_ALL, 0)
    gen = spawn(ka, system, ka.KA_STAGE_GENERATE)
    pipe = compose(ka, comp, gen)
    s, q = ka.ka_request(pipe, ka.make_msg(seed=5, gen_n=1 << 26))
    s, m = ka.ka_receive(q, 0)
    assert s in (ka.KA_E_TIMEOUT, 0)
    if s == ka.KA_E_TIMEOUT:
        s, m = ka.ka_receive(q, -1)
    assert s == 0 and m.count == 1 << 26
    ka.ka_ref_release(m.refs[0])
    for a in (pipe, comp, gen):
        ka.ka_actor_release(a)


def test_concurrent_requesters(ka, system):
    comp = spawn(ka, system, ka.KA_STAGE_COMPACT, ka.KA_PRED_MOD_NE0, 7)
    errors = []

    def worker(tid):
        try:
            for i in range(20):
                n = 1000 + 997 * (tid * 20 + i)
                x = ki.uniform_u32(tid * 1000 + i, n)
                out = np.zeros(n, dtype=np.uint32)
                s, q = ka.ka_request(comp, ka.make_msg(h_in=x, h_out=out))
                assert s == 0
                s, m = ka.ka_receive(q)
                assert s == 0
                y, k = oracle.compact(x, "mod_ne0", 7)
                assert m.count == k and np.array_equal(out[:k], y)
                for j in range(m.n_refs):
                    ka.ka_ref_release(m.refs[j])
        except Exception as e:  # pragma: no cover - reported below
            errors.append(repr(e))

    ts = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors
    ka.ka_actor_release(comp)


def three_actor(ka, sys_h, mask):
    pred = spawn(ka, sys_h, ka.KA_STAGE_PREDICATE, ka.KA_PRED_AND_MASK_EQ0, mask)
    scan = spawn(ka, sys_h, ka.KA_STAGE_EXSCAN)
    scat = spawn(ka, sys_h, ka.KA_STAGE_SCATTER)
    return compose(ka, scat, scan, pred), (pred, scan, scat)


def test_results_received_in_reverse_order(ka, system):
    """Requests that finish while nobody waits on them are fulfilled by the
    completion thread; receiving them later, in reverse order, gives each its
    own result."""
    pipe, parts = three_actor(ka, system, 3)
    inputs, reqs = [], []
    for i in range(16):
        x = ki.uniform_u32(100 + i, 3000 + 4099 * i)
        d_x = to_dev(x)
        s, rx = ka.ka_ref_wrap(system, d_x, x.size, x.size)
        assert s == 0
        s, q = ka.ka_request(pipe, ka.make_msg([rx]))
        assert s == 0
        inputs.append((x, d_x, rx))
        reqs.append(q)
    torch.cuda.synchronize()
    for (x, _, rx), q in reversed(list(zip(inputs, reqs))):
        s, m = ka.ka_receive(q)
        assert s == 0
        y, k = oracle.compact(x, "and_mask_eq0", 3)
        assert m.count == k and np.array_equal(result_data(ka, m.refs[0], k), y)
        for j in range(m.n_refs):
            ka.ka_ref_release(m.refs[j])
        ka.ka_ref_release(rx)
    assert ka.ka_system_pool_bytes(system)[1] == 0
    for a in (pipe,) + parts:
        ka.ka_actor_release(a)


def test_threads_share_composite_with_device_refs(ka, system):
    """Four threads drive one composite over device references: requests run
    on the requesting thread while its actors are idle and through the
    mailboxes and the dispatcher thread otherwise; every result matches the
    oracle and the pool is empty afterwards."""
    pipe, parts = three_actor(ka, system, 1)
    cases = []
    for t in range(4):
        for i in range(12):
            x = ki.uniform_u32(7000 + 100 * t + i, 1 + 2749 * (t * 12 + i))
            cases.append((t, x, to_dev(x)))
    torch.cuda.synchronize()
    errors = []

    def worker(tid):
        try:
            for t, x, d_x in cases:
                if t != tid:
                    continue
                s, rx = ka.ka_ref_wrap(system, d_x, x.size, x.size)
                assert s == 0
                s, q = ka.ka_request(pipe, ka.make_msg([rx]))
                assert s == 0
                s, m = ka.ka_receive(q)
                assert s == 0
                y, k = oracle.compact(x, "and_mask_eq0", 1)
                assert m.count == k and np.array_equal(result_data(ka, m.refs[0], k), y)
                for j in range(m.n_refs):
                    ka.ka_ref_release(m.refs[j])
                ka.ka_ref_release(rx)
        except Exception as e:  # pragma: no cover - reported below
            errors.append(repr(e))

    ts = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors
    assert ka.ka_system_pool_bytes(system)[1] == 0
    for a in (pipe,) + parts:
        ka.ka_actor_release(a)


def test_receiver_that_blocks_gets_result(ka, system):
    """A request that outlasts the receiver's spin window (a Mandelbrot stage
    of 8192 x 4096 pixels, up to 2000 steps each) is fulfilled by the
    completion thread and wakes the blocked receiver."""
    w, h, iters = 8192, 4096, 2000
    a = spawn(ka, system, ka.KA_STAGE_MANDELBROT, w, iters, h)
    for _ in range(2):
        s, q = ka.ka_request(a, ka.make_msg())
        assert s == 0
        s, m = ka.ka_receive(q)
        assert s == 0 and m.count == w * h
        for j in range(m.n_refs):
            ka.ka_ref_release(m.refs[j])
    assert ka.ka_system_pool_bytes(system)[1] == 0
    ka.ka_actor_release(a)


def test_destroy_with_requests_in_flight_makes_every_handle_stale(ka):
    """Destroying a system with requests still in flight (force) finishes or
    fails them; afterwards its request, reference and actor handles return
    KA_E_STALE instead of touching freed state, and a new system works."""
    s, sys_h = ka.ka_system_create(0)
    assert s == 0
    gen = spawn(ka, sys_h, ka.KA_STAGE_GENERATE)
    comp = spawn(ka, sys_h, ka.KA_STAGE_COMPACT, ka.KA_PRED_LT, 1 << 31)
    pipe = compose(ka, comp, gen)
    reqs = []
    for i in range(8):
        s, q = ka.ka_request(pipe, ka.make_msg(seed=i, gen_n=1 << 22))
        assert s == 0
        reqs.append(q)
    s, rx = ka.ka_ref_alloc(sys_h, 1 << 20)
    assert s == 0
    assert ka.ka_system_destroy(sys_h, 1) == 0
    for q in reqs:
        assert ka.ka_receive(q, 0)[0] == ka.KA_E_STALE
    assert ka.ka_ref_release(rx) == ka.KA_E_STALE
    assert ka.ka_ref_info(rx)[0] == ka.KA_E_STALE
    assert ka.ka_request(pipe, ka.make_msg(seed=1, gen_n=16))[0] == ka.KA_E_STALE
    for a in (pipe, gen, comp):
        assert ka.ka_actor_release(a) == ka.KA_E_STALE
    assert ka.ka_system_destroy(sys_h, 1) == ka.KA_E_STALE
    # a fresh system is unaffected
    s, sys2 = ka.ka_system_create(0)
    assert s == 0
    g2 = spawn(ka, sys2, ka.KA_STAGE_GENERATE)
    s, q = ka.ka_request(g2, ka.make_msg(seed=3, gen_n=1000))
    s, m = ka.ka_receive(q)
    assert s == 0 and m.count == 1000
    ka.ka_ref_release(m.refs[0])
    ka.ka_actor_release(g2)
    assert ka.ka_system_destroy(sys2, 0) == 0


def test_receive_time_out_bounds_the_wait(ka, system):
    """A time-out of 0 polls (returns at once, not after the spin window);
    a short time-out on a long request expires; then the result arrives."""
    import time
    a = spawn(ka, system, ka.KA_STAGE_MANDELBROT, 8192, 2000, 4096)  # about 25 ms of GPU work
    s, q = ka.ka_request(a, ka.make_msg())
    assert s == 0
    t0 = time.perf_counter()
    s, _ = ka.ka_receive(q, 0)
    dt = time.perf_counter() - t0
    assert s == ka.KA_E_TIMEOUT and dt < 1e-3, dt
    t0 = time.perf_counter()
    s, _ = ka.ka_receive(q, 300_000)  # 0.3 ms
    dt = time.perf_counter() - t0
    assert s == ka.KA_E_TIMEOUT and dt < 5e-3, dt
    s, m = ka.ka_receive(q, -1)
    assert s == 0 and m.count == 8192 * 4096
    for j in range(m.n_refs):
        ka.ka_ref_release(m.refs[j])
    ka.ka_actor_release(a)


@pytest.mark.parametrize("flags", [0, 1])
def test_bench_loops_count_like_the_oracle(ka, system, flags):
    """The native timing loops (direct chain, with either wait, and the
    request loop) compute the same result length as the oracle."""
    n = (1 << 18) + 3
    x = ki.uniform_u32(21, n)
    d_x = to_dev(x)
    spec = [(ka.KA_STAGE_COMPACT, ka.KA_PRED_LT, ki.threshold_for(0.4), 0)]
    s, sec, k_direct = ka.ka_bench_direct_chain(spec, d_x, n, 5, flags=flags)
    assert s == 0 and sec > 0
    comp = spawn(ka, system, ka.KA_STAGE_COMPACT, ka.KA_PRED_LT, ki.threshold_for(0.4))
    s, rx = ka.ka_ref_wrap(system, d_x, n, n)
    assert s == 0
    s, sec, k_actor = ka.ka_bench_request_loop(comp, ka.make_msg([rx]), 5, 1)
    assert s == 0
    _, k = oracle.compact(x, "lt", ki.threshold_for(0.4))
    assert k_direct == k_actor == k
    ka.ka_ref_release(rx)
    ka.ka_actor_release(comp)
