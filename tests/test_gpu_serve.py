"""The serving loop through the C ABI: a Poisson trace of 1-4 stage pipelines
over fresh seeded arrays, under continuous batching and under plain
per-request launches. Every request's result equals the oracle's pipeline
over the same input (alone), whatever it shared the GPU with (in the mix);
admission respects the budget; oversized requests are rejected."""
import ctypes

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


@pytest.fixture()
def system(ka):
    s, h = ka.ka_system_create(0)
    assert s == 0, ka.ka_strerror(s)
    yield h
    assert ka.ka_system_destroy(h, 1) == 0


def stage_spec(ka, st):
    if st.kind == "map_hash":
        return (ka.PRED["all"], 0, ka.KA_XFORM_HASH)
    return (ka.PRED[st.pred], st.param, ka.KA_XFORM_NONE)


def trace(ka, rate, duration, lo, hi, seed_off=0, max_requests=None):
    tr = ki.config_serve(rate, duration, lo, hi, master_seed=ki.MASTER_SEED + 5 + seed_off,
                         max_requests=max_requests)
    stages = [[stage_spec(ka, ki.PIPELINE4[int(k)]) for k in tr.stage_kind[r][:tr.n_stages[r]]]
              for r in range(len(tr.n))]
    return tr, stages, ka.serve_requests(tr.arrival_s, tr.n, tr.seeds, stages)


def expected(tr, r):
    """The oracle's result for request r alone: (data, count)."""
    st = [ki.PIPELINE4[int(k)] for k in tr.stage_kind[r][:tr.n_stages[r]]]
    y = oracle.pipeline(oracle.generate(int(tr.seeds[r]), int(tr.n[r])), st)[-1]
    return y, len(y)


@pytest.mark.parametrize("mode,flags", [(0, 0), (0, 1), (1, 0), (2, 0), (2, 1)])
def test_every_result_matches_the_oracle(ka, system, mode, flags):
    """flags 1 (KA_SERVE_BATCH_LONE): ticks of one request are batched too;
    else they run as that request's plain launches."""
    tr, stages, reqs = trace(ka, 4000.0, 0.1, 8, 18)
    n = len(tr.n)
    assert n > 200
    # value mode for every 7th request: its data comes back too
    outs = {}
    for r in range(0, n, 7):
        buf = np.zeros(int(tr.n[r]) + 1, dtype=np.uint32)
        outs[r] = buf
        reqs[r].h_out = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
        reqs[r].h_out_cap = buf.size
    s, res, stats = ka.serve(system, reqs, mode=mode, flags=flags)
    assert s == 0, ka.ka_strerror(s)
    assert stats.elements == int(np.sum(tr.n)) and stats.rejected == 0
    for r in range(n):
        y, k = expected(tr, r)
        assert res[r].status == 0 and res[r].count == k, (r, res[r].status, res[r].count, k)
        assert res[r].done_s >= res[r].admit_s >= tr.arrival_s[r] - 1e-3
        if r in outs:
            assert np.array_equal(outs[r][:k], y) and outs[r][k] == 0
    if mode != 1:
        assert stats.iterations < n  # requests shared batched launches
    else:
        assert stats.iterations == n
    if mode == 1 or flags:
        assert stats.lone_ticks == 0
    if mode == 0:
        # every tick was one graph launch, or one request's plain launches
        assert stats.graph_launches + stats.lone_ticks == stats.iterations
        assert stats.graph_launches > 0
    else:
        assert stats.graph_launches == 0


@pytest.mark.parametrize("flags", [0, 1])
def test_same_result_alone_and_in_the_mix(ka, system, flags):
    """A request served alone (as a tick of its own: plain launches, or batched
    with flags 1) and inside a busy trace gives the same count and data."""
    tr, stages, reqs = trace(ka, 20000.0, 0.05, 10, 20, seed_off=1)
    s, mix, _ = ka.serve(system, reqs, mode=0)
    assert s == 0
    for r in [0, len(tr.n) // 2, len(tr.n) - 1]:
        one = ka.serve_requests([0.0], [tr.n[r]], [tr.seeds[r]], [stages[r]])
        buf_one = np.zeros(int(tr.n[r]), dtype=np.uint32)
        one[0].h_out = buf_one.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
        one[0].h_out_cap = buf_one.size
        s, alone, st1 = ka.serve(system, one, mode=0, flags=flags)
        assert st1.lone_ticks == (0 if flags else 1)
        assert s == 0 and alone[0].status == 0 and mix[r].status == 0
        assert alone[0].count == mix[r].count
        y, k = expected(tr, r)
        assert alone[0].count == k and np.array_equal(buf_one[:k], y)


def test_budget_admission_and_rejection(ka, system):
    tr, stages, reqs = trace(ka, 50000.0, 0.01, 14, 18, seed_off=2)
    budget = 4 << 20  # 4 MiB: at most a few requests of up to 1 MiB each at once
    big = ka.serve_requests([0.0], [3 << 20], [5], [[(ka.PRED["lt"], 7, 0)]])
    s, res, stats = ka.serve(system, reqs, mode=0, budget_bytes=budget)
    assert s == 0
    assert stats.peak_bytes <= budget and stats.rejected == 0
    for r in range(len(tr.n)):
        _, k = expected(tr, r)
        assert res[r].status == 0 and res[r].count == k
    s, res, stats = ka.serve(system, big, mode=1, budget_bytes=budget)
    assert s == 0 and stats.rejected == 1 and res[0].status == ka.KA_E_BUDGET


def test_invalid_stage_is_reported(ka, system):
    reqs = ka.serve_requests([0.0, 0.0], [1000, 1000], [1, 2], [[(ka.PRED["mod_ne0"], 0, 0)], [(ka.PRED["ne"], 0, 0)]])
    s, res, _ = ka.serve(system, reqs, mode=0)
    assert s == 0
    assert res[0].status == ka.KA_E_ARG
    assert res[1].status == 0 and res[1].count == oracle.compact(oracle.generate(2, 1000), "ne", 0)[1]


@pytest.mark.parametrize("mode,flags", [(0, 0), (1, 0)])
def test_full_size_trace_sampled(ka, mode, flags):
    """The timed serving workload itself (20 000 requests/s for 1 s, sizes
    2^10..2^24, 1-4 stages, a 64 GiB budget): every request succeeds, every
    element is counted, and a deterministic sample (the four largest requests
    and 24 spread over the trace) returns the oracle's data."""
    s, sysh = ka.ka_system_create(0, budget_bytes=64 << 30)
    assert s == 0, ka.ka_strerror(s)
    try:
        tr = ki.config_serve(20000.0, 1.0)
        stages = [[stage_spec(ka, ki.PIPELINE4[int(k)]) for k in tr.stage_kind[r][:tr.n_stages[r]]]
                  for r in range(len(tr.n))]
        reqs = ka.serve_requests(tr.arrival_s, tr.n, tr.seeds, stages)
        n = len(tr.n)
        assert n > 15000 and int(np.max(tr.n)) > (1 << 23)
        sample = sorted(set(np.argsort(tr.n)[-4:].tolist()) | set(np.linspace(0, n - 1, 24).astype(int).tolist()))
        outs = {}
        for r in sample:
            buf = np.zeros(int(tr.n[r]) + 1, dtype=np.uint32)
            outs[r] = buf
            reqs[r].h_out = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
            reqs[r].h_out_cap = buf.size
        s, res, stats = ka.serve(sysh, reqs, mode=mode, flags=flags)
        assert s == 0, ka.ka_strerror(s)
        assert stats.elements == int(np.sum(tr.n)) and stats.rejected == 0
        assert all(res[r].status == 0 for r in range(n))
        for r in sample:
            y, k = expected(tr, r)
            assert res[r].count == k, (r, res[r].count, k)
            assert np.array_equal(outs[r][:k], y) and outs[r][k] == 0, r
    finally:
        assert ka.ka_system_destroy(sysh, 1) == 0
