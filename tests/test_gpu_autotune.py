"""The autotuner on the GPU: for the compaction, the scan and the batch kernel,
ka_autotune returns a supported shape it timed (positive time), ka_tile_for
then reports that shape, the cache file holds it and a fresh process reloads
it, and the kernels launched with no tile (so on the tuned shape) still match
the oracle bit for bit."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import ka_inputs as ki  # noqa: E402
import oracle  # noqa: E402
from gpu_util import Workspace, empty, stream, to_dev, to_host, word  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
REGISTER_SHAPES = {(128, 4), (128, 8), (128, 16), (256, 4), (256, 8), (256, 16), (512, 4), (512, 8), (512, 16),
                   (1024, 4), (1024, 8)}
TMA_SHAPES = {(256, 16), (512, 16), (768, 16)}
BATCH_ONLY_SHAPES = {(704, 16)}  # the batch kernel also has this shape
BATCH_KEY = 1 << 17  # every batch looks up the entry stored under this size


@pytest.fixture(scope="module")
def ka(cuda_ok):
    import paper_1709_07781_gb300 as m
    return m


def reload_in_fresh_process(path, kernel, n):
    """ka_tile_for in a new process before and after ka_autotune_load(path)."""
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import paper_1709_07781_gb300 as ka\n"
            "s0, before = ka.ka_tile_for(%d, %d)\n"
            "s1 = ka.ka_autotune_load(%r)\n"
            "s2, after = ka.ka_tile_for(%d, %d)\n"
            "print(s0, s1, s2, before[0], before[1], after[0], after[1])\n") % (ROOT, kernel, n, path, kernel, n)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    v = [int(t) for t in r.stdout.split()]
    assert v[:3] == [0, 0, 0]
    return (v[3], v[4]), (v[5], v[6])


def tune(ka, kernel, n, path):
    s, shape, us = ka.ka_autotune(kernel, n, path, stream())
    assert s == 0, ka.ka_strerror(s)
    assert shape in REGISTER_SHAPES | TMA_SHAPES | (BATCH_ONLY_SHAPES if kernel == ka.KA_KERNEL_BATCH else set())
    assert us > 0.0
    return shape, us


def cached_entry(path, kernel):
    with open(path) as fh:
        entries = json.load(fh)["entries"]
    mine = [e for e in entries if e["kernel"] == kernel]
    assert mine, entries
    return mine


def test_autotune_compaction(ka, tmp_path):
    n = 1 << 24
    path = str(tmp_path / "tune.json")
    shape, _ = tune(ka, ka.KA_KERNEL_COMPACT, n, path)
    assert ka.ka_tile_for(ka.KA_KERNEL_COMPACT, n) == (0, shape)
    assert any((e["block"], e["ipt"]) == shape for e in cached_entry(path, ka.KA_KERNEL_COMPACT))
    before, after = reload_in_fresh_process(path, ka.KA_KERNEL_COMPACT, n)
    assert after == shape
    assert before == (768, 16)  # the default a process without the cache uses
    # the compaction with no tile runs on the tuned shape and matches the oracle
    for s_ in (0.01, 0.5):
        x = ki.uniform_u32(600 + int(100 * s_), n)
        ws = Workspace(ka, n, (128, 4))  # sized for the smallest tile: fits any tuned shape
        out, cnt = empty(n + 16), empty(1)
        assert ka.ka_compact(to_dev(x), n, None, ka.PRED["lt"], ki.threshold_for(s_), 0, out, cnt, ws.ptr,
                             ws.nbytes, None, stream()) == 0
        torch.cuda.synchronize()
        assert ws.status(ka) == 0
        want, k = oracle.compact(x, "lt", ki.threshold_for(s_))
        assert word(cnt) == k and np.array_equal(to_host(out, k), want)


def test_autotune_scan(ka, tmp_path):
    n = (1 << 24) + 3
    path = str(tmp_path / "tune.json")
    shape, _ = tune(ka, ka.KA_KERNEL_SCAN, n, path)
    assert ka.ka_tile_for(ka.KA_KERNEL_SCAN, n) == (0, shape)
    assert any((e["block"], e["ipt"]) == shape for e in cached_entry(path, ka.KA_KERNEL_SCAN))
    _, after = reload_in_fresh_process(path, ka.KA_KERNEL_SCAN, n)
    assert after == shape
    f = (ki.uniform_u32(610, n) & np.uint32(1)).astype(np.uint32)
    ws = Workspace(ka, n, (128, 4))
    out, total = empty(n), empty(1)
    assert ka.ka_exclusive_scan(to_dev(f), n, None, out, total, ws.ptr, ws.nbytes, None, stream()) == 0
    torch.cuda.synchronize()
    assert ws.status(ka) == 0
    want, tot = oracle.exclusive_scan(f)
    assert word(total) == tot and np.array_equal(to_host(out, n), want)


def test_autotune_batch(ka, tmp_path):
    from test_gpu_batch import check, run_batch
    path = str(tmp_path / "tune.json")
    shape, _ = tune(ka, ka.KA_KERNEL_BATCH, 1 << 24, path)
    assert shape in TMA_SHAPES | REGISTER_SHAPES | BATCH_ONLY_SHAPES
    assert ka.ka_tile_for(ka.KA_KERNEL_BATCH, BATCH_KEY) == (0, shape)
    assert any((e["block"], e["ipt"]) == shape for e in cached_entry(path, ka.KA_KERNEL_BATCH))
    _, after = reload_in_fresh_process(path, ka.KA_KERNEL_BATCH, BATCH_KEY)
    assert after == shape
    rng = np.random.default_rng(620)
    sizes = [int(v) for v in rng.integers(1, 200_000, size=40)]
    xs = [ki.uniform_u32(621 + i, m) for i, m in enumerate(sizes)]
    preds = [("lt", ki.threshold_for(float(rng.uniform(0.01, 0.99)))) for _ in sizes]
    dst, counts, _ = run_batch(ka, xs, preds)  # no tile: the tuned shape
    check(xs, preds, None, dst, counts)
