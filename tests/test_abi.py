"""The C ABI library without a GPU: it loads, exports every entry point that
include/ka.h declares, and its host-only calls behave (no kernel runs here)."""
import ctypes
import os
import re
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ka.h")


@pytest.fixture(scope="module")
def ka():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1709_07781_gb300 as m
    return m


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(ka_[a-z0-9_]+)\s*\(", text)
    return sorted({n for n in names if not n.endswith("_fn")})


def test_every_declared_symbol_is_exported(ka):
    names = declared_functions()
    assert len(names) >= 40
    lib = ctypes.CDLL(ka._lib.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding covers every one of them under the same name
    assert set(names) <= set(ka._lib.DECLARED), set(names) - set(ka._lib.DECLARED)


def declared_arity():
    """Parameter count of every function prototype in include/ka.h."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    text = re.sub(r"#[^\n]*", "", text)
    out = {}
    for m in re.finditer(r"\b(ka_[a-z0-9_]+)\s*\(([^()]*)\)\s*;", text):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_signatures_match_the_header(ka):
    """Every ctypes prototype has as many arguments as the C declaration."""
    arity = declared_arity()
    assert len(arity) >= 40
    wrong = {n: (len(ka._lib._SIGS[n][1]), k) for n, k in arity.items()
             if n in ka._lib._SIGS and len(ka._lib._SIGS[n][1]) != k}
    assert not wrong, wrong


def test_strerror_and_version(ka):
    assert ka.ka_version() >= 100
    assert "timed out" in ka.ka_strerror(ka.KA_E_DEVICE_TIMEOUT)
    for code in ka._lib.STATUS:
        assert ka.ka_strerror(code) != "unknown status"


def test_workspace_size(ka):
    s, b = ka.ka_workspace_size(1 << 28)
    assert s == 0 and b >= 256 + 8 * ((1 << 28) // 512)
    s, b2 = ka.ka_workspace_size(1 << 28, (256, 16))
    assert s == 0 and 256 + 8 * ((1 << 28) // 4096) <= b2 < b
    assert ka.ka_workspace_size(1 << 33)[0] == ka.KA_E_ARG
    assert ka.ka_workspace_size(100, (100, 4))[0] == ka.KA_E_ARG


def test_default_tiles(ka):
    assert ka.ka_tile_for(ka.KA_KERNEL_COMPACT, 1 << 28) == (0, (768, 16))
    assert ka.ka_tile_for(ka.KA_KERNEL_SCAN, 1 << 28) == (0, (512, 16))
    assert ka.ka_tile_for(ka.KA_KERNEL_BATCH, 1 << 17) == (0, (704, 16))
    s, t = ka.ka_tile_for(ka.KA_KERNEL_COMPACT, 1 << 20)
    assert s == 0 and t[0] * t[1] <= 4096


def test_batch_only_shape(ka, tmp_path):
    """(704, 16) is a shape of the batch kernel (five stages) and of no other:
    a batch workspace takes it, a single-array workspace refuses it, and a
    tuning cache entry naming it is taken for the batch kernel and skipped
    for the compaction."""
    s, nbytes = ka.ka_batch_workspace_size(16, 1 << 20, (704, 16))
    assert s == 0 and nbytes > 0
    s, _ = ka.ka_workspace_size(1 << 20, (704, 16))
    assert s == ka.KA_E_ARG
    assert ka.ka_batch_workspace_size(16, 1 << 20, (640, 16))[0] == ka.KA_E_ARG
    before = ka.ka_tile_for(ka.KA_KERNEL_COMPACT, 1 << 30)
    p = tmp_path / "tune.json"
    p.write_text('{"entries": [\n  {"kernel": %d, "bucket": 30, "block": 704, "ipt": 16, "us": 1.0},\n'
                 '  {"kernel": %d, "bucket": 17, "block": 704, "ipt": 16, "us": 1.0}\n]}\n'
                 % (ka.KA_KERNEL_COMPACT, ka.KA_KERNEL_BATCH))
    assert ka.ka_autotune_load(str(p)) == 0
    assert ka.ka_tile_for(ka.KA_KERNEL_COMPACT, 1 << 30) == before
    assert ka.ka_tile_for(ka.KA_KERNEL_BATCH, 1 << 17) == (0, (704, 16))


def test_autotune_cache_roundtrip(ka, tmp_path):
    p = tmp_path / "tune.json"
    p.write_text('{"entries": [\n  {"kernel": 0, "bucket": 17, "block": 128, "ipt": 8, "us": 3.5}\n]}\n')
    assert ka.ka_autotune_load(str(p)) == 0
    assert ka.ka_tile_for(ka.KA_KERNEL_COMPACT, 1 << 17) == (0, (128, 8))
    assert ka.ka_autotune_load(str(tmp_path / "missing.json")) == ka.KA_E_ARG


def test_kernel_predicates_match_the_oracle_definition(ka):
    """The kernels' canonical predicates (x < p<<28 for the top-bits test, the
    division-free multiple test) agree with the oracle's plain definitions."""
    import oracle
    import ka_inputs as ki
    xs = list(map(int, ki.uniform_u32(5, 3000))) + [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 12, 0x7FFFFFFF, 0x80000000,
                                                   0xFFFFFFFF, 0xFFFFFFFE, 0xFFFFFFFD, 0xFFFFFFFC, 3 * 1431655765]
    cases = [("and_mask_eq0", 3), ("lt", 12345), ("popc_odd", 0), ("ne", 7), ("ne", 0), ("all", 0)]
    cases += [("topbits_lt", p) for p in (0, 1, 7, 8, 15, 16, 100)]
    cases += [("mod_ne0", d) for d in (1, 2, 3, 4, 5, 6, 7, 12, 24, 96, 1000, 65536, 2**31, 2**31 + 1,
                                       0xFFFFFFFF, 0xFFFFFFFE)]
    for pred, param in cases:
        for x in xs:
            s, got = ka.ka_debug_pred_keep(ka.PRED[pred], param, x)
            assert s == 0
            assert got == oracle.keep(pred, param, x), (pred, param, x)
    assert ka.ka_debug_pred_keep(ka.KA_PRED_MOD_NE0, 0, 5)[0] == ka.KA_E_ARG


def test_references_cannot_be_serialised(ka):
    buf = ctypes.create_string_buffer(16)
    n = ctypes.c_uint64(0)
    assert ka.lib.ka_ref_serialize(None, buf, 16, ctypes.byref(n)) == ka.KA_E_NOT_SERIALIZABLE


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No fallback: importing the package without libka.so raises."""
    import shutil
    pkg = os.path.join(ROOT, "paper_1709_07781_gb300")
    dst = tmp_path / "paper_1709_07781_gb300"
    shutil.copytree(pkg, dst, ignore=shutil.ignore_patterns("_build", "__pycache__"))
    r = subprocess.run([sys.executable, "-c", "import paper_1709_07781_gb300"], cwd=str(tmp_path),
                       capture_output=True, text=True)
    assert r.returncode != 0 and "libka.so is not built" in r.stderr


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1709_07781_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "ka_oracle" not in text, f


def test_host_stream_scratch_size_and_refusals(ka):
    """ka_compact_host's sizing and the argument checks it makes before any
    device work: three rotating buffer sets (input and one output per
    predicate) of whole 256-byte blocks, then the compaction workspace."""
    r256 = lambda b: (b + 255) // 256 * 256  # noqa: E731
    for chunk, p in ((1 << 24, 3), (1000, 1), (4, 4)):
        s, b = ka.ka_compact_host_scratch_size(chunk, p)
        ws = ka.ka_workspace_size(chunk)[1]
        assert s == 0 and b == 3 * (1 + p) * r256(4 * chunk) + 3 * 256 + r256(ws)
    assert ka.ka_compact_host_scratch_size(0, 2) == ka.ka_compact_host_scratch_size(1 << 24, 2)
    assert ka.ka_compact_host_scratch_size(1 << 24, 0)[0] == ka.KA_E_ARG
    assert ka.ka_compact_host_scratch_size(1 << 24, 5)[0] == ka.KA_E_ARG
    assert ka.ka_compact_host_scratch_size(1 << 32, 1)[0] == ka.KA_E_ARG
    x = np.arange(16, dtype=np.uint32)
    out = [np.zeros(16, dtype=np.uint32)]
    lt = ka.PRED["lt"]
    _, b = ka.ka_compact_host_scratch_size(1024, 1)
    fake = 1 << 40  # never dereferenced: every call below is refused first
    assert ka.ka_compact_host(x, 16, [lt], [5], [0], out, 1024, fake, b - 1)[0] == ka.KA_E_WORKSPACE
    assert ka.ka_compact_host(x, 16, [lt], [5], [0], out, 1024, fake + 8, b)[0] == ka.KA_E_ARG
    assert ka.ka_compact_host(x, 16, [lt], [5], [9], out, 1024, fake, b)[0] == ka.KA_E_ARG
    assert ka.ka_compact_host(None, 16, [lt], [5], [0], out, 1024, fake, b)[0] == ka.KA_E_ARG
    assert ka.ka_compact_host(x, 16, [lt], [5], [0], [None], 1024, fake, b)[0] == ka.KA_E_ARG
    assert ka.ka_compact_host(x, 16, [], [], [], [], 1024, fake, b)[0] == ka.KA_E_ARG
    # n = 0 needs no device work: every count is 0
    assert ka.ka_compact_host(x, 0, [lt, lt], [5, 6], [0, 0], out * 2, 1024, fake, 1 << 40) == (0, [0, 0])


def test_bench_direct_chain_refuses_unknown_flags(ka):
    """Argument checks come before any CUDA call."""
    spec = [(ka.KA_STAGE_EMPTY, 0, 0, 0)]
    assert ka.ka_bench_direct_chain(spec, None, 16, 1, flags=2)[0] == ka.KA_E_ARG
    assert ka.ka_bench_direct_chain(spec, None, 16, 0, flags=ka.KA_BENCH_WAIT_TAG)[0] == ka.KA_E_ARG


def test_last_cuda_error_names_the_failure(ka):
    """Without a GPU, a call that needs the device returns KA_E_CUDA, and
    ka_last_cuda_error gives the CUDA error behind it."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    s, _ = ka.ka_system_create(0)
    assert s == ka.KA_E_CUDA
    assert ka.ka_last_cuda_error() != 0


def test_launch_caches_are_keyed_by_device(ka):
    """The occupancy and resident-grid caches hold one value per device
    ordinal: a second device computes its own, a failed computation (a value
    <= 0) is not kept, and an ordinal outside the table is never cached."""
    s, out = ka.ka_debug_device_cache([0, 1, 0, 1, 2, 0], [10, 20, 99, 99, 30, 99])
    assert s == 0 and out == [10, 20, 10, 20, 30, 10]
    s, out = ka.ka_debug_device_cache([3, 3, 3], [-1, 7, 9])
    assert s == 0 and out == [-1, 7, 7]
    s, out = ka.ka_debug_device_cache([70, 70, -1, -1], [5, 6, 4, 8])
    assert s == 0 and out == [5, 6, 4, 8]
