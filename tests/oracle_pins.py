"""Pins for the CPU oracle: checks against facts that do not come from the oracle.

Each check raises AssertionError when the currently loaded oracle library is
wrong. They are used by test_oracle_pins.py on the real oracle and by
test_oracle_mutations.py on copies of it with a planted mistake, to show that a
plausible slip anywhere in the oracle fails at least one pin.

What each pin rests on:
  * generator   - published SplitMix64 check values (tests/golden).
  * compaction  - exhaustive search on tiny inputs: the unique index subset whose
                  members all pass the test and whose non-members all fail it;
                  numpy boolean-mask selection (a library routine) on larger data;
                  invariants (count = number of kept entries, stable subsequence).
  * predicates  - hand-picked values whose answer is fixed by arithmetic
                  (bit patterns, multiples of 3, the threshold boundary).
  * scan        - all-ones gives 0, 1, 2, ...; all-zeros gives zeros; numpy
                  cumsum (library) with mod 2^32 wrap; first differences.
  * hash map    - recovery of x by the modular inverse of 2654435761 found by
                  Newton iteration; h(0) = 0, h(1) = 2654435761.
  * interleave  - numpy strided slices.
"""
from __future__ import annotations

import itertools
import os

import numpy as np

import oracle
import ka_inputs as ki

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden_splitmix():
    with open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) as fh:
        lines = [ln.strip() for ln in fh if ln.strip() and not ln.startswith("#")]
    seed = int(lines[0].split()[1])
    return seed, [int(v) for v in lines[1:]]


def check_generator():
    seed, vals = _golden_splitmix()
    got = [oracle.splitmix64(seed, i) for i in range(len(vals))]
    assert got == vals, (got, vals)
    x = oracle.generate(seed, len(vals))
    assert [int(v) for v in x] == [v >> 32 for v in vals]


def numpy_keep(pred, param, x):
    """Independent vectorised form of each keep test (numpy operators)."""
    x = np.asarray(x, dtype=np.uint32)
    if pred == "and_mask_eq0":
        return (x & np.uint32(param)) == 0
    if pred == "lt":
        return x < np.uint32(param)
    if pred == "topbits_lt":
        return (x >> np.uint32(28)) < np.uint32(param)
    if pred == "popc_odd":
        return (np.bitwise_count(x) & 1) == 1
    if pred == "mod_ne0":
        return (x % np.uint32(param)) != 0
    if pred == "ne":
        return x != np.uint32(param)
    if pred == "all":
        return np.ones(x.shape, dtype=bool)
    raise ValueError(pred)


def check_predicate_values():
    cases = [
        ("and_mask_eq0", 3, 4, 1), ("and_mask_eq0", 3, 5, 0), ("and_mask_eq0", 3, 0, 1),
        ("and_mask_eq0", 3, 0xFFFFFFFC, 1), ("and_mask_eq0", 3, 0xFFFFFFFE, 0),
        ("lt", 1000, 999, 1), ("lt", 1000, 1000, 0), ("lt", 0, 0, 0), ("lt", 0xFFFFFFFF, 0xFFFFFFFE, 1),
        ("topbits_lt", 8, 0x7FFFFFFF, 1), ("topbits_lt", 8, 0x80000000, 0),
        ("topbits_lt", 8, 0xF0000000, 0), ("topbits_lt", 1, 0x0FFFFFFF, 1), ("topbits_lt", 1, 0x10000000, 0),
        ("popc_odd", 0, 0, 0), ("popc_odd", 0, 1, 1), ("popc_odd", 0, 3, 0), ("popc_odd", 0, 7, 1),
        ("popc_odd", 0, 0x80000000, 1), ("popc_odd", 0, 0xFFFFFFFF, 0), ("popc_odd", 0, 0x80000001, 0),
        ("mod_ne0", 3, 9, 0), ("mod_ne0", 3, 10, 1), ("mod_ne0", 3, 0, 0), ("mod_ne0", 3, 0xFFFFFFFF, 0),
        ("mod_ne0", 3, 0xFFFFFFFE, 1), ("mod_ne0", 7, 49, 0),
        ("ne", 0, 0, 1 - 1), ("ne", 0, 5, 1), ("ne", 5, 5, 0),
        ("all", 0, 0, 1), ("all", 0, 0xFFFFFFFF, 1), ("all", 7, 7, 1),
    ]
    for pred, param, x, want in cases:
        got = oracle.keep(pred, param, x)
        assert got == want, (pred, param, hex(x), got, want)
    # a zero modulus is rejected, not evaluated
    assert oracle.keep("mod_ne0", 0, 5) == -1


def _exhaustive_subset(x, keepmask):
    """The unique subset S of indices with every member kept and every
    non-member removed, found by trying all 2^n subsets; returns x[S] in order."""
    n = len(x)
    found = []
    for bits in range(1 << n):
        ok = True
        for i in range(n):
            inside = (bits >> i) & 1
            if inside != int(keepmask[i]):
                ok = False
                break
        if ok:
            found.append([x[i] for i in range(n) if (bits >> i) & 1])
    assert len(found) == 1
    return found[0]


def check_compaction_exhaustive(max_n=12, search_n=8):
    # every keep/remove pattern up to max_n entries: removed entries are 0 and
    # kept entries distinct non-zero values, so 'ne 0' keeps exactly the pattern.
    # Up to search_n entries the expectation comes from the subset search; above
    # it, from the pattern itself (the non-zero entries in index order).
    for n in range(0, max_n + 1):
        for pattern in range(1 << n):
            mask = [(pattern >> i) & 1 for i in range(n)]
            x = [(i + 1) * 2654435 % 1000003 + 1 if mask[i] else 0 for i in range(n)]
            want = _exhaustive_subset(x, mask) if n <= search_n else [v for v, m in zip(x, mask) if m]
            y, k = oracle.compact(np.array(x, dtype=np.uint32), "ne", 0)
            assert k == sum(mask) and list(map(int, y)) == want, (n, pattern, y, want)


def check_compaction_small_exhaustive_values():
    # all arrays of length <= 5 over a small alphabet that straddles each
    # predicate's boundary, checked against the exhaustive subset search.
    alphabet = [0, 1, 2, 3, 4, 7, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFF]
    preds = [("and_mask_eq0", 3), ("lt", 4), ("topbits_lt", 8), ("popc_odd", 0), ("mod_ne0", 3), ("ne", 3)]
    for pred, param in preds:
        for n in range(0, 4):
            for tup in itertools.product(alphabet, repeat=n):
                x = np.array(tup, dtype=np.uint32)
                mask = numpy_keep(pred, param, x)
                want = _exhaustive_subset(list(map(int, x)), list(map(int, mask)))
                y, k = oracle.compact(x, pred, param)
                assert k == len(want) and list(map(int, y)) == want, (pred, tup)


def _is_stable_subsequence(y, x):
    j = 0
    for v in x:
        if j < len(y) and y[j] == v:
            j += 1
    return j == len(y)


def check_compaction_library(n=20000, seed=11):
    x = ki.uniform_u32(seed, n)
    for pred, param in [("and_mask_eq0", 3), ("lt", ki.threshold_for(0.5)), ("topbits_lt", 8),
                        ("popc_odd", 0), ("mod_ne0", 3), ("ne", int(x[17])), ("all", 0)]:
        mask = numpy_keep(pred, param, x)
        y, k = oracle.compact(x, pred, param)
        assert k == int(mask.sum())
        assert np.array_equal(y, x[mask])
        assert _is_stable_subsequence(list(map(int, y[:500])), list(map(int, x)))
        f = oracle.predicate_map(x, pred, param)
        assert np.array_equal(f.astype(bool), mask)


def check_scan():
    for n in [0, 1, 2, 5, 1000]:
        o, total = oracle.exclusive_scan(np.ones(n, dtype=np.uint32))
        assert total == n and np.array_equal(o, np.arange(n, dtype=np.uint32))
        o, total = oracle.exclusive_scan(np.zeros(n, dtype=np.uint32))
        assert total == 0 and not o.any()
    v = ki.uniform_u32(5, 4096)
    o, total = oracle.exclusive_scan(v)
    ref = np.concatenate([[0], np.cumsum(v.astype(np.uint64))]) % (1 << 32)
    assert np.array_equal(o, ref[:-1].astype(np.uint32)) and total == int(ref[-1])
    assert np.array_equal((o[1:] - o[:-1]).astype(np.uint32), v[:-1])
    # wrap mod 2^32
    o, total = oracle.exclusive_scan(np.array([0xFFFFFFFF, 2, 5], dtype=np.uint32))
    assert list(map(int, o)) == [0, 0xFFFFFFFF, 1] and total == 6


def check_three_phase(n=5000):
    x = ki.uniform_u32(21, n)
    for pred, param in [("and_mask_eq0", 3), ("lt", 123456789), ("popc_odd", 0)]:
        f, o, total, y = oracle.three_phase(x, pred, param)
        mask = numpy_keep(pred, param, x)
        assert total == int(mask.sum())
        assert np.array_equal(y, x[mask])
        assert np.array_equal(o, (np.cumsum(mask) - mask).astype(np.uint32))


def _inverse_mod_2_32(a):
    """Newton iteration for the inverse of an odd a mod 2^32: each step doubles
    the number of correct low bits (x <- x (2 - a x))."""
    x = a  # correct to 3 bits for odd a
    for _ in range(5):
        x = (x * (2 - a * x)) % (1 << 32)
    assert (a * x) % (1 << 32) == 1
    return x


def check_hash():
    a = 2654435761
    inv = _inverse_mod_2_32(a)
    x = ki.uniform_u32(31, 50000)
    h = oracle.map_hash(x)
    back = ((h.astype(np.uint64) * np.uint64(inv)) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    assert np.array_equal(back, x)
    h = oracle.map_hash(np.array([0, 1, 2, 0xFFFFFFFF], dtype=np.uint32))
    assert list(map(int, h)) == [0, a, (2 * a) % (1 << 32), (1 << 32) - a]
    # bijection: no two distinct inputs collide
    assert np.unique(oracle.map_hash(np.arange(1 << 16, dtype=np.uint32))).size == 1 << 16


def check_interleave():
    a, b = ki.index_pairs(1000, 0.3)
    idx = oracle.prepare_index(a, b)
    assert np.array_equal(idx[0::2], a) and np.array_equal(idx[1::2], b)
    y, k = oracle.fuse_fills_literals(a, b)
    assert k == int((a != 0).sum() + (b != 0).sum())
    assert np.array_equal(y, idx[idx != 0])


def _binom_ok(k, n, p, sigmas=6.0):
    sd = (n * p * (1 - p)) ** 0.5
    return abs(k - n * p) <= sigmas * sd + 1


def check_selectivity():
    # keep (x & 3) == 0 keeps ~1/4; x < floor(s 2^32) keeps ~s; the 4-stage
    # pipeline keeps ~1/2, ~1/2, ~2/3 per compaction stage.
    n = 1 << 16
    x = ki.uniform_u32(1, n)
    _, k = oracle.compact(x, "and_mask_eq0", 3)
    assert _binom_ok(k, n, 0.25)
    for s in (0.01, 0.5, 0.99):
        _, k = oracle.compact(x, "lt", ki.threshold_for(s))
        assert _binom_ok(k, n, s)
    outs = oracle.pipeline(x, ki.PIPELINE4)
    sizes = [n] + [o.size for o in outs]
    assert sizes[1] == n
    assert _binom_ok(sizes[2], sizes[1], 0.5)
    assert _binom_ok(sizes[3], sizes[2], 0.5)
    assert _binom_ok(sizes[4], sizes[3], 2.0 / 3.0)


def _one_point(cr, ci, max_iter):
    """Escape count of the single point c = cr + ci i (a 1 x 1 image)."""
    return int(oracle.mandelbrot(1, 1, cr, ci, cr + 1.0, ci + 1.0, max_iter)[0, 0])


def check_mandelbrot_points():
    """Escape counts that follow from the orbit of z <- z^2 + c by hand (all
    values are small integers, exact in single precision), with the rule
    "step while |z|^2 <= 4": c = 1: 0, 1, 2, 5 -> 3 steps; c = 2: 0, 2, 6 -> 2;
    c = 3: 0, 3 -> 1; c = -2: 0, -2, 2, 2, ... stays on |z|^2 = 4 -> never
    escapes; c = -1: 0, -1, 0, ... bounded; c = 0: bounded; c = i: 0, i, -1 + i,
    -i, -1 + i, ... bounded; c = -i by symmetry; c = 1 + i: 0, 1 + i, 1 + 3i
    (|z|^2 = 10) -> 2 steps; c = -1 + i: 0, -1 + i, -1 - i, -1 + 3i -> 3 steps;
    c = 0.25 (the cusp, converges to 1/2) bounded."""
    m = 50
    cases = [((1.0, 0.0), 3), ((2.0, 0.0), 2), ((3.0, 0.0), 1), ((-2.0, 0.0), m), ((-1.0, 0.0), m),
             ((0.0, 0.0), m), ((0.0, 1.0), m), ((0.0, -1.0), m), ((1.0, 1.0), 2), ((0.25, 0.0), m),
             ((-3.0, 0.0), 1), ((0.0, 2.0), 2), ((-1.0, 1.0), 3)]
    for (cr, ci), k in cases:
        assert _one_point(cr, ci, m) == k, (cr, ci, _one_point(cr, ci, m), k)
    assert _one_point(0.0, 0.0, 0) == 0 and _one_point(0.0, 0.0, 1) == 1


def check_mandelbrot_image_properties():
    """Image-level facts: pixel (x, y) is the point re_min + x dre, im_min + y dim
    (a 1 x 1 image at that point gives the same count); conjugate points escape
    after the same number of steps (negating ci negates every zi exactly); a
    larger iteration limit only raises counts that reached the smaller limit."""
    region = (-2.0, -1.25, 0.5, 1.25)
    img = oracle.mandelbrot(40, 30, *region, 100)
    assert img.shape == (30, 40) and img.max() == 100 and img.min() <= 3
    dre = np.float32(np.float32(0.5 - -2.0) / np.float32(40))
    dim = np.float32(np.float32(1.25 - -1.25) / np.float32(30))
    for (x, y) in [(0, 0), (39, 29), (17, 11), (25, 3)]:
        cr = float(np.float32(np.float32(-2.0) + np.float32(x) * dre))
        ci = float(np.float32(np.float32(-1.25) + np.float32(y) * dim))
        assert img[y, x] == _one_point(cr, ci, 100)
    rng = np.random.default_rng(3)
    for cr, ci in rng.uniform(-2.0, 1.0, size=(200, 2)).astype(np.float32):
        assert _one_point(float(cr), float(ci), 200) == _one_point(float(cr), float(-ci), 200)
    hi = oracle.mandelbrot(40, 30, *region, 300)
    assert np.array_equal(np.minimum(hi, 100), img)


ALL_PINS = [check_generator, check_predicate_values, check_compaction_exhaustive,
            check_compaction_small_exhaustive_values, check_compaction_library, check_scan,
            check_three_phase, check_hash, check_interleave, check_selectivity, check_mandelbrot_points,
            check_mandelbrot_image_properties]
