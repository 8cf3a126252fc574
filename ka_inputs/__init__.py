"""Seeded synthetic inputs for the stream-compaction pipelines.

This module is shared by the CPU oracle's tests, the GPU parity tests and the
benchmark. It holds none of the compaction arithmetic: only a counter-based
random stream and the recipes that turn it into workload descriptions (array
sizes, predicate names and parameters, per-instance thresholds, arrival times).

Random stream: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014). The counter-based form used everywhere in this
repository is

    splitmix64(seed, i) = mix64(seed + (i + 1) * 0x9E3779B97F4A7C15  mod 2^64)
    mix64(z): z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
              z = (z ^ (z >> 27)) * 0x94D049BB133111EB
              return z ^ (z >> 31)

so splitmix64(seed, i) is the (i+1)-th output of the sequential generator whose
state starts at `seed`. A uint32 input element is the high half of it.

The paper measures its indexing pipeline on VAST log data and its overhead on
matrix multiplication; neither is a public dataset on this path, so every
workload here is synthetic uint32 data of the sizes and selectivities listed in
`CONFIGS` below.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB

# Predicate names understood by both sides; each side maps them to its own ids.
PREDICATES = ("and_mask_eq0", "lt", "topbits_lt", "popc_odd", "mod_ne0", "ne")


def splitmix64(seed: int, idx) -> np.ndarray:
    """Counter-based SplitMix64 outputs for the given indices (uint64 array)."""
    i = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (i + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix64_one(seed: int, i: int) -> int:
    return int(splitmix64(seed, np.array([i], dtype=np.uint64))[0])


def uniform_u32(seed: int, n: int, start: int = 0) -> np.ndarray:
    """n uint32 values x_i = hi32(splitmix64(seed, start + i)), uniform over [0, 2^32)."""
    if n == 0:
        return np.zeros(0, dtype=np.uint32)
    idx = np.arange(start, start + n, dtype=np.uint64)
    return (splitmix64(seed, idx) >> np.uint64(32)).astype(np.uint32)


def uniform_f64(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1): the top 53 bits of splitmix64(seed, i) scaled by 2^-53."""
    idx = np.arange(n, dtype=np.uint64)
    return (splitmix64(seed, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def substream(master_seed: int, k: int) -> int:
    """Seed of the k-th independent sub-stream of a master seed."""
    return splitmix64_one(master_seed, k)


def threshold_for(selectivity: float) -> int:
    """t = floor(s * 2^32), clamped to [0, 2^32 - 1]: keep x < t keeps about s of uniform data."""
    t = int(math.floor(selectivity * 4294967296.0))
    return max(0, min(t, 0xFFFFFFFF))


def log_uniform_sizes(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """n = floor(2^U), U ~ U[lo, hi), clamped to [2^lo, 2^hi]."""
    u = uniform_f64(seed, count)
    n = np.floor(np.exp2(lo + (hi - lo) * u)).astype(np.int64)
    return np.clip(n, 1 << lo, 1 << hi)


# ---------------------------------------------------------------------------
# Workload recipes (one per benchmark configuration).
# ---------------------------------------------------------------------------

MASTER_SEED = 0x1709_0778_1000_0001


@dataclass(frozen=True)
class Stage:
    """One stage of a pipeline: 'map_hash' or a keep-predicate ('compact')."""
    kind: str                  # "map_hash" | "compact"
    pred: str = ""             # predicate name for "compact"
    param: int = 0


# The four stages of the 4-stage composed pipeline: hash map, then keep
# (h >> 28) < 8, keep popcount(h) odd, keep h % 3 != 0.
PIPELINE4 = (
    Stage("map_hash"),
    Stage("compact", "topbits_lt", 8),
    Stage("compact", "popc_odd", 0),
    Stage("compact", "mod_ne0", 3),
)


@dataclass
class Workload:
    name: str
    n: int
    seed: int
    stages: tuple = ()
    extra: dict = field(default_factory=dict)


def config_single(n: int = 1 << 20, seed: int = 1) -> Workload:
    """Single compaction pipeline: keep (x & 3) == 0 (about 25 % selectivity)."""
    return Workload("single_and3_n%d" % n, n, seed, (Stage("compact", "and_mask_eq0", 3),))


def config_large(selectivity: float, n: int = 1 << 28, seed: int = 2) -> Workload:
    """Large single compaction: keep x < t with t = floor(s * 2^32)."""
    t = threshold_for(selectivity)
    return Workload("large_lt_s%g_n%d" % (selectivity, n), n, seed,
                    (Stage("compact", "lt", t),), {"selectivity": selectivity, "t": t})


def config_pipeline4(n: int = 1 << 26, seed: int = 3) -> Workload:
    return Workload("pipeline4_n%d" % n, n, seed, PIPELINE4)


@dataclass
class BatchSpec:
    """Independent compaction instances: sizes, data seeds and thresholds."""
    n: np.ndarray          # int64 sizes
    seeds: np.ndarray      # uint64 data seeds
    t: np.ndarray          # uint32 thresholds (keep x < t)
    selectivity: np.ndarray


def config_batch(count: int = 4096, lo: int = 8, hi: int = 20,
                 master_seed: int = MASTER_SEED + 4) -> BatchSpec:
    """Batched instances: n_i log-uniform in [2^lo, 2^hi], s_i ~ U[0.01, 0.99)."""
    sizes = log_uniform_sizes(substream(master_seed, 0), count, lo, hi)
    seeds = splitmix64(substream(master_seed, 1), np.arange(count, dtype=np.uint64))
    s = 0.01 + 0.98 * uniform_f64(substream(master_seed, 2), count)
    t = np.array([threshold_for(v) for v in s], dtype=np.uint64).astype(np.uint32)
    return BatchSpec(sizes, seeds, t, s)


@dataclass
class ServeTrace:
    """Poisson request trace: arrival time (s), size, data seed and stage list per request."""
    arrival_s: np.ndarray
    n: np.ndarray
    seeds: np.ndarray
    n_stages: np.ndarray
    stage_kind: np.ndarray     # int8 [R, 4]: index into PIPELINE4 for each stage slot


def config_serve(rate_hz: float = 20000.0, duration_s: float = 60.0, lo: int = 10,
                 hi: int = 24, master_seed: int = MASTER_SEED + 5,
                 max_requests: int | None = None) -> ServeTrace:
    """Poisson arrivals; each request is 1-4 stages drawn from the 4-stage pipeline's set."""
    expected = int(rate_hz * duration_s * 1.2) + 64
    u = uniform_f64(substream(master_seed, 0), expected)
    gaps = -np.log1p(-u) / rate_hz
    arrival = np.cumsum(gaps)
    arrival = arrival[arrival < duration_s]
    r = arrival.size if max_requests is None else min(arrival.size, max_requests)
    arrival = arrival[:r]
    sizes = log_uniform_sizes(substream(master_seed, 1), r, lo, hi)
    seeds = splitmix64(substream(master_seed, 2), np.arange(r, dtype=np.uint64))
    n_stages = 1 + np.minimum((uniform_f64(substream(master_seed, 3), r) * 4).astype(np.int64), 3)
    kinds = np.minimum((uniform_f64(substream(master_seed, 4), r * 4) * 4).astype(np.int64), 3)
    return ServeTrace(arrival, sizes, seeds, n_stages, kinds.reshape(r, 4).astype(np.int8))


def index_pairs(k: int, zero_fraction: float, seed: int = 7):
    """Chunk ids and literals (k each) for the interleave-then-remove-zeros step.

    Both arrays are uniform uint32 with a controlled fraction of entries forced
    to zero (the value the compaction removes).
    """
    a = uniform_u32(seed, k)
    b = uniform_u32(seed + 1, k)
    za = uniform_f64(substream(seed, 2), k) < zero_fraction
    zb = uniform_f64(substream(seed, 3), k) < zero_fraction
    a = np.where(za, np.uint32(0), a).astype(np.uint32)
    b = np.where(zb, np.uint32(0), b).astype(np.uint32)
    return a, b
