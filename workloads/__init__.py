"""Seeded synthetic inputs for the static-index workloads (paper Section 8.1).

This module only draws numbers. It holds none of the index method's
arithmetic (no sorting into a layout, no search) and is the one piece of code
that both the CUDA path's tests/bench and the CPU oracle's tests use.

Workload shapes follow Section 8.1 of the paper (unique, uniformly drawn build
keys; probe batches drawn from the build set in random order; ranges of a
fixed width starting at a uniform offset) and Section 8.9 (Zipf-skewed probes).

Unique keys without a dedupe sort
---------------------------------
A key set of n unique values, uniform over a domain [0, 2^B), is drawn as
``keys[j] = perm(j)`` for j = 0..n-1, where ``perm`` is a seeded bijection of
[0, 2^B) (a few rounds of multiply-by-odd and xor-shift, each a bijection mod
2^B).  A value known NOT to be in the build set is ``perm(j)`` for some
j >= n, so "misses drawn uniformly from values not in the build set" is
``perm(uniform integer in [n, 2^B))`` -- exactly uniform over the complement.
rowID j belongs to keys[j] (generation order), so key order is random with
respect to rowIDs.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "SEED_BASE",
    "seed_for",
    "unique_keys",
    "point_probes",
    "ranges_with_expected_rows",
    "zipf_ranks",
    "zipf_expected_distinct",
    "duplicate_keys",
]

#: Base of every seed; each workload mixes in its config id and size.
SEED_BASE = 0x9E3779B97F4A7C15

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def seed_for(config_id: int, size_log2: int, salt: int = 0) -> int:
    """Deterministic 64-bit seed for (config, size, salt)."""
    return (SEED_BASE ^ (config_id << 8) ^ size_log2 ^ (salt << 20)) & 0xFFFFFFFFFFFFFFFF


def _splitmix64(x: int) -> int:
    x = (x + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return z ^ (z >> 31)


class _Bijection:
    """A seeded bijection of [0, 2^bits): rounds of x += a; x *= odd; x ^= x >> s.

    Every step is invertible modulo 2^bits (an odd multiplier has an inverse
    mod 2^bits; a right xor-shift by s >= 1 is invertible), so the composition
    is a permutation of the domain.
    """

    def __init__(self, bits: int, seed: int):
        assert 8 <= bits <= 64
        self.bits = bits
        self.mask = np.uint64((1 << bits) - 1) if bits < 64 else _M64
        s = seed
        self.rounds = []
        for shift in (bits // 2 - 1, bits // 2 - 3, bits // 2 + 1):
            s = _splitmix64(s)
            add = s & ((1 << bits) - 1)
            s = _splitmix64(s)
            mul = (s | 1) & ((1 << bits) - 1)
            self.rounds.append((np.uint64(add), np.uint64(mul), np.uint64(shift)))

    def __call__(self, j: np.ndarray) -> np.ndarray:
        x = j.astype(np.uint64, copy=True)
        with np.errstate(over="ignore"):
            for add, mul, shift in self.rounds:
                x += add
                x &= self.mask
                x *= mul
                x &= self.mask
                x ^= x >> shift
        return x


def _domain_bits(key_bits: int) -> int:
    # u32 keys: uniform over [0, 2^32); u64 keys: uniform over [0, 2^63)
    # (the 64-bit workload of the paper's Section 8.7 as shaped for this library).
    if key_bits == 32:
        return 32
    if key_bits == 64:
        return 63
    raise ValueError("key_bits must be 32 or 64")


def _dtype(key_bits: int):
    return np.uint32 if key_bits == 32 else np.uint64


def unique_keys(n: int, key_bits: int, seed: int) -> np.ndarray:
    """n unique keys, uniform over the key domain, in random (generation) order.

    rowID j is meant to be paired with keys[j].
    """
    dom = _domain_bits(key_bits)
    if n > (1 << dom):
        raise ValueError("more unique keys than the domain holds")
    perm = _Bijection(dom, seed)
    return perm(np.arange(n, dtype=np.uint64)).astype(_dtype(key_bits))


def _miss_values(n: int, m: int, key_bits: int, seed: int, rng) -> np.ndarray:
    dom = _domain_bits(key_bits)
    perm = _Bijection(dom, seed)
    j = rng.integers(n, 1 << dom, size=m, dtype=np.uint64, endpoint=False)
    return perm(j).astype(_dtype(key_bits))


def zipf_ranks(n: int, m: int, s: float, rng) -> np.ndarray:
    """m draws of a rank in 1..n with P(r) proportional to r^-s (inverse CDF).

    This is the textbook Zipf law the paper's Section 8.9 counts with: at
    s = 1.25, 2^25 draws over 2^28 keys touch about 1.2 M distinct keys.
    """
    if n <= 0:
        return np.zeros(0, dtype=np.int64)
    cdf = np.cumsum(np.arange(1, n + 1, dtype=np.float64) ** (-s))
    cdf /= cdf[-1]
    u = rng.random(m)
    r = np.searchsorted(cdf, u, side="left") + 1
    return np.minimum(r, n).astype(np.int64)


def zipf_expected_distinct(n: int, draws: int, s: float, chunk: int = 1 << 24) -> float:
    """E[#distinct ranks] after `draws` Zipf(s) draws over 1..n: sum_r 1-(1-p_r)^draws."""
    h = 0.0
    for a in range(1, n + 1, chunk):
        r = np.arange(a, min(n, a + chunk - 1) + 1, dtype=np.float64)
        h += float(np.sum(r ** (-s)))
    tot = 0.0
    for a in range(1, n + 1, chunk):
        r = np.arange(a, min(n, a + chunk - 1) + 1, dtype=np.float64)
        p = r ** (-s) / h
        tot += float(np.sum(-np.expm1(draws * np.log1p(-p))))
    return tot


def point_probes(keys: np.ndarray, m: int, hit_rate: float, key_bits: int,
                 key_seed: int, seed: int, dist: str = "uniform",
                 zipf_s: float = 0.99) -> np.ndarray:
    """m probes: round(m*hit_rate) hits drawn from `keys`, the rest misses, shuffled.

    Hits are uniform over the build keys (`dist="uniform"`) or Zipf(zipf_s)
    over ranks, rank r mapping to keys[r-1] (generation order, so random in key
    space).  Misses are uniform over the values NOT in the build set; this
    needs `key_seed`, the seed `keys` was drawn with by `unique_keys`.
    """
    rng = np.random.default_rng(seed)
    n = len(keys)
    n_hit = int(round(m * hit_rate)) if n > 0 else 0
    if dist == "uniform":
        idx = rng.integers(0, max(n, 1), size=n_hit)
    elif dist == "zipf":
        idx = zipf_ranks(n, n_hit, zipf_s, rng) - 1
    else:
        raise ValueError(dist)
    hits = keys[idx] if n_hit else np.zeros(0, dtype=_dtype(key_bits))
    misses = _miss_values(n, m - n_hit, key_bits, key_seed, rng)
    q = np.concatenate([hits.astype(_dtype(key_bits)), misses])
    rng.shuffle(q)
    return q


def ranges_with_expected_rows(n: int, m: int, expected_rows: float, key_bits: int,
                              seed: int):
    """m inclusive ranges [L, L+w] whose expected result size is `expected_rows`.

    With n unique keys uniform over a domain of D values the density is n/D,
    so w + 1 = expected_rows * D / n.  L is uniform in [0, D-1-w].
    Returns (lo, hi, w).
    """
    rng = np.random.default_rng(seed)
    D = 1 << _domain_bits(key_bits)
    w = max(0, int(round(expected_rows * D / max(n, 1))) - 1)
    w = min(w, D - 1)
    lo = rng.integers(0, D - w, size=m, dtype=np.uint64, endpoint=False)
    hi = lo + np.uint64(w)
    t = _dtype(key_bits)
    return lo.astype(t), hi.astype(t), w


def duplicate_keys(n_distinct: int, replicas: int, key_bits: int, seed: int) -> np.ndarray:
    """Each of n_distinct unique keys repeated `replicas` times, shuffled (Section 8.11)."""
    base = unique_keys(n_distinct, key_bits, seed)
    rng = np.random.default_rng(seed ^ 0x5DEECE66D)
    k = np.repeat(base, replicas)
    rng.shuffle(k)
    return k
