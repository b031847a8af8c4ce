"""The seeded input generators: uniqueness, hit rates, range widths, Zipf law."""
import numpy as np
import pytest

import workloads as W


@pytest.mark.parametrize("bits", [32, 64])
def test_unique_keys_unique_in_domain_and_deterministic(bits):
    seed = W.seed_for(1, 16)
    k = W.unique_keys(1 << 16, bits, seed)
    assert len(np.unique(k)) == len(k)
    if bits == 64:
        assert int(k.max()) < (1 << 63)
    assert np.array_equal(k, W.unique_keys(1 << 16, bits, seed))
    assert not np.array_equal(k, W.unique_keys(1 << 16, bits, seed + 1))
    # roughly uniform: each eighth of the domain gets about 1/8 of the keys
    top = (1 << 32) if bits == 32 else (1 << 63)
    h, _ = np.histogram(k.astype(np.float64), bins=8, range=(0, float(top)))
    assert np.all(np.abs(h / len(k) - 1 / 8) < 0.01)


@pytest.mark.parametrize("bits", [32, 64])
def test_point_probes_hit_rate_and_misses_absent(bits):
    seed = W.seed_for(2, 14)
    keys = W.unique_keys(1 << 14, bits, seed)
    q = W.point_probes(keys, 1 << 15, 0.5, bits, seed, 99)
    present = np.isin(q, keys)
    assert present.sum() == 1 << 14  # exactly half
    # hits and misses are interleaved, not blocked
    assert 0.4 < present[: 1 << 12].mean() < 0.6
    q2 = W.point_probes(keys, 1 << 12, 1.0, bits, seed, 5)
    assert np.isin(q2, keys).all()


def test_ranges_expected_rows():
    n = 1 << 18
    keys = np.sort(W.unique_keys(n, 32, 3))
    for E in (1, 16, 256):
        lo, hi, w = W.ranges_with_expected_rows(n, 1 << 14, E, 32, 11)
        assert np.all(hi.astype(np.int64) - lo.astype(np.int64) == w)
        cnt = np.searchsorted(keys, hi, side="right") - np.searchsorted(keys, lo, side="left")
        assert abs(cnt.mean() / E - 1) < 0.05


def test_zipf_law_matches_section89_counts():
    # Section 8.9 reports, for 2^25 Zipf probes over 2^28 keys, 1,201,800 distinct
    # keys queried at exponent 1.25 and 8016 at exponent 2.0.  Under the textbook
    # law P(r) ~ r^-s the expected distinct counts must agree to well under 1%.
    e125 = W.zipf_expected_distinct(1 << 28, 1 << 25, 1.25)
    e200 = W.zipf_expected_distinct(1 << 28, 1 << 25, 2.0)
    assert abs(e125 / 1201800 - 1) < 0.005
    assert abs(e200 / 8016 - 1) < 0.005


def test_zipf_sampler_matches_its_law():
    rng = np.random.default_rng(17)
    n, draws = 1 << 20, 1 << 20
    r = W.zipf_ranks(n, draws, 1.25, rng)
    assert r.min() >= 1 and r.max() <= n
    want = W.zipf_expected_distinct(n, draws, 1.25)
    assert abs(len(np.unique(r)) / want - 1) < 0.01
    # rank 1 frequency ~ 1/H(n, s)
    h = np.sum(np.arange(1, n + 1, dtype=np.float64) ** -1.25)
    assert abs(np.mean(r == 1) * h - 1) < 0.02
