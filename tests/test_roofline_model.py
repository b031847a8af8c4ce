"""The algorithmic-bytes model of a k-ary lookup (bench.eks_bytes_per_lookup)
against a replay of the descents on the oracle's layout.

A lower_bound descent depends only on r = #keys < x, r in [0, n], so the n + 1
values of r enumerate every path.  The model claims that every path visits every
full level once, and that exactly b + ceil(b / (k-1)) of them (b bottom keys)
reach the partial bottom level.  The replay walks each path on the layout the
oracle builds by recursive in-order fill (no closed form involved) and counts.
"""
import numpy as np
import pytest

import bench
import oracle


def _replay(n, k):
    keys = np.arange(1, n + 1, dtype=np.uint64) * 2  # key i = 2(i+1): x = 2r+1 has r keys below
    lk, _ = oracle.layout_arrays(keys, np.arange(n, dtype=np.uint32), oracle.EYTZINGER_KARY, k)
    lk = [int(v) for v in lk]
    sizes = bench.kary_level_sizes(n, k)
    m = len(sizes) - 1
    top = n - sizes[-1]  # first slot of the bottom level
    visits = [0] * (m + 1)
    for r in range(n + 1):
        x = 2 * r + 1
        s, level = 0, 0
        while s < n:
            visits[level] += 1
            node = [lk[t] if t < n else 1 << 64 for t in range(s, s + k - 1)]
            c = sum(1 for v in node if v < x)
            s = s * k + (c + 1) * (k - 1)
            level += 1
        assert level >= m  # every path passes all full levels
    return visits, top


@pytest.mark.parametrize("n,k", [(100, 5), (1000, 5), (624, 5), (625, 5), (3000, 9), (777, 3),
                                 (4000, 17), (2 ** 12 + 9, 2)])
def test_reach_of_every_level_matches_the_model(n, k):
    visits, top = _replay(n, k)
    sizes = bench.kary_level_sizes(n, k)
    m = len(sizes) - 1
    assert sum(sizes) == n and top == k ** m - 1
    for l in range(m):
        assert visits[l] == n + 1, l
    b = sizes[-1]
    assert visits[m] == b + -(-b // (k - 1))
    # the model's probability for the bottom level, with nothing resident
    # (hit rate 0: no rowID sectors, so every request counted is a node read)
    _, reqs = bench.eks_bytes_per_lookup(n, k, 8, 0.0, 0)
    node = -(-(k - 1) * 8 // 32) * 32
    expect = m + visits[m] / (n + 1)
    assert abs(reqs.get(node, 0.0) - expect) < 1e-9
