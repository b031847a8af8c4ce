"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each test checks the oracle against something the paper prints or the
mathematics fixes: the worked example of Figures 8, 10 and 11, the closed-form
permutations of Sections 4 and 6.1, search-tree invariants, the Section 5.1
level property, and brute force on tiny inputs.  No GPU is needed.
"""
import itertools
import random

import numpy as np
import pytest

import oracle
from conftest import read_golden


def floor_log(x, k):
    """Largest l with k**l <= x (x >= 1), in exact integer arithmetic."""
    l, p = 0, 1
    while p * k <= x:
        p *= k
        l += 1
    return l


def pprime_closed_form(t, n, k):
    """Source rank of Eytzinger slot t, Section 6.1 (k = 2: Section 4).

    Two readings of the printed equations are applied: the case labels of p'(t)
    are exchanged (the bottom level, t >= k^m - 1, takes i + floor(i/(k-1)); the
    upper levels take the corrected p(t)), and the level is floor(log_k(t + 1)).
    """
    m = floor_log(n, k)
    top = k ** m - 1
    b = n - top
    if t >= top:
        i = t - top
        return i + i // (k - 1)
    l = floor_log(t + 1, k)
    i = t - (k ** l - 1)
    p = k ** (m - l - 1) * (1 + i + i // (k - 1)) - 1
    return p + min(b, (k - 1) * (p + 1))


# ---------------------------------------------------------------- worked example

def test_fig10_ternary_order_and_levels():
    g = read_golden("fig10_ternary.txt")
    keys = np.array(g["sorted"], dtype=np.uint32)
    rows = np.arange(len(keys), dtype=np.uint32)
    # feed the dataset in a scrambled order: the oracle has to sort it first
    perm = np.random.default_rng(1).permutation(len(keys))
    lk, lr = oracle.layout_arrays(keys[perm], rows[perm], oracle.EYTZINGER_KARY, 3)
    assert lk.tolist() == g["ternary"]
    # level of slot t in the ternary tree: levels hold 2, 6, 18, ... slots
    lvl = [floor_log(t + 1, 3) for t in range(len(keys))]
    assert lvl == g["ternary_level"]
    # level of each sorted entry = level of the slot that holds its rank
    sr = oracle.layout_slot_rank(len(keys), 3)
    level_of_rank = [0] * len(keys)
    for t, r in enumerate(sr):
        level_of_rank[int(r)] = lvl[t]
    assert level_of_rank == g["sorted_level"]


def _eks_descent(layout_keys, k, x):
    """Section 6.2 point lookup: count pivots < x, jump to i*k + (c+1)*(k-1)."""
    n = len(layout_keys)
    s, visited, counts = 0, [], []
    while s < n:
        visited.append(s)
        piv = [int(layout_keys[s + j]) for j in range(k - 1) if s + j < n]
        if x in piv:
            return visited, counts, s + piv.index(x)
        c = sum(1 for p in piv if p < x)
        counts.append(c)
        s = s * k + (c + 1) * (k - 1)
    return visited, counts, None


def test_fig11_ternary_lookup_path():
    g10 = read_golden("fig10_ternary.txt")
    g = read_golden("fig11_ternary_lookup9.txt")
    keys = np.array(g10["sorted"], dtype=np.uint32)
    lk, _ = oracle.layout_arrays(keys, np.arange(15, dtype=np.uint32),
                                 oracle.EYTZINGER_KARY, 3)
    visited, counts, found = _eks_descent(lk, 3, g["probe"][0])
    assert visited == g["node_offsets"]
    assert counts == g["pivots_less"]
    assert found == g["found_offset"][0]
    assert lk[found] == g["probe"][0]


def test_sec5_ebs_example_and_range():
    g10 = read_golden("fig10_ternary.txt")
    g = read_golden("sec5_ebs_range_9_12.txt")
    keys = np.array(g10["sorted"], dtype=np.uint32)
    rows = np.arange(15, dtype=np.uint32)
    lk, _ = oracle.layout_arrays(keys, rows, oracle.EYTZINGER)
    one_based = [None] + lk.tolist()
    assert one_based[1] == g["root"][0]
    assert one_based[2] == g["slot2"][0]
    assert one_based[3] == g["slot3"][0]
    assert one_based[5] == g["slot5"][0]
    sk, sr = oracle.sort_pairs(keys, rows)
    off, out = oracle.range_lookup(sk, sr, np.array(g["range_lo"], np.uint32),
                                   np.array(g["range_hi"], np.uint32))
    assert off.tolist() == [0, 4]
    assert sk[np.searchsorted(sk, 9):][:4].tolist() == g["range_keys"]
    assert [int(keys[r]) for r in out] == g["range_keys"]


def test_sec4_n17_full_levels_and_bottom():
    # Section 4, Figure 7: n = 17 gives m = floor(log2(n+1)) = 4 full levels and
    # b = n - (2^m - 1) = 2 bottom-level entries, which sit in the last slots and
    # come from sorted positions 0 and 2 (stride 2 from offset 0).
    n = 17
    assert floor_log(n + 1, 2) == 4 and n - (2 ** 4 - 1) == 2
    sr = oracle.layout_slot_rank(n, 2)
    assert sr[15] == 0 and sr[16] == 2


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("M", range(1, 15))
def test_sec4_perfect_tree_formula(M):
    # Section 4: for n = 2^M - 1 slot t holds sorted position 2^{M-l-1}(1+2i) - 1.
    n = 2 ** M - 1
    sr = oracle.layout_slot_rank(n, 2)
    t = np.arange(n, dtype=np.int64)
    l = np.array([floor_log(int(x) + 1, 2) for x in t], dtype=np.int64)
    i = t - (2 ** l - 1)
    p = (2 ** (M - l - 1)) * (1 + 2 * i) - 1
    assert np.array_equal(sr.astype(np.int64), p)


def _sizes_for(k):
    s = set(range(1, 260))
    for e in (2, 3, 4):
        for d in (-2, -1, 0, 1, 2):
            v = k ** e + d
            if 1 <= v <= 40000:
                s.add(v)
    return sorted(s)


@pytest.mark.parametrize("k", [2, 3, 4, 5, 7, 8, 9, 16, 17, 32, 33])
def test_sec61_general_formula_equals_inorder_fill(k):
    for n in _sizes_for(k):
        sr = oracle.layout_slot_rank(n, k)
        want = [pprime_closed_form(t, n, k) for t in range(n)]
        assert sr.tolist() == want, (k, n)


def test_sec61_k2_reduces_to_sec4():
    # Section 6.1 states that k = 2 gives back the Section 4 equations; with the
    # Section 4 choice m = floor(log2(n+1)) the same ranks come out.
    for n in range(1, 600):
        m = floor_log(n + 1, 2)
        b = n - (2 ** m - 1)
        got = []
        for t in range(n):
            if t >= 2 ** m - 1:
                got.append(2 * (t - (2 ** m - 1)))
            else:
                l = floor_log(t + 1, 2)
                i = t - (2 ** l - 1)
                p = 2 ** (m - l - 1) * (1 + 2 * i) - 1
                got.append(p + min(b, p + 1))
        assert got == oracle.layout_slot_rank(n, 2).tolist(), n


# ---------------------------------------------------------------- invariants

def _subtree_rank_bounds(sr, n, k):
    """(min, max) rank in each node's subtree, by a bottom-up pass over nodes."""
    nodes = (n + k - 2) // (k - 1)
    lo = [None] * nodes
    hi = [None] * nodes
    for j in reversed(range(nodes)):
        first = j * (k - 1)
        ranks = [int(sr[s]) for s in range(first, min(first + k - 1, n))]
        vals = list(ranks)
        for c in range(k):
            ch = j * k + 1 + c
            if ch < nodes:
                vals += [lo[ch], hi[ch]]
        lo[j], hi[j] = min(vals), max(vals)
    return lo, hi


@pytest.mark.parametrize("k", [2, 3, 5, 9, 17])
def test_layout_is_search_tree(k):
    rng = random.Random(k)
    for n in [1, 2, 3, k - 1, k, k + 1, k * k - 1, k * k, 97, 500, rng.randint(600, 3000)]:
        sr = oracle.layout_slot_rank(n, k)
        # a permutation of the ranks
        assert sorted(sr.tolist()) == list(range(n))
        # slots are ascending within every level, and within every node
        lvl_start = 0
        size = k - 1
        while lvl_start < n:
            seg = sr[lvl_start:min(n, lvl_start + size)].tolist()
            assert seg == sorted(seg)
            lvl_start += size
            size *= k
        # child c of node j lies strictly between pivots c-1 and c of node j
        lo, hi = _subtree_rank_bounds(sr, n, k)
        nodes = len(lo)
        for j in range(nodes):
            first = j * (k - 1)
            piv = [int(sr[s]) for s in range(first, min(first + k - 1, n))]
            for c in range(k):
                ch = j * k + 1 + c
                if ch >= nodes:
                    continue
                if c > 0:
                    assert lo[ch] > piv[c - 1]
                if c < len(piv):
                    assert hi[ch] < piv[c]
                else:
                    # only a full node has a child right of its last pivot
                    assert len(piv) == k - 1 and c == k - 1


def test_sec51_three_qualifying_means_more_below():
    # Section 5.1: if at least three entries of one Eytzinger level fall in the
    # range, every deeper full level holds strictly more of them.
    rng = np.random.default_rng(5)
    for n in [2 ** 10 - 1, 2 ** 12 - 1, 3000]:
        sr = oracle.layout_slot_rank(n, 2)
        m_full = floor_log(n + 1, 2)  # levels 0..m_full-1 are full
        for _ in range(300):
            a = int(rng.integers(0, n))
            b = int(rng.integers(a, min(n, a + 200)))
            per_level = []
            for l in range(m_full):
                seg = sr[2 ** l - 1: 2 ** (l + 1) - 1]
                per_level.append(int(np.sum((seg >= a) & (seg <= b))))
            for l in range(m_full - 1):
                if per_level[l] >= 3:
                    assert per_level[l + 1] > per_level[l]


# ---------------------------------------------------------------- results vs brute force

def _brute_point(keys, rows, x):
    js = [j for j in range(len(keys)) if keys[j] == x]
    return rows[min(js)] if js else oracle.MISS


def _brute_range(keys, rows, L, U):
    if L > U:
        return []
    sel = sorted((int(keys[j]), j) for j in range(len(keys)) if L <= keys[j] <= U)
    return [int(rows[j]) for _, j in sel]


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_results_equal_brute_force(dtype):
    rng = np.random.default_rng(7)
    top = np.iinfo(dtype).max
    for n in [0, 1, 2, 5, 16, 33, 100]:
        # small value alphabet -> many duplicates; include the extremes
        vals = np.array([0, 1, 2, 3, 5, 8, 13, top - 1, top], dtype=dtype)
        keys = vals[rng.integers(0, len(vals), size=n)]
        rows = rng.permutation(10 * n + 1)[:n].astype(np.uint32)
        sk, sr = oracle.sort_pairs(keys, rows)
        probes = np.array(sorted(set(vals.tolist()) | {4, 6, 7, 100}), dtype=dtype)
        got = oracle.point_lookup(sk, sr, probes)
        assert got.tolist() == [_brute_point(keys, rows, int(x)) for x in probes]
        pairs = list(itertools.product(probes.tolist(), repeat=2))
        lo = np.array([p[0] for p in pairs], dtype=dtype)
        hi = np.array([p[1] for p in pairs], dtype=dtype)
        off, out = oracle.range_lookup(sk, sr, lo, hi)
        for i, (L, U) in enumerate(pairs):
            assert out[off[i]:off[i + 1]].tolist() == _brute_range(keys, rows, L, U)


def test_threads_do_not_change_results():
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 2 ** 63, size=50000, dtype=np.uint64)
    rows = np.arange(50000, dtype=np.uint32)
    sk, sr = oracle.sort_pairs(keys, rows)
    q = np.concatenate([keys[:20000], rng.integers(0, 2 ** 63, size=20000, dtype=np.uint64)])
    a = oracle.point_lookup(sk, sr, q, threads=1)
    b = oracle.point_lookup(sk, sr, q, threads=4)
    assert np.array_equal(a, b)
    lo = q[:10000]
    hi = lo + np.uint64(2 ** 50)
    o1, r1 = oracle.range_lookup(sk, sr, lo, hi, threads=1)
    o2, r2 = oracle.range_lookup(sk, sr, lo, hi, threads=4)
    assert np.array_equal(o1, o2) and np.array_equal(r1, r2)
