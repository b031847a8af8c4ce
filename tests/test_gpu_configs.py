"""Parity at the workload sizes the benchmark runs (Section 8.1 shapes).

  * 2^16 uint32 keys, sorted and Eytzinger, 2^20 probes (all hits): every output
    against the oracle.
  * 2^26 uint64 keys, 2^27 probes at hit rate 0.5 (uniform, and Zipf(0.99) hits):
    every output of every layout against the oracle (the answer does not depend on
    the layout, so the oracle runs once per probe set), in the launch
    configuration the benchmark times.
  * 2^28 uint64 keys: the hybrid build's layout against the oracle's in-order
    fill, slot by slot; and with unique keys and rowID j for key j, a hit on
    keys[j] must return j and every miss GI_MISS -- a property that holds at any
    size.
  * 2^26 uint32 keys, 2^24 ranges with 1, 16 and 256 expected rows: every offset
    and every row against the oracle (for 256 rows, about 2^32 rows per layout,
    compared in chunks of 2^20 ranges).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2506_01576_gb300 as gi
import workloads as W

pytestmark = pytest.mark.gpu

from gpu_util import DEV, to_dev, to_host  # noqa: E402

THREADS = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global THREADS
    from paper_2506_01576_gb300 import _build
    _build.build()
    gi.load()
    torch.cuda.set_device(DEV)
    THREADS = oracle.hardware_threads()


def _point_dev(idx, q_dev, m):
    out = torch.empty(m, dtype=torch.int32, device=DEV)
    gi.gi_point_lookup(idx, q_dev, out)
    torch.cuda.synchronize()
    return to_host(out, np.uint32)


def test_small_config_u32_sorted_and_eytzinger():
    n, m = 1 << 16, 1 << 20
    seed = W.seed_for(0, 16)
    keys = W.unique_keys(n, 32, seed)
    rows = np.arange(n, dtype=np.uint32)
    q = W.point_probes(keys, m, 1.0, 32, seed, seed + 1)
    sk, sr = oracle.sort_pairs(keys, rows)
    want = oracle.point_lookup(sk, sr, q, THREADS)
    assert not np.any(want == oracle.MISS)
    qd = to_dev(q)
    for layout in (gi.GI_SORTED, gi.GI_EYTZINGER):
        idx = gi.gi_build(to_dev(keys), to_dev(rows), layout | gi.GI_KEY_U32, 0)
        assert np.array_equal(_point_dev(idx, qd, m), want)
        gi.gi_destroy(idx)


@pytest.fixture(scope="module")
def big_u64():
    n, m = 1 << 26, 1 << 27
    seed = W.seed_for(1, 26)
    keys = W.unique_keys(n, 64, seed)
    rows = np.arange(n, dtype=np.uint32)
    sk, sr = oracle.sort_pairs(keys, rows)
    return n, m, seed, keys, rows, sk, sr


LARGE_LAYOUTS = [(gi.GI_SORTED, 0), (gi.GI_EYTZINGER, 2)] + [
    (gi.GI_EYTZINGER_KARY, k) for k in (4, 8, 16, 32, 5, 9, 17, 33)]


@pytest.mark.parametrize("dist", ["uniform", "zipf"])
def test_large_config_u64_every_layout(big_u64, dist):
    n, m, seed, keys, rows, sk, sr = big_u64
    q = W.point_probes(keys, m, 0.5, 64, seed, seed + (2 if dist == "zipf" else 1), dist=dist)
    want = oracle.point_lookup(sk, sr, q, THREADS)
    assert abs(np.mean(want != oracle.MISS) - 0.5) < 1e-6
    kd, rd, qd = to_dev(keys), to_dev(rows), to_dev(q)
    layouts = LARGE_LAYOUTS if dist == "uniform" else [(gi.GI_SORTED, 0), (gi.GI_EYTZINGER_KARY, 9)]
    for layout, k in layouts:
        idx = gi.gi_build(kd, rd, layout | gi.GI_KEY_U64, k)
        assert gi.gi_footprint_bytes(idx) == n * 12 + (8 if layout == gi.GI_EYTZINGER else 0)
        got = _point_dev(idx, qd, m)
        bad = np.flatnonzero(got != want)
        assert bad.size == 0, (layout, k, bad[:5], got[bad[:5]], want[bad[:5]])
        gi.gi_destroy(idx)


def test_layout_at_scale_matches_inorder_fill(big_u64):
    n, m, seed, keys, rows, sk, sr = big_u64
    kd, rd = to_dev(keys), to_dev(rows)
    for layout, k in ((gi.GI_EYTZINGER, 2), (gi.GI_EYTZINGER_KARY, 9), (gi.GI_EYTZINGER_KARY, 16)):
        idx = gi.gi_build(kd, rd, layout | gi.GI_KEY_U64, k)
        lk = torch.empty(n, dtype=torch.int64, device=DEV)
        lr = torch.empty(n, dtype=torch.int32, device=DEV)
        gi.gi_copy_layout(idx, lk, lr)
        r = oracle.layout_slot_rank(n, k).astype(np.int64)
        assert np.array_equal(to_host(lk, np.uint64), sk[r])
        assert np.array_equal(to_host(lr, np.uint32), sr[r])
        gi.gi_destroy(idx)


def test_layout_at_2e28_hybrid_matches_inorder_fill():
    """2^28 u64 keys, k = 5: the default build takes the hybrid sort (two MSD
    scatters on the 8-bit windows below the highest differing bit, 65536 buckets of
    about 4096 pairs, each sorted in shared memory and written into the layout), in
    fewer launches than the LSD sort's eight passes would take; every slot's key and
    rowID against the oracle's in-order fill."""
    n = 1 << 28
    keys = W.unique_keys(n, 64, W.seed_for(1, 28))
    rows = np.arange(n, dtype=np.uint32)
    kd, rd = to_dev(keys), to_dev(rows)
    c0 = gi.gi_launch_count()
    idx = gi.gi_build(kd, rd, gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64, 5)
    launches = gi.gi_launch_count() - c0
    del kd, rd
    assert launches <= 13, launches  # the LSD path takes at least 8 passes + 6 other launches
    lk = torch.empty(n, dtype=torch.int64, device=DEV)
    lr = torch.empty(n, dtype=torch.int32, device=DEV)
    gi.gi_copy_layout(idx, lk, lr)
    gi.gi_destroy(idx)
    got_k, got_r = to_host(lk, np.uint64), to_host(lr, np.uint32)
    del lk, lr
    sk, sr = oracle.sort_pairs(keys, rows)
    r = oracle.layout_slot_rank(n, 5)
    assert np.array_equal(got_k, sk[r])
    assert np.array_equal(got_r, sr[r])


def test_largest_build_size_property():
    n, m = 1 << 28, 1 << 24
    seed = W.seed_for(1, 28)
    keys = W.unique_keys(n, 64, seed)
    rng = np.random.default_rng(3)
    j = rng.integers(0, n, size=m // 2)
    miss = W.point_probes(keys, m // 2, 0.0, 64, seed, 9)  # values not in the key set
    q = np.concatenate([keys[j], miss])
    want = np.concatenate([j.astype(np.uint32), np.full(m // 2, oracle.MISS, np.uint32)])
    kd = to_dev(keys)
    rd = torch.arange(n, dtype=torch.int32, device=DEV)
    qd = to_dev(q)
    del keys
    for layout, k in ((gi.GI_SORTED, 0), (gi.GI_EYTZINGER, 2), (gi.GI_EYTZINGER_KARY, 9)):
        idx = gi.gi_build(kd, rd, layout | gi.GI_KEY_U64, k)
        assert np.array_equal(_point_dev(idx, qd, m), want), (layout, k)
        gi.gi_destroy(idx)


@pytest.fixture(scope="module")
def ranges_u32():
    n, m = 1 << 26, 1 << 24
    seed = W.seed_for(2, 26)
    keys = W.unique_keys(n, 32, seed)
    rows = np.arange(n, dtype=np.uint32)
    sk, sr = oracle.sort_pairs(keys, rows)
    return n, m, seed, keys, rows, sk, sr


RANGE_LAYOUTS = ((gi.GI_SORTED, 0), (gi.GI_EYTZINGER, 2), (gi.GI_EYTZINGER_KARY, 16),
                 (gi.GI_EYTZINGER_KARY, 17))


@pytest.mark.parametrize("E", [1, 16])
def test_range_config_u32(ranges_u32, E):
    n, m, seed, keys, rows, sk, sr = ranges_u32
    lo, hi, w = W.ranges_with_expected_rows(n, m, E, 32, seed + E)
    woff, wrows = oracle.range_lookup(sk, sr, lo, hi, THREADS)
    assert abs(float(woff[-1]) / m / E - 1) < 0.02
    kd, rd, lod, hid = to_dev(keys), to_dev(rows), to_dev(lo), to_dev(hi)
    for layout, k in RANGE_LAYOUTS:
        idx = gi.gi_build(kd, rd, layout | gi.GI_KEY_U32, k)
        off = torch.empty(m + 1, dtype=torch.int64, device=DEV)
        gi.gi_range_lookup(idx, lod, hid, off)
        total = int(off[-1].item())
        out = torch.empty(total, dtype=torch.int32, device=DEV)
        gi.gi_range_lookup(idx, lod, hid, off, out)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(off, np.uint64), woff), (layout, k)
        assert np.array_equal(to_host(out, np.uint32), wrows), (layout, k)
        del out
        gi.gi_destroy(idx)


def test_range_config_u32_256_rows_every_row(ranges_u32):
    """E = 256: about 2^32 rows (16 GiB) per layout.  Every offset and every row of
    every layout is compared with the oracle, 2^20 ranges at a time: the oracle
    answers one chunk, and each layout's CSR slice for it is copied back and
    compared."""
    n, m, seed, keys, rows, sk, sr = ranges_u32
    E = 256
    lo, hi, w = W.ranges_with_expected_rows(n, m, E, 32, seed + E)
    kd, rd, lod, hid = to_dev(keys), to_dev(rows), to_dev(lo), to_dev(hi)
    outs = []
    for layout, k in RANGE_LAYOUTS:
        idx = gi.gi_build(kd, rd, layout | gi.GI_KEY_U32, k)
        off = torch.empty(m + 1, dtype=torch.int64, device=DEV)
        gi.gi_range_lookup(idx, lod, hid, off)
        total = int(off[-1].item())
        out = torch.empty(total, dtype=torch.int32, device=DEV)
        gi.gi_range_lookup(idx, lod, hid, off, out)
        torch.cuda.synchronize()
        gi.gi_destroy(idx)
        outs.append((layout, k, to_host(off, np.uint64).astype(np.int64), out))
    assert abs(float(outs[0][2][-1]) / m / E - 1) < 0.02
    chunk = 1 << 20
    for a in range(0, m, chunk):
        b = min(m, a + chunk)
        coff, crows = oracle.range_lookup(sk, sr, lo[a:b], hi[a:b], THREADS)
        for layout, k, o, out in outs:
            assert np.array_equal(o[a:b + 1] - o[a], coff.astype(np.int64)), (layout, k, a)
            got = to_host(out[int(o[a]):int(o[b])], np.uint32)
            assert np.array_equal(got, crows), (layout, k, a)
    del outs
