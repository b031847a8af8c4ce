"""Batched form vs the CPU oracle, index by index.

Thousands of independent indexes of uneven size are built by one segmented
radix sort + permutation and probed by one persistent launch.  Every index's
layout and every probe's rowID must equal what the oracle gives for that index
alone (integers: exact).  Also: the build + lookup sequence captured in a CUDA
graph and replayed gives the same answers, and the full batched workload shape
(4096 indexes, 2^8..2^20 keys, 2^10..2^18 probes at hit rate 0.75) on a sample
of indexes.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2506_01576_gb300 as gi
import workloads as W

pytestmark = pytest.mark.gpu

from gpu_util import DEV, to_dev, to_host  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2506_01576_gb300 import _build
    _build.build()
    gi.load()
    torch.cuda.set_device(DEV)


def _make_batch(sizes, bits, seed, dup=False):
    keys, rows = [], []
    for i, n in enumerate(sizes):
        if dup and n:
            k = W.duplicate_keys(max(1, n // 3), 3, bits, seed + i)[:n]
            if len(k) < n:
                k = np.concatenate([k, k[: n - len(k)]])
        else:
            k = W.unique_keys(n, bits, seed + i)
        keys.append(k)
        rows.append(np.random.default_rng(seed + i).permutation(n).astype(np.uint32))
    off = np.zeros(len(sizes) + 1, dtype=np.uint64)
    np.cumsum(np.array(sizes, dtype=np.uint64), out=off[1:])
    return keys, rows, off


def _probes(keys, bits, per_index, seed):
    qs = []
    for i, k in enumerate(keys):
        m = per_index[i]
        if len(k):
            q = W.point_probes(k, m, 0.75, bits, W.seed_for(9, 9, i), seed + i)
        else:
            q = np.random.default_rng(seed + i).integers(0, 2 ** (bits - 1), size=m).astype(k.dtype)
        qs.append(q.astype(np.uint64 if bits == 64 else np.uint32))
    qoff = np.zeros(len(keys) + 1, dtype=np.uint64)
    np.cumsum(np.array([len(q) for q in qs], dtype=np.uint64), out=qoff[1:])
    return qs, qoff


def _check(batch, keys, rows, qs, qoff, out, layout, k, check_layout=True, which=None):
    got = to_host(out, np.uint32)
    for i in (range(len(keys)) if which is None else which):
        sk, sr = oracle.sort_pairs(keys[i], rows[i])
        want = oracle.point_lookup(sk, sr, qs[i])
        seg = got[int(qoff[i]):int(qoff[i + 1])]
        assert np.array_equal(seg, want), ("index", i, len(keys[i]))
        if check_layout and len(keys[i]):
            n = len(keys[i])
            kk = torch.empty(n, dtype=torch.int64 if keys[i].dtype == np.uint64 else torch.int32, device=DEV)
            rr = torch.empty(n, dtype=torch.int32, device=DEV)
            gi.gi_batch_copy_index(batch, i, kk, rr)
            ok, orr = oracle.layout_arrays(keys[i], rows[i],
                                           oracle.EYTZINGER_KARY if layout == gi.GI_EYTZINGER_KARY else oracle.SORTED, k)
            assert np.array_equal(to_host(kk, keys[i].dtype), ok), ("layout", i)
            assert np.array_equal(to_host(rr, np.uint32), orr), ("layout rows", i)


@pytest.mark.parametrize("bits", [64, 32])
@pytest.mark.parametrize("layout,k", [(gi.GI_EYTZINGER_KARY, 5), (gi.GI_EYTZINGER_KARY, 9),
                                      (gi.GI_EYTZINGER_KARY, 3), (gi.GI_EYTZINGER_KARY, 17),
                                      (gi.GI_SORTED, 0)])
def test_batch_equals_oracle_per_index(bits, layout, k):
    rng = np.random.default_rng(bits + k)
    sizes = [0, 1, 2, 3, 7, 100, 3071, 3072, 3073, 5000] + list(rng.integers(0, 40000, size=30))
    sizes += [70000, 0, 6]
    keys, rows, off = _make_batch(sizes, bits, 100 + k)
    per_index = list(rng.integers(0, 3000, size=len(sizes)))
    qs, qoff = _probes(keys, bits, per_index, 7)
    flag = gi.GI_KEY_U64 if bits == 64 else gi.GI_KEY_U32
    batch = gi.gi_batch_create(off, layout | flag, k)
    kd = to_dev(np.concatenate(keys)) if off[-1] else torch.empty(0, device=DEV)
    rd = to_dev(np.concatenate(rows))
    gi.gi_batch_build(batch, kd, rd)
    qd = to_dev(np.concatenate(qs))
    qod = to_dev(qoff)
    out = torch.full((int(qoff[-1]),), -5, dtype=torch.int32, device=DEV)
    gi.gi_batch_point_lookup(batch, qd, qod, out)
    gi.gi_batch_sync(batch)
    _check(batch, keys, rows, qs, qoff, out, layout, k)
    # knobs change the schedule, not the answer
    for opt, v in ((gi.GI_BATCH_OPT_CHUNK, 96), (gi.GI_BATCH_OPT_BLOCKS_PER_SM, 1),
                   (gi.GI_BATCH_OPT_SMEM_BUDGET, 0), (gi.GI_BATCH_OPT_SMEM_BUDGET, 40960)):
        gi.gi_batch_set_option(batch, opt, v)
        out.fill_(-5)
        gi.gi_batch_point_lookup(batch, qd, qod, out)
        gi.gi_batch_sync(batch)
        _check(batch, keys, rows, qs, qoff, out, layout, k, check_layout=False)
    gi.gi_batch_destroy(batch)


def test_batch_duplicates_and_rebuild():
    rng = np.random.default_rng(3)
    sizes = list(rng.integers(1, 9000, size=25))
    keys, rows, off = _make_batch(sizes, 64, 55, dup=True)
    qs, qoff = _probes(keys, 64, [500] * len(sizes), 8)
    batch = gi.gi_batch_create(off, gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64, 5)
    kd, rd = to_dev(np.concatenate(keys)), to_dev(np.concatenate(rows))
    qd, qod = to_dev(np.concatenate(qs)), to_dev(qoff)
    out = torch.empty(int(qoff[-1]), dtype=torch.int32, device=DEV)
    for _ in range(2):  # a second build over the same buffers gives the same index
        gi.gi_batch_build(batch, kd, rd)
        gi.gi_batch_point_lookup(batch, qd, qod, out)
        gi.gi_batch_sync(batch)
        _check(batch, keys, rows, qs, qoff, out, gi.GI_EYTZINGER_KARY, 5)
    gi.gi_batch_destroy(batch)


def test_batch_build_and_lookup_replay_from_a_cuda_graph():
    rng = np.random.default_rng(11)
    sizes = list(rng.integers(0, 20000, size=64))
    keys, rows, off = _make_batch(sizes, 64, 77)
    qs, qoff = _probes(keys, 64, list(rng.integers(0, 4000, size=64)), 9)
    batch = gi.gi_batch_create(off, gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64, 5)
    kd, rd = to_dev(np.concatenate(keys)), to_dev(np.concatenate(rows))
    qd, qod = to_dev(np.concatenate(qs)), to_dev(qoff)
    out = torch.full((int(qoff[-1]),), -5, dtype=torch.int32, device=DEV)
    s = torch.cuda.Stream()
    gi.gi_batch_set_stream(batch, s)
    # warm-up outside the capture (lazy module loading)
    with torch.cuda.stream(s):
        gi.gi_batch_build(batch, kd, rd)
        gi.gi_batch_point_lookup(batch, qd, qod, out)
    s.synchronize()
    out.fill_(-5)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        gi.gi_batch_build(batch, kd, rd)
        gi.gi_batch_point_lookup(batch, qd, qod, out)
    for _ in range(2):
        out.fill_(-5)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        gi.gi_batch_sync(batch)
        _check(batch, keys, rows, qs, qoff, out, gi.GI_EYTZINGER_KARY, 5, check_layout=False)
    gi.gi_batch_destroy(batch)


def test_batched_workload_shape_sampled():
    # 4096 indexes, sizes log-uniform 2^8..2^20, probes log-uniform 2^10..2^18 at hit
    # rate 0.75; 48 indexes (including the largest and smallest) checked fully
    rng = np.random.default_rng(2024)
    B = 4096
    sizes = np.exp2(rng.uniform(8, 20, size=B)).astype(np.int64)
    nq = np.exp2(rng.uniform(10, 18, size=B)).astype(np.int64)
    off = np.zeros(B + 1, dtype=np.uint64)
    np.cumsum(sizes.astype(np.uint64), out=off[1:])
    keys = [W.unique_keys(int(n), 64, W.seed_for(3, 20, i)) for i, n in enumerate(sizes)]
    rows = [np.arange(n, dtype=np.uint32) for n in sizes]
    qs, qoff = _probes(keys, 64, list(nq), 13)
    batch = gi.gi_batch_create(off, gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64, 5)
    kd, rd = to_dev(np.concatenate(keys)), to_dev(np.concatenate(rows))
    qd, qod = to_dev(np.concatenate(qs)), to_dev(qoff)
    out = torch.empty(int(qoff[-1]), dtype=torch.int32, device=DEV)
    gi.gi_batch_build(batch, kd, rd)
    gi.gi_batch_point_lookup(batch, qd, qod, out)
    gi.gi_batch_sync(batch)
    which = sorted(set([int(np.argmax(sizes)), int(np.argmin(sizes))] +
                       list(rng.choice(B, size=46, replace=False))))
    _check(batch, keys, rows, qs, qoff, out, gi.GI_EYTZINGER_KARY, 5, check_layout=True, which=which)
    assert gi.gi_batch_footprint_bytes(batch) == int(off[-1]) * 12
    gi.gi_batch_destroy(batch)


@pytest.mark.parametrize("bits", [64, 32])
@pytest.mark.parametrize("layout,k", [(gi.GI_EYTZINGER_KARY, 5), (gi.GI_SORTED, 0), (gi.GI_EYTZINGER_KARY, 17),
                                      (gi.GI_EYTZINGER_KARY, 2)])
def test_batch_build_plans_every_path(bits, layout, k):
    # the build sorts each index by a plan chosen on the device from the bits in
    # which its keys differ: whole index in one CTA (<= 5120 pairs), one MSD scatter
    # on a window of its highest significant bits + bucket sort, or the LSD passes
    # when a window bucket would exceed 5120 pairs.  One batch holds every case: tiny, uniform, skewed (almost
    # all keys in one MSD bucket), all keys equal, heavy duplicates, narrow ranges.
    dt = np.uint64 if bits == 64 else np.uint32
    top = np.iinfo(dt).max
    rng = np.random.default_rng(bits + k)
    keys = [
        W.unique_keys(4000, bits, 1),                                        # whole
        W.unique_keys(60000, bits, 2),                                       # MSD
        np.concatenate([np.arange(9000, dtype=dt), np.array([top], dt)]),    # skewed: LSD
        np.full(6000, 12345, dt),                                            # all equal: LSD
        W.duplicate_keys(1500, 8, bits, 3)[:12000].astype(dt),               # duplicates: MSD
        rng.integers(0, 1 << 10, size=20000).astype(dt),                     # narrow: MSD on low bits
        np.zeros(0, dt), np.array([7], dt), W.unique_keys(5120, bits, 4),    # empty, one, largest whole
        W.unique_keys(5121, bits, 6),                                        # just above: MSD
        W.unique_keys(100000, bits, 5),
    ]
    rows = [rng.permutation(len(x)).astype(np.uint32) for x in keys]
    off = np.zeros(len(keys) + 1, dtype=np.uint64)
    np.cumsum(np.array([len(x) for x in keys], dtype=np.uint64), out=off[1:])
    qs, qoff = _probes(keys, bits, [3000] * len(keys), 17)
    flag = gi.GI_KEY_U64 if bits == 64 else gi.GI_KEY_U32
    batch = gi.gi_batch_create(off, layout | flag, k)
    gi.gi_batch_build(batch, to_dev(np.concatenate(keys)), to_dev(np.concatenate(rows)))
    out = torch.full((int(qoff[-1]),), -5, dtype=torch.int32, device=DEV)
    gi.gi_batch_point_lookup(batch, to_dev(np.concatenate(qs)), to_dev(qoff), out)
    gi.gi_batch_sync(batch)
    _check(batch, keys, rows, qs, qoff, out, layout, k)
    gi.gi_batch_destroy(batch)


@pytest.mark.parametrize("sizes", [[100000], [0], [0, 0, 7000, 0], [1]])
def test_batch_degenerate_shapes(sizes):
    # one index, only empty indexes, empty indexes around one: every plan kernel and
    # ticket map must cope with indexes that have no tiles
    keys, rows, off = _make_batch(sizes, 64, 61)
    qs, qoff = _probes(keys, 64, [700] * len(sizes), 19)
    batch = gi.gi_batch_create(off, gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64, 9)
    kd = to_dev(np.concatenate(keys)) if off[-1] else torch.empty(0, dtype=torch.int64, device=DEV)
    rd = to_dev(np.concatenate(rows)) if off[-1] else torch.empty(0, dtype=torch.int32, device=DEV)
    gi.gi_batch_build(batch, kd, rd)
    out = torch.full((int(qoff[-1]),), -5, dtype=torch.int32, device=DEV)
    gi.gi_batch_point_lookup(batch, to_dev(np.concatenate(qs)), to_dev(qoff), out)
    gi.gi_batch_sync(batch)
    _check(batch, keys, rows, qs, qoff, out, gi.GI_EYTZINGER_KARY, 9)
    gi.gi_batch_destroy(batch)


@pytest.mark.parametrize("bits", [64, 32])
def test_batch_reserved_rowid_reported_by_sync(bits):
    # the reserved rowID is found in whichever pass first reads the caller's rowIDs:
    # the bucket sort of a whole index, the MSD scatter, or the first LSD pass
    dt = np.uint64 if bits == 64 else np.uint32
    keys = [W.unique_keys(3000, bits, 1),                                  # whole
            W.unique_keys(60000, bits, 2),                                 # MSD
            np.concatenate([np.arange(9000, dtype=dt), np.array([np.iinfo(dt).max], dt)]),  # LSD
            np.full(6000, 12345, dt)]                                      # all equal: LSD
    off = np.zeros(len(keys) + 1, dtype=np.uint64)
    np.cumsum(np.array([len(x) for x in keys], dtype=np.uint64), out=off[1:])
    flag = gi.GI_KEY_U64 if bits == 64 else gi.GI_KEY_U32
    batch = gi.gi_batch_create(off, gi.GI_EYTZINGER_KARY | flag, 5)
    kd = to_dev(np.concatenate(keys))
    for bad in range(len(keys)):
        rows = [np.arange(len(x), dtype=np.uint32) for x in keys]
        rows[bad][len(keys[bad]) // 2] = gi.GI_MISS
        gi.gi_batch_build(batch, kd, to_dev(np.concatenate(rows)))
        with pytest.raises(gi.GIError) as e:
            gi.gi_batch_sync(batch)
        assert e.value.code == gi.GI_ERR_INVALID, bad
    # reported once; a clean build afterwards syncs without error and is correct
    rows = [np.random.default_rng(i).permutation(len(x)).astype(np.uint32) for i, x in enumerate(keys)]
    gi.gi_batch_build(batch, kd, to_dev(np.concatenate(rows)))
    qs, qoff = _probes(keys, bits, [2000] * len(keys), 23)
    out = torch.full((int(qoff[-1]),), -5, dtype=torch.int32, device=DEV)
    gi.gi_batch_point_lookup(batch, to_dev(np.concatenate(qs)), to_dev(qoff), out)
    gi.gi_batch_sync(batch)
    _check(batch, keys, rows, qs, qoff, out, gi.GI_EYTZINGER_KARY, 5)
    gi.gi_batch_destroy(batch)


def _check_mixed(batch, keys, rows, qs, qoff, out, ks, check_layout=True):
    """Per index: lookups vs the oracle, and the layout of its own fan-out
    (0: sorted; 2: the binary tree in 0-based in-order fill; k: k-ary)."""
    got = to_host(out, np.uint32)
    for i in range(len(keys)):
        sk, sr = oracle.sort_pairs(keys[i], rows[i])
        assert np.array_equal(got[int(qoff[i]):int(qoff[i + 1])], oracle.point_lookup(sk, sr, qs[i])), \
            ("index", i, len(keys[i]), ks[i])
        if check_layout and len(keys[i]):
            n = len(keys[i])
            kk = torch.empty(n, dtype=torch.int64 if keys[i].dtype == np.uint64 else torch.int32, device=DEV)
            rr = torch.empty(n, dtype=torch.int32, device=DEV)
            gi.gi_batch_copy_index(batch, i, kk, rr)
            lay = oracle.SORTED if ks[i] == 0 else oracle.EYTZINGER_KARY
            ok, orr = oracle.layout_arrays(keys[i], rows[i], lay, max(int(ks[i]), 2))
            assert np.array_equal(to_host(kk, keys[i].dtype), ok), ("layout", i, ks[i])
            assert np.array_equal(to_host(rr, np.uint32), orr), ("layout rows", i, ks[i])


@pytest.mark.parametrize("bits", [64, 32])
def test_batch_fanout_per_index_equals_oracle(bits):
    """Each index of one batch has its own fan-out (sorted, 2, 3, 5, 9, 17), over
    every build plan (whole index in one CTA, MSD + buckets, LSD fallback), in one
    build and one lookup launch; then the same batch with other fan-outs."""
    dt = np.uint64 if bits == 64 else np.uint32
    rng = np.random.default_rng(bits)
    keys = [W.unique_keys(4000, bits, 1), W.unique_keys(60000, bits, 2),
            np.concatenate([np.arange(9000, dtype=dt), np.array([np.iinfo(dt).max], dt)]),  # LSD
            W.duplicate_keys(1500, 8, bits, 3)[:12000].astype(dt), np.zeros(0, dt), np.array([7], dt),
            W.unique_keys(5120, bits, 4), W.unique_keys(100000, bits, 5)]
    keys += [W.unique_keys(int(n), bits, 10 + i) for i, n in enumerate(rng.integers(1, 30000, size=16))]
    rows = [rng.permutation(len(x)).astype(np.uint32) for x in keys]
    off = np.zeros(len(keys) + 1, dtype=np.uint64)
    np.cumsum(np.array([len(x) for x in keys], dtype=np.uint64), out=off[1:])
    qs, qoff = _probes(keys, bits, list(rng.integers(100, 3000, size=len(keys))), 31)
    flag = gi.GI_KEY_U64 if bits == 64 else gi.GI_KEY_U32
    batch = gi.gi_batch_create(off, gi.GI_EYTZINGER_KARY | flag, 5)
    kd, rd = to_dev(np.concatenate(keys)), to_dev(np.concatenate(rows))
    qd, qod = to_dev(np.concatenate(qs)), to_dev(qoff)
    out = torch.full((int(qoff[-1]),), -5, dtype=torch.int32, device=DEV)
    cycle = np.array([0, 2, 3, 5, 9, 17], dtype=np.uint32)
    for shift in (0, 3):
        ks = cycle[(np.arange(len(keys)) + shift) % len(cycle)]
        gi.gi_batch_set_fanouts(batch, ks)
        assert np.array_equal(gi.gi_batch_get_fanouts(batch, len(keys)), ks)
        gi.gi_batch_build(batch, kd, rd)
        out.fill_(-5)
        gi.gi_batch_point_lookup(batch, qd, qod, out)
        gi.gi_batch_sync(batch)
        _check_mixed(batch, keys, rows, qs, qoff, out, ks)
        for opt, v in ((gi.GI_BATCH_OPT_SMEM_BUDGET, 40960), (gi.GI_BATCH_OPT_CHUNK, 96)):
            gi.gi_batch_set_option(batch, opt, v)
            out.fill_(-5)
            gi.gi_batch_point_lookup(batch, qd, qod, out)
            gi.gi_batch_sync(batch)
            _check_mixed(batch, keys, rows, qs, qoff, out, ks, check_layout=False)
        gi.gi_batch_set_option(batch, gi.GI_BATCH_OPT_SMEM_BUDGET, 0)
        gi.gi_batch_set_option(batch, gi.GI_BATCH_OPT_CHUNK, 2048)
    with pytest.raises(gi.GIError) as e:
        gi.gi_batch_set_fanouts(batch, np.full(len(keys), 4, np.uint32))
    assert e.value.code == gi.GI_ERR_INVALID
    gi.gi_batch_destroy(batch)


def test_batch_fanout_automatic_and_graph_replay():
    """NULL fan-outs choose by size class (k = 3 up to 2^12 u64 keys, k = 5 above,
    when nothing is recorded); the mixed batch's build + lookup replayed from a
    CUDA graph gives the oracle's answers."""
    gi.gi_batch_fanout_table_clear()
    rng = np.random.default_rng(12)
    sizes = [int(x) for x in np.exp2(rng.uniform(8, 20, size=40)).astype(np.int64)]
    keys, rows, off = _make_batch(sizes, 64, 81)
    qs, qoff = _probes(keys, 64, list(rng.integers(0, 4000, size=len(sizes))), 10)
    batch = gi.gi_batch_create(off, gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64, 5)
    gi.gi_batch_set_fanouts(batch, None)
    ks = gi.gi_batch_get_fanouts(batch, len(sizes))
    want = [3 if n <= (1 << 12) else 5 for n in sizes]
    assert list(ks) == want
    kd, rd = to_dev(np.concatenate(keys)), to_dev(np.concatenate(rows))
    qd, qod = to_dev(np.concatenate(qs)), to_dev(qoff)
    out = torch.full((int(qoff[-1]),), -5, dtype=torch.int32, device=DEV)
    s = torch.cuda.Stream()
    gi.gi_batch_set_stream(batch, s)
    with torch.cuda.stream(s):
        gi.gi_batch_build(batch, kd, rd)
        gi.gi_batch_point_lookup(batch, qd, qod, out)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        gi.gi_batch_build(batch, kd, rd)
        gi.gi_batch_point_lookup(batch, qd, qod, out)
    for _ in range(2):
        out.fill_(-5)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        gi.gi_batch_sync(batch)
        _check_mixed(batch, keys, rows, qs, qoff, out, ks)
    gi.gi_batch_destroy(batch)


def test_batch_fanout_tuner():
    """gi_batch_tune_fanouts times every candidate fan-out per size class and keeps
    the fastest per class; with GI_TUNE_APPLY the batch ends built with them (its
    answers still the oracle's), with GI_TUNE_RECORD a later batch's automatic
    choice follows the record."""
    gi.gi_batch_fanout_table_clear()
    rng = np.random.default_rng(5)
    sizes = [int(x) for x in np.exp2(rng.uniform(8, 18, size=60)).astype(np.int64)]
    keys, rows, off = _make_batch(sizes, 64, 91)
    qs, qoff = _probes(keys, 64, list(rng.integers(500, 3000, size=len(sizes))), 12)
    batch = gi.gi_batch_create(off, gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64, 5)
    kd, rd = to_dev(np.concatenate(keys)), to_dev(np.concatenate(rows))
    qd, qod = to_dev(np.concatenate(qs)), to_dev(qoff)
    ks, cms = gi.gi_batch_tune_fanouts(batch, len(sizes), kd, rd, qd, qod, reps=2,
                                       flags=gi.GI_TUNE_APPLY | gi.GI_TUNE_RECORD)
    cls = [int(np.floor(np.log2(n))) for n in sizes]
    cand = [2, 3, 5, 9, 17]
    for i, c in enumerate(cls):
        assert cms[c].min() > 0
        assert ks[i] == cand[int(np.argmin(cms[c]))]  # the fastest candidate of its class
    assert np.array_equal(gi.gi_batch_get_fanouts(batch, len(sizes)), ks)
    out = torch.full((int(qoff[-1]),), -5, dtype=torch.int32, device=DEV)
    gi.gi_batch_point_lookup(batch, qd, qod, out)
    gi.gi_batch_sync(batch)
    _check_mixed(batch, keys, rows, qs, qoff, out, ks, check_layout=False)
    # a new batch of the same sizes takes the recorded choices automatically
    b2 = gi.gi_batch_create(off, gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64, 5)
    gi.gi_batch_set_fanouts(b2, None)
    assert np.array_equal(gi.gi_batch_get_fanouts(b2, len(sizes)), ks)
    gi.gi_batch_destroy(b2)
    gi.gi_batch_fanout_table_clear()
    gi.gi_batch_destroy(batch)
