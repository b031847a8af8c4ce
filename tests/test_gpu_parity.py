"""GPU path vs CPU oracle, element by element, through the C ABI.

Every output is integer: results must be bit-identical (rowIDs, CSR offsets,
CSR rows and their order), and the built layout must equal the oracle's
in-order fill slot by slot.  Sizes span several radix tiles (4096 u32 / 3072 u64
keys per tile) with ragged tails, every fan-out the library compiles plus two it
does not (generic kernel), unique and duplicate-heavy key sets, and the edge
cases: empty index, one key, probes at 0 and at the key maximum, empty and
inverted ranges, ranges covering everything.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2506_01576_gb300 as gi
import workloads as W

pytestmark = pytest.mark.gpu

from gpu_util import DEV, build, layout_arrays, point, ranges, to_dev  # noqa: E402

LAYOUTS = [(gi.GI_SORTED, 0), (gi.GI_EYTZINGER, 2)] + [
    (gi.GI_EYTZINGER_KARY, k) for k in (3, 4, 5, 8, 9, 16, 17, 32, 33, 2, 6)]
SIZES = [0, 1, 2, 3, 7, 31, 100, 1000, 3071, 3072, 4097, 12289, 50000]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2506_01576_gb300 import _build
    _build.build()
    gi.load()
    torch.cuda.set_device(DEV)


def _oracle_layout(keys, rows, layout, k):
    return oracle.layout_arrays(keys, rows, {gi.GI_SORTED: oracle.SORTED, gi.GI_EYTZINGER: oracle.EYTZINGER,
                                             gi.GI_EYTZINGER_KARY: oracle.EYTZINGER_KARY}[layout], k)


def _probe_set(keys, dtype, rng):
    top = np.iinfo(dtype).max
    extra = np.array([0, 1, top, top - 1], dtype=dtype)
    rnd = rng.integers(0, top, size=2000, dtype=dtype, endpoint=True)
    near = (keys[: 500] + dtype(1)) if len(keys) else np.zeros(0, dtype)
    return np.concatenate([keys, extra, rnd, near]).astype(dtype)


def _range_set(keys, dtype, rng):
    top = np.iinfo(dtype).max
    sk = np.sort(keys)
    m = 600
    a = rng.integers(0, top, size=m, dtype=dtype, endpoint=True)
    w = rng.integers(0, 2 ** (8 * np.dtype(dtype).itemsize - 6), size=m, dtype=dtype)
    with np.errstate(over="ignore"):
        b = a + w  # wraps on overflow
    b = np.where(b < a, top, b).astype(dtype)
    lo = [a]
    hi = [b]
    if len(sk):
        i = rng.integers(0, len(sk), size=200)
        j = np.minimum(i + rng.integers(0, 40, size=200), len(sk) - 1)
        lo.append(sk[i]); hi.append(sk[j])               # exact key bounds
        lo.append(sk[j]); hi.append(sk[i])               # inverted (empty unless equal)
    lo.append(np.array([0, top, 0, 5, top], dtype=dtype))
    hi.append(np.array([top, top, 0, 4, 0], dtype=dtype))  # everything, max only, min only, empty, inverted
    return np.concatenate(lo).astype(dtype), np.concatenate(hi).astype(dtype)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("layout,k", LAYOUTS)
def test_unique_keys_all_sizes(dtype, layout, k):
    bits = 8 * np.dtype(dtype).itemsize
    rng = np.random.default_rng(1234 + k)
    for n in SIZES:
        keys = W.unique_keys(n, bits, W.seed_for(7, n % 64, k))
        rows = rng.permutation(n).astype(np.uint32)
        idx = build(keys, rows, layout, k)
        inf = gi.gi_get_info(idx)
        assert inf.n == n and inf.unique == 1
        assert gi.gi_footprint_bytes(idx) == n * (np.dtype(dtype).itemsize + 4) + (
            np.dtype(dtype).itemsize if layout == gi.GI_EYTZINGER else 0)
        lk, lr = layout_arrays(idx, n, dtype)
        ok, orr = _oracle_layout(keys, rows, layout, k)
        assert np.array_equal(lk, ok) and np.array_equal(lr, orr), ("layout", n)
        sk, sr = oracle.sort_pairs(keys, rows)
        q = _probe_set(keys, dtype, rng)
        assert np.array_equal(point(idx, q), oracle.point_lookup(sk, sr, q)), ("point", n)
        lo, hi = _range_set(keys, dtype, rng)
        off, rr = ranges(idx, lo, hi)
        woff, wrr = oracle.range_lookup(sk, sr, lo, hi)
        assert np.array_equal(off, woff), ("offsets", n)
        assert np.array_equal(rr, wrr), ("rows", n)
        gi.gi_destroy(idx)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("layout,k", [(gi.GI_SORTED, 0), (gi.GI_EYTZINGER, 2),
                                      (gi.GI_EYTZINGER_KARY, 3), (gi.GI_EYTZINGER_KARY, 9),
                                      (gi.GI_EYTZINGER_KARY, 16), (gi.GI_EYTZINGER_KARY, 33),
                                      (gi.GI_EYTZINGER_KARY, 7)])
def test_duplicate_keys(dtype, layout, k):
    # duplicates: first entry in input order wins a point lookup; ranges list all of
    # them in (key, input position) order (Section 8.11)
    rng = np.random.default_rng(99)
    top = np.iinfo(dtype).max
    for n, alphabet in [(50, 3), (1000, 37), (9000, 500), (20000, 20000)]:
        vals = np.unique(rng.integers(0, top, size=alphabet, dtype=dtype, endpoint=True))
        vals[0] = 0
        keys = vals[rng.integers(0, len(vals), size=n)]
        rows = rng.permutation(n).astype(np.uint32)
        idx = build(keys, rows, layout, k)
        assert gi.gi_get_info(idx).unique == (1 if len(np.unique(keys)) == n else 0)
        lk, lr = layout_arrays(idx, n, dtype)
        ok, orr = _oracle_layout(keys, rows, layout, k)
        assert np.array_equal(lk, ok) and np.array_equal(lr, orr)
        sk, sr = oracle.sort_pairs(keys, rows)
        q = np.concatenate([vals, _probe_set(keys[:100], dtype, rng)]).astype(dtype)
        assert np.array_equal(point(idx, q), oracle.point_lookup(sk, sr, q))
        lo, hi = _range_set(keys, dtype, rng)
        lo = np.concatenate([lo, vals[:50]]).astype(dtype)
        hi = np.concatenate([hi, vals[:50]]).astype(dtype)
        off, rr = ranges(idx, lo, hi)
        woff, wrr = oracle.range_lookup(sk, sr, lo, hi)
        assert np.array_equal(off, woff) and np.array_equal(rr, wrr)
        gi.gi_destroy(idx)


def test_all_equal_keys_skip_every_radix_pass():
    # every digit trivial: no radix pass runs, the input order is the sorted order
    for dtype in (np.uint32, np.uint64):
        keys = np.full(5000, 12345, dtype=dtype)
        rows = np.arange(5000, dtype=np.uint32)[::-1].copy()
        for layout, k in [(gi.GI_SORTED, 0), (gi.GI_EYTZINGER, 2), (gi.GI_EYTZINGER_KARY, 9)]:
            idx = build(keys, rows, layout, k)
            lk, lr = layout_arrays(idx, 5000, dtype)
            ok, orr = _oracle_layout(keys, rows, layout, k)
            assert np.array_equal(lk, ok) and np.array_equal(lr, orr)
            assert point(idx, np.array([12345, 1], dtype=dtype)).tolist() == [4999, gi.GI_MISS]
            gi.gi_destroy(idx)


@pytest.mark.parametrize("layout,k", [(gi.GI_EYTZINGER, 2), (gi.GI_EYTZINGER_KARY, 9),
                                      (gi.GI_EYTZINGER_KARY, 17), (gi.GI_EYTZINGER_KARY, 5)])
@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_every_knob_gives_identical_results(layout, k, dtype):
    # group size, interleaving, shared-memory pinning, block size, persistent grid,
    # prefetch and early exit change the schedule, never the answer (Sections 6.2, 7)
    bits = 8 * np.dtype(dtype).itemsize
    n = 70001
    keys = W.unique_keys(n, bits, 5)
    rows = np.arange(n, dtype=np.uint32)
    q = W.point_probes(keys, 100000, 0.5, bits, 5, 6)
    sk, sr = oracle.sort_pairs(keys, rows)
    want = oracle.point_lookup(sk, sr, q)
    idx = build(keys, rows, layout, k)
    groups = [g for g in (1, 2, 4, 8, 16, 32) if layout == gi.GI_EYTZINGER_KARY
              and _supported(idx, g)] or [None]
    configs = []
    for g in groups:
        for pt in (1, 2, 4):
            configs.append(dict(group=g, pt=pt, smem=0, block=256, bpsm=0, pf=0, ee=1))
    configs += [dict(group=groups[-1], pt=2, smem=3, block=256, bpsm=2, pf=0, ee=1),
                dict(group=groups[0], pt=1, smem=4, block=512, bpsm=1, pf=0, ee=0),
                dict(group=groups[-1], pt=4, smem=2, block=128, bpsm=0, pf=0, ee=1),
                dict(group=groups[0], pt=2, smem=0, block=64, bpsm=4, pf=0, ee=0)]
    if layout == gi.GI_EYTZINGER:
        configs += [dict(group=None, pt=p, smem=s, block=256, bpsm=b, pf=f, ee=1)
                    for f in (2, 3, 4) for p in (1, 4) for (s, b) in ((0, 0), (8, 2))]
    for c in configs:
        if c["group"] is not None:
            gi.gi_set_option(idx, gi.GI_OPT_GROUP, c["group"])
        gi.gi_set_option(idx, gi.GI_OPT_PER_THREAD, c["pt"])
        try:
            gi.gi_set_option(idx, gi.GI_OPT_SMEM_LEVELS, c["smem"])
        except gi.GIError:  # that many levels do not fit in shared memory
            gi.gi_set_option(idx, gi.GI_OPT_SMEM_LEVELS, 2)
        gi.gi_set_option(idx, gi.GI_OPT_BLOCK, c["block"])
        gi.gi_set_option(idx, gi.GI_OPT_BLOCKS_PER_SM, c["bpsm"])
        gi.gi_set_option(idx, gi.GI_OPT_PREFETCH, c["pf"])
        gi.gi_set_option(idx, gi.GI_OPT_EARLY_EXIT, c["ee"])
        assert np.array_equal(point(idx, q), want), c
    gi.gi_sync(idx)
    gi.gi_destroy(idx)


def _supported(idx, g):
    try:
        gi.gi_set_option(idx, gi.GI_OPT_GROUP, g)
        return True
    except gi.GIError:
        return False


def test_host_buffers_equal_device_buffers():
    # the staged host-memory path (pinned and pageable) returns what the device path does
    n, m = 200003, 3 * (1 << 22) + 77  # several staging chunks with a ragged tail
    keys = W.unique_keys(n, 64, 11)
    rows = np.arange(n, dtype=np.uint32)
    q = W.point_probes(keys, m, 0.5, 64, 11, 12)
    sk, sr = oracle.sort_pairs(keys, rows)
    want = oracle.point_lookup(sk, sr, q, threads=oracle.hardware_threads())
    idx = gi.gi_build(keys, rows, gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64, 9)  # host inputs
    out = np.empty(m, dtype=np.uint32)
    gi.gi_point_lookup(idx, q, out)  # pageable host memory
    assert np.array_equal(out, want)
    qp = torch.from_numpy(q.view(np.int64)).pin_memory()
    op = torch.empty(m, dtype=torch.int32).pin_memory()
    gi.gi_point_lookup(idx, qp, op)
    assert np.array_equal(op.numpy().view(np.uint32), want)
    lo = q[:5000]
    hi = lo + np.uint64(1 << 48)
    woff, wrr = oracle.range_lookup(sk, sr, lo, hi)
    off = np.empty(len(lo) + 1, dtype=np.uint64)
    gi.gi_range_lookup(idx, lo, hi, off)
    rr = np.empty(int(off[-1]), dtype=np.uint32)
    gi.gi_range_lookup(idx, lo, hi, off, rr)
    assert np.array_equal(off, woff) and np.array_equal(rr, wrr)
    gi.gi_destroy(idx)


@pytest.mark.parametrize("layout,k", [(gi.GI_EYTZINGER_KARY, 5), (gi.GI_SORTED, 0), (gi.GI_EYTZINGER, 0)])
def test_host_range_fill_pipeline(layout, k):
    # more than 2^22 rows into host memory: the fill runs in 8 chunks of ranges, each
    # chunk's rows copied back while the next is filled; a ragged range count,
    # empty ranges and one range bigger than a chunk
    n = (1 << 21) + 5
    keys = W.unique_keys(n, 64, 41)
    rows = np.random.default_rng(4).permutation(n).astype(np.uint32)
    sk, sr = oracle.sort_pairs(keys, rows)
    m = 40003
    lo, hi, _ = W.ranges_with_expected_rows(n, m, 160, 64, 43)
    lo[7], hi[7] = hi[7], lo[7]          # lo > hi: empty
    lo[9], hi[9] = 0, np.uint64(1 << 62)  # about half of all keys
    woff, wrr = oracle.range_lookup(sk, sr, lo, hi)
    assert woff[-1] > (1 << 22)
    idx = build(keys, rows, layout, k)
    for pinned in (False, True):
        alloc = (lambda a: torch.from_numpy(a).pin_memory().numpy()) if pinned else (lambda a: a)
        off = alloc(np.zeros(m + 1, dtype=np.uint64))
        out = alloc(np.zeros(int(woff[-1]), dtype=np.uint32))
        gi.gi_range_lookup(idx, alloc(lo.copy()), alloc(hi.copy()), off, out)
        assert np.array_equal(off, woff) and np.array_equal(out, wrr), pinned
        # device offsets, host rows
        offd = torch.empty(m + 1, dtype=torch.int64, device=DEV)
        out2 = alloc(np.zeros(int(woff[-1]), dtype=np.uint32))
        gi.gi_range_lookup(idx, to_dev(lo), to_dev(hi), offd, out2)
        assert np.array_equal(out2, wrr), pinned
    gi.gi_destroy(idx)


def test_reserved_rowid_rejected_and_streams():
    keys = np.arange(100, dtype=np.uint32)
    rows = np.arange(100, dtype=np.uint32)
    rows[57] = gi.GI_MISS
    with pytest.raises(gi.GIError) as e:
        build(keys, rows, gi.GI_EYTZINGER)
    assert e.value.code == gi.GI_ERR_INVALID
    # a built index follows the thread's default stream and can be moved to another
    s = torch.cuda.Stream()
    gi.gi_set_stream(None, s)
    try:
        rows[57] = 57
        idx = build(keys, rows, gi.GI_EYTZINGER_KARY, 9)
        with torch.cuda.stream(s):
            out = torch.empty(100, dtype=torch.int32, device=DEV)
            gi.gi_point_lookup(idx, to_dev(keys), out)
        s.synchronize()
        assert out.cpu().numpy().tolist() == list(range(100))
        gi.gi_set_stream(idx, None)
        assert point(idx, keys).tolist() == list(range(100))
        gi.gi_destroy(idx)
    finally:
        gi.gi_set_stream(None, None)


def _pin(a):
    return torch.from_numpy(a).pin_memory().numpy()


@pytest.mark.parametrize("sizes", [(1 << 24) + 11, 300007])
def test_build_from_page_locked_host_memory(sizes):
    # page-locked keys: the histogram pass copies them over the bus as it counts;
    # page-locked rowIDs: the first sort pass reads them where they are.  Every
    # combination of pinned / pageable / device inputs gives the oracle's layout;
    # 2^24 + 11 u64 keys take the hybrid sort, 300007 the LSD sort.
    n = sizes
    keys = W.unique_keys(n, 64, 13)
    rows = np.random.default_rng(8).permutation(n).astype(np.uint32)
    ok, orr = _oracle_layout(keys, rows, gi.GI_EYTZINGER_KARY, 5)
    kinds = {"pinned": _pin, "pageable": lambda a: a.copy(), "device": to_dev}
    for kk, rk in (("pinned", "pinned"), ("pinned", "pageable"), ("pageable", "pinned"),
                   ("device", "pinned"), ("pinned", "device")):
        idx = gi.gi_build(kinds[kk](keys), kinds[rk](rows), gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64, 5)
        lk, lr = layout_arrays(idx, n, np.uint64)
        assert np.array_equal(lk, ok) and np.array_equal(lr, orr), (kk, rk)
        gi.gi_destroy(idx)


@pytest.mark.parametrize("equal_keys", [False, True])
def test_reserved_rowid_rejected_from_page_locked_rows(equal_keys):
    # the check runs in the pass that reads the input rowIDs (or on its own when
    # every key is equal and no pass runs), also when they are read over the bus
    n = 5000
    keys = np.full(n, 7, np.uint64) if equal_keys else W.unique_keys(n, 64, 3)
    rows = np.arange(n, dtype=np.uint32)
    rows[n - 1] = gi.GI_MISS
    for lay, k in ((gi.GI_SORTED, 0), (gi.GI_EYTZINGER_KARY, 5)):
        for src in (_pin, lambda a: a.copy(), to_dev):
            with pytest.raises(gi.GIError) as e:
                gi.gi_build(src(keys), src(rows), lay | gi.GI_KEY_U64, k)
            assert e.value.code == gi.GI_ERR_INVALID
    rows[n - 1] = n - 1
    idx = gi.gi_build(_pin(keys), _pin(rows), gi.GI_SORTED | gi.GI_KEY_U64, 0)
    assert gi.gi_get_info(idx).unique == (0 if equal_keys else 1)
    gi.gi_destroy(idx)


def test_probes_roofline_kernels_run():
    buf = torch.zeros(1 << 24, dtype=torch.int32, device=DEV)
    sink = torch.zeros(1, dtype=torch.int64, device=DEV)
    for c in (16, 32, 64, 128, 256):
        gi.gi_probe_random_sectors(buf, c, 1 << 20, 7, sink)
    for g in (1, 2, 16, 32, 64):
        gi.gi_coalescing_probe(buf, 1 << 16, g, 64, 3, sink)
    torch.cuda.synchronize()
    with pytest.raises(gi.GIError):
        gi.gi_probe_random_sectors(buf, 48, 10, 1, sink)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("layout,k", [(gi.GI_EYTZINGER, 2), (gi.GI_EYTZINGER_KARY, 5),
                                      (gi.GI_EYTZINGER_KARY, 16), (gi.GI_EYTZINGER_KARY, 33),
                                      (gi.GI_EYTZINGER_KARY, 6)])
def test_range_fill_by_level_runs_equals_by_rank(dtype, layout, k):
    # Section 5 level-by-level fill (warp switch at 32 slots per level, Section 5.1)
    # and the per-rank map write the same CSR; widths from a few rows to thousands
    bits = 8 * np.dtype(dtype).itemsize
    n = 200003
    keys = W.unique_keys(n, bits, 41)
    rows = np.random.default_rng(1).permutation(n).astype(np.uint32)
    sk, sr = oracle.sort_pairs(keys, rows)
    idx = build(keys, rows, layout, k)
    for E in (1, 5, 40, 300, 3000):
        lo, hi, _ = W.ranges_with_expected_rows(n, 4000, E, bits, E)
        woff, wrr = oracle.range_lookup(sk, sr, lo, hi)
        for fill in (0, 1):
            gi.gi_set_option(idx, gi.GI_OPT_RANGE_FILL, fill)
            off, rr = ranges(idx, lo, hi)
            assert np.array_equal(off, woff) and np.array_equal(rr, wrr), (E, fill)
    gi.gi_destroy(idx)


@pytest.mark.parametrize("replicas", [1, 4, 64, 1024])
def test_duplicate_keys_all_occurrences_by_point_range(replicas):
    # Section 8.11 / Fig 25: with duplicates a point query returns every occurrence,
    # i.e. the range [x, x]; occurrences come in input order
    n_distinct = max(1, 100000 // replicas)
    keys = W.duplicate_keys(n_distinct, replicas, 64, 5)
    rows = np.arange(len(keys), dtype=np.uint32)
    sk, sr = oracle.sort_pairs(keys, rows)
    probes = np.concatenate([np.unique(keys)[:3000], W.unique_keys(500, 64, 999)]).astype(np.uint64)
    woff, wrr = oracle.range_lookup(sk, sr, probes, probes)
    for layout, k in ((gi.GI_SORTED, 0), (gi.GI_EYTZINGER, 2), (gi.GI_EYTZINGER_KARY, 9)):
        idx = build(keys, rows, layout, k)
        off, rr = ranges(idx, probes, probes)
        assert np.array_equal(off, woff) and np.array_equal(rr, wrr), (layout, k)
        # the point lookup returns the first occurrence (input order)
        first = point(idx, probes)
        want_first = np.where(np.diff(woff) > 0, wrr[np.minimum(woff[:-1], len(wrr) - 1).astype(np.int64)], gi.GI_MISS)
        assert np.array_equal(first, want_first.astype(np.uint32))
        gi.gi_destroy(idx)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("layout,k", [(gi.GI_SORTED, 0), (gi.GI_EYTZINGER, 2), (gi.GI_EYTZINGER_KARY, 3),
                                      (gi.GI_EYTZINGER_KARY, 5), (gi.GI_EYTZINGER_KARY, 9),
                                      (gi.GI_EYTZINGER_KARY, 17), (gi.GI_EYTZINGER_KARY, 4)])
def test_local_lookup_reordering_changes_nothing(dtype, layout, k):
    # Section 7.4: probes sorted per CTA tile, results restored to probe order;
    # ragged last tile, duplicate keys, Zipf-skewed and pre-sorted probes
    bits = 8 * np.dtype(dtype).itemsize
    for n, dup in ((123457, False), (50000, True)):
        keys = W.duplicate_keys(n // 5, 5, bits, 3) if dup else W.unique_keys(n, bits, 3)
        rows = np.arange(len(keys), dtype=np.uint32)
        sk, sr = oracle.sort_pairs(keys, rows)
        idx = build(keys, rows, layout, k)
        gi.gi_set_option(idx, gi.GI_OPT_REORDER, 1)
        for q in (W.point_probes(np.unique(keys), 10007, 0.5, bits, 3, 4, dist="zipf", zipf_s=1.25),
                  np.sort(W.point_probes(np.unique(keys), 20000, 0.5, bits, 3, 5)),
                  np.array([0, np.iinfo(dtype).max], dtype=dtype)):
            assert np.array_equal(point(idx, q.astype(dtype)), oracle.point_lookup(sk, sr, q.astype(dtype)))
        gi.gi_destroy(idx)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("dist", ["uniform", "narrow", "dups", "dups64", "cluster", "skewed"])
def test_hybrid_msd_build_equals_plain_lsd_build(dtype, dist):
    # GI_BUILD_HYBRID scatters by the top digit(s) and sorts each bucket in shared
    # memory (the default does so only from 2^24 u64 keys up); GI_BUILD_LSD forces
    # the plain LSD passes.  Both must give the oracle's layout.  narrow: the top digits are trivial; dups: 16 copies of every key
    # (stability); dups64: 64 copies, more than a sub-bucket may hold for count
    # ranking, so every bucket's split gives up and the ballot passes sort it; cluster: 20000 keys share their top 16 bits, so one level-2 bucket
    # is too big for a CTA and the build falls back to LSD after the first scatter;
    # skewed: 70% of the keys below 2^16, so the hybrid sort is not tried at all.
    bits = 8 * np.dtype(dtype).itemsize
    top = np.iinfo(dtype).max
    n = (1 << 21) + 12345
    rng = np.random.default_rng(17)
    if dist == "uniform":
        keys = W.unique_keys(n, bits, 8)
    elif dist == "narrow":
        keys = rng.integers(0, 1 << 24, size=n).astype(dtype)
    elif dist == "dups":
        keys = W.duplicate_keys(n // 16, 16, bits, 8)
        n = len(keys)
    elif dist == "dups64":
        keys = W.duplicate_keys(n // 64, 64, bits, 9)
        n = len(keys)
    elif dist == "cluster":
        keys = rng.integers(0, top, size=n, dtype=dtype, endpoint=True)
        hi = dtype(0xABCD) << dtype(bits - 16)
        keys[:20000] = hi | rng.integers(0, 1 << (bits - 16), size=20000, dtype=np.uint64).astype(dtype)
        rng.shuffle(keys)
    else:
        keys = np.where(rng.random(n) < 0.7, rng.integers(0, 1 << 16, size=n).astype(dtype),
                        rng.integers(0, top, size=n, dtype=dtype, endpoint=True))
    rows = rng.permutation(n).astype(np.uint32)
    sk, sr = oracle.sort_pairs(keys, rows)
    q = np.concatenate([keys[rng.integers(0, n, size=20000)],
                        rng.integers(0, top, size=5000, dtype=dtype, endpoint=True)])
    want = oracle.point_lookup(sk, sr, q)
    unique = bool(np.all(sk[1:] != sk[:-1]))
    for layout, k in ((gi.GI_SORTED, 0), (gi.GI_EYTZINGER_KARY, 5)):
        ok, orr = _oracle_layout(keys, rows, layout, k)
        for flag in (gi.GI_BUILD_HYBRID, gi.GI_BUILD_LSD):
            idx = build(keys, rows, layout | flag, k)
            lk, lr = layout_arrays(idx, n, dtype)
            assert np.array_equal(lk, ok) and np.array_equal(lr, orr), (layout, flag)
            assert np.array_equal(point(idx, q), want), (layout, flag)
            assert bool(gi.gi_get_info(idx).unique) == unique, (layout, flag)
            gi.gi_destroy(idx)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("layout,k", [(gi.GI_EYTZINGER, 0), (gi.GI_EYTZINGER_KARY, 3), (gi.GI_EYTZINGER_KARY, 9),
                                      (gi.GI_EYTZINGER_KARY, 17), (gi.GI_EYTZINGER_KARY, 4),
                                      (gi.GI_EYTZINGER_KARY, 33)])
def test_hybrid_build_writes_every_layout(dtype, layout, k):
    # the bucket sort writes each key straight to its slot in the layout (the
    # 32-bit rank -> slot map, specialised for k = 2, 3, 5, 9, 17, generic otherwise);
    # the extreme keys 0 and the maximum are in the input, n just above 2^20
    bits = 8 * np.dtype(dtype).itemsize
    top = np.iinfo(dtype).max
    n = (1 << 20) + 3
    keys = W.unique_keys(n, bits, 31)
    keys[:2] = [0, top]
    keys = np.unique(keys)
    n = len(keys)
    rng = np.random.default_rng(5)
    keys = keys[rng.permutation(n)]
    rows = rng.permutation(n).astype(np.uint32)
    ok, orr = _oracle_layout(keys, rows, layout, k)
    for flag in (gi.GI_BUILD_HYBRID, gi.GI_BUILD_LSD):
        idx = build(keys, rows, layout | flag, k)
        lk, lr = layout_arrays(idx, n, dtype)
        assert np.array_equal(lk, ok) and np.array_equal(lr, orr), flag
        info = gi.gi_get_info(idx)
        assert info.unique == 1
        gi.gi_destroy(idx)


@pytest.mark.parametrize("n,hybrid_launches", [((1 << 18) + 1000, 5), ((1 << 21) + 1000, 13), (1 << 24, 13)])
@pytest.mark.parametrize("layout,k", [(gi.GI_EYTZINGER_KARY, 5), (gi.GI_SORTED, 0)])
def test_default_build_takes_the_hybrid_sort_from_2e18_u64(layout, k, n, hybrid_launches):
    # the default path from the size where it starts to pay, 2^18 u64 keys.  The
    # launch count shows which sort ran.  Hybrid with two windows: the pass finding
    # the differing bits, the window's counts + scan, two MSD passes, one
    # per-bucket histogram + scan, the bucket lists by size class, one bucket-sort
    # launch per class = 13 kernels; with one window (2^18 + 1000 keys: ~1030-pair
    # buckets after the first scatter) 3 + 1 MSD pass + 1 bucket-sort launch = 5.
    # LSD: histogram, scan, 8 passes and the permutation or duplicate check = 11.
    keys = W.unique_keys(n, 64, 77)
    rows = np.random.default_rng(3).permutation(n).astype(np.uint32)
    ok, orr = _oracle_layout(keys, rows, layout, k)
    for flag, launches in ((0, hybrid_launches), (gi.GI_BUILD_LSD, 11)):
        c0 = gi.gi_launch_count()
        idx = build(keys, rows, layout | flag, k)
        assert gi.gi_launch_count() - c0 == launches, flag
        lk, lr = layout_arrays(idx, n, np.uint64)
        assert np.array_equal(lk, ok) and np.array_equal(lr, orr), flag
        gi.gi_destroy(idx)


def test_build_flags_are_exclusive():
    keys = np.arange(10, dtype=np.uint64)
    rows = np.arange(10, dtype=np.uint32)
    with pytest.raises(gi.GIError) as e:
        build(keys, rows, gi.GI_SORTED | gi.GI_BUILD_LSD | gi.GI_BUILD_HYBRID, 0)
    assert e.value.code == gi.GI_ERR_INVALID


@pytest.mark.parametrize("layout,k", [(gi.GI_EYTZINGER_KARY, 5), (gi.GI_SORTED, 0)])
def test_hybrid_buckets_above_4096_take_the_512_thread_sort(layout, k):
    # 2^20 uniform keys plus a cluster of 4400 keys that agree on every bit from
    # bit 13 up: the cluster and ~512 uniform keys share one bucket after both MSD
    # windows (the first 8 bits below bit 62, then 3 more: its level-1 bucket holds
    # ~8700 pairs), ~4900 pairs, which takes the bucket sort's 512-thread class (up
    # to 5120 pairs); random low 13 bits within the cluster
    rng = np.random.default_rng(23)
    base = rng.integers(0, 1 << 62, size=1, dtype=np.uint64)[0] & ~np.uint64(0x1FFF)
    cluster = base | np.arange(4400, dtype=np.uint64)
    keys = np.unique(np.concatenate([W.unique_keys(1 << 20, 64, 29), cluster]))
    n = len(keys)
    keys = keys[rng.permutation(n)]
    rows = rng.permutation(n).astype(np.uint32)
    ok, orr = _oracle_layout(keys, rows, layout, k)
    # hybrid: 8 launches before the bucket sort, then one per size class (the
    # cluster's bucket in the 5120-pair class, the ~512-pair buckets in the
    # smallest), 13 in all; LSD: 11
    for flag, launches in ((gi.GI_BUILD_HYBRID, 13), (gi.GI_BUILD_LSD, 11)):
        c0 = gi.gi_launch_count()
        idx = build(keys, rows, layout | flag, k)
        assert gi.gi_launch_count() - c0 == launches, flag  # the hybrid sort did run
        lk, lr = layout_arrays(idx, n, np.uint64)
        assert np.array_equal(lk, ok) and np.array_equal(lr, orr), flag
        gi.gi_destroy(idx)


def test_default_build_skips_the_speculative_pass_when_the_top_byte_is_trivial():
    # 2^24 u64 keys below 2^32: the build queues its MSD pass on the window below the
    # highest differing bit before the host sees any counts; the keys differ in only
    # four bytes, where the LSD sort is used, so the window counting marks the window
    # trivial and the pass returns at once; the LSD passes sort from the input
    # (the pass finding the differing bits, window counts + scan, the no-op pass,
    # the digit counts + scan, 4 passes, permutation = 11 launches)
    n = 1 << 24
    keys = W.unique_keys(n, 32, 91).astype(np.uint64)
    rows = np.random.default_rng(3).permutation(n).astype(np.uint32)
    rows[5] = gi.GI_MISS  # the LSD's first pass still checks the input rowIDs
    with pytest.raises(gi.GIError):
        build(keys, rows, gi.GI_EYTZINGER_KARY, 5)
    rows[5] = n + 7
    ok, orr = _oracle_layout(keys, rows, gi.GI_EYTZINGER_KARY, 5)
    c0 = gi.gi_launch_count()
    idx = build(keys, rows, gi.GI_EYTZINGER_KARY, 5)
    assert gi.gi_launch_count() - c0 == 11
    lk, lr = layout_arrays(idx, n, np.uint64)
    assert np.array_equal(lk, ok) and np.array_equal(lr, orr)
    gi.gi_destroy(idx)
