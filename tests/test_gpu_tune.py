"""The autotuner (gi_tune, gi_batch_tune) against the CPU oracle.

The knobs it sweeps change the schedule of a lookup, never its result, so after
tuning every lookup must still equal the oracle's (integers: exact).  Also: the
chosen values are the ones the index then reports, a report-only call leaves the
index as it was, and the table hands a recorded size class's values to other
indexes of that class and to no other.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2506_01576_gb300 as gi
import workloads as W

pytestmark = pytest.mark.gpu

from gpu_util import DEV, build, point, to_dev  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2506_01576_gb300 import _build
    _build.build()
    gi.load()
    torch.cuda.set_device(DEV)
    gi.gi_tune_table_clear()
    yield
    gi.gi_tune_table_clear()


def _options(idx):
    return [gi.gi_get_option(idx, o) for o in range(1, 11)]


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("layout,k", [(gi.GI_SORTED, 0), (gi.GI_EYTZINGER, 2), (gi.GI_EYTZINGER_KARY, 5),
                                      (gi.GI_EYTZINGER_KARY, 9), (gi.GI_EYTZINGER_KARY, 17),
                                      (gi.GI_EYTZINGER_KARY, 7)])
def test_tuned_lookups_equal_the_oracle(dtype, layout, k):
    bits = 8 * np.dtype(dtype).itemsize
    n = 300007
    keys = W.unique_keys(n, bits, 31)
    rows = np.random.default_rng(31).permutation(n).astype(np.uint32)
    q = W.point_probes(keys, 200003, 0.5, bits, 31, 32)
    sk, sr = oracle.sort_pairs(keys, rows)
    want = oracle.point_lookup(sk, sr, q)
    idx = build(keys, rows, layout, k)
    before = _options(idx)
    # report only: the index keeps its settings
    r = gi.gi_tune(idx, to_dev(q), 2, 0)
    assert _options(idx) == before
    assert r.trials >= 2 and r.passes >= 1
    assert r.best_ms <= r.start_ms
    assert [r.start_options[o] for o in range(1, 11) if o != gi.GI_OPT_RANGE_FILL] == \
        [before[o - 1] for o in range(1, 11) if o != gi.GI_OPT_RANGE_FILL]
    # applied: the index reports the chosen values and still answers exactly
    r = gi.gi_tune(idx, to_dev(q), 2, gi.GI_TUNE_APPLY)
    got = _options(idx)
    for o in range(1, 11):
        if o != gi.GI_OPT_RANGE_FILL:
            assert got[o - 1] == r.options[o], o
    assert np.array_equal(point(idx, q), want)
    gi.gi_sync(idx)
    gi.gi_destroy(idx)


def test_table_hands_a_size_class_its_values():
    gi.gi_tune_table_clear()
    lay = gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64
    keys = W.unique_keys(1 << 18, 64, 41)  # size class 18: n in [2^18, 2^19)
    rows = np.arange(len(keys), dtype=np.uint32)
    q = W.point_probes(keys, 1 << 18, 0.5, 64, 41, 42)
    idx = build(keys, rows, gi.GI_EYTZINGER_KARY, 5)
    defaults = _options(idx)
    r = gi.gi_tune(idx, to_dev(q), 2, gi.GI_TUNE_RECORD)  # recorded, not applied
    rec = gi.gi_tune_table_get(lay, 5, (1 << 18) + 12345)
    assert rec is not None
    assert [rec[o] for o in range(1, 11) if o != gi.GI_OPT_RANGE_FILL] == \
        [r.options[o] for o in range(1, 11) if o != gi.GI_OPT_RANGE_FILL]
    assert gi.gi_tune_table_get(lay, 5, 1 << 19) is None      # another class
    assert gi.gi_tune_table_get(lay, 9, 1 << 18) is None      # another k
    assert gi.gi_tune_table_get(gi.GI_EYTZINGER_KARY | gi.GI_KEY_U32, 5, 1 << 18) is None
    # the recorded index and a new one of the same class take every automatic knob
    # from the table; an explicit setting wins over it
    n2 = (1 << 18) + 77777
    keys2 = W.unique_keys(n2, 64, 43)
    rows2 = np.arange(n2, dtype=np.uint32)
    idx2 = build(keys2, rows2, gi.GI_EYTZINGER_KARY, 5)
    for x in (idx, idx2):
        got = _options(x)
        for o in range(1, 11):
            if o not in (gi.GI_OPT_RANGE_FILL, gi.GI_OPT_SMEM_LEVELS):
                assert got[o - 1] == rec[o], (o, got, rec)
    gi.gi_set_option(idx2, gi.GI_OPT_BLOCK, 64 if rec[gi.GI_OPT_BLOCK] != 64 else 128)
    assert gi.gi_get_option(idx2, gi.GI_OPT_BLOCK) != rec[gi.GI_OPT_BLOCK]
    q2 = W.point_probes(keys2, 100000, 0.5, 64, 43, 44)
    sk, sr = oracle.sort_pairs(keys2, rows2)
    assert np.array_equal(point(idx2, q2), oracle.point_lookup(sk, sr, q2))
    # another class keeps the defaults
    keys3 = W.unique_keys(1 << 17, 64, 45)
    idx3 = build(keys3, np.arange(1 << 17, dtype=np.uint32), gi.GI_EYTZINGER_KARY, 5)
    assert gi.gi_get_option(idx3, gi.GI_OPT_GROUP) == defaults[gi.GI_OPT_GROUP - 1]
    gi.gi_tune_table_clear()
    assert _options(idx) == defaults
    for x in (idx, idx2, idx3):
        gi.gi_destroy(x)


def test_tune_rejects_host_probes_and_empty_input():
    keys = W.unique_keys(5000, 64, 51)
    idx = build(keys, np.arange(5000, dtype=np.uint32), gi.GI_EYTZINGER_KARY, 5)
    before = _options(idx)
    with pytest.raises(gi.GIError) as e:
        gi.gi_tune(idx, keys[:100].copy(), 1, gi.GI_TUNE_APPLY)
    assert e.value.code == gi.GI_ERR_INVALID
    with pytest.raises(gi.GIError) as e:
        gi.gi_tune(idx, torch.empty(0, dtype=torch.int64, device=DEV), 1, gi.GI_TUNE_APPLY)
    assert e.value.code == gi.GI_ERR_INVALID
    assert _options(idx) == before
    gi.gi_destroy(idx)


def test_batch_tune_keeps_results():
    rng = np.random.default_rng(61)
    sizes = list(rng.integers(0, 30000, size=40)) + [70000, 1, 0]
    keys = [W.unique_keys(int(n), 64, 600 + i) for i, n in enumerate(sizes)]
    rows = [np.arange(len(x), dtype=np.uint32) for x in keys]
    off = np.zeros(len(sizes) + 1, dtype=np.uint64)
    np.cumsum(np.array(sizes, dtype=np.uint64), out=off[1:])
    qs = [W.point_probes(x, 2000, 0.75, 64, 700 + i, 800 + i) if len(x) else
          np.arange(2000, dtype=np.uint64) for i, x in enumerate(keys)]
    qoff = np.zeros(len(sizes) + 1, dtype=np.uint64)
    np.cumsum(np.array([len(x) for x in qs], dtype=np.uint64), out=qoff[1:])
    batch = gi.gi_batch_create(off, gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64, 5)
    gi.gi_batch_build(batch, to_dev(np.concatenate(keys)), to_dev(np.concatenate(rows)))
    qd, qod = to_dev(np.concatenate(qs)), to_dev(qoff)
    r = gi.gi_batch_tune(batch, qd, qod, 2)
    assert r.trials >= 2 and r.best_ms <= r.start_ms
    assert r.start_options[gi.GI_BATCH_OPT_CHUNK] == 2048
    out = torch.full((int(qoff[-1]),), -5, dtype=torch.int32, device=DEV)
    gi.gi_batch_point_lookup(batch, qd, qod, out)
    gi.gi_batch_sync(batch)
    got = out.cpu().numpy().view(np.uint32)
    for i in range(len(sizes)):
        sk, sr = oracle.sort_pairs(keys[i], rows[i])
        assert np.array_equal(got[int(qoff[i]):int(qoff[i + 1])], oracle.point_lookup(sk, sr, qs[i])), i
    gi.gi_batch_destroy(batch)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_build_tuned_picks_a_layout_and_answers_exactly(dtype):
    gi.gi_tune_table_clear()
    bits = 8 * np.dtype(dtype).itemsize
    n = (1 << 16) + 123
    keys = W.unique_keys(n, bits, 71)
    rows = np.random.default_rng(71).permutation(n).astype(np.uint32)
    q = W.point_probes(keys, 1 << 17, 0.5, bits, 71, 72)
    kf = gi.GI_KEY_U64 if bits == 64 else gi.GI_KEY_U32
    idx, r = gi.gi_build_tuned(to_dev(keys), to_dev(rows), kf, to_dev(q), 2,
                               gi.GI_TUNE_APPLY | gi.GI_TUNE_RECORD)
    info = gi.gi_get_info(idx)
    assert (info.layout, info.k) in {(gi.GI_SORTED, 0), (gi.GI_EYTZINGER, 2), (gi.GI_EYTZINGER_KARY, 3),
                                     (gi.GI_EYTZINGER_KARY, 5), (gi.GI_EYTZINGER_KARY, 9),
                                     (gi.GI_EYTZINGER_KARY, 17)}
    assert info.n == n and info.key_bytes == bits // 8
    for o in range(1, 11):
        if o != gi.GI_OPT_RANGE_FILL:
            assert gi.gi_get_option(idx, o) == r.options[o], o
    sk, sr = oracle.sort_pairs(keys, rows)
    assert np.array_equal(point(idx, q), oracle.point_lookup(sk, sr, q))
    # the layout, k and knobs of the size class are recorded
    assert gi.gi_tune_table_layout(kf, n) == (info.layout, info.k if info.layout == gi.GI_EYTZINGER_KARY else 0)
    assert gi.gi_tune_table_layout(kf, n * 4) is None
    assert gi.gi_tune_table_get(kf | info.layout, info.k, n) is not None
    gi.gi_destroy(idx)
    gi.gi_tune_table_clear()
    assert gi.gi_tune_table_layout(kf, n) is None
