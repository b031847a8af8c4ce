"""Out-of-memory handling, made on the host: gi_debug_fail_alloc makes one of the
library's device allocations report out-of-memory without allocating (no GPU is
driven out of memory).  Every call that meets it must return GI_ERR_NOMEM, free
what it had taken, and leave the library usable: the next call gives the
oracle's answer.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2506_01576_gb300 as gi
import workloads as W

pytestmark = pytest.mark.gpu

from gpu_util import DEV, point, to_dev  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2506_01576_gb300 import _build
    _build.build()
    gi.load()
    torch.cuda.set_device(DEV)
    yield
    gi.gi_debug_fail_alloc(-1)


def _attempt(fn, after):
    gi.gi_debug_fail_alloc(after)
    try:
        return fn(), None
    except gi.GIError as e:
        return None, e
    finally:
        gi.gi_debug_fail_alloc(-1)


@pytest.mark.parametrize("n,flags", [(300001, 0), ((1 << 24) + 5, 0), (5000, gi.GI_BUILD_LSD), (0, 0)])
def test_every_build_allocation_can_fail_cleanly(n, flags):
    keys = W.unique_keys(n, 64, 81)
    rows = np.arange(n, dtype=np.uint32)
    kd = to_dev(keys) if n else torch.empty(0, dtype=torch.int64, device=DEV)
    rd = to_dev(rows) if n else torch.empty(0, dtype=torch.int32, device=DEV)
    q = W.point_probes(keys, 50000, 0.5, 64, 81, 82) if n else np.arange(100, dtype=np.uint64)
    sk, sr = oracle.sort_pairs(keys, rows)
    want = oracle.point_lookup(sk, sr, q)
    failures = 0
    for after in range(0, 32):
        idx, err = _attempt(lambda: gi.gi_build(kd, rd, gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64 | flags, 5), after)
        if err is not None:
            assert err.code == gi.GI_ERR_NOMEM, (after, str(err))
            failures += 1
            continue
        # the hook lay beyond the build's allocations: a complete, correct index
        assert np.array_equal(point(idx, q), want)
        gi.gi_destroy(idx)
        break
    else:
        pytest.fail("the build never completed")
    assert failures >= 2  # the status word and the index arrays at least
    idx = gi.gi_build(kd, rd, gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64 | flags, 5)
    assert np.array_equal(point(idx, q), want)
    gi.gi_destroy(idx)


def test_staging_and_range_scratch_failures_leave_the_index_usable():
    n = 200003
    keys = W.unique_keys(n, 64, 83)
    rows = np.arange(n, dtype=np.uint32)
    sk, sr = oracle.sort_pairs(keys, rows)
    idx = gi.gi_build(to_dev(keys), to_dev(rows), gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64, 9)
    # host probes go through staging buffers allocated on first use
    q = W.point_probes(keys, (1 << 22) + 999, 0.5, 64, 83, 84)
    want = oracle.point_lookup(sk, sr, q)
    out = np.empty(len(q), dtype=np.uint32)
    for after in range(0, 6):
        _, err = _attempt(lambda: gi.gi_point_lookup(idx, q, out), after)
        if err is not None:
            assert err.code == gi.GI_ERR_NOMEM, str(err)
    out[:] = 0
    gi.gi_point_lookup(idx, q, out)
    assert np.array_equal(out, want)
    # device ranges: the scratch of the count pass
    lo, hi, _ = W.ranges_with_expected_rows(n, 100000, 4.0, 64, 85)
    lod, hid = to_dev(lo), to_dev(hi)
    off = torch.empty(len(lo) + 1, dtype=torch.int64, device=DEV)
    _, err = _attempt(lambda: gi.gi_range_lookup(idx, lod, hid, off), 0)
    assert err is not None and err.code == gi.GI_ERR_NOMEM
    gi.gi_range_lookup(idx, lod, hid, off)
    total = int(off[-1].item())
    rws = torch.empty(max(total, 1), dtype=torch.int32, device=DEV)
    gi.gi_range_lookup(idx, lod, hid, off, rws)
    wo, wr = oracle.range_lookup(sk, sr, lo, hi)
    assert np.array_equal(off.cpu().numpy().view(np.uint64), wo)
    assert np.array_equal(rws[:total].cpu().numpy().view(np.uint32), wr)
    gi.gi_sync(idx)
    gi.gi_destroy(idx)
