"""The allocation-free range lookup matches the regular one.

gi_range_lookup_noalloc serves callers that may not allocate device memory
themselves or through this library -- a query engine whose pool allocator owns
the whole GPU, or a caller that cannot let an allocation call block or
synchronise the device mid-query.  Its scratch lives in a fixed array inside the
library, so its results must equal gi_range_lookup's exactly (integer CSR
output: offsets and rowIDs, bit for bit), on every call, including two calls in
a row that reuse the same array.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import paper_2506_01576_gb300 as gi
import workloads as W

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2506_01576_gb300 import _build
    _build.build()
    gi.load()
    torch.cuda.set_device(DEV)


def _dev(a):
    return torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a.view(np.int32)).to(DEV)


def _regular(idx, lo, hi):
    m = lo.numel()
    off = torch.empty(m + 1, dtype=torch.int64, device=DEV)
    gi.gi_range_lookup(idx, lo, hi, off)
    rows = torch.empty(max(int(off[-1].item()), 1), dtype=torch.int32, device=DEV)
    gi.gi_range_lookup(idx, lo, hi, off, rows)
    torch.cuda.synchronize()
    return off.cpu().numpy(), rows.cpu().numpy()[: int(off[-1].item())]


def _noalloc(idx, lo, hi, capacity):
    m = lo.numel()
    off = torch.full((m + 1,), -1, dtype=torch.int64, device=DEV)
    gi.gi_range_lookup_noalloc(idx, lo, hi, off)  # offsets only
    total = int(off[-1].item())
    assert total <= capacity
    rows = torch.full((max(capacity, 1),), -7, dtype=torch.int32, device=DEV)
    gi.gi_range_lookup_noalloc(idx, lo, hi, off, rows)
    torch.cuda.synchronize()
    return off.cpu().numpy(), rows.cpu().numpy()[:total]


@pytest.mark.parametrize("layout,k,bits", [(gi.GI_EYTZINGER_KARY, 5, 64), (gi.GI_EYTZINGER_KARY, 16, 32),
                                           (gi.GI_EYTZINGER, 2, 64), (gi.GI_SORTED, 0, 32)])
def test_noalloc_equals_regular_two_calls_in_a_row(layout, k, bits):
    n = 300_001
    keys = W.unique_keys(n, bits, 21)
    rows = np.arange(n, dtype=np.uint32)
    flag = gi.GI_KEY_U64 if bits == 64 else gi.GI_KEY_U32
    idx = gi.gi_build(_dev(keys), _dev(rows), layout | flag, k)
    for call, (m, E, seed) in enumerate([(gi.GI_NOALLOC_MAX_RANGES, 4.0, 1), (70_001, 40.0, 2)]):
        lo, hi, _ = W.ranges_with_expected_rows(n, m, E, bits, seed)
        lo[:5] = hi[:5] + 1  # a few inverted (empty) ranges
        tlo, thi = _dev(lo), _dev(hi)
        off_r, rows_r = _regular(idx, tlo, thi)
        off_n, rows_n = _noalloc(idx, tlo, thi, len(rows_r))
        assert np.array_equal(off_n, off_r), "offsets differ on call %d" % call
        assert np.array_equal(rows_n, rows_r), "rows differ on call %d" % call
    gi.gi_destroy(idx)


def test_noalloc_rejects_what_it_cannot_do_without_allocating():
    keys = W.unique_keys(1000, 64, 3)
    idx = gi.gi_build(_dev(keys), _dev(np.arange(1000, dtype=np.uint32)),
                      gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64, 9)
    # more ranges than the fixed scratch holds: a clear error, nothing launched
    m = gi.GI_NOALLOC_MAX_RANGES + 1
    big = torch.zeros(m, dtype=torch.int64, device=DEV)
    off = torch.empty(m + 1, dtype=torch.int64, device=DEV)
    with pytest.raises(gi.GIError) as e:
        gi.gi_range_lookup_noalloc(idx, big, big, off)
    assert e.value.code == gi.GI_ERR_INVALID and "maximum" in str(e.value)
    # host buffers would need staging memory: refused
    lo = np.zeros(4, dtype=np.uint64)
    with pytest.raises(gi.GIError) as e:
        gi.gi_range_lookup_noalloc(idx, lo, lo, np.zeros(5, dtype=np.uint64))
    assert e.value.code == gi.GI_ERR_INVALID
    # empty batch
    off0 = torch.full((1,), -1, dtype=torch.int64, device=DEV)
    gi.gi_range_lookup_noalloc(idx, torch.empty(0, dtype=torch.int64, device=DEV),
                               torch.empty(0, dtype=torch.int64, device=DEV), off0)
    torch.cuda.synchronize()
    assert int(off0[0].item()) == 0
    gi.gi_destroy(idx)
