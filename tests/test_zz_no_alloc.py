"""The allocation-free range lookup matches the regular one.

gi_range_lookup_noalloc serves callers that may not allocate device memory
themselves or through this library -- a query engine whose pool allocator owns
the whole GPU, or a caller that cannot let an allocation call block or
synchronise the device mid-query.  Its scratch lives in a fixed array inside the
library, so its results must equal gi_range_lookup's exactly (integer CSR
output: offsets and rowIDs, bit for bit), on every call, including two calls in
a row that reuse the same array.  This file is collected last on purpose.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import torch

import oracle
import paper_2506_01576_gb300 as gi
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

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
    rows = torch.full((max(capacity, 1),), -7, dtype=torch.int32, device=DEV)
    torch.cuda.synchronize()
    # any allocation the library made from here on would fail (a host-side test
    # hook: nothing is allocated and no GPU fault is involved); the calls succeed
    gi.gi_debug_fail_alloc(0)
    try:
        gi.gi_range_lookup_noalloc(idx, lo, hi, off)  # offsets only
        total = int(off[-1].item())
        assert total <= capacity
        gi.gi_range_lookup_noalloc(idx, lo, hi, off, rows)
        torch.cuda.synchronize()
    finally:
        gi.gi_debug_fail_alloc(-1)
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


def test_regular_call_after_noalloc_recounts():
    """Regular offsets-only call, then a noalloc call with other bounds into the
    same offsets array, then the regular call with rows and the first bounds: the
    last call must count again (the offsets were overwritten), not reuse the
    first call's counts.  Checked against the oracle."""
    n = 50_000
    keys = W.unique_keys(n, 64, 5)
    rows = np.arange(n, dtype=np.uint32)
    idx = gi.gi_build(_dev(keys), _dev(rows), gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64, 5)
    m = 4096
    lo1, hi1, _ = W.ranges_with_expected_rows(n, m, 3.0, 64, 11)
    lo2, hi2, _ = W.ranges_with_expected_rows(n, m, 30.0, 64, 12)
    sk, sr = oracle.sort_pairs(keys, rows)
    want_off, want_rows = oracle.range_lookup(sk, sr, lo1, hi1)
    t1, u1, t2, u2 = _dev(lo1), _dev(hi1), _dev(lo2), _dev(hi2)
    off = torch.empty(m + 1, dtype=torch.int64, device=DEV)
    gi.gi_range_lookup(idx, t1, u1, off)  # first call of the two-call protocol
    total1 = int(off[-1].item())
    assert total1 == int(want_off[-1])
    gi.gi_range_lookup_noalloc(idx, t2, u2, off)  # overwrites off with other counts
    torch.cuda.synchronize()
    out = torch.full((max(total1, 1),), -7, dtype=torch.int32, device=DEV)
    gi.gi_range_lookup(idx, t1, u1, off, out)  # same pointers as the first call
    torch.cuda.synchronize()
    assert np.array_equal(off.cpu().numpy().view(np.uint64), want_off)
    assert np.array_equal(out.cpu().numpy().view(np.uint32)[:total1], want_rows)
    gi.gi_destroy(idx)


def test_first_call_during_capture_is_refused():
    """In a fresh process the first call looks up the scratch array's address;
    during a stream capture that is refused with a clear error, and the same call
    made outside the capture then works."""
    code = textwrap.dedent("""
        import sys
        sys.path.insert(0, %r)
        import numpy as np, torch
        import paper_2506_01576_gb300 as gi, workloads as W
        gi.load()
        dev = torch.device("cuda:0")
        torch.cuda.set_device(dev)
        keys = W.unique_keys(1000, 64, 3)
        t = lambda a: torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a.view(np.int32)).to(dev)
        idx = gi.gi_build(t(keys), t(np.arange(1000, dtype=np.uint32)), gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64, 5)
        lo = t(np.sort(keys)[:16].copy())
        off = torch.empty(17, dtype=torch.int64, device=dev)
        s = torch.cuda.Stream()
        gi.gi_set_stream(idx, s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        err = None
        with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
            try:
                gi.gi_range_lookup_noalloc(idx, lo, lo, off)
            except gi.GIError as e:
                err = e
        assert err is not None and err.code == gi.GI_ERR_INVALID and "capture" in str(err), err
        gi.gi_range_lookup_noalloc(idx, lo, lo, off)
        torch.cuda.synchronize()
        assert int(off[-1].item()) == 16
        gi.gi_destroy(idx)
        print("capture refusal ok")
    """) % ROOT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "capture refusal ok" in r.stdout, r.stdout + r.stderr
