"""Serving form: continuous batching over resident indexes.

Each request's answer must equal the oracle's for its index, and a request must
get the same bits when served alone and when it arrives among hundreds of
others from several client threads (integer outputs: the stated tolerance is
zero).  Admission by arena memory is exercised with an arena far smaller than
the offered work, and a request larger than the whole arena is refused.
"""
import threading

import numpy as np
import pytest
import torch

import oracle
import paper_2506_01576_gb300 as gi
import workloads as W

pytestmark = pytest.mark.gpu

from gpu_util import DEV, to_dev  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2506_01576_gb300 import _build
    _build.build()
    gi.load()
    torch.cuda.set_device(DEV)


def _resident(sizes, layout, k, bits=64):
    idx, ref = [], []
    for i, n in enumerate(sizes):
        keys = W.unique_keys(n, bits, W.seed_for(4, 0, i))
        rows = np.random.default_rng(i).permutation(n).astype(np.uint32)
        flag = gi.GI_KEY_U64 if bits == 64 else gi.GI_KEY_U32
        idx.append(gi.gi_build(to_dev(keys), to_dev(rows), layout | flag, k))
        ref.append((keys,) + oracle.sort_pairs(keys, rows))
    return idx, ref


def _make_request(ref, rng, i, bits=64):
    keys, sk, sr = ref[i]
    m = int(np.exp2(rng.uniform(0, 12)))
    dt = np.uint64 if bits == 64 else np.uint32
    if rng.random() < 0.8:
        q = W.point_probes(keys, m, 0.5, bits, W.seed_for(4, 0, i), int(rng.integers(1 << 30)))
        return ("point", i, q.astype(dt))
    n = len(keys)
    lo, hi, _ = W.ranges_with_expected_rows(n, m, 16, bits, int(rng.integers(1 << 30)))
    return ("range", i, lo.astype(dt), hi.astype(dt))


class _Pending:
    def __init__(self, server, req, pinned=False):
        self.req = req
        alloc = (lambda a: torch.from_numpy(a).pin_memory().numpy()) if pinned else (lambda a: a)
        if req[0] == "point":
            self.q = alloc(req[2].copy())
            self.out = alloc(np.full(len(self.q), 7, dtype=np.uint32))
            self.ticket = gi.gi_server_submit(server, req[1], gi.GI_REQ_POINT, self.q, out_rowids=self.out)
        else:
            self.lo, self.hi = alloc(req[2].copy()), alloc(req[3].copy())
            self.off = alloc(np.zeros(len(self.lo) + 1, dtype=np.uint64))
            self.cap = 64 * len(self.lo) + 64
            self.rows = alloc(np.zeros(self.cap, dtype=np.uint32))
            self.ticket = gi.gi_server_submit(server, req[1], gi.GI_REQ_RANGE, self.lo, out_rowids=self.rows,
                                              hi=self.hi, out_offsets=self.off, rows_capacity=self.cap)

    def result(self, server):
        st, t0, t1 = gi.gi_server_wait(server, self.ticket)
        assert st == gi.GI_OK and t1 >= t0 > 0
        if self.req[0] == "point":
            return (self.out.copy(),)
        return (self.off.copy(), self.rows[: int(self.off[-1])].copy())


def _want(ref, req):
    keys, sk, sr = ref[req[1]]
    if req[0] == "point":
        return (oracle.point_lookup(sk, sr, req[2]),)
    return oracle.range_lookup(sk, sr, req[2], req[3])


@pytest.mark.parametrize("layout,k", [(gi.GI_EYTZINGER_KARY, 5), (gi.GI_SORTED, 0), (gi.GI_EYTZINGER_KARY, 9)])
def test_each_result_same_alone_and_in_the_mix(layout, k):
    idx, ref = _resident([1 << 12, 5000, 1 << 15, 70001, 1 << 18, 3, 1, 200000], layout, k)
    server = gi.gi_server_create(idx, 64 << 20, 3)
    rng = np.random.default_rng(k + 1)
    probes = [_make_request(ref, rng, int(rng.integers(0, len(idx)))) for _ in range(6)]
    alone = []
    for req in probes:  # alone: nothing else in flight
        p = _Pending(server, req)
        alone.append(p.result(server))
    for req, a in zip(probes, alone):
        for x, y in zip(a, _want(ref, req)):
            assert np.array_equal(x, y)
    # in the mix: four client threads submit 600 requests, the probes among them
    mix = [_make_request(ref, rng, int(rng.integers(0, len(idx)))) for _ in range(600)]
    for j, req in enumerate(probes):
        mix.insert(50 + 97 * j, req)
    results = [None] * len(mix)
    errors = []

    def client(part):
        try:
            pend = [(j, _Pending(server, mix[j], pinned=(j % 2 == 0))) for j in part]
            for j, p in pend:
                results[j] = p.result(server)
        except Exception as e:  # pragma: no cover - reported below
            errors.append(e)

    ts = [threading.Thread(target=client, args=(list(range(c, len(mix), 4)),)) for c in range(4)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors
    for req, res in zip(mix, results):
        for x, y in zip(res, _want(ref, req)):
            assert np.array_equal(x, y)
    for j, req in enumerate(probes):
        res = results[50 + 97 * j]  # where probe j was inserted
        for x, y in zip(res, alone[j]):
            assert np.array_equal(x, y), "a request changed when served in the mix"
    batches, requests, admitted = gi.gi_server_stats(server)
    assert requests == len(mix) + len(probes) and batches >= 2
    gi.gi_server_destroy(server)
    for ix in idx:
        gi.gi_destroy(ix)


def test_pinned_and_pageable_buffers_mixed():
    """Page-locked host buffers are copied by the copy engine one by one, pageable
    ones gathered into the batch's staging copy: requests that mix the two (pinned
    probes with pageable results and the reverse, one pinned bound with one
    pageable, pinned probes at an address that is not 8-byte aligned, a small
    pinned request, which is staged anyway) all answer as the oracle does."""
    idx, ref = _resident([1 << 12, 70001], gi.GI_EYTZINGER_KARY, 5)
    server = gi.gi_server_create(idx, 64 << 20, 3)
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    rng = np.random.default_rng(77)
    pend = []
    for case in range(8):
        i = case % 2
        keys, sk, sr = ref[i]
        m = 2100 + 37 * case if case < 7 else 700  # above / below the size staged anyway
        q = W.point_probes(keys, m, 0.5, 64, W.seed_for(4, 1, case), 11 + case)
        if case in (0, 1, 2):
            qin = pin(q.copy()) if case != 1 else q.copy()
            out = np.full(m, 7, np.uint32) if case != 1 else pin(np.full(m, 7, np.uint32))
            if case == 2:  # pinned probes 4 bytes past an 8-byte boundary
                raw = pin(np.zeros(8 * m + 8, np.uint8))
                qin = np.ndarray((m,), dtype=np.uint64, buffer=raw, offset=4)
                qin[:] = q
                out = pin(np.full(m, 7, np.uint32))
            t = gi.gi_server_submit(server, i, gi.GI_REQ_POINT, qin, out_rowids=out)
            pend.append(("point", t, out, (oracle.point_lookup(sk, sr, q),), qin))
        else:
            lo, hi, _ = W.ranges_with_expected_rows(len(keys), m, 16, 64, int(rng.integers(1 << 30)))
            lo, hi = lo.astype(np.uint64), hi.astype(np.uint64)
            a = pin(lo.copy()) if case % 2 else lo.copy()
            b = hi.copy() if case == 3 else pin(hi.copy())  # cases 5, 7: both pinned
            cap = 64 * m + 64
            off = pin(np.zeros(m + 1, np.uint64)) if case > 5 else np.zeros(m + 1, np.uint64)
            rows = np.zeros(cap, np.uint32)
            t = gi.gi_server_submit(server, i, gi.GI_REQ_RANGE, a, out_rowids=rows, hi=b, out_offsets=off,
                                    rows_capacity=cap)
            pend.append(("range", t, (off, rows), oracle.range_lookup(sk, sr, lo, hi), (a, b)))
    for kind, t, got, want, _keep in pend:
        st, t0, t1 = gi.gi_server_wait(server, t)
        assert st == gi.GI_OK
        if kind == "point":
            assert np.array_equal(got, want[0])
        else:
            off, rows = got
            assert np.array_equal(off, want[0])
            assert np.array_equal(rows[: int(off[-1])], want[1])
    gi.gi_server_destroy(server)
    for ix in idx:
        gi.gi_destroy(ix)


def test_admission_waits_for_arena_memory():
    # a 1 MiB arena: most requests have to wait for earlier ones to free memory
    idx, ref = _resident([1 << 16, 1 << 14], gi.GI_EYTZINGER_KARY, 5)
    server = gi.gi_server_create(idx, 1 << 20, 2)
    rng = np.random.default_rng(2)
    reqs = [_make_request(ref, rng, i % 2) for i in range(200)]
    pend = [_Pending(server, r) for r in reqs]
    for p in pend:
        for x, y in zip(p.result(server), _want(ref, p.req)):
            assert np.array_equal(x, y)
    # bigger than the whole arena: refused at submit
    big = np.zeros(1 << 18, dtype=np.uint64)
    with pytest.raises(gi.GIError) as e:
        gi.gi_server_submit(server, 0, gi.GI_REQ_POINT, big, out_rowids=np.zeros(1 << 18, np.uint32))
    assert e.value.code == gi.GI_ERR_NOMEM
    gi.gi_server_destroy(server)
    for ix in idx:
        gi.gi_destroy(ix)


def test_range_larger_than_its_buffer_reports_capacity():
    idx, ref = _resident([1 << 16], gi.GI_EYTZINGER_KARY, 5)
    server = gi.gi_server_create(idx, 16 << 20, 2)
    keys, sk, sr = ref[0]
    lo = np.array([0, 0], dtype=np.uint64)
    hi = np.array([2 ** 63, 2 ** 62], dtype=np.uint64)
    off = np.zeros(3, dtype=np.uint64)
    rows = np.zeros(10, dtype=np.uint32)
    t = gi.gi_server_submit(server, 0, gi.GI_REQ_RANGE, lo, out_rowids=rows, hi=hi, out_offsets=off,
                            rows_capacity=10)
    st, _, _ = gi.gi_server_wait(server, t)
    assert st == gi.GI_ERR_CAPACITY
    woff, _ = oracle.range_lookup(sk, sr, lo, hi)
    assert np.array_equal(off, woff)
    gi.gi_server_destroy(server)
    gi.gi_destroy(idx[0])


@pytest.mark.parametrize("threads", [1, 4])
def test_native_replay_results_match_oracle(threads):
    """The native load generators (gi_server_replay, gi_replay_serial) submit the
    same trace; every request has its own host buffers, and every answer equals the
    oracle's, from the server and from the one-at-a-time baseline alike."""
    idx, ref = _resident([1 << 14, 70001, 1 << 17], gi.GI_EYTZINGER_KARY, 5)
    rng = np.random.default_rng(40 + threads)
    trace = [_make_request(ref, rng, int(rng.integers(0, len(idx)))) for _ in range(300)]

    def buffers():
        out = []
        for req in trace:
            if req[0] == "point":
                out.append((req[1], gi.GI_REQ_POINT, req[2].copy(), np.full(len(req[2]), 7, np.uint32),
                            None, None, 0))
            else:
                cap = 64 * len(req[2]) + 64
                out.append((req[1], gi.GI_REQ_RANGE, req[2].copy(), np.zeros(cap, np.uint32), req[3].copy(),
                            np.zeros(len(req[2]) + 1, np.uint64), cap))
        return out

    arrival = np.sort(rng.integers(0, 20_000_000, size=len(trace))).astype(np.int64)  # within 20 ms
    server = gi.gi_server_create(idx, 64 << 20, 3)
    for replay in ("server", "serial"):
        bufs = buffers()
        if replay == "server":
            lat, st, wall = gi.gi_server_replay(server, bufs, arrival, threads)
        else:
            lat, st, wall = gi.gi_replay_serial(idx, bufs, arrival)
        assert (st == gi.GI_OK).all() and (lat >= 0).all() and wall > 0
        for req, b in zip(trace, bufs):
            want = _want(ref, req)
            if req[0] == "point":
                assert np.array_equal(b[3], want[0])
            else:
                off = b[5]
                assert np.array_equal(off, want[0])
                assert np.array_equal(b[3][: int(off[-1])], want[1])
    gi.gi_server_destroy(server)
    for ix in idx:
        gi.gi_destroy(ix)
