"""CPU oracle for the static index -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  The product path (the CUDA library and
its binding) never does, and this package never imports the product.

Everything here is a plain restatement of the paper's definitions:

* ``sort_pairs``      -- key-value sort by (key, input position) (Section 3).
* ``point_lookup``    -- lower_bound on the sorted array; rowID on a match,
                         ``MISS`` otherwise (Sections 1, 3).
* ``range_lookup``    -- lower_bound(L) then a forward scan while key <= U,
                         as CSR (offsets, rowIDs) in ascending key order
                         (Section 1, inclusive bounds).
* ``layout_slot_rank``-- the Eytzinger (k = 2) and k-ary Eytzinger order as the
                         in-order fill of the complete k-ary tree stored level
                         by level (Sections 3, 4, 6; Figs 5, 10).
* ``layout_arrays``   -- the index's arrays for a layout, built from the above.

The compute lives in ``oracle.cpp`` (std::sort, std::lower_bound, a linear
scan, a recursive fill); this file only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

MISS = 0xFFFFFFFF

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
# GI_ORACLE_LIB names another build of oracle.cpp to load instead; the mutation
# tests load copies with a planted mistake this way, to show that the pins fail
_OVERRIDE = os.environ.get("GI_ORACLE_LIB")
_LIB = _OVERRIDE or os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (g++, host only)."""
    if _OVERRIDE:
        return _LIB
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC,
                               "-o", tmp, "-pthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P, U64, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
        lib.or_sort_pairs.argtypes = [P, P, U64, I, P, P]
        lib.or_point_lookup.argtypes = [P, P, U64, I, P, U64, P, I]
        lib.or_range_offsets.argtypes = [P, U64, I, P, P, U64, P, I]
        lib.or_range_fill.argtypes = [P, P, U64, I, P, P, U64, P, P, I]
        lib.or_layout_slot_rank.argtypes = [U64, ctypes.c_uint32, P]
        lib.or_hardware_threads.argtypes = []
        for f in (lib.or_sort_pairs, lib.or_point_lookup, lib.or_range_offsets,
                  lib.or_range_fill, lib.or_layout_slot_rank, lib.or_hardware_threads):
            f.restype = I
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _kb(a: np.ndarray) -> int:
    if a.dtype == np.uint32:
        return 4
    if a.dtype == np.uint64:
        return 8
    raise TypeError("keys must be uint32 or uint64, got %s" % a.dtype)


def hardware_threads() -> int:
    return int(_load().or_hardware_threads())


def sort_pairs(keys: np.ndarray, rowids: np.ndarray):
    """(sorted keys, rowIDs in the same order); equal keys keep input order."""
    keys = np.ascontiguousarray(keys)
    rowids = np.ascontiguousarray(rowids, dtype=np.uint32)
    n = len(keys)
    assert len(rowids) == n
    sk = np.empty_like(keys)
    sr = np.empty(n, dtype=np.uint32)
    rc = _load().or_sort_pairs(_ptr(keys), _ptr(rowids), n, _kb(keys), _ptr(sk), _ptr(sr))
    assert rc == 0
    return sk, sr


def point_lookup(skeys: np.ndarray, srows: np.ndarray, queries: np.ndarray,
                 threads: int = 1) -> np.ndarray:
    """rowID of the first entry (in sorted order) whose key equals each probe, else MISS."""
    queries = np.ascontiguousarray(queries, dtype=skeys.dtype)
    out = np.empty(len(queries), dtype=np.uint32)
    rc = _load().or_point_lookup(_ptr(skeys), _ptr(srows), len(skeys), _kb(skeys),
                                 _ptr(queries), len(queries), _ptr(out), threads)
    assert rc == 0
    return out


def range_lookup(skeys: np.ndarray, srows: np.ndarray, lo: np.ndarray, hi: np.ndarray,
                 threads: int = 1):
    """CSR result of inclusive ranges [lo_i, hi_i]: (offsets[m+1] u64, rowIDs u32)."""
    lo = np.ascontiguousarray(lo, dtype=skeys.dtype)
    hi = np.ascontiguousarray(hi, dtype=skeys.dtype)
    m = len(lo)
    assert len(hi) == m
    off = np.empty(m + 1, dtype=np.uint64)
    lib = _load()
    rc = lib.or_range_offsets(_ptr(skeys), len(skeys), _kb(skeys), _ptr(lo), _ptr(hi), m,
                              _ptr(off), threads)
    assert rc == 0
    rows = np.empty(int(off[m]), dtype=np.uint32)
    rc = lib.or_range_fill(_ptr(skeys), _ptr(srows), len(skeys), _kb(skeys), _ptr(lo),
                           _ptr(hi), m, _ptr(off), _ptr(rows), threads)
    assert rc == 0
    return off, rows


def layout_slot_rank(n: int, k: int) -> np.ndarray:
    """slot_rank[s] = sorted rank held by slot s of the k-ary Eytzinger array (k=2: EBS)."""
    out = np.empty(n, dtype=np.uint64)
    rc = _load().or_layout_slot_rank(n, k, _ptr(out))
    assert rc == 0, "in-order fill did not hand out exactly n ranks"
    return out


SORTED, EYTZINGER, EYTZINGER_KARY = 0, 1, 2


def layout_arrays(keys: np.ndarray, rowids: np.ndarray, layout: int, k: int = 2):
    """(keys, rowIDs) of the index in the given layout, slot 0 first.

    For EYTZINGER the arrays are the 0-based slots t = 0..n-1 (the paper stores
    slot t at 1-based position t+1 behind an empty slot 0).
    """
    sk, sr = sort_pairs(keys, rowids)
    if layout == SORTED:
        return sk, sr
    kk = 2 if layout == EYTZINGER else k
    r = layout_slot_rank(len(sk), kk).astype(np.int64)
    return sk[r], sr[r]
