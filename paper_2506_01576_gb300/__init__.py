"""Python binding of libgi (include/gi.h): a static GPU index over (key, rowID)
pairs in sorted, Eytzinger or k-ary Eytzinger order, for GB300 (sm_103a).

The functions keep the C names and only marshal arguments: buffers may be torch
tensors (CUDA or CPU) or numpy arrays; their data pointers go straight to the C
library, which runs every step on the GPU.  There is no CPU fallback: if
libgi.so is missing or fails to load, importing the binding's entry points
raises.

    idx = gi_build(keys, rowids, GI_EYTZINGER_KARY | GI_KEY_U64, 9)
    gi_point_lookup(idx, probes, out)          # out: uint32 rowIDs or GI_MISS
    gi_range_lookup(idx, lo, hi, offsets)       # offsets: m+1 uint64
    gi_range_lookup(idx, lo, hi, offsets, rows) # rows: offsets[m] uint32
    gi_destroy(idx)
"""
from __future__ import annotations

import ctypes
import os

__all__ = [
    "GI_SORTED", "GI_EYTZINGER", "GI_EYTZINGER_KARY", "GI_KEY_U32", "GI_KEY_U64", "GI_MISS",
    "GI_BUILD_LSD", "GI_BUILD_HYBRID",
    "GI_OK", "GI_ERR_INVALID", "GI_ERR_NOMEM", "GI_ERR_CUDA", "GI_ERR_TIMEOUT",
    "GI_OPT_GROUP", "GI_OPT_PER_THREAD", "GI_OPT_SMEM_LEVELS", "GI_OPT_BLOCK",
    "GI_OPT_BLOCKS_PER_SM", "GI_OPT_PREFETCH", "GI_OPT_EARLY_EXIT", "GI_OPT_HOT_LEVELS", "GI_OPT_RANGE_FILL", "GI_OPT_REORDER",
    "GIError", "Index", "gi_info", "lib_path", "load",
    "gi_build", "gi_point_lookup", "gi_range_lookup", "gi_destroy", "gi_set_stream", "gi_sync",
    "gi_last_error", "gi_footprint_bytes", "gi_get_info", "gi_copy_layout", "gi_set_option", "gi_get_option",
    "gi_probe_random_sectors", "gi_coalescing_probe", "gi_launch_count",
    "gi_range_lookup_noalloc", "GI_NOALLOC_MAX_RANGES",
    "Batch", "gi_batch_create", "gi_batch_set_stream", "gi_batch_build", "gi_batch_point_lookup",
    "gi_batch_sync", "gi_batch_copy_index", "gi_batch_set_option", "gi_batch_footprint_bytes",
    "gi_batch_destroy", "gi_batch_set_fanouts", "gi_batch_get_fanouts", "gi_batch_tune_fanouts",
    "gi_batch_fanout_table_clear", "GI_BATCH_OPT_CHUNK", "GI_BATCH_OPT_BLOCKS_PER_SM", "GI_BATCH_OPT_SMEM_BUDGET",
    "Server", "gi_request", "gi_server_create", "gi_server_submit", "gi_server_wait", "gi_server_stats",
    "gi_server_destroy", "GI_REQ_POINT", "GI_REQ_RANGE", "GI_ERR_CAPACITY",
    "make_requests", "gi_server_replay", "gi_replay_serial",
    "gi_tune_result", "gi_tune", "gi_tune_table_get", "gi_tune_table_clear", "gi_batch_tune",
    "GI_TUNE_APPLY", "GI_TUNE_RECORD", "gi_build_tuned", "gi_tune_table_layout", "gi_debug_fail_alloc",
]

GI_SORTED, GI_EYTZINGER, GI_EYTZINGER_KARY = 0, 1, 2
GI_KEY_U32, GI_KEY_U64 = 0x000, 0x100
GI_BUILD_LSD = 0x10000
GI_BUILD_HYBRID = 0x20000
GI_OK, GI_ERR_INVALID, GI_ERR_NOMEM, GI_ERR_CUDA, GI_ERR_TIMEOUT, GI_ERR_CAPACITY = 0, 1, 2, 3, 4, 5
GI_REQ_POINT, GI_REQ_RANGE = 0, 1
GI_MISS = 0xFFFFFFFF
GI_NOALLOC_MAX_RANGES = 1 << 20
GI_BATCH_OPT_CHUNK, GI_BATCH_OPT_BLOCKS_PER_SM, GI_BATCH_OPT_SMEM_BUDGET = 1, 2, 3
GI_TUNE_APPLY, GI_TUNE_RECORD = 1, 2
(GI_OPT_GROUP, GI_OPT_PER_THREAD, GI_OPT_SMEM_LEVELS, GI_OPT_BLOCK, GI_OPT_BLOCKS_PER_SM,
 GI_OPT_PREFETCH, GI_OPT_EARLY_EXIT, GI_OPT_HOT_LEVELS, GI_OPT_RANGE_FILL, GI_OPT_REORDER) = range(1, 11)

_HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(_HERE, "libgi.so")
_lib = None


class GIError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("gi error %d: %s" % (code, msg))
        self.code = code


class gi_request(ctypes.Structure):
    _fields_ = [("index", ctypes.c_uint32), ("kind", ctypes.c_uint32), ("m", ctypes.c_uint64),
                ("keys", ctypes.c_void_p), ("hi", ctypes.c_void_p), ("out_rowids", ctypes.c_void_p),
                ("out_offsets", ctypes.c_void_p), ("rows_capacity", ctypes.c_uint64)]


class gi_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("layout", ctypes.c_int32), ("k", ctypes.c_uint32),
                ("key_bytes", ctypes.c_uint32), ("unique", ctypes.c_uint32),
                ("levels", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("keys", ctypes.c_void_p), ("rowids", ctypes.c_void_p),
                ("footprint_bytes", ctypes.c_uint64)]


class gi_tune_result(ctypes.Structure):
    _fields_ = [("start_options", ctypes.c_int64 * 11), ("options", ctypes.c_int64 * 11),
                ("start_ms", ctypes.c_double), ("best_ms", ctypes.c_double),
                ("trials", ctypes.c_uint32), ("passes", ctypes.c_uint32)]


def load(build_if_missing: bool = False):
    """Load libgi.so (optionally compiling it first).  Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        from . import _build
        _build.build()
    if not os.path.exists(lib_path):
        raise ImportError("libgi.so is not built (%s); run __graft_entry__.build()" % lib_path)
    lib = ctypes.CDLL(lib_path)
    P, U64, U32, I, I64 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_int64
    sig = {
        "gi_build": (I, [P, P, U64, I, U32, ctypes.POINTER(P)]),
        "gi_point_lookup": (I, [P, P, U64, P]),
        "gi_range_lookup": (I, [P, P, P, U64, P, P]),
        "gi_destroy": (None, [P]),
        "gi_set_stream": (I, [P, P]),
        "gi_sync": (I, [P]),
        "gi_last_error": (ctypes.c_char_p, []),
        "gi_footprint_bytes": (U64, [P]),
        "gi_get_info": (I, [P, ctypes.POINTER(gi_info)]),
        "gi_copy_layout": (I, [P, P, P]),
        "gi_set_option": (I, [P, I, I64]),
        "gi_get_option": (I, [P, I, ctypes.POINTER(I64)]),
        "gi_probe_random_sectors": (I, [P, U64, U32, U64, U64, P, P]),
        "gi_coalescing_probe": (I, [P, U64, U32, U32, U32, U64, P, P]),
        "gi_launch_count": (U64, []),
        "gi_range_lookup_noalloc": (I, [P, P, P, U64, P, P]),
        "gi_batch_create": (I, [P, ctypes.c_uint32, I, U32, ctypes.POINTER(P)]),
        "gi_batch_set_stream": (I, [P, P]),
        "gi_batch_build": (I, [P, P, P]),
        "gi_batch_point_lookup": (I, [P, P, P, U64, P]),
        "gi_batch_sync": (I, [P]),
        "gi_batch_copy_index": (I, [P, U32, P, P]),
        "gi_batch_set_option": (I, [P, I, I64]),
        "gi_batch_footprint_bytes": (U64, [P]),
        "gi_batch_destroy": (None, [P]),
        "gi_batch_set_fanouts": (I, [P, P]),
        "gi_batch_get_fanouts": (I, [P, P]),
        "gi_batch_tune_fanouts": (I, [P, P, P, P, P, U64, U32, I, P, P]),
        "gi_batch_fanout_table_clear": (None, []),
        "gi_server_create": (I, [ctypes.POINTER(P), U32, U64, U32, ctypes.POINTER(P)]),
        "gi_server_submit": (I, [P, ctypes.POINTER(gi_request), ctypes.POINTER(U64)]),
        "gi_server_wait": (I, [P, U64, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "gi_server_stats": (I, [P, ctypes.POINTER(U64), ctypes.POINTER(U64), ctypes.POINTER(U64)]),
        "gi_server_destroy": (None, [P]),
        "gi_server_replay": (I, [P, ctypes.POINTER(gi_request), P, U64, U32, P, P,
                                 ctypes.POINTER(ctypes.c_double)]),
        "gi_replay_serial": (I, [ctypes.POINTER(P), U32, ctypes.POINTER(gi_request), P, U64, P, P,
                                 ctypes.POINTER(ctypes.c_double)]),
        "gi_tune": (I, [P, P, U64, U32, I, ctypes.POINTER(gi_tune_result)]),
        "gi_tune_table_get": (I, [I, U32, U64, ctypes.POINTER(I64), ctypes.POINTER(I)]),
        "gi_tune_table_clear": (None, []),
        "gi_batch_tune": (I, [P, P, P, U64, U32, ctypes.POINTER(gi_tune_result)]),
        "gi_build_tuned": (I, [P, P, U64, I, P, U64, U32, I, ctypes.POINTER(P),
                               ctypes.POINTER(gi_tune_result)]),
        "gi_tune_table_layout": (I, [I, U64, ctypes.POINTER(I), ctypes.POINTER(U32), ctypes.POINTER(I)]),
        "gi_debug_fail_alloc": (None, [I64]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != GI_OK:
        raise GIError(rc, load().gi_last_error().decode(errors="replace"))


def _ptr(x):
    """Data pointer of a torch tensor / numpy array (contiguous), an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):  # torch.Tensor
        if not x.is_contiguous():
            raise ValueError("buffers must be contiguous")
        return x.data_ptr()
    if hasattr(x, "__array_interface__"):  # numpy
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("buffers must be contiguous")
        return x.__array_interface__["data"][0]
    raise TypeError("unsupported buffer type %r" % type(x))


def _len(x) -> int:
    if hasattr(x, "numel"):
        return int(x.numel())
    return int(len(x))


def _stream_handle(stream):
    if stream is None or isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


class Index:
    """Handle of a built index (owns the C gi_index*)."""

    def __init__(self, handle: int, keepalive=None):
        self._h = handle

    @property
    def handle(self) -> int:
        if not self._h:
            raise GIError(GI_ERR_INVALID, "index was destroyed")
        return self._h

    def info(self) -> gi_info:
        return gi_get_info(self)

    def close(self):
        if self._h:
            load().gi_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gi_build(keys, rowids, layout: int, k: int = 0) -> Index:
    lib = load()
    n = _len(keys)
    if _len(rowids) != n:
        raise ValueError("keys and rowids differ in length")
    out = ctypes.c_void_p()
    _check(lib.gi_build(_ptr(keys), _ptr(rowids), n, layout, k, ctypes.byref(out)))
    return Index(out.value)


def gi_point_lookup(index: Index, queries, out_rowids) -> None:
    m = _len(queries)
    if _len(out_rowids) < m:
        raise ValueError("out_rowids too small")
    _check(load().gi_point_lookup(index.handle, _ptr(queries), m, _ptr(out_rowids)))


def gi_range_lookup(index: Index, lo, hi, out_offsets, out_rowids=None) -> None:
    m = _len(lo)
    if _len(hi) != m or _len(out_offsets) < m + 1:
        raise ValueError("lo/hi lengths differ or out_offsets is shorter than m+1")
    _check(load().gi_range_lookup(index.handle, _ptr(lo), _ptr(hi), m, _ptr(out_offsets),
                                  _ptr(out_rowids)))


def gi_range_lookup_noalloc(index: Index, lo, hi, out_offsets, out_rowids=None) -> None:
    """gi_range_lookup without any allocation: device buffers only, at most
    GI_NOALLOC_MAX_RANGES ranges, scratch in a fixed array inside the library."""
    m = _len(lo)
    if _len(hi) != m or _len(out_offsets) < m + 1:
        raise ValueError("lo/hi lengths differ or out_offsets is shorter than m+1")
    _check(load().gi_range_lookup_noalloc(index.handle, _ptr(lo), _ptr(hi), m, _ptr(out_offsets),
                                          _ptr(out_rowids)))


class Batch:
    """Handle of a batch of indexes (owns the C gi_batch*)."""

    def __init__(self, handle: int, B: int):
        self._h = handle
        self.B = B

    @property
    def handle(self) -> int:
        if not self._h:
            raise GIError(GI_ERR_INVALID, "batch was destroyed")
        return self._h

    def close(self):
        if self._h:
            load().gi_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gi_batch_create(key_offsets, layout: int, k: int = 0) -> Batch:
    """key_offsets: host uint64 array of B+1 offsets into the concatenated pairs."""
    import numpy as np
    ko = np.ascontiguousarray(key_offsets, dtype=np.uint64)
    out = ctypes.c_void_p()
    _check(load().gi_batch_create(_ptr(ko), len(ko) - 1, layout, k, ctypes.byref(out)))
    return Batch(out.value, len(ko) - 1)


def gi_batch_set_stream(batch: Batch, stream) -> None:
    _check(load().gi_batch_set_stream(batch.handle, _stream_handle(stream)))


def gi_batch_build(batch: Batch, keys, rowids) -> None:
    _check(load().gi_batch_build(batch.handle, _ptr(keys), _ptr(rowids)))


def gi_batch_point_lookup(batch: Batch, queries, query_offsets, out_rowids) -> None:
    _check(load().gi_batch_point_lookup(batch.handle, _ptr(queries), _ptr(query_offsets),
                                        _len(queries), _ptr(out_rowids)))


def gi_batch_sync(batch: Batch) -> None:
    _check(load().gi_batch_sync(batch.handle))


def gi_batch_copy_index(batch: Batch, i: int, keys_out=None, rowids_out=None) -> None:
    _check(load().gi_batch_copy_index(batch.handle, i, _ptr(keys_out), _ptr(rowids_out)))


def gi_batch_set_option(batch: Batch, option: int, value: int) -> None:
    _check(load().gi_batch_set_option(batch.handle, option, value))


def gi_batch_footprint_bytes(batch: Batch) -> int:
    return int(load().gi_batch_footprint_bytes(batch.handle))


def gi_batch_destroy(batch: Batch) -> None:
    batch.close()


def gi_batch_set_fanouts(batch: Batch, ks=None) -> None:
    """Fan-out of every index (0 sorted, 2, 3, 5, 9, 17); None: by size class."""
    import numpy as _np
    arr = None if ks is None else _np.ascontiguousarray(ks, dtype=_np.uint32)
    _check(load().gi_batch_set_fanouts(batch.handle, None if arr is None else arr.ctypes.data))


def gi_batch_get_fanouts(batch: Batch, B: int):
    import numpy as _np
    out = _np.zeros(B, dtype=_np.uint32)
    _check(load().gi_batch_get_fanouts(batch.handle, out.ctypes.data))
    return out


def gi_batch_tune_fanouts(batch: Batch, B: int, keys, rowids, queries, query_offsets, reps: int = 0,
                          flags: int = 0):
    """Per-size-class fan-out tuner; returns (chosen fan-outs [B], class_ms [64, 5])."""
    import numpy as _np
    ks = _np.zeros(B, dtype=_np.uint32)
    cms = _np.zeros(64 * 5, dtype=_np.float64)
    _check(load().gi_batch_tune_fanouts(batch.handle, _ptr(keys), _ptr(rowids), _ptr(queries),
                                        _ptr(query_offsets), _len(queries), reps, flags,
                                        ks.ctypes.data, cms.ctypes.data))
    return ks, cms.reshape(64, 5)


def gi_batch_fanout_table_clear() -> None:
    load().gi_batch_fanout_table_clear()


class Server:
    """Handle of a serving engine (owns the C gi_server*)."""

    def __init__(self, handle: int, keep):
        self._h = handle
        self._keep = keep  # the served Index handles must outlive the server

    @property
    def handle(self) -> int:
        if not self._h:
            raise GIError(GI_ERR_INVALID, "server was destroyed")
        return self._h

    def close(self):
        if self._h:
            load().gi_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gi_server_create(indexes, arena_bytes: int, max_inflight: int = 3) -> Server:
    arr = (ctypes.c_void_p * len(indexes))(*[ix.handle for ix in indexes])
    out = ctypes.c_void_p()
    _check(load().gi_server_create(arr, len(indexes), arena_bytes, max_inflight, ctypes.byref(out)))
    return Server(out.value, list(indexes))


def gi_server_submit(server: Server, index: int, kind: int, keys, out_rowids=None, hi=None,
                     out_offsets=None, rows_capacity: int = 0) -> int:
    """Queue a request on host buffers; returns its ticket."""
    r = gi_request(index, kind, _len(keys), _ptr(keys), _ptr(hi), _ptr(out_rowids), _ptr(out_offsets),
                   rows_capacity)
    t = ctypes.c_uint64()
    _check(load().gi_server_submit(server.handle, ctypes.byref(r), ctypes.byref(t)))
    return int(t.value)


def gi_server_wait(server: Server, ticket: int):
    """Block until the request completes; returns (status, submit_ns, done_ns)."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    rc = load().gi_server_wait(server.handle, ticket, ctypes.byref(a), ctypes.byref(b))
    if rc not in (GI_OK, GI_ERR_CAPACITY):
        _check(rc)
    return rc, int(a.value), int(b.value)


def make_requests(reqs):
    """A ctypes array of gi_request from tuples (index, kind, keys, out_rowids, hi,
    out_offsets, rows_capacity) of host buffers (torch CPU tensors or numpy arrays)."""
    arr = (gi_request * len(reqs))()
    for i, (index, kind, keys, out_rowids, hi, out_offsets, cap) in enumerate(reqs):
        arr[i] = gi_request(index, kind, _len(keys), _ptr(keys), _ptr(hi), _ptr(out_rowids),
                            _ptr(out_offsets), cap)
    return arr


def gi_server_replay(server: Server, requests, arrival_ns, threads: int = 4):
    """Open-loop replay from native threads: request i at arrival_ns[i] (int64 numpy
    array).  Returns (latency_ns, status, wall_s); latency -1 if not accepted."""
    import numpy as _np
    arr = requests if isinstance(requests, ctypes.Array) else make_requests(requests)
    n = len(arr)
    arrival = _np.ascontiguousarray(arrival_ns, dtype=_np.int64)
    lat = _np.zeros(n, dtype=_np.int64)
    st = _np.zeros(n, dtype=_np.int32)
    wall = ctypes.c_double()
    rc = load().gi_server_replay(server.handle, arr, arrival.ctypes.data, n, threads, lat.ctypes.data,
                                 st.ctypes.data, ctypes.byref(wall))
    _check(rc)
    return lat, st, float(wall.value)


def gi_replay_serial(indexes, requests, arrival_ns):
    """The baseline of gi_server_replay: one native thread, the plain calls, one
    request at a time.  Returns (latency_ns, status, wall_s)."""
    import numpy as _np
    arr = requests if isinstance(requests, ctypes.Array) else make_requests(requests)
    n = len(arr)
    ix = (ctypes.c_void_p * len(indexes))(*[i.handle for i in indexes])
    arrival = _np.ascontiguousarray(arrival_ns, dtype=_np.int64)
    lat = _np.zeros(n, dtype=_np.int64)
    st = _np.zeros(n, dtype=_np.int32)
    wall = ctypes.c_double()
    rc = load().gi_replay_serial(ix, len(indexes), arr, arrival.ctypes.data, n, lat.ctypes.data,
                                 st.ctypes.data, ctypes.byref(wall))
    _check(rc)
    return lat, st, float(wall.value)


def gi_server_stats(server: Server):
    a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().gi_server_stats(server.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return int(a.value), int(b.value), int(c.value)


def gi_server_destroy(server: Server) -> None:
    server.close()


def gi_destroy(index: Index) -> None:
    index.close()


def gi_set_stream(index, stream) -> None:
    _check(load().gi_set_stream(index.handle if index is not None else None,
                                _stream_handle(stream)))


def gi_sync(index: Index) -> None:
    _check(load().gi_sync(index.handle))


def gi_last_error() -> str:
    return load().gi_last_error().decode(errors="replace")


def gi_footprint_bytes(index: Index) -> int:
    return int(load().gi_footprint_bytes(index.handle))


def gi_get_info(index: Index) -> gi_info:
    inf = gi_info()
    _check(load().gi_get_info(index.handle, ctypes.byref(inf)))
    return inf


def gi_copy_layout(index: Index, keys_out=None, rowids_out=None) -> None:
    _check(load().gi_copy_layout(index.handle, _ptr(keys_out), _ptr(rowids_out)))


def gi_set_option(index: Index, option: int, value: int) -> None:
    _check(load().gi_set_option(index.handle, option, value))


def gi_get_option(index: Index, option: int) -> int:
    v = ctypes.c_int64()
    _check(load().gi_get_option(index.handle, option, ctypes.byref(v)))
    return int(v.value)


def gi_tune(index: Index, queries, reps: int = 0, flags: int = GI_TUNE_APPLY) -> gi_tune_result:
    r = gi_tune_result()
    _check(load().gi_tune(index.handle, _ptr(queries), _len(queries), reps, flags, ctypes.byref(r)))
    return r


def gi_tune_table_get(layout: int, k: int, n: int):
    """The autotuner table's options for (layout | key width, k, n), or None."""
    opts = (ctypes.c_int64 * 11)()
    found = ctypes.c_int()
    _check(load().gi_tune_table_get(layout, k, n, opts, ctypes.byref(found)))
    return list(opts) if found.value else None


def gi_build_tuned(keys, rowids, key_flags: int, queries, reps: int = 0,
                   flags: int = GI_TUNE_APPLY):
    """Build in every layout / k, tune each on `queries`, keep the fastest:
    returns (Index, gi_tune_result)."""
    r = gi_tune_result()
    h = ctypes.c_void_p()
    _check(load().gi_build_tuned(_ptr(keys), _ptr(rowids), _len(keys), key_flags, _ptr(queries),
                                 _len(queries), reps, flags, ctypes.byref(h), ctypes.byref(r)))
    return Index(h.value, (keys, rowids)), r


def gi_tune_table_layout(key_flags: int, n: int):
    """The recorded (layout, k) for the size class of n, or None."""
    lay, k, found = ctypes.c_int(), ctypes.c_uint32(), ctypes.c_int()
    _check(load().gi_tune_table_layout(key_flags, n, ctypes.byref(lay), ctypes.byref(k), ctypes.byref(found)))
    return (lay.value, k.value) if found.value else None


def gi_tune_table_clear() -> None:
    load().gi_tune_table_clear()


def gi_batch_tune(batch: Batch, queries, query_offsets, reps: int = 0) -> gi_tune_result:
    r = gi_tune_result()
    _check(load().gi_batch_tune(batch.handle, _ptr(queries), _ptr(query_offsets), _len(queries),
                                reps, ctypes.byref(r)))
    return r


def gi_probe_random_sectors(buf, chunk_bytes: int, loads: int, seed: int, sink, stream=None) -> None:
    nbytes = buf.numel() * buf.element_size()
    _check(load().gi_probe_random_sectors(_ptr(buf), nbytes, chunk_bytes, loads, seed, _ptr(sink),
                                          _stream_handle(stream)))


def gi_coalescing_probe(buf, threads: int, group: int, steps: int, seed: int, sink,
                        stream=None) -> None:
    _check(load().gi_coalescing_probe(_ptr(buf), _len(buf), threads, group, steps, seed,
                                      _ptr(sink), _stream_handle(stream)))


def gi_debug_fail_alloc(after: int) -> None:
    """Test hook: the library's device allocation after `after` more succeeds fails
    with out-of-memory (once); after < 0 disarms."""
    load().gi_debug_fail_alloc(after)


def gi_launch_count() -> int:
    return int(load().gi_launch_count())
