"""Helpers for the GPU tests: numpy <-> torch CUDA buffers of unsigned types."""
import numpy as np
import torch

import paper_2506_01576_gb300 as gi

DEV = torch.device("cuda:0")

_SIGNED = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64}


def to_dev(a: np.ndarray) -> torch.Tensor:
    """Copy an unsigned numpy array to a CUDA tensor of the signed type of equal width."""
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(_SIGNED[a.dtype])).to(DEV)


def to_host(t: torch.Tensor, dtype) -> np.ndarray:
    return t.cpu().numpy().view(dtype)


def empty_u32(n: int) -> torch.Tensor:
    return torch.empty(max(n, 1), dtype=torch.int32, device=DEV)[:n] if n else torch.empty(0, dtype=torch.int32, device=DEV)


def empty_u64(n: int) -> torch.Tensor:
    return torch.empty(n, dtype=torch.int64, device=DEV)


def key_flag(dtype) -> int:
    return gi.GI_KEY_U64 if np.dtype(dtype) == np.uint64 else gi.GI_KEY_U32


def build(keys: np.ndarray, rows: np.ndarray, layout: int, k: int = 0):
    return gi.gi_build(to_dev(keys), to_dev(rows), layout | key_flag(keys.dtype), k)


def point(idx, q: np.ndarray) -> np.ndarray:
    out = torch.empty(len(q), dtype=torch.int32, device=DEV)
    gi.gi_point_lookup(idx, to_dev(q), out)
    torch.cuda.synchronize()
    return to_host(out, np.uint32)


def ranges(idx, lo: np.ndarray, hi: np.ndarray):
    tlo, thi = to_dev(lo), to_dev(hi)
    off = empty_u64(len(lo) + 1)
    gi.gi_range_lookup(idx, tlo, thi, off)
    total = int(off[-1].item())
    rows = torch.empty(max(total, 1), dtype=torch.int32, device=DEV)
    gi.gi_range_lookup(idx, tlo, thi, off, rows)
    torch.cuda.synchronize()
    return to_host(off, np.uint64), to_host(rows, np.uint32)[:total]


def layout_arrays(idx, n: int, dtype):
    k = torch.empty(n, dtype=torch.int64 if np.dtype(dtype) == np.uint64 else torch.int32, device=DEV)
    r = torch.empty(n, dtype=torch.int32, device=DEV)
    if n:
        gi.gi_copy_layout(idx, k, r)
    return to_host(k, dtype), to_host(r, np.uint32)
