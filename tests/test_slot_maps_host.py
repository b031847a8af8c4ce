"""The CUDA path's closed-form slot maps, run on the host, against the paper.

slot_to_rank (p'(t), Sections 4 and 6.1), its inverse rank_to_slot, and the
32-bit level-table map slot_of_rank that the bucket sort and the range fill use
are __host__ __device__ functions; `slotmap_probe.cu` exposes them to this test.
They are checked against the formula of Section 6.1 as restated in
test_oracle_pins (Python integers, no overflow) at sampled ranks for index
sizes up to 2^32 - 1, beyond what a GPU test can build, and exhaustively as a
bijection for small sizes.  No GPU is needed.
"""
import ctypes
import os
import random
import subprocess

import pytest

from test_oracle_pins import pprime_closed_form

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
PKG = os.path.join(ROOT, "paper_2506_01576_gb300")
OUT = os.path.join(HERE, "_build", "libslotprobe.so")
SRC = os.path.join(HERE, "slotmap_probe.cu")


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return "nvcc"


@pytest.fixture(scope="module")
def probe():
    from paper_2506_01576_gb300 import _build
    lib = _build.build()  # libgi.so: the probe links its host make_geom
    deps = [SRC, os.path.join(PKG, "csrc", "gi_internal.cuh"), lib]
    if not os.path.exists(OUT) or os.path.getmtime(OUT) < max(os.path.getmtime(d) for d in deps):
        os.makedirs(os.path.dirname(OUT), exist_ok=True)
        cmd = [_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
               "-shared", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
               "-I" + os.path.join(ROOT, "include"), "-I" + os.path.join(PKG, "csrc"),
               SRC, "-o", OUT + ".tmp", "-L" + PKG, "-lgi", "-Xlinker", "-rpath=" + PKG]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        os.replace(OUT + ".tmp", OUT)
    p = ctypes.CDLL(OUT)
    U64, U32 = ctypes.c_uint64, ctypes.c_uint32
    p.sp_slot_to_rank.restype = U64
    p.sp_slot_to_rank.argtypes = [U64, U32, U64]
    p.sp_rank_to_slot.restype = U64
    p.sp_rank_to_slot.argtypes = [U64, U32, U64]
    p.sp_slot_of_rank.restype = U32
    p.sp_slot_of_rank.argtypes = [U64, U32, U32, ctypes.c_int]
    return p


def _ranks(n, k, rng):
    """Boundary ranks (ends, bottom-level edges, node edges) and random ones."""
    top = 1
    while top * k <= n:
        top *= k
    top -= 1
    b = n - top
    cand = {0, 1, n - 1, n - 2, b - 1, b, b + 1, top, top - 1, (b // (k - 1)) * k, n // 2}
    cand |= {rng.randrange(n) for _ in range(300)}
    return sorted(r for r in cand if 0 <= r < n)


@pytest.mark.parametrize("k", [2, 3, 4, 5, 9, 16, 17, 33])
def test_maps_equal_the_paper_formula_up_to_2_32(probe, k):
    rng = random.Random(k)
    sizes = [1, 2, k - 1, k, k + 1, 1000, 2 ** 20 + 7, 2 ** 26, 2 ** 31 - 1, 2 ** 31, 2 ** 32 - 1]
    p = k
    while p < 2 ** 32:  # around every power of k: the tree just full / one key into a new level
        sizes += [p - 2, p - 1, p, p + 1]
        p *= k
    for n in sorted({s for s in sizes if 1 <= s < 2 ** 32}):
        for r in _ranks(n, k, rng):
            t = probe.sp_slot_of_rank(n, k, r, 0)
            assert pprime_closed_form(t, n, k) == r, (n, k, r, t)
            assert probe.sp_rank_to_slot(n, k, r) == t, (n, k, r)
            assert probe.sp_slot_to_rank(n, k, t) == r, (n, k, t)
            if k in (2, 3, 5, 9, 17):
                assert probe.sp_slot_of_rank(n, k, r, 1) == t, (n, k, r)


@pytest.mark.parametrize("k", [2, 3, 5, 7, 9, 17])
def test_slot_of_rank_is_a_bijection_for_small_n(probe, k):
    for n in list(range(1, 300)) + [k ** 3 - 1, k ** 3, k ** 3 + 1]:
        slots = [probe.sp_slot_of_rank(n, k, r, 0) for r in range(n)]
        assert sorted(slots) == list(range(n)), (n, k)
