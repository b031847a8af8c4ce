"""Max-key padding of the key array covers every read the lookups make (CPU).

The lookup kernels read whole k-ary nodes without per-pivot bounds checks: a
node starting at slot s < n is read as k-1 keys, slots s .. s+k-2, and slots at
or past n must hold the maximum key (written by the build from the end of the
layout's keys to the end of the allocation).  Shared-memory staging copies the
slots of whole top levels, rounded to whole nodes and to 16 bytes.  This checks,
for every fan-out k = 2..33 and both key widths, at n = k^m - 1, k^m, k^m + 1 and
a few other sizes up to 2^32, that each such read ends inside the allocation and
that every slot it touches at or past n lies in the padded region.  The sizes come
from csrc/gi_alloc.h, compiled with the host compiler; the reads are restated here
from the kernels' addressing (node starts are multiples of k-1)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _sizes():
    cases = set()
    for k in range(2, 34):
        p = k
        while p <= (1 << 32):
            for n in (p - 1, p, p + 1):
                if 1 <= n < (1 << 32):
                    cases.add((n, k))
            p *= k
        for n in (1, 2, 3, 5, 63, 64, 65, 1000, (1 << 26) + 7, (1 << 32) - 1):
            cases.add((n, k))
    return sorted(cases)


def _probe(triples):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    os.makedirs(os.path.join(HERE, "_build"), exist_ok=True)
    exe = os.path.join(HERE, "_build", "alloc_probe")
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-I" + os.path.join(ROOT, "paper_2506_01576_gb300", "csrc"),
                        os.path.join(HERE, "alloc_probe.cpp"), "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    inp = "".join("%d %d %d\n" % t for t in triples)
    r = subprocess.run([exe], input=inp, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    return [tuple(int(v) for v in line.split()) for line in r.stdout.splitlines()]


def _kary_reach(n, k):
    """Last key slot read by a node read: the last node start below n, plus k-2."""
    node = k - 1
    last_start = (n - 1) // node * node
    return last_start + node - 1


def _staging_reach(n, k, kb):
    """Last key slot of the deepest staging (every level, whole nodes, 16-byte rounding)."""
    node = k - 1
    whole = (n + node - 1) // node * node
    nbytes = (whole * kb + 15) // 16 * 16
    return nbytes // kb - 1


def test_padding_covers_every_node_read():
    cases = _sizes()
    triples = [(n, kb, 0) for n, k in cases for kb in (4, 8)]
    triples += [(n, kb, 1) for n in sorted({n for n, _ in cases}) for kb in (4, 8)]
    out = dict(zip(triples, _probe(triples)))
    checked = 0
    for n, k in cases:
        for kb in (4, 8):
            used, alloc = out[(n, kb, 0)]
            assert used == n * kb
            slots = alloc // kb  # whole key slots in the allocation
            for reach in (_kary_reach(n, k), _staging_reach(n, k, kb)):
                assert reach < slots, (n, k, kb, reach, slots)
                # every slot read at or past n is padding: [used, alloc) in bytes
                assert reach < n or (n * kb >= used and (reach + 1) * kb <= alloc)
                checked += 1
    for n in sorted({n for n, _ in cases}):
        for kb in (4, 8):
            used, alloc = out[(n, kb, 1)]
            # Eytzinger: 1-based slots 1..n are read (slot 0 is the empty slot)
            assert used == (n + 1) * kb and n < alloc // kb
    assert checked > 4000
