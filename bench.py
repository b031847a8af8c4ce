"""Benchmark: point lookups/s on a static index of 2^26 uint64 keys (EKS vs BS).

One step is one pass of the whole hot path over one batch of synthetic input:
  build    gi_build of 2^26 unique uint64 keys (uniform in [0, 2^63), rowIDs
           0..n-1): radix sort + k-ary Eytzinger permutation;
  point    gi_point_lookup of 2^27 uint64 probes, hit rate 0.5, uniform;
  range    gi_range_lookup of 2^22 inclusive ranges with 16 expected rows each
           (count + scan + fill into CSR).
value = point lookups in the step / step time (device clock, CUDA events, max
over ranks).  Inputs (0.5 GiB keys, 1 GiB probes) are larger than L2, so no
extra flush is needed between steps.

Extra fields: lookup-only throughput of EKS and of textbook BS on the same
index keys (the "EKS vs BS" of the metric), the roofline of the lookup kernel
against the measured HBM copy bandwidth and against a random-access probe run
in the same process, an end-to-end number through the C ABI with host buffers,
and the CPU oracle timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "point lookups/s @2^26 u64 keys, EKS vs textbook BS; % of HBM sector roofline"
UNIT = "lookups/s"


# ---------------------------------------------------------------- helpers
def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-log", type=int, default=26)
    ap.add_argument("--m-log", type=int, default=27)
    ap.add_argument("--ranges-log", type=int, default=22)
    ap.add_argument("--range-rows", type=float, default=16.0)
    ap.add_argument("--k", type=int, default=5, help="EKS fan-out")
    ap.add_argument("--layout", default="eks", choices=["eks", "ebs", "bs"],
                    help="layout built and probed in the timed step")
    ap.add_argument("--group", type=int, default=-1)
    ap.add_argument("--per-thread", type=int, default=-1)
    ap.add_argument("--smem-levels", type=int, default=-1)
    ap.add_argument("--blocks-per-sm", type=int, default=-1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-probe", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="timed steps only (for profiler launch lists)")
    ap.add_argument("--no-legs", action="store_true", help="skip the ranges / batched / serving legs")
    ap.add_argument("--workload", default="point",
                    choices=["point", "batched", "ranges", "dups", "skew", "serve", "sizes", "tune"],
                    help="point: the 2^26-key step (default); batched: 4096 indexes in one graph; "
                         "ranges: 2^24 ranges on 2^26 u32 keys; dups: replicated keys, point = range [x, x]")
    ap.add_argument("--batch-k", type=int, default=5)
    ap.add_argument("--serve-indexes", type=int, default=64)
    ap.add_argument("--serve-min-log", type=int, default=20)
    ap.add_argument("--serve-max-log", type=int, default=27)
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--serve-rates", default="1000,4000,16000,64000,128000,256000")
    ap.add_argument("--batch-indexes", type=int, default=4096)
    ap.add_argument("--probe-sweep", action="store_true",
                    help="print random-access throughput over buffer sizes (L2 vs HBM) and exit")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled while the timed region runs.

    One nvidia-smi process in loop mode (every `interval_ms`) runs from start()
    to stop(); samples are stamped on arrival, and summary() keeps those that
    arrived between begin() and end() (the timed region).
    """

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 50):
        self.gpu = gpu_index
        self.interval_ms = interval_ms
        self.samples = []  # (arrival time, fields)
        self.window = (0.0, float("inf"))
        self._proc = None
        self._t = None

    def _read(self):
        for line in self._proc.stdout:
            line = line.strip()
            if line:
                self.samples.append((time.monotonic(), [x.strip() for x in line.split(",")]))

    def start(self):
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", str(self.interval_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self._proc = None
        return self

    def begin(self):
        self.window = (time.monotonic(), float("inf"))

    def end(self):
        self.window = (self.window[0], time.monotonic())

    def stop(self):
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()
            self._t.join(timeout=5)

    def summary(self):
        t0, t1 = self.window
        inside = [f for t, f in self.samples if t0 <= t <= t1]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(s[0]) for s in inside if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in inside if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in inside for i in range(4)
                          if len(s) > 3 + i and s[3 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(inside)}


def step_config(a, world):
    """The benchmark step's workload (the same dict for both arms)."""
    return {"workload": "build 2^%d unique u64 keys (%s) + 2^%d point probes (hit 0.5, "
                        "uniform) + 2^%d ranges (%.0f expected rows) per step"
                        % (a.n_log, "EKS k=%d" % a.k if a.layout == "eks" else a.layout.upper(),
                           a.m_log, a.ranges_log, a.range_rows),
            "n_keys": 1 << a.n_log, "point_probes": 1 << a.m_log, "ranges": 1 << a.ranges_log,
            "layout": a.layout.upper(), "k": a.k if a.layout == "eks" else None,
            "l2": "inputs larger than L2 (no flush)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def kary_level_sizes(n: int, k: int):
    """Keys per level of the complete k-ary tree of n keys (last level partial)."""
    if n == 0:
        return []
    m, p = 0, 1
    while p <= n // k:
        p *= k
        m += 1
    sizes = [(k - 1) * k ** l for l in range(m)]
    sizes.append(n - (p - 1))
    return sizes


def eks_bytes_per_lookup(n: int, k: int, key_bytes: int, hit_rate: float, l2_bytes: int):
    """Algorithmic DRAM bytes of one k-ary lookup, and the random requests by size.

    Levels whose cumulative key bytes fit in L2 are counted as resident.  Every
    lookup visits all full levels; it reaches the partial bottom level iff its
    gap borders a bottom key: (b + bottom nodes) of the n + 1 gaps.  Each visited
    level reads one node (k-1 keys, rounded up to 32-byte sectors).  A hit reads
    one rowID sector.  Probe and result stream once (key + 4 bytes).
    """
    sizes = kary_level_sizes(n, k)
    node = math.ceil((k - 1) * key_bytes / 32) * 32
    cum, reqs = 0, {}
    for l, sz in enumerate(sizes):
        cum += sz * key_bytes
        if cum <= l2_bytes:
            continue
        if l < len(sizes) - 1:
            p = 1.0
        else:
            b = sz
            p = (b + math.ceil(b / (k - 1))) / (n + 1)
        reqs[node] = reqs.get(node, 0.0) + p
    reqs[32] = reqs.get(32, 0.0) + hit_rate
    nbytes = sum(sz * c for sz, c in reqs.items()) + key_bytes + 4
    return nbytes, reqs


def max_over_ranks(ms: float, device="cpu") -> float:
    """The slowest rank's time: the whole job is done only when every replica is."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, steps: int, ms: float) -> float:
    """Whole-job rate: units every rank processed over the slowest rank's time."""
    return units_per_rank * world * steps / (ms / 1e3)


# ---------------------------------------------------------------- our arm
def run_ours(a):
    import torch
    import torch.distributed as dist

    import paper_2506_01576_gb300 as gi

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    gi.load()
    n, m, mr = 1 << a.n_log, 1 << a.m_log, 1 << a.ranges_log
    seed = W.seed_for(1, a.n_log, rank)
    keys = W.unique_keys(n, 64, seed)
    rows = np.arange(n, dtype=np.uint32)
    q = W.point_probes(keys, m, 0.5, 64, seed, seed + 1)
    lo, hi, w = W.ranges_with_expected_rows(n, mr, a.range_rows, 64, seed + 2)
    dv = lambda x: torch.from_numpy(x.view(np.int64) if x.dtype == np.uint64 else x.view(np.int32)).to(dev)
    kd, rd, qd, lod, hid = dv(keys), dv(rows), dv(q), dv(lo), dv(hi)
    out = torch.empty(m, dtype=torch.int32, device=dev)
    off = torch.empty(mr + 1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    gi.gi_set_stream(None, stream)
    layout = {"eks": gi.GI_EYTZINGER_KARY, "ebs": gi.GI_EYTZINGER, "bs": gi.GI_SORTED}[a.layout] | gi.GI_KEY_U64

    def configure(idx):
        for opt, v in ((gi.GI_OPT_GROUP, a.group if a.layout == "eks" else -1),
                       (gi.GI_OPT_PER_THREAD, a.per_thread),
                       (gi.GI_OPT_SMEM_LEVELS, a.smem_levels),
                       (gi.GI_OPT_BLOCKS_PER_SM, a.blocks_per_sm)):
            gi.gi_set_option(idx, opt, v)

    # size the range output once (the same ranges every step)
    idx = gi.gi_build(kd, rd, layout, a.k)
    gi.gi_range_lookup(idx, lod, hid, off)
    total_rows = int(off[-1].item())
    rout = torch.empty(max(total_rows, 1), dtype=torch.int32, device=dev)
    gi.gi_destroy(idx)

    ev_pt = []

    def step(timed):
        idx = gi.gi_build(kd, rd, layout, a.k)
        configure(idx)
        if timed:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        gi.gi_point_lookup(idx, qd, out)
        if timed:
            e1.record(stream)
            ev_pt.append((e0, e1))
        gi.gi_range_lookup(idx, lod, hid, off, rout)  # single call: count + scan + fill
        gi.gi_destroy(idx)  # waits for the stream

    clk = ClockSampler(local).start()  # the sampler's start-up overlaps the warm-up
    for _ in range(a.warmup):
        step(False)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = gi.gi_launch_count()
    clk.begin()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(a.steps):
        step(True)
    t1.record(stream)
    torch.cuda.synchronize()
    clk.end()
    clk.stop()
    launches = gi.gi_launch_count() - l0
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(t0.elapsed_time(t1), dev if world > 1 and dist.get_backend() == "nccl" else "cpu")
    ms_step = ms / a.steps
    value = job_throughput(m, world, a.steps, ms)
    pt_ms = float(np.mean([e0.elapsed_time(e1) for e0, e1 in ev_pt]))

    # parity spot check of the timed configuration (results are integers: exact)
    res = {}
    if rank == 0 and not a.no_extras:
        res = extras(a, gi, torch, dev, kd, rd, qd, out, keys, q, n, m, pt_ms, configure, layout,
                     total_rows, lo, hi)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": step_config(a, world), "range_rows_total": total_rows,
        "clocks": clk.summary(), "gpu_launches": int(launches),
    }
    line.update(res)
    print(json.dumps(line), flush=True)


def extras(a, gi, torch, dev, kd, rd, qd, out, keys, q, n, m, pt_ms, configure, layout, total_rows,
           lo, hi):
    """Lookup-only rates, roofline, e2e through host buffers, CPU oracle."""
    import oracle
    stream = torch.cuda.current_stream()

    def ev_time(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    res = {}
    # ---- lookup-only: EKS (timed configuration), textbook BS, EBS
    idx = gi.gi_build(kd, rd, layout, a.k)
    configure(idx)
    eks_ms = ev_time(lambda: gi.gi_point_lookup(idx, qd, out))
    opts = {name: gi.gi_get_option(idx, o) for name, o in
            (("group", gi.GI_OPT_GROUP), ("per_thread", gi.GI_OPT_PER_THREAD),
             ("smem_levels", gi.GI_OPT_SMEM_LEVELS), ("block", gi.GI_OPT_BLOCK),
             ("blocks_per_sm", gi.GI_OPT_BLOCKS_PER_SM), ("hot_levels", gi.GI_OPT_HOT_LEVELS))}
    gi.gi_point_lookup(idx, qd, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    gi.gi_destroy(idx)
    bs = gi.gi_build(kd, rd, gi.GI_SORTED | gi.GI_KEY_U64, 0)
    bs_ms = ev_time(lambda: gi.gi_point_lookup(bs, qd, out))
    gi.gi_destroy(bs)
    eb = gi.gi_build(kd, rd, gi.GI_EYTZINGER | gi.GI_KEY_U64, 0)
    gi.gi_set_option(eb, gi.GI_OPT_PER_THREAD, 4)
    ebs_ms = ev_time(lambda: gi.gi_point_lookup(eb, qd, out))
    gi.gi_destroy(eb)
    # sampled parity: probes whose rowID is known without the oracle
    rng = np.random.default_rng(0)
    samp = rng.choice(m, size=1 << 16, replace=False)
    sk_idx = np.argsort(keys, kind="stable")
    sk = keys[sk_idx]
    r = np.searchsorted(sk, q[samp])
    hit = (r < n) & (sk[np.minimum(r, n - 1)] == q[samp])
    want = np.where(hit, sk_idx[np.minimum(r, n - 1)].astype(np.uint32), np.uint32(0xFFFFFFFF))
    parity_ok = bool(np.array_equal(got[samp], want))
    res["lookup_only"] = {
        "eks_lookups_per_s": m / (eks_ms / 1e3), "eks_ms": eks_ms, "eks_kernel_ms_in_step": pt_ms,
        "bs_lookups_per_s": m / (bs_ms / 1e3), "bs_ms": bs_ms,
        "ebs_lookups_per_s": m / (ebs_ms / 1e3), "ebs_ms": ebs_ms,
        "speedup_eks_vs_bs": bs_ms / eks_ms, "eks_config": opts,
        "sampled_parity_65536": parity_ok,
    }
    # ---- roofline of the dominant kernel (EKS point lookup)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    bpl, reqs = eks_bytes_per_lookup(n, a.k, 8, 0.5, l2)
    achieved = bpl * m / (pt_ms / 1e3) / 1e9
    res["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                       "frac": achieved / hbm, "traffic": recorded_traffic(a, m, opts["hot_levels"], opts["block"]),
                       "peak_source": "measured" if peaks else "fallback",
                       "kernel": "k_eks_point", "algorithmic_bytes_per_lookup": bpl,
                       "random_requests_per_lookup": reqs, "l2_bytes": l2}
    if not a.no_probe:
        buf = torch.empty(16 << 30, dtype=torch.uint8, device=dev)
        sink = torch.zeros(1, dtype=torch.int64, device=dev)
        rate = {}
        for c in sorted(set(list(reqs.keys()) + [32])):
            loads = 1 << 28
            t = ev_time(lambda: gi.gi_probe_random_sectors(buf, c, loads, 7, sink, stream), reps=3)
            rate[c] = loads / (t / 1e3)
        del buf
        torch.cuda.empty_cache()
        t_per = sum(cnt / rate[c] for c, cnt in reqs.items())
        bound = 1.0 / t_per
        res["roofline"]["random_access"] = {
            "probe_chunks_per_s": {str(c): v for c, v in rate.items()},
            "bound_lookups_per_s": bound, "frac": (m / (pt_ms / 1e3)) / bound,
            "note": "bound = 1 / sum(requests_of_size_s / measured random-chunk rate at s)"}
    # ---- e2e through the C ABI with pinned host buffers
    if not a.no_e2e:
        nk = len(keys)
        hk = torch.from_numpy(keys.view(np.int64)).pin_memory()
        hr = torch.arange(nk, dtype=torch.int32).pin_memory()
        hq = torch.from_numpy(q.view(np.int64)).pin_memory()
        ho = torch.empty(m, dtype=torch.int32).pin_memory()
        mr = 1 << a.ranges_log
        lo, hi, _ = W.ranges_with_expected_rows(n, mr, a.range_rows, 64, W.seed_for(1, a.n_log, 0) + 2)
        hlo = torch.from_numpy(lo.view(np.int64)).pin_memory()
        hhi = torch.from_numpy(hi.view(np.int64)).pin_memory()
        hoff = torch.empty(mr + 1, dtype=torch.int64).pin_memory()
        hrows = torch.empty(max(total_rows, 1), dtype=torch.int32).pin_memory()

        def e2e_step():
            idx = gi.gi_build(hk, hr, layout, a.k)
            configure(idx)
            gi.gi_point_lookup(idx, hq, ho)
            gi.gi_range_lookup(idx, hlo, hhi, hoff, hrows)  # count + scan + fill, staged
            gi.gi_destroy(idx)
            return int(hoff[-1])

        for _ in range(2):  # warm-up: the first calls set up the staging buffers
            e2e_step()
        # each step timed on the host clock; the median of 5 (a step is ~15 ms, so
        # one descheduled host thread would otherwise move a 3-step mean by 2x)
        reps = 5
        times = []
        for _ in range(reps):
            t0 = time.perf_counter()
            total = e2e_step()
            times.append(time.perf_counter() - t0)
        dt = float(np.median(times))
        res["e2e"] = {"value": m / dt, "unit": UNIT,
                      "h2d_bytes_per_step": nk * 8 + nk * 4 + m * 8 + 2 * mr * 8,
                      "d2h_bytes_per_step": m * 4 + (mr + 1) * 8 + total * 4,
                      "ms_per_step": dt * 1e3, "ms_per_step_each": [round(x * 1e3, 3) for x in times],
                      "stat": "median of %d steps after 2 warm-up steps" % reps, "host_buffers": "pinned"}
    # ---- the other forms of the path, each at a stated size (after the timed region)
    if not a.no_legs:
        res["ranges"] = ranges_leg(gi, torch, dev)
        bt = batched_measure(gi, torch, dev, 1024, 5, 5, 3, tune=False, per_index=True)
        bt["note"] = "1024 of the 4096 indexes of the batched workload (same size law)"
        res["batched"] = bt
        meta, runs = serving_sweep(gi, torch, dev, 8, 20, 24, [2000.0, 64000.0], 0.5, 400,
                                   serial_max_requests=4000)
        meta["note"] = ("8 resident indexes of 2^20..2^24 u64 keys (the serving workload's request "
                        "mix and arrival law at two offered loads)")
        res["serving"] = {**meta, "runs": runs}
    # ---- CPU oracle on the host cores (bounded sample)
    if not a.no_cpu:
        res["cpu_baseline"] = cpu_oracle_sample(keys, q, lo, hi, n, m, a)
    return res


def recorded_traffic(a, m, hot_levels, block):
    """DRAM bytes of one k_eks_point launch from the committed ncu summary, or None.

    Valid only for the configuration it was captured on (2^26 u64 keys, k = 5,
    2^27 probes, default knobs, the same number of evict-last levels and block size) and while
    the kernel source is unchanged.
    """
    import hashlib
    if (a.layout, a.k, a.n_log, a.m_log, a.group, a.per_thread, a.smem_levels,
            a.blocks_per_sm) != ("eks", 5, 26, 27, -1, -1, -1, -1):
        return None
    try:
        txt = open(os.path.join(ROOT, "profiles", "k_eks_point_u64_k5_2e26.md")).read()
        rec = dict(l.split(": ", 1) for l in txt.splitlines()
                   if l.startswith(("traffic_full_launch_bytes:", "kernel_source_sha256:",
                                    "hot_levels:", "block:")))
        h = hashlib.sha256()
        for f in ("gi_point_impl.cuh", "gi_eks_inst.cuh"):
            h.update(open(os.path.join(ROOT, "paper_2506_01576_gb300", "csrc", f), "rb").read())
        if h.hexdigest() != rec["kernel_source_sha256"].strip():
            return None
        if int(rec["hot_levels"]) != int(hot_levels) or int(rec["block"]) != int(block):
            return None
        return int(rec["traffic_full_launch_bytes"])
    except Exception:
        return None


def oracle_step_estimate(oracle, keys, rows, sk, sr, q, lo, hi, threads, rng,
                         sort_sample, point_sample, range_sample):
    """Seconds of one benchmark step on the oracle, from timed samples: std::sort of
    `sort_sample` pairs (one thread) scaled to n by n log n; std::lower_bound of
    `point_sample` probes over the full sorted index on `threads` threads, scaled
    to the probe count; the ranges (lower_bound + forward scan, CSR) of
    `range_sample` ranges on `threads` threads, scaled to the range count."""
    n, m, mr = len(keys), len(q), len(lo)
    j = int(rng.integers(0, n - sort_sample + 1))
    t0 = time.perf_counter()
    oracle.sort_pairs(keys[j:j + sort_sample], rows[j:j + sort_sample])
    t_sort = time.perf_counter() - t0
    i = int(rng.integers(0, m - point_sample + 1))
    t0 = time.perf_counter()
    oracle.point_lookup(sk, sr, q[i:i + point_sample], threads)
    t_pt = time.perf_counter() - t0
    r = int(rng.integers(0, mr - range_sample + 1))
    t0 = time.perf_counter()
    oracle.range_lookup(sk, sr, lo[r:r + range_sample], hi[r:r + range_sample], threads)
    t_rg = time.perf_counter() - t0
    return (t_sort * (n / sort_sample) * (math.log2(n) / math.log2(sort_sample))
            + t_pt * (m / point_sample) + t_rg * (mr / range_sample))


def oracle_sample_text(n, m, mr, threads, sort_sample, point_sample, range_sample):
    return ("std::sort of 2^%d pairs (1 thread, scaled n log n to 2^%d) + std::lower_bound of "
            "2^%d probes on %d threads (scaled to 2^%d) + 2^%d ranges, lower_bound and scan, on "
            "%d threads (scaled to 2^%d)"
            % (int(math.log2(sort_sample)), int(math.log2(n)), int(math.log2(point_sample)),
               threads, int(math.log2(m)), int(math.log2(range_sample)), threads, int(math.log2(mr))))


def oracle_lookup_rates(oracle, sk, sr, q, threads, sample=1 << 20):
    """std::lower_bound lookups/s of the oracle on 1 thread and on `threads` threads
    (the same 2^20-probe sample of the workload's probes, over the full index)."""
    x = q[:sample]
    t0 = time.perf_counter()
    oracle.point_lookup(sk, sr, x, 1)
    t1 = time.perf_counter()
    oracle.point_lookup(sk, sr, x, threads)
    t2 = time.perf_counter()
    return {"lookups_per_s_1_thread": len(x) / (t1 - t0),
            "lookups_per_s_all_threads": len(x) / (t2 - t1), "threads": threads,
            "sample_probes": len(x)}


def cpu_oracle_sample(keys, q, lo, hi, n, m, a, sort_sample=1 << 22, point_sample=1 << 21,
                      range_sample=1 << 17):
    """The oracle as it stands on the host cores: one sampled step, scaled."""
    import oracle
    threads = oracle.hardware_threads()
    rows = np.arange(n, dtype=np.uint32)
    sk, sr = oracle.sort_pairs(keys, rows)  # full index, untimed
    mr = len(lo)
    range_sample = min(range_sample, mr)
    est = oracle_step_estimate(oracle, keys, rows, sk, sr, q, lo, hi, threads,
                               np.random.default_rng(0), sort_sample, point_sample, range_sample)
    return {"value": m / est, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": oracle_sample_text(n, m, mr, threads, sort_sample, point_sample, range_sample),
            "est_step_s": est, "point_lookups": oracle_lookup_rates(oracle, sk, sr, q, threads)}


# ---------------------------------------------------------------- reference arm
def run_reference(a):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    n, m, mr = 1 << a.n_log, 1 << a.m_log, 1 << a.ranges_log
    seed = W.seed_for(1, a.n_log, 0)
    keys = W.unique_keys(n, 64, seed)
    q = W.point_probes(keys, m, 0.5, 64, seed, seed + 1)
    lo, hi, _ = W.ranges_with_expected_rows(n, mr, a.range_rows, 64, seed + 2)
    rows = np.arange(n, dtype=np.uint32)
    threads = oracle.hardware_threads()
    sk, sr = oracle.sort_pairs(keys, rows)
    sort_sample, point_sample, range_sample = min(1 << 21, n), min(1 << 20, m), min(1 << 16, mr)
    rng = np.random.default_rng(1)

    def step():
        return oracle_step_estimate(oracle, keys, rows, sk, sr, q, lo, hi, threads, rng,
                                    sort_sample, point_sample, range_sample)

    for _ in range(a.warmup):
        step()
    t0 = time.perf_counter()
    ests = [step() for _ in range(a.steps)]
    wall = (time.perf_counter() - t0) / a.steps  # the sampled step as timed
    est = float(np.mean(ests))
    value = m / est
    sample = ("each step a sample, scaled to the full step (est_full_step_ms): "
              + oracle_sample_text(n, m, mr, threads, sort_sample, point_sample, range_sample))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": wall * 1e3, "est_full_step_ms": est * 1e3,
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "impl": "reference", "config": step_config(a, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample,
                             "point_lookups": oracle_lookup_rates(oracle, sk, sr, q, threads)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def probe_sweep():
    """Random 32 B / 128 B loads over buffers from 8 MiB to 16 GiB (one line each)."""
    import torch

    import paper_2506_01576_gb300 as gi
    gi.load()
    dev = torch.device("cuda", 0)
    sink = torch.zeros(1, dtype=torch.int64, device=dev)
    for mb in (8, 32, 64, 96, 112, 128, 160, 256, 1024, 16384):
        buf = torch.ones(mb << 20, dtype=torch.uint8, device=dev)
        for c in (32, 128):
            loads = 1 << 27
            for _ in range(2):
                gi.gi_probe_random_sectors(buf, c, loads, 3, sink)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            gi.gi_probe_random_sectors(buf, c, loads, 5, sink)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            print(json.dumps({"buffer_mib": mb, "chunk_bytes": c, "chunks_per_s": loads / ms * 1e3,
                              "GBps": loads * c / ms / 1e6}), flush=True)
        del buf


def batched_measure(gi, torch, dev, B, k, steps, warmup, tune=False, per_index=True, seed=2024,
                    mixed=True):
    """B independent indexes (2^8..2^20 u64 keys, log-uniform) with 2^10..2^18 probes
    each at hit rate 0.75: build + lookup of all of them as one CUDA graph
    (gi_batch_*), against one gi_build + gi_point_lookup per index.  Returns a dict."""
    rng = np.random.default_rng(seed)
    sizes = np.exp2(rng.uniform(8, 20, size=B)).astype(np.int64)
    nq = np.exp2(rng.uniform(10, 18, size=B)).astype(np.int64)
    off = np.zeros(B + 1, dtype=np.uint64)
    np.cumsum(sizes.astype(np.uint64), out=off[1:])
    keys = np.concatenate([W.unique_keys(int(n), 64, W.seed_for(3, 20, i)) for i, n in enumerate(sizes)])
    qs = []
    for i, n in enumerate(sizes):
        k0 = int(off[i])
        qs.append(W.point_probes(keys[k0:k0 + int(n)], int(nq[i]), 0.75, 64, W.seed_for(3, 20, i), 17 + i))
    q = np.concatenate(qs)
    qoff = np.zeros(B + 1, dtype=np.uint64)
    np.cumsum(nq.astype(np.uint64), out=qoff[1:])
    m = int(qoff[-1])
    kd = torch.from_numpy(keys.view(np.int64)).to(dev)
    rd = torch.arange(len(keys), dtype=torch.int32, device=dev)
    qd = torch.from_numpy(q.view(np.int64)).to(dev)
    qod = torch.from_numpy(qoff.view(np.int64)).to(dev)
    out = torch.empty(m, dtype=torch.int32, device=dev)
    layout = gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64
    batch = gi.gi_batch_create(off, layout, k)
    s = torch.cuda.Stream()
    gi.gi_batch_set_stream(batch, s)
    with torch.cuda.stream(s):
        gi.gi_batch_build(batch, kd, rd)
        gi.gi_batch_point_lookup(batch, qd, qod, out)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    c0 = gi.gi_launch_count()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        gi.gi_batch_build(batch, kd, rd)
        gi.gi_batch_point_lookup(batch, qd, qod, out)
    kernels_per_replay = gi.gi_launch_count() - c0  # kernel nodes captured in the graph

    def ev(fn, reps):
        with torch.cuda.stream(s):  # replays and launches both go to stream s
            for _ in range(warmup):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                fn()
            e1.record(s)
            e1.synchronize()
        return e0.elapsed_time(e1) / reps

    clk = ClockSampler(0).start()
    for _ in range(3):  # warm replays while the sampler starts
        g.replay()
    torch.cuda.synchronize()
    clk.begin()
    graph_ms = ev(lambda: g.replay(), steps)
    clk.end()
    clk.stop()
    gi.gi_batch_sync(batch)
    got = out.cpu().numpy().view(np.uint32)
    lookup_ms = ev(lambda: gi.gi_batch_point_lookup(batch, qd, qod, out), steps)
    build_ms = ev(lambda: gi.gi_batch_build(batch, kd, rd), max(2, steps // 2))
    # sampled parity without the oracle: per index, sorted keys and numpy searchsorted
    samp_ok = True
    for i in rng.choice(B, size=min(B, 64), replace=False):
        k0, k1, q0, q1 = int(off[i]), int(off[i + 1]), int(qoff[i]), int(qoff[i + 1])
        order = np.argsort(keys[k0:k1], kind="stable")
        sk = keys[k0:k1][order]
        r = np.searchsorted(sk, q[q0:q1])
        rc = np.minimum(r, len(sk) - 1)
        hit = (r < len(sk)) & (sk[rc] == q[q0:q1])
        want = np.where(hit, (order[rc] + k0).astype(np.uint32), np.uint32(0xFFFFFFFF))
        samp_ok &= bool(np.array_equal(got[q0:q1], want))
    # per-index fan-outs: the automatic choice by size class, then the tuner's
    # per-class choice; each captured and replayed as its own graph
    fan = {}
    if mixed:
        def graph_ms_now():
            gg = torch.cuda.CUDAGraph()
            with torch.cuda.stream(s):
                gi.gi_batch_build(batch, kd, rd)
                gi.gi_batch_point_lookup(batch, qd, qod, out)
            s.synchronize()
            with torch.cuda.graph(gg, stream=s, capture_error_mode="relaxed"):
                gi.gi_batch_build(batch, kd, rd)
                gi.gi_batch_point_lookup(batch, qd, qod, out)
            t = ev(lambda: gg.replay(), steps)
            gi.gi_batch_sync(batch)
            return t, out.cpu().numpy().view(np.uint32)

        def parts_now():
            return (ev(lambda: gi.gi_batch_build(batch, kd, rd), max(2, steps // 2)),
                    ev(lambda: gi.gi_batch_point_lookup(batch, qd, qod, out), steps))

        gi.gi_batch_fanout_table_clear()
        gi.gi_batch_set_fanouts(batch, None)
        ks_auto = gi.gi_batch_get_fanouts(batch, B)
        t_auto, got_auto = graph_ms_now()
        b_auto, l_auto = parts_now()
        ks_t, cms = gi.gi_batch_tune_fanouts(batch, B, kd, rd, qd, qod, reps=3, flags=gi.GI_TUNE_APPLY)
        t_tuned, got_tuned = graph_ms_now()
        b_tuned, l_tuned = parts_now()
        classes = {}
        for c in range(64):
            if cms[c].max() > 0:
                classes["2^%d" % c] = {"chosen_k": int([2, 3, 5, 9, 17][int(np.argmin(cms[c]))]),
                                       "ms_by_k": {str(k): round(float(v), 4)
                                                   for k, v in zip((2, 3, 5, 9, 17), cms[c])}}
        fan = {"graph_step_ms_auto_fanouts": t_auto, "graph_step_ms_tuned_fanouts": t_tuned,
               "build_ms_auto_fanouts": b_auto, "lookup_ms_auto_fanouts": l_auto,
               "build_ms_tuned_fanouts": b_tuned, "lookup_ms_tuned_fanouts": l_tuned,
               "lookups_per_s_tuned_fanouts": m / (t_tuned / 1e3),
               "auto_fanout_counts": {str(k): int((ks_auto == k).sum()) for k in (2, 3, 5, 9, 17)},
               "tuned_per_class": classes,
               "results_identical_to_k5": bool(np.array_equal(got_auto, got) and np.array_equal(got_tuned, got))}
        gi.gi_batch_set_fanouts(batch, np.full(B, k, np.uint32))
        gi.gi_batch_build(batch, kd, rd)
    tuned = None
    if tune:  # the autotuner on the same probes (the graph keeps the defaults)
        r = gi.gi_batch_tune(batch, qd, qod)
        names = {gi.GI_BATCH_OPT_CHUNK: "chunk", gi.GI_BATCH_OPT_BLOCKS_PER_SM: "blocks_per_sm",
                 gi.GI_BATCH_OPT_SMEM_BUDGET: "smem_budget"}
        tuned = {"lookup_ms": ev(lambda: gi.gi_batch_point_lookup(batch, qd, qod, out), steps),
                 "start": {v: int(r.start_options[o]) for o, v in names.items()},
                 "chosen": {v: int(r.options[o]) for o, v in names.items()}, "trials": int(r.trials)}
    # one index at a time through the single-index API
    per_ms, same = None, None
    if per_index:
        gi.gi_set_stream(None, s)
        out2 = torch.empty(m, dtype=torch.int32, device=dev)

        def one_by_one():
            for i in range(B):
                k0, k1 = int(off[i]), int(off[i + 1])
                q0, q1 = int(qoff[i]), int(qoff[i + 1])
                idx = gi.gi_build(kd[k0:k1], rd[k0:k1], layout, k)
                gi.gi_point_lookup(idx, qd[q0:q1], out2[q0:q1])
                gi.gi_destroy(idx)

        torch.cuda.synchronize()
        t0 = time.perf_counter()
        one_by_one()
        torch.cuda.synchronize()
        per_ms = (time.perf_counter() - t0) * 1e3
        same = bool(np.array_equal(got, out2.cpu().numpy().view(np.uint32)))
        gi.gi_set_stream(None, None)
    gi.gi_batch_destroy(batch)
    return {"indexes": B, "keys_total": int(off[-1]), "probes_total": m, "k": k,
            "graph_step_ms": graph_ms, "build_ms": build_ms, "lookup_ms": lookup_ms,
            "lookups_per_s": m / (graph_ms / 1e3), "lookup_only_per_s": m / (lookup_ms / 1e3),
            "lookup_tuned": tuned, "per_index_launches_ms": per_ms,
            "speedup_vs_per_index": per_ms and per_ms / graph_ms,
            "per_index_results_identical": same, "sampled_parity_64_indexes": samp_ok,
            "kernels_per_graph": int(kernels_per_replay), "clocks": clk.summary(), **fan}


def run_batched(a):
    """The batched form (the survey's C4): 4096 indexes, one JSON line."""
    import torch

    import paper_2506_01576_gb300 as gi
    gi.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    r = batched_measure(gi, torch, dev, a.batch_indexes, a.batch_k, a.steps, a.warmup,
                        tune=not a.no_extras, per_index=not a.no_extras)
    B, m = r["indexes"], r["probes_total"]
    print(json.dumps({
        "metric": "batched lookups/s (%d indexes, 2^8..2^20 u64 keys, 2^10..2^18 probes each, hit 0.75)" % B,
        "value": r["lookups_per_s"], "unit": UNIT, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": r["graph_step_ms"], "higher_is_better": True, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "batched build + lookup, one CUDA graph", "indexes": B,
                   "keys_total": r["keys_total"], "probes_total": m, "k": a.batch_k},
        "gpu_launches": r["kernels_per_graph"] * a.steps, **r}), flush=True)


def _ev_ms(torch, fn, reps, warm=2):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def ranges_leg(gi, torch, dev, E=16, steps=5, layouts=None):
    """2^26 unique u32 keys, 2^24 inclusive ranges with E expected rows (CSR output),
    one call (count + scan + fill) per layout; sampled parity by numpy."""
    n, m = 1 << 26, 1 << 24
    seed = W.seed_for(2, 26)
    keys = W.unique_keys(n, 32, seed)
    kd = torch.from_numpy(keys.view(np.int32)).to(dev)
    rd = torch.arange(n, dtype=torch.int32, device=dev)
    lo, hi, w = W.ranges_with_expected_rows(n, m, E, 32, seed + E)
    lod, hid = torch.from_numpy(lo.view(np.int32)).to(dev), torch.from_numpy(hi.view(np.int32)).to(dev)
    off = torch.empty(m + 1, dtype=torch.int64, device=dev)
    order = np.argsort(keys, kind="stable")
    sk = keys[order]
    samp = np.random.default_rng(5).choice(m, size=4096, replace=False)
    out = {}
    for name, layout, k in layouts or (("sorted", gi.GI_SORTED, 0), ("EBS", gi.GI_EYTZINGER, 2),
                                       ("EKS k=16", gi.GI_EYTZINGER_KARY, 16)):
        idx = gi.gi_build(kd, rd, layout | gi.GI_KEY_U32, k)
        gi.gi_range_lookup(idx, lod, hid, off)
        total = int(off[-1].item())
        rows = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
        ms = _ev_ms(torch, lambda: gi.gi_range_lookup(idx, lod, hid, off, rows), steps)
        o = off.cpu().numpy().view(np.uint64)
        rr = rows.cpu().numpy().view(np.uint32)
        ok = True
        for i in samp:
            a, b = np.searchsorted(sk, lo[i], "left"), np.searchsorted(sk, hi[i], "right")
            ok &= bool(o[i + 1] - o[i] == b - a) and bool(np.array_equal(rr[o[i]:o[i + 1]], order[a:b]))
        out[name] = {"ms": ms, "ranges_per_s": m / ms * 1e3, "rows_per_s": total / ms * 1e3, "rows": total,
                     "sampled_parity_4096": ok}
        del rows
        gi.gi_destroy(idx)
    return {"n_keys": n, "key": "u32", "ranges": m, "expected_rows": E, "width": int(w), "layouts": out}


def run_ranges(a):
    """2^26 unique u32 keys, 2^24 inclusive ranges with 1, 16 and 256 expected rows,
    CSR output, for the sorted, Eytzinger and k-ary (16, 17) layouts and both
    range-fill strategies; one JSON line per case (count + scan + fill, one call)."""
    import torch

    import paper_2506_01576_gb300 as gi
    gi.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n, m = 1 << 26, 1 << 24
    seed = W.seed_for(2, 26)
    keys = W.unique_keys(n, 32, seed)
    kd = torch.from_numpy(keys.view(np.int32)).to(dev)
    rd = torch.arange(n, dtype=torch.int32, device=dev)
    for E in (1, 16, 256):
        lo, hi, w = W.ranges_with_expected_rows(n, m, E, 32, seed + E)
        lod, hid = torch.from_numpy(lo.view(np.int32)).to(dev), torch.from_numpy(hi.view(np.int32)).to(dev)
        off = torch.empty(m + 1, dtype=torch.int64, device=dev)
        for layout, k, fills in ((gi.GI_SORTED, 0, (0,)), (gi.GI_EYTZINGER, 2, (0, 1)),
                                 (gi.GI_EYTZINGER_KARY, 16, (0, 1)), (gi.GI_EYTZINGER_KARY, 17, (0, 1))):
            idx = gi.gi_build(kd, rd, layout | gi.GI_KEY_U32, k)
            gi.gi_range_lookup(idx, lod, hid, off)
            total = int(off[-1].item())
            out = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
            for fill in fills:
                gi.gi_set_option(idx, gi.GI_OPT_RANGE_FILL, fill)
                # a single call with the output: count + scan + fill
                ms = _ev_ms(torch, lambda: gi.gi_range_lookup(idx, lod, hid, off, out), a.steps)
                cnt_ms = _ev_ms(torch, lambda: gi.gi_range_lookup(idx, lod, hid, off), a.steps)
                print(json.dumps({"workload": "ranges", "E": E, "width": w,
                                  "layout": {0: "sorted", 1: "EBS", 2: "EKS"}[layout], "k": k,
                                  "fill": "level runs" if fill else "rank map", "ranges": m,
                                  "rows": total, "ms": ms, "count_scan_ms": cnt_ms,
                                  "ranges_per_s": m / ms * 1e3, "rows_per_s": total / ms * 1e3,
                                  "ms_per_expected_hit_per_2e18_ranges": ms / E / 64}), flush=True)
            del out
            gi.gi_destroy(idx)


def run_sizes(a):
    """Point lookups and builds over the index size: n = 2^10 .. 2^28 unique u64 keys,
    2^27 probes (hit rate 0.5, uniform) per size, textbook BS, EBS and EKS with
    k = 4, 5, 8, 9, 16, 17; build time of the k = 5 layout (hybrid sort and plain
    LSD) and of the sorted layout.  One JSON line per size."""
    import torch

    import paper_2506_01576_gb300 as gi
    gi.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    m = 1 << a.m_log
    out = torch.empty(m, dtype=torch.int32, device=dev)
    lo_log, hi_log = 10, 28
    for nl in range(lo_log, hi_log + 1):
        n = 1 << nl
        seed = W.seed_for(5, nl)
        keys = W.unique_keys(n, 64, seed)
        q = W.point_probes(keys, m, 0.5, 64, seed, seed + 1)
        kd = torch.from_numpy(keys.view(np.int64)).to(dev)
        rd = torch.arange(n, dtype=torch.int32, device=dev)
        qd = torch.from_numpy(q.view(np.int64)).to(dev)
        U = gi.GI_KEY_U64
        line = {"workload": "sizes", "n_log": nl, "probes": m, "lookups_per_s": {}, "build_ms": {}}
        for name, lay, k in (("BS", gi.GI_SORTED, 0), ("EBS", gi.GI_EYTZINGER, 0),
                             ("EKS4", gi.GI_EYTZINGER_KARY, 4), ("EKS5", gi.GI_EYTZINGER_KARY, 5),
                             ("EKS8", gi.GI_EYTZINGER_KARY, 8), ("EKS9", gi.GI_EYTZINGER_KARY, 9),
                             ("EKS16", gi.GI_EYTZINGER_KARY, 16), ("EKS17", gi.GI_EYTZINGER_KARY, 17)):
            idx = gi.gi_build(kd, rd, lay | U, k)
            ms = _ev_ms(torch, lambda: gi.gi_point_lookup(idx, qd, out), a.steps)
            line["lookups_per_s"][name] = m / ms * 1e3
            gi.gi_destroy(idx)
        for name, lay, k in (("EKS5", gi.GI_EYTZINGER_KARY, 5),
                             ("EKS5_lsd", gi.GI_EYTZINGER_KARY | gi.GI_BUILD_LSD, 5),
                             ("sorted", gi.GI_SORTED, 0)):
            line["build_ms"][name] = _ev_ms(
                torch, lambda: gi.gi_destroy(gi.gi_build(kd, rd, lay | U, k)), max(3, a.steps // 3))
        print(json.dumps(line), flush=True)
        del kd, rd, qd


_OPT_NAMES = {1: "group", 2: "per_thread", 3: "smem_levels", 4: "block", 5: "blocks_per_sm",
              6: "prefetch", 7: "early_exit", 8: "hot_levels", 9: "range_fill", 10: "reorder"}


def run_tune(a):
    """The autotuner (gi_tune) over the index size: n = 2^10 .. 2^28 unique u64 keys
    (even powers), 2^27 probes (hit rate 0.5, uniform); BS, EBS and EKS k = 5, 9, 17,
    each timed with the default knobs and with the knobs gi_tune picks on a 2^22-probe
    sample, and the fastest layout per size either way (the paper's composite
    strategy, Section 9); then the layout, k and knobs gi_build_tuned picks on the same
    sample.  One JSON line per size."""
    import torch

    import paper_2506_01576_gb300 as gi
    gi.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    m = 1 << a.m_log
    out = torch.empty(m, dtype=torch.int32, device=dev)
    for nl in range(10, 29, 2):
        n = 1 << nl
        seed = W.seed_for(5, nl)
        keys = W.unique_keys(n, 64, seed)
        q = W.point_probes(keys, m, 0.5, 64, seed, seed + 1)
        kd = torch.from_numpy(keys.view(np.int64)).to(dev)
        rd = torch.arange(n, dtype=torch.int32, device=dev)
        qd = torch.from_numpy(q.view(np.int64)).to(dev)
        sample = qd[: min(m, 1 << 22)]
        line = {"workload": "tune", "n_log": nl, "probes": m, "tune_sample": int(sample.numel()),
                "default": {}, "tuned": {}, "knobs": {}, "trials": {}, "tune_s": {}}
        for name, lay, k in (("BS", gi.GI_SORTED, 0), ("EBS", gi.GI_EYTZINGER, 0),
                             ("EKS5", gi.GI_EYTZINGER_KARY, 5), ("EKS9", gi.GI_EYTZINGER_KARY, 9),
                             ("EKS17", gi.GI_EYTZINGER_KARY, 17)):
            idx = gi.gi_build(kd, rd, lay | gi.GI_KEY_U64, k)
            ms = _ev_ms(torch, lambda: gi.gi_point_lookup(idx, qd, out), a.steps)
            line["default"][name] = m / ms * 1e3
            t0 = time.perf_counter()
            r = gi.gi_tune(idx, sample, 0, gi.GI_TUNE_APPLY)
            line["tune_s"][name] = time.perf_counter() - t0
            ms = _ev_ms(torch, lambda: gi.gi_point_lookup(idx, qd, out), a.steps)
            line["tuned"][name] = m / ms * 1e3
            line["knobs"][name] = {_OPT_NAMES[o]: int(r.options[o]) for o in range(1, 11)
                                   if r.options[o] != r.start_options[o]}
            line["trials"][name] = int(r.trials)
            gi.gi_destroy(idx)
        line["fastest_default"] = max(line["default"], key=line["default"].get)
        line["fastest_tuned"] = max(line["tuned"], key=line["tuned"].get)
        # the layout and k chosen by the library itself (gi_build_tuned)
        t0 = time.perf_counter()
        idx, r = gi.gi_build_tuned(kd, rd, gi.GI_KEY_U64, sample)
        info = gi.gi_get_info(idx)
        ms = _ev_ms(torch, lambda: gi.gi_point_lookup(idx, qd, out), a.steps)
        line["build_tuned"] = {"layout": {0: "sorted", 1: "EBS", 2: "EKS"}[info.layout], "k": int(info.k),
                               "lookups_per_s": m / ms * 1e3, "seconds": time.perf_counter() - t0}
        gi.gi_destroy(idx)
        print(json.dumps(line), flush=True)
        del kd, rd, qd, sample


def run_dups(a):
    """Section 8.11 / Fig 25 shape: 2^26 u64 keys, each distinct key replicated r
    times; 2^20 point queries as ranges [x, x] returning every occurrence."""
    import torch

    import paper_2506_01576_gb300 as gi
    gi.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n, m = 1 << 26, 1 << 20
    for r in (1, 4, 16, 64, 256, 1024):
        keys = W.duplicate_keys(n // r, r, 64, 7)
        kd = torch.from_numpy(keys.view(np.int64)).to(dev)
        rd = torch.arange(len(keys), dtype=torch.int32, device=dev)
        rng = np.random.default_rng(r)
        q = keys[rng.integers(0, len(keys), size=m)]
        qd = torch.from_numpy(q.view(np.int64)).to(dev)
        off = torch.empty(m + 1, dtype=torch.int64, device=dev)
        for layout, k in ((gi.GI_SORTED, 0), (gi.GI_EYTZINGER, 2), (gi.GI_EYTZINGER_KARY, 5),
                          (gi.GI_EYTZINGER_KARY, 9)):
            idx = gi.gi_build(kd, rd, layout | gi.GI_KEY_U64, k)
            gi.gi_range_lookup(idx, qd, qd, off)
            total = int(off[-1].item())
            out = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
            ms = _ev_ms(torch, lambda: gi.gi_range_lookup(idx, qd, qd, off, out), a.steps)
            print(json.dumps({"workload": "duplicates", "replicas": r, "layout": {0: "sorted", 1: "EBS", 2: "EKS"}[layout],
                              "k": k, "queries": m, "rows": total, "ms": ms,
                              "queries_per_s": m / ms * 1e3, "rows_per_s": total / ms * 1e3}), flush=True)
            del out
            gi.gi_destroy(idx)
        del kd, rd


def run_skew(a):
    """Sections 8.9-8.10 shapes on 2^26 u64 keys: 2^25 probes at hit rate 0.5 with
    hits uniform, Zipf(s) for s up to 2.0, or the uniform probes pre-sorted; BS, EBS,
    EKS single (k = 5) and EKS group (k = 9, 8 lanes), each with and without local
    lookup reordering.  One JSON line per case."""
    import torch

    import paper_2506_01576_gb300 as gi
    gi.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n, m = 1 << 26, 1 << 25
    seed = W.seed_for(1, 26)
    keys = W.unique_keys(n, 64, seed)
    kd = torch.from_numpy(keys.view(np.int64)).to(dev)
    rd = torch.arange(n, dtype=torch.int32, device=dev)
    out = torch.empty(m, dtype=torch.int32, device=dev)
    configs = [("BS", gi.GI_SORTED, 0, {}), ("EBS", gi.GI_EYTZINGER, 2, {gi.GI_OPT_PER_THREAD: 4}),
               ("EKS single k=5", gi.GI_EYTZINGER_KARY, 5, {gi.GI_OPT_GROUP: 1}),
               ("EKS group k=9", gi.GI_EYTZINGER_KARY, 9, {gi.GI_OPT_GROUP: 8})]
    built = {}
    for name, layout, k, opts in configs:
        built[name] = gi.gi_build(kd, rd, layout | gi.GI_KEY_U64, k)
        for o, v in opts.items():
            gi.gi_set_option(built[name], o, v)
    dists = [("uniform", 0.0)] + [("zipf", s) for s in (0.5, 0.99, 1.25, 1.5, 2.0)] + [("sorted", 0.0)]
    for dname, zs in dists:
        q = W.point_probes(keys, m, 0.5, 64, seed, seed + 5, dist="zipf" if dname == "zipf" else "uniform",
                           zipf_s=zs if zs else 0.99)
        if dname == "sorted":
            q = np.sort(q)
        qd = torch.from_numpy(q.view(np.int64)).to(dev)
        for name, layout, k, opts in configs:
            idx = built[name]
            for ro in (0, 1):
                gi.gi_set_option(idx, gi.GI_OPT_REORDER, ro)
                ms = _ev_ms(torch, lambda: gi.gi_point_lookup(idx, qd, out), a.steps)
                print(json.dumps({"workload": "skew", "probes": dname, "zipf_s": zs, "index": name,
                                  "reorder": ro, "ms": ms, "lookups_per_s": m / ms * 1e3}), flush=True)
        del qd
    for v in built.values():
        gi.gi_destroy(v)


def serving_sweep(gi, torch, dev, n_indexes, min_log, max_log, rates, seconds, pool_size, repeats=1,
                  serial_max_requests=20000, seed=77, threads=4):
    """The serving form at several offered loads, driven by the library's native
    open-loop load generator: resident indexes of log-uniform sizes (u64 keys, EKS
    k = 5), Poisson arrivals, requests of 1..2^16 probes (log-uniform), 80% point
    (hit rate 0.5), 20% range (16 expected rows).  For each load: the continuous-
    batching server (gi_server_replay) and, as the baseline, one request at a time
    through the plain calls (gi_replay_serial; its schedule cut to the first
    `serial_max_requests` arrivals past its capacity).  Returns one dict per run."""
    rng = np.random.default_rng(seed)
    sizes = np.exp2(rng.uniform(min_log, max_log, size=n_indexes)).astype(np.int64)
    idx, pool = [], []
    layout = gi.GI_EYTZINGER_KARY | gi.GI_KEY_U64
    per_index = max(4, pool_size // n_indexes)
    pin = lambda x: torch.from_numpy(x.view(np.int64)).pin_memory()
    for i, n in enumerate(sizes):
        keys = W.unique_keys(int(n), 64, W.seed_for(5, 27, i))
        kd = torch.from_numpy(keys.view(np.int64)).to(dev)
        rd = torch.arange(int(n), dtype=torch.int32, device=dev)
        idx.append(gi.gi_build(kd, rd, layout, 5))
        del kd, rd
        for _ in range(per_index):
            m = int(np.exp2(rng.uniform(0, 16)))
            if rng.random() < 0.8:
                q = W.point_probes(keys, m, 0.5, 64, W.seed_for(5, 27, i), int(rng.integers(1 << 30)))
                pool.append((i, gi.GI_REQ_POINT, pin(q), torch.empty(m, dtype=torch.int32).pin_memory(),
                             None, None, 0))
            else:
                lo, hi, _ = W.ranges_with_expected_rows(int(n), m, 16, 64, int(rng.integers(1 << 30)))
                cap = 32 * m + 1024
                pool.append((i, gi.GI_REQ_RANGE, pin(lo), torch.empty(cap, dtype=torch.int32).pin_memory(),
                             pin(hi), torch.empty(m + 1, dtype=torch.int64).pin_memory(), cap))
        del keys
    torch.cuda.synchronize()
    order = rng.permutation(len(pool))
    sizes_m = np.array([p[2].numel() for p in pool])
    mean_m = float(np.mean(sizes_m))
    results = []

    def schedule(rate, rep, limit=None):
        r2 = np.random.default_rng(int(rate) * 7 + rep)
        cnt = int(rate * seconds * 1.2) + 16
        t = np.cumsum(r2.exponential(1.0 / rate, size=cnt))
        t = t[t < seconds]
        if limit is not None:
            t = t[:limit]
        which = order[np.arange(len(t)) % len(pool)]
        reqs = gi.make_requests([pool[j] for j in which])
        return reqs, (t * 1e9).astype(np.int64), int(sizes_m[which].sum())

    def summary(mode, rate, rep, lat, st, wall, probes, nreq):
        ok = lat >= 0
        l = lat[ok] / 1e6
        return {"mode": mode, "offered_requests_per_s": rate, "offered_lookups_per_s": rate * mean_m,
                "repeat": rep, "requests": int(nreq), "lookups_per_s": probes / wall,
                "requests_per_s": nreq / wall, "p50_ms": float(np.percentile(l, 50)),
                "p99_ms": float(np.percentile(l, 99)), "wall_s": wall,
                "capacity_exceeded": int((st == gi.GI_ERR_CAPACITY).sum())}

    server = gi.gi_server_create(idx, 2 << 30, 3)
    for rate in rates:
        for rep in range(repeats):
            reqs, arr, probes = schedule(rate, rep)
            lat, st, wall = gi.gi_server_replay(server, reqs, arr, threads)
            results.append(summary("server", rate, rep, lat, st, wall, probes, len(arr)))
    gi.gi_server_destroy(server)
    for rate in rates:
        for rep in range(repeats):
            reqs, arr, probes = schedule(rate, rep, serial_max_requests)
            lat, st, wall = gi.gi_replay_serial(idx, reqs, arr)
            results.append(summary("one at a time", rate, rep, lat, st, wall, probes, len(arr)))
    for ix in idx:
        gi.gi_destroy(ix)
    meta = {"indexes": n_indexes, "keys_total": int(sizes.sum()), "index_log2_range": [min_log, max_log],
            "mean_probes_per_request": mean_m, "request_pool": len(pool), "seconds_per_load": seconds,
            "submit_threads": threads}
    return meta, results


def run_serving(a):
    """Serving form (the survey's C5): 64 resident indexes of 2^20..2^27 u64 keys, an
    offered-load sweep past saturation, every load twice; one JSON line per run."""
    import torch

    import paper_2506_01576_gb300 as gi
    gi.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rates = [float(x) for x in a.serve_rates.split(",")]
    meta, results = serving_sweep(gi, torch, dev, a.serve_indexes, a.serve_min_log, a.serve_max_log, rates,
                                  a.serve_seconds, 3000, repeats=2)
    for r in results:
        r.update(meta)
        r["workload"] = "serve"
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    args = parse()
    if args.workload == "serve":
        run_serving(args)
    elif args.workload == "skew":
        run_skew(args)
    elif args.workload == "ranges":
        run_ranges(args)
    elif args.workload == "dups":
        run_dups(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "sizes":
        run_sizes(args)
    elif args.workload == "tune":
        run_tune(args)
    elif args.probe_sweep:
        probe_sweep()
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
