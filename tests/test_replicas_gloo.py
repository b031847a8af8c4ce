"""The multi-GPU form is N independent replicas (one index per rank, no data-path
collective).  Its only cross-rank step is the timing: every rank's time is
reduced with MAX and the whole-job rate counts every rank's lookups.  Checked
here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 20.0][rank]  # the second replica is slower
    got = bench.max_over_ranks(ms)
    rate = bench.job_throughput(1 << 27, world, 10, got)
    q.put((rank, got, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_slowest_time_and_total_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, rate in res:
        assert got == 20.0
        assert rate == pytest.approx((1 << 27) * 2 * 10 / 0.020)


def test_single_process_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(7.0) == 7.0
    assert bench.job_throughput(100, 1, 2, 1000.0) == 200.0
