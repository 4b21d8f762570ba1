"""The multi-rank timing logic of bench.py (one replica per GPU; the job's
time is the slowest rank's; value sums the ranks) on two gloo ranks, CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [1200.0, 1500.0][rank]                       # rank 1 is slower
    m = bench.max_over_ranks(ms, world, device="cpu")
    v = bench.job_throughput(5 * 30, m, world)
    q.put((rank, m, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [1500.0, 1500.0]
    assert out[0][2] == pytest.approx(2 * 150 / 1.5) and out[0][2] == out[1][2]


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_throughput(100, 2000.0, 1) == pytest.approx(50.0)
