"""Host logic of the multi-GPU replica benchmark, on CPU with gloo ranks.

Each rank runs an independent replica; the only exchange is the gather of
every rank's timed-region length, and the whole-job value is all units over
the slowest rank."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = 100.0 + 50.0 * rank  # rank 1 is the slowest
    times = bench.gather_times(ms, world, "cpu")
    value, ms_per_step = bench.aggregate(None, times, 10)
    q.put((rank, times, value, ms_per_step))
    dist.destroy_process_group()


def test_two_gloo_replicas_aggregate_over_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, times, value, ms_per_step in out:
        assert times == [100.0, 150.0]
        # 2 replicas x 10 steps over the slowest rank's 150 ms
        assert value == pytest.approx(2 * 10 / 0.150)
        assert ms_per_step == pytest.approx(15.0)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.gather_times(12.5, 1, "cpu") == [12.5]
    value, ms_per_step = bench.aggregate(None, [12.5], 5)
    assert value == pytest.approx(400.0) and ms_per_step == pytest.approx(2.5)
