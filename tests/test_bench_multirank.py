"""Host logic of the multi-rank benchmark on CPU: two gloo ranks, the job time is
the slowest rank's and the throughput counts every rank's solves (weak scaling,
no collective on the data path)."""
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


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [4000.0, 5000.0][rank]
    m = bench.reduce_max(local_ms)
    rate = bench.whole_job_rate(world, 2, m)
    out[rank] = (m, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_slowest_time_and_count_all_solves():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        m, rate = out[r]
        assert m == 5000.0
        assert rate == pytest.approx(2 * 2 * 1000.0 / 5000.0)


def test_single_process_reduce_is_identity():
    import bench
    assert bench.reduce_max(12.5) == 12.5
    assert bench.whole_job_rate(1, 3, 6000.0) == pytest.approx(0.5)
