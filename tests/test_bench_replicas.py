"""The multi-GPU path of bench.py (independent replicas, weak scaling): the whole-job value is
the items of all ranks over the slowest rank's time.  Run as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench.dist_env() == (ws, rank, rank)
    local_ms = [120.0, 200.0][rank]      # rank 1 is the slow one
    dist.barrier()
    value, max_ms = bench.job_throughput(local_ms, items_per_rank=1024, steps=10, ws=ws)
    out[rank] = (value, max_ms)
    dist.destroy_process_group()


def test_job_throughput_takes_the_slowest_rank_over_two_gloo_ranks():
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(ws):
        value, max_ms = res[r]
        assert max_ms == pytest.approx(200.0)
        assert value == pytest.approx(2 * 1024 * 10 / 0.2)


def test_job_throughput_single_rank():
    import bench
    value, ms = bench.job_throughput(50.0, 100, 4, 1)
    assert ms == 50.0 and value == pytest.approx(100 * 4 / 0.05)
