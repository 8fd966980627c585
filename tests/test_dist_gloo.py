"""The multi-rank path of bench.py on the CPU: two gloo ranks, each with its
own boxes, agree on the job's step time (the maximum over ranks) and the
whole-job rate (all ranks' boxes over that time)."""
from __future__ import annotations

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
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 135.5][rank]
    agg = bench.aggregate_step_ms(ms, world, torch.device("cpu"))
    dist.barrier()
    out[rank] = agg
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == out[1] == 135.5
        nbox = 512
        assert abs(2 * nbox / (out[0] / 1e3) - 7557.19) < 0.1   # whole-job boxes/s for 2 ranks


def test_single_rank_passthrough():
    import torch
    import bench
    assert bench.aggregate_step_ms(42.0, 1, torch.device("cpu")) == 42.0
