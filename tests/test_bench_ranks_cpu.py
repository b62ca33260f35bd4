"""The multi-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1, each a replica with
its own device time and unit count; the job's time is the slowest rank's and its units the
sum (weak scaling, no collective on the data path)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, u = bench.aggregate_over_ranks(100.0 + 50.0 * rank, 7 + rank, dist, "cpu")
    out[rank] = (t, u)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_max_time_sum_units():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        assert dict(out) == {0: (150.0, 15), 1: (150.0, 15)}


def test_single_rank_aggregation_is_identity():
    import bench

    assert bench.aggregate_over_ranks(12.5, 3, None, "cpu") == (12.5, 3)
