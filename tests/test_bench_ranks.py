"""The bench's multi-rank logic on CPU: two gloo ranks each time their own
array (weak scaling, no data-path collective); every rank ends up with the
slowest rank's timings and rank 0's whole-job throughput counts both ranks'
bytes over that time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [1.0 + rank, 10.0 - rank, 3.0 * (rank + 1)]
        got = bench.max_over_ranks(mine, "cpu", world)
        out[rank] = (got, bench.aggregate_gbs(1e9, world, got[0]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_max_and_aggregate():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(2):
            got, gbs = out[r]
            assert got == [2.0, 10.0, 6.0]
            assert gbs == pytest.approx(2 * 1e9 / 2.0 / 1e6)
