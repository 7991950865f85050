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


def test_reference_arm_line(monkeypatch):
    # the reference arm (the oracle on host cores) prints one line with the
    # contract's keys on rank 0 and nothing elsewhere; the oracle timing is
    # replaced by fixed samples so the test stays fast
    import types

    samples = iter([{"value": v, "sample": "stub", "cores": 8, "cpu": "stub cpu", "seconds": 1.0}
                    for v in (1.0, 2.0, 4.0, 6.0)])
    seen = []

    def stub(rows=bench.CPU_ROWS, threads=0, x=None):
        seen.append((rows, threads, None if x is None else x.shape))
        return next(samples)

    monkeypatch.setattr(bench, "cpu_baseline", stub)
    args = types.SimpleNamespace(steps=2, warmup=2)
    assert bench.run_reference(args, 1, 2) is None
    line = bench.run_reference(args, 0, 2)
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] == 5.0 and line["n_gpus"] == 2 and line["steps"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == 5.0
    assert line["cpu_baseline"]["cores"] == 8
    # the same sample as the GPU arm's cpu_baseline: the field's first rows,
    # on all cores
    assert all(r == bench.CPU_ROWS and t == 0 and shp == (bench.CPU_ROWS, 4096)
               for r, t, shp in seen)
    assert line["e2e"] == {"value": 5.0, "unit": "GB/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    for k in ("unit", "warmup", "higher_is_better", "scaling", "vs_baseline", "dtype", "data",
              "config"):
        assert k in line


def test_cpu_model_named():
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()


def test_committed_traffic_figures_are_read():
    # the roofline's `traffic` comes from the committed ncu summary: the
    # dominant kernel (the sweep) has a per-launch DRAM figure close to one
    # read of the 64 MiB input (no re-reads); a kernel changed since its
    # capture has none (null in the bench line)
    xb = 4096 * 4096 * 4
    assert xb <= bench._traffic("profile") < 1.1 * xb
    for k in ("encode", "decode"):
        t = bench._traffic(k)
        assert t is None or (isinstance(t, int) and t > 0), k
    assert bench._traffic("no_such_kernel") is None
