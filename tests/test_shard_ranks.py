"""Sharding one array over ranks, on CPU (two and three gloo ranks).

Each rank takes a contiguous block range (block_ranges), builds its shard
container from the oracle's packets of those blocks (the halo block before
the range fixes the first block's stream decision), exchanges its payload
size with the others (all-gather), and rank 0 merges the gathered shards
(merge_host).  The merged container must equal the oracle's single-call
container byte for byte, and every shard must decode on its own to its
slice of the array.  This checks the range split, the exchange step and the
offset rebase without a GPU; tests/test_gpu_shard.py runs the kernels.
"""
import os
import socket
import struct

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_1303_4994_gb300 import shard as S


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _oracle_shard(x, N, mode, num, den, code, b0, b1):
    """A shard container (the sub-array's container) from the oracle's
    packets of blocks [b0, b1) of x."""
    n = x.size
    pk = O.encode_blocks(x, N, mode, num, den, code, b0, b1)
    ns = min(b1 * N, n) - b0 * N
    head = bytearray(O.encode(x[:0], N, mode, num, den, code)[:40])
    struct.pack_into("<Q", head, 20, ns)
    payload = b"".join(pk)
    struct.pack_into("<Q", head, 28, len(payload))
    table = b""
    if mode == O.MODE_FQ:
        offs = np.cumsum([0] + [len(p) // 4 for p in pk[:-1]])
        table = struct.pack(f"<{len(pk)}I", *offs.tolist())
        table += b"\0" * (S.table_bytes(len(pk)) - len(table))
    return bytes(head) + table + payload


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(5)
        results = []
        for dt, N, n, mode, rate, code in ((np.float32, 64, 64 * 37 + 13, O.MODE_FQ, (1, 1), 900),
                                           (np.int16, 128, 128 * 29, O.MODE_FR, (4, 1), 0),
                                           (np.float64, 64, 64 * 40 + 1, O.MODE_FQ, (1, 1), 1536)):
            x = (np.cumsum(rng.standard_normal(n)) * 300).astype(dt)
            nb = (n + N - 1) // N
            b0, b1 = S.block_ranges(nb, world)[rank]
            mine = _oracle_shard(x, N, mode, rate[0], rate[1], code, b0, b1)
            fq = mode == O.MODE_FQ
            pay = S.payload_bytes(len(mine), b1 - b0, fq)
            off, total, sizes = S.exchange_payload_sizes(pay)
            # this shard decodes on its own to its slice of the array
            ns = min(b1 * N, n) - b0 * N
            y = O.decode(mine, dt, ns)
            full = O.encode(x, N, mode, rate[0], rate[1], code)
            yf = O.decode(full, dt, n)
            own = bool(np.array_equal(y.view(np.uint8), yf[b0 * N:b0 * N + ns].view(np.uint8)))
            gathered = [None] * world
            dist.all_gather_object(gathered, (mine, (b0, b1)))
            merged = S.merge_host([g[0] for g in gathered], [g[1] for g in gathered], n, fq)
            results.append((own, merged == full, off == sum(sizes[:rank]), total == sum(sizes)))
        out[rank] = results
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_shard_exchange_merge(world):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(world):
            assert all(all(v) for v in out[r]), out[r]


def test_block_ranges_and_halo():
    assert S.block_ranges(10, 3) == [(0, 3), (3, 6), (6, 10)]
    assert S.block_ranges(2, 3) == [(0, 0), (0, 1), (1, 2)]
    assert S.halo_elements(1000, 64, 0, 4) == (0, 256)
    assert S.halo_elements(1000, 64, 4, 16) == (192, 1000)
    assert S.exclusive_offsets([5, 0, 7]) == ([0, 5, 5], 12)
