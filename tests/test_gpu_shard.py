"""GPU parity of sharded encoding (one array split into block ranges).

apax_encode_shard encodes a block range from the range's samples and the
halo block before it; its container is the sub-array's own container, so it
decodes alone; apax_merge_shards and apax_shard_rebase assemble the shards
into the container a single apax_encode call writes, byte for byte, which
is also the oracle's.  The multi-rank test runs two processes (gloo for the
exchange of payload sizes); both drive their kernels on this one GPU, and
no kernel waits for another.
"""
import os
import socket

import numpy as np
import pytest
import torch

import oracle as O
from paper_1303_4994_gb300 import apax as A
from paper_1303_4994_gb300 import build as B
from paper_1303_4994_gb300 import shard as S
from paper_1303_4994_gb300 import synth

pytestmark = pytest.mark.gpu

TT = {np.dtype(np.int16): torch.int16, np.dtype(np.int32): torch.int32,
      np.dtype(np.float32): torch.float32, np.dtype(np.float64): torch.float64}


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    A.lib()
    torch.cuda.init()


def _shards(xt, n, p, ranges):
    out = []
    for b0, b1 in ranges:
        e0, e1 = S.halo_elements(n, p.block_size, b0, b1)
        out.append(A.encode_shard(xt[e0:e1].contiguous(), n, p, b0, b1))
    return out


@pytest.mark.parametrize("case", ["f32_fq", "i16_fr", "f64_fq", "f32_fr_predict", "t1_fr", "field"])
@pytest.mark.parametrize("k", [2, 3, 7])
def test_shards_merge_to_single_call(case, k):
    rng = np.random.default_rng(hash((case, k)) % 1000)
    if case == "f32_fq":
        x, N, p = (np.cumsum(rng.standard_normal(256 * 300 + 77)).astype(np.float32), 256,
                   A.params(256, A.FIXED_QUALITY, (1, 1), 1100))
    elif case == "i16_fr":
        x, N, p = synth.sensor_trace(64 * 900 + 5, seed=4), 64, A.params(64, A.FIXED_RATE, (4, 1))
    elif case == "f64_fq":
        x, N, p = (np.cumsum(rng.standard_normal(1000 * 50 + 3)).astype(np.float64), 1000,
                   A.params(1000, A.FIXED_QUALITY, (1, 1), 2560))
    elif case == "f32_fr_predict":
        x, N, p = (np.cumsum(rng.standard_normal(256 * 200)).astype(np.float32), 256,
                   A.params(256, A.FIXED_RATE, (6, 1), 0, A.SEARCH_PREDICT))
    elif case == "t1_fr":  # shards of 40,000 blocks: the block-per-thread encoder
        x, N, p = synth.sensor_trace(64 * 40000 * k, seed=5), 64, A.params(64, A.FIXED_RATE, (4, 1))
    else:
        x, N, p = synth.grf2d(1024, 1024, seed=7).reshape(-1), 256, A.params(256, A.FIXED_QUALITY,
                                                                              (1, 1), 2048)
    n = x.size
    nb = (n + N - 1) // N
    xt = torch.from_numpy(x).cuda()
    dc = A.TORCH_CODE[xt.dtype]
    whole = A.encode(xt, N, p.mode, (p.rate_num, p.rate_den), p.atten_code, search=p.search)
    want = O.encode(x, N, p.mode, p.rate_num, p.rate_den, p.atten_code, threads=0,
                    search=p.search)
    assert whole.cpu().numpy().tobytes() == want
    ranges = S.block_ranges(nb, k)
    shards = _shards(xt, n, p, ranges)
    merged = A.merge_shards(shards, ranges, dc, n, p)
    assert merged.cpu().numpy().tobytes() == want
    host = S.merge_host([c.cpu().numpy().tobytes() for c in shards], ranges, n,
                        p.mode == A.FIXED_QUALITY)
    assert host == want
    # every shard decodes on its own to its slice of the array
    y = A.decode(whole, xt.dtype, n)
    for c, (b0, b1) in zip(shards, ranges):
        ns = A.shard_elements(n, N, b0, b1)
        ys = A.decode(c, xt.dtype, ns)
        assert torch.equal(ys.view(torch.uint8), y[b0 * N:b0 * N + ns].view(torch.uint8))
    # distributed form: a rebased shard table is the whole container's slice
    if p.mode == A.FIXED_QUALITY:
        fq = True
        pays = [S.payload_bytes(c.numel(), b1 - b0, fq) for c, (b0, b1) in zip(shards, ranges)]
        offs, _ = S.exclusive_offsets(pays)
        tab = np.frombuffer(want, np.uint32, nb, 40)
        for c, (b0, b1), o in zip(shards, ranges, offs):
            A.shard_rebase(c, b1 - b0, o // 4)
            got = np.frombuffer(c.cpu().numpy().tobytes(), np.uint32, b1 - b0, 40)
            assert np.array_equal(got, tab[b0:b1])


def test_shard_argument_checks():
    x = torch.zeros(1000, dtype=torch.float32, device="cuda")
    p = A.params(64, A.FIXED_QUALITY, (1, 1), 0)
    for b0, b1 in ((3, 3), (5, 2), (0, 17)):  # empty, reversed, past the 16 blocks
        with pytest.raises(A.ApaxError) as e:
            A.encode_shard(x, 1000, p, b0, b1)
        assert e.value.status == -1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        B.build()
        A.lib()
        x = synth.grf2d(1024, 2048, seed=8).reshape(-1)
        N, p = 256, A.params(256, A.FIXED_QUALITY, (1, 1), 1792)
        n, nb = x.size, (x.size + 255) // 256
        b0, b1 = S.block_ranges(nb, world)[rank]
        e0, e1 = S.halo_elements(n, N, b0, b1)
        xt = torch.from_numpy(x[e0:e1].copy()).cuda()  # this rank holds only its range
        c = A.encode_shard(xt, n, p, b0, b1)
        pay = S.payload_bytes(c.numel(), b1 - b0, True)
        off, total, sizes = S.exchange_payload_sizes(pay)  # the exchange step
        A.shard_rebase(c, b1 - b0, off // 4)
        torch.cuda.synchronize()
        gathered = [None] * world
        dist.all_gather_object(gathered, (c.cpu().numpy().tobytes(), (b0, b1)))
        ok = True
        if rank == 0:
            want = O.encode(x, N, O.MODE_FQ, 1, 1, 1792, threads=0)
            tab = np.frombuffer(want, np.uint32, nb, 40)
            poff = 40 + S.table_bytes(nb)
            for cb, (c0, c1) in gathered:
                ok &= np.array_equal(np.frombuffer(cb, np.uint32, c1 - c0, 40), tab[c0:c1])
            pays = [cb[40 + S.table_bytes(c1 - c0):] for cb, (c0, c1) in gathered]
            ok &= b"".join(pays) == want[poff:]
            ok &= total == len(want) - poff
        out[rank] = bool(ok)
    finally:
        dist.destroy_process_group()


def test_two_processes_exchange_and_rebase():
    ctx = torch.multiprocessing.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        assert out[0] and out[1]
