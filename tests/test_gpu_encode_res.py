"""GPU parity of the fixed-quality encoder that keeps each block in registers
(int8, int16 and float32 blocks of at most 256 samples, arrays of more than
4,096 blocks): byte-identical containers against the oracle.

It decides each block's stream on its own registers and hands the decision
to the next team, so the cases cross every boundary that exchange has: team
pairs inside a warp, warps inside a CTA, the halo block before each tile,
the first block of the array, shards whose first block is not the array's,
ragged last blocks, blocks whose threads hold fewer groups than others, and
streams that change from block to block; both format options as well.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1303_4994_gb300 import apax as A
from paper_1303_4994_gb300 import build as B
from paper_1303_4994_gb300 import shard as S

pytestmark = pytest.mark.gpu

NP = {1: np.int8, 2: np.int16, 4: np.float32}


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    A.lib()
    torch.cuda.init()


def _mixed(dt, n, rng):
    """Blocks alternating between noise, a random walk, a parabola and a
    Nyquist-band tone, in runs of varying length, so that the stream each
    block chooses changes often."""
    t = np.arange(n, dtype=np.float64)
    kind = (t // (64 * (1 + (t // 5000) % 3))) % 4
    v = np.where(kind == 0, rng.standard_normal(n),
                 np.where(kind == 1, np.cumsum(rng.standard_normal(n)) * 0.3,
                          np.where(kind == 2, 1e-4 * ((t % 97) - 40) ** 2,
                                   (-1.0) ** t * (5 + np.sin(t * 0.01)))))
    if dt == 4:
        return (v * np.exp(rng.uniform(-6, 6))).astype(np.float32)
    info = np.iinfo(NP[dt])
    amp = 20 if dt == 1 else 3000
    return np.clip(np.rint(v * amp), info.min, info.max).astype(NP[dt])


@pytest.mark.parametrize("dt", [1, 2, 4])
@pytest.mark.parametrize("N", [64, 100, 136, 256])
def test_register_encoder_parity(dt, N):
    rng = np.random.default_rng(dt * 1000 + N)
    nb = 4096 + 700 + int(rng.integers(0, 300))
    n = N * nb - int(rng.integers(0, N))  # a ragged last block
    x = _mixed(dt, n, rng)
    xt = torch.from_numpy(x).cuda()
    for code in (0, 300, 1536, int(rng.integers(0, 4096))):
        want = O.encode(x, N, O.MODE_FQ, 1, 1, code, threads=0)
        got = A.encode(xt, N, A.FIXED_QUALITY, (1, 1), code)
        gb = got.cpu().numpy().tobytes()
        assert len(gb) == len(want)
        if gb != want:
            diff = np.nonzero(np.frombuffer(gb, np.uint8) != np.frombuffer(want, np.uint8))[0]
            raise AssertionError(f"code {code}: container differs at byte {diff[0]} of {len(want)}")


@pytest.mark.parametrize("fmt", [A.FORMAT_GROUP8, A.FORMAT_SUM_STREAM,
                                 A.FORMAT_GROUP8 | A.FORMAT_SUM_STREAM])
def test_register_encoder_formats(fmt):
    rng = np.random.default_rng(fmt)
    for dt, N in ((4, 256), (2, 64), (1, 136)):
        n = N * 5000 + 33
        x = _mixed(dt, n, rng)
        want = O.encode(x, N, O.MODE_FQ, 1, 1, 700, threads=0, fmt=fmt)
        got = A.encode(torch.from_numpy(x).cuda(), N, A.FIXED_QUALITY, (1, 1), 700, fmt=fmt)
        assert got.cpu().numpy().tobytes() == want, (dt, N)


def test_register_encoder_shards():
    # shards of 5,000+ blocks: the first tile's halo is the block before the
    # shard, read from the caller's halo element range
    rng = np.random.default_rng(9)
    N = 256
    x = _mixed(4, N * 15000 + 77, rng)
    n, nb = x.size, (x.size + N - 1) // N
    xt = torch.from_numpy(x).cuda()
    p = A.params(N, A.FIXED_QUALITY, (1, 1), 2048)
    want = O.encode(x, N, O.MODE_FQ, 1, 1, 2048, threads=0)
    ranges = S.block_ranges(nb, 3)
    shards = []
    for b0, b1 in ranges:
        e0, e1 = S.halo_elements(n, N, b0, b1)
        shards.append(A.encode_shard(xt[e0:e1].contiguous(), n, p, b0, b1))
    assert A.merge_shards(shards, ranges, A.F32, n, p).cpu().numpy().tobytes() == want


def test_register_encoder_nonfinite_and_device_code():
    N = 256
    x = np.cumsum(np.random.default_rng(3).standard_normal(N * 6000)).astype(np.float32)
    x[N * 4321 + 17] = np.nan
    xt = torch.from_numpy(x).cuda()
    r = A.encode_status(xt, A.params(N, A.FIXED_QUALITY, (1, 1), 512))
    assert r.status == -8
    # the code read on the device (profile -> encode without a host round trip)
    x[N * 4321 + 17] = 0.0
    xt = torch.from_numpy(x).cuda()
    pws, pts, summ = A.profile_buffers(xt, N, 16)
    A.profile_into(xt, N, list(A.DEFAULT_CANDIDATES), 0.9999, pws, pts, summ)
    p = A.params(N, A.FIXED_QUALITY)
    out = torch.empty(A.encoded_size(A.F32, x.size, p), dtype=torch.uint8, device="cuda")
    ws = torch.empty(A.workspace_size(A.F32, x.size, p), dtype=torch.uint8, device="cuda")
    res = A.new_result("cuda")
    A.encode_into(xt, p, out, ws, res, summary=summ)
    rr = A.read_result(res)
    code = int(A.read_summary(summ).recommended_code)
    assert rr.status == 0
    assert out[:rr.bytes].cpu().numpy().tobytes() == O.encode(x, N, O.MODE_FQ, 1, 1, code, threads=0)
