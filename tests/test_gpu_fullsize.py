"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times.  The GPU runs the whole array; the oracle's threaded drivers (the same
per-block routines on every host core, contiguous block ranges) produce the
whole expected result, compared byte for byte and bit for bit:

* float32 4096 x 4096 k^-3 field: profile (16 codes, r >= 0.9999) ->
  fixed-quality encode at the recommended code read on the device -> decode.
  All 16 profile points (bytes, the six sums, r) and the recommendation equal
  the oracle's profile of the whole array; the container equals the oracle's
  container; the decoded array equals the oracle's decode.
* float64 512^3 field (1 GiB, one call each): the same at r >= 0.99999.
* int16 sensor trace replicated 64 times, fixed rate 4:1: the container
  equals the oracle's container of the whole replica, and every copy after
  the first repeats the first copy's packets except its first packet, whose
  lag decision sees the previous copy's last block; the decode is lossless
  against the oracle's.
* 40,000 blocks of float32 (the block-per-thread decoder's size): block
  ranges decode to the whole array's values, the containers equal the
  oracle's, and a reserved stream selector is reported as corrupt.
"""
import struct

import numpy as np
import pytest
import torch

import oracle as O
from paper_1303_4994_gb300 import apax as A
from paper_1303_4994_gb300 import build as B
from paper_1303_4994_gb300 import synth

pytestmark = pytest.mark.gpu
N = 256


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    A.lib()
    torch.cuda.init()


def _packets(container: bytes, nb: int, mode: int, budget: int = 0):
    """Packets of a container (offset table for fixed quality, j*B otherwise)."""
    poff = 40 + (((4 * nb + 7) // 8) * 8 if mode == 1 else 0)
    if mode == 1:
        tab = np.frombuffer(container, dtype=np.uint32, count=nb, offset=40).astype(np.int64)
        starts = poff + 4 * tab
    else:
        starts = poff + budget * np.arange(nb, dtype=np.int64)
    out = []
    for j in range(nb):
        h0 = int(np.frombuffer(container, dtype=np.uint32, count=1, offset=int(starts[j]))[0])
        plen = h0 >> 14
        out.append(container[int(starts[j]):int(starts[j]) + plen])
    return out


def _profiled_fq_parity(x, dtype, target, fmt=0):
    """Profile -> fixed-quality encode at the recommended code -> decode on
    the whole array, each result against the oracle's whole-array result."""
    n = x.size
    xt = torch.from_numpy(x).cuda()
    nc = 16
    pws, pts, summ = A.profile_buffers(xt, N, nc)
    A.profile_into(xt, N, list(A.DEFAULT_CANDIDATES), target, pws, pts, summ, fmt=fmt)
    p = A.params(N, A.FIXED_QUALITY, fmt=fmt)
    tcode = A.F32 if dtype == np.float32 else A.F64
    out = torch.empty(A.encoded_size(tcode, n, p), dtype=torch.uint8, device="cuda")
    ws = torch.empty(A.workspace_size(tcode, n, p), dtype=torch.uint8, device="cuda")
    res = A.new_result("cuda")
    A.encode_into(xt, p, out, ws, res, summary=summ)
    torch.cuda.synchronize()
    sm = A.read_summary(summ)
    r = A.read_result(res)
    assert sm.status == 0 and r.status == 0
    code = int(sm.recommended_code)
    gpts = A.read_points(pts, nc)
    point = gpts[sm.recommended]
    assert point.code == code and point.r >= target
    assert point.bytes == r.bytes  # exact size prediction
    del ws, pws
    # every profile point of the whole array, bit for bit
    opts, orec, omiss = O.profile(x, N, list(A.DEFAULT_CANDIDATES), target, threads=0, fmt=fmt)
    assert sm.recommended == orec and bool(sm.flags & 1) == omiss
    for g, o in zip(gpts, opts):
        assert (g.code, g.bytes) == (o.code, o.bytes)
        for f in ("sx", "sy", "sxx", "sxy", "syy", "sdd", "r"):
            assert struct.pack("<d", getattr(g, f)) == struct.pack("<d", getattr(o, f)), (g.code, f)
    # the whole container and the whole decoded array
    cont = out[:r.bytes].cpu().numpy().tobytes()
    want = O.encode(x, N, O.MODE_FQ, 1, 1, code, threads=0, fmt=fmt)
    assert len(cont) == len(want)
    assert cont == want
    y = A.decode(out[:r.bytes], torch.float32 if dtype == np.float32 else torch.float64, n)
    del out
    ui = np.uint32 if dtype == np.float32 else np.uint64
    yo = O.decode(want, dtype, n, threads=0)
    assert np.array_equal(y.cpu().numpy().view(ui), yo.view(ui))
    return point


def test_field_4096_full_size_parity():
    _profiled_fq_parity(synth.grf2d(4096, 4096, seed=1).reshape(-1), np.float32, 0.9999)


def test_field_4096_full_size_parity_version2():
    # the same workload in a version-2 container (groups of 8, the sum
    # stream): the team sweep sizes the packets, the pre-pass picks streams
    _profiled_fq_parity(synth.grf2d(4096, 4096, seed=1).reshape(-1), np.float32, 0.9999,
                        fmt=A.FORMAT_GROUP8 | A.FORMAT_SUM_STREAM)


def test_nyquist_replica_version2_parity():
    # 1,024 copies of the Nyquist-band int16 trace, lossless, in every
    # format: the sum stream's decoder paths at 1,024 x 1,024 blocks
    x = np.tile(synth.nyquist_trace(), 1024)
    xt = torch.from_numpy(x).cuda()
    for fmt in (A.FORMAT_SUM_STREAM, A.FORMAT_GROUP8 | A.FORMAT_SUM_STREAM):
        c = A.encode(xt, 256, A.FIXED_QUALITY, (1, 1), 0, fmt=fmt)
        want = O.encode(x, 256, O.MODE_FQ, 1, 1, 0, threads=0, fmt=fmt)
        assert c.cpu().numpy().tobytes() == want
        y = A.decode(c, torch.int16, x.size)
        assert torch.equal(y, xt)  # lossless


def test_field3d_512_full_size_parity():
    # the 1 GiB float64 simulation field, encoded and decoded in one call each
    x = synth.field3d(512, seed=2).reshape(-1)
    point = _profiled_fq_parity(x, np.float64, 0.99999)
    assert point.code > 0  # a lossy setting was chosen


def test_sensor_replica_repeats_packets():
    trace = synth.sensor_trace()
    reps = 64
    x = np.tile(trace, reps)
    xt = torch.from_numpy(x).cuda()
    ct = A.encode(xt, N, A.FIXED_RATE, (4, 1), 0)
    c = ct.cpu().numpy().tobytes()
    assert c == O.encode(x, N, O.MODE_FR, 4, 1, 0, threads=0)  # the whole replica
    y = A.decode(ct, torch.int16, x.size).cpu().numpy()
    np.testing.assert_array_equal(y, O.decode(c, np.int16, x.size, threads=0))
    single = O.encode(trace, N, O.MODE_FR, 4, 1, 0)
    budget = 128  # 256 int16 samples at 4:1
    nb1 = trace.size // N
    assert len(c) == 40 + reps * nb1 * budget
    pk = _packets(c, reps * nb1, 0, budget)
    first = _packets(single, nb1, 0, budget)
    assert pk[:nb1] == first
    seam = O.encode_blocks(x, N, O.MODE_FR, 4, 1, 0, nb1, nb1 + 1)[0]
    for k in range(1, reps):
        assert pk[k * nb1] == seam  # its lag decision sees the previous copy
        assert pk[k * nb1 + 1:(k + 1) * nb1] == first[1:]


def test_large_array_block_range_and_corruption():
    # enough blocks for the block-per-thread decoder: a block range decodes
    # to the same values as the whole array, and a reserved stream selector
    # in one packet is reported as corrupt
    rng = np.random.default_rng(43)
    nb = 40000
    x = np.cumsum(rng.standard_normal(nb * N)).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    for mode, rate, code in ((A.FIXED_QUALITY, (1, 1), 640), (A.FIXED_RATE, (4, 1), 0)):
        c = A.encode(xt, N, mode, rate, code)
        full = A.decode(c, torch.float32, x.size)
        for b0, b1 in ((0, nb), (1000, 35000), (nb - 33000, nb)):
            part = A.decode_blocks(c, torch.float32, x.size, b0, b1, N)
            assert torch.equal(part.view(torch.int32), full[b0 * N:b1 * N].view(torch.int32))
        # the whole container and decode against the oracle
        cont = c.cpu().numpy().tobytes()
        assert cont == O.encode(x, N, mode, rate[0], rate[1], code, threads=0), mode
        yo = O.decode(cont, np.float32, x.size, threads=0)
        assert np.array_equal(full.cpu().numpy().view(np.uint32), yo.view(np.uint32))
        # packet 12345's selector set to the reserved value 3
        bad = bytearray(cont)
        poff = 40 + (((4 * nb + 7) // 8) * 8 if mode == A.FIXED_QUALITY else 0)
        start = poff + (4 * int(np.frombuffer(cont, np.uint32, 1, 40 + 4 * 12345)[0])
                        if mode == A.FIXED_QUALITY else 256 * 12345)
        bad[start] |= 3
        _, r = A.decode(torch.frombuffer(bad, dtype=torch.uint8).cuda(), torch.float32, x.size,
                        check=False)
        assert r.status == -9


@pytest.mark.parametrize("kind", ["noise", "walk", "sine"])
def test_block_per_thread_decode_selector_loops(kind):
    # 40,000 blocks of 64 int16 samples (the block-per-thread decoder): white
    # noise, a random walk and a slow sinusoid make nearly every block take
    # stream 0, 1 and 2 respectively, so warps see one selector (the
    # per-selector loops); the few others mix within their warps
    rng = np.random.default_rng({"noise": 51, "walk": 52, "sine": 53}[kind])
    nb, n64 = 40000, 64
    n = nb * n64 - 17  # ragged last block
    if kind == "noise":
        x = rng.integers(-3000, 3000, n).astype(np.int16)
    elif kind == "walk":
        x = np.clip(np.cumsum(rng.integers(-300, 301, n)), -32768, 32767).astype(np.int16)
    else:
        t = np.arange(n)
        x = np.rint(20000 * np.sin(t * 0.002) + rng.normal(0, 0.3, n)).astype(np.int16)
    xt = torch.from_numpy(x).cuda()
    c = A.encode(xt, n64, A.FIXED_QUALITY, (1, 1), 0)
    cont = c.cpu().numpy().tobytes()
    pk = _packets(cont, nb, 1)
    sel = np.array([p[0] & 3 for p in pk])
    want_s = {"noise": 0, "walk": 1, "sine": 2}[kind]
    assert (sel == want_s).mean() > 0.9, np.bincount(sel, minlength=3)
    y = A.decode(c, torch.int16, n).cpu().numpy()
    np.testing.assert_array_equal(y, x)  # code 0 is lossless for int16
    assert cont == O.encode(x, n64, O.MODE_FQ, 1, 1, 0, threads=0)
