"""GPU parity of the second container version against the oracle: BFPE
groups of 8 and the sum stream (alone and together), through the C ABI.

Bit-exact bar as for version 1: byte-identical containers, bit-identical
decoded arrays, identical profile points.  Cases: every element type, both
modes and both fixed-rate searches, block sizes from 64 to 16,384 (teams of
8 and of 32, the block-per-thread decoder), ragged tails and arrays of one
sample, data near the Nyquist frequency (where the sum stream wins) and
smooth data (where it does not), block ranges, the batched and sharded
paths, the profiler's byte counts, and the header rules (a sum-stream
packet in a container that does not allow it is corrupt).
"""
import struct

import numpy as np
import pytest
import torch

import oracle as O
from paper_1303_4994_gb300 import apax as A
from paper_1303_4994_gb300 import build as B
from paper_1303_4994_gb300 import shard as S
from paper_1303_4994_gb300 import synth

pytestmark = pytest.mark.gpu

NP = {1: np.int8, 2: np.int16, 3: np.int32, 4: np.float32, 5: np.float64}
TT = {1: torch.int8, 2: torch.int16, 3: torch.int32, 4: torch.float32, 5: torch.float64}
UINT = {1: np.uint8, 2: np.uint16, 3: np.uint32, 4: np.uint32, 5: np.uint64}
G8, SUM = A.FORMAT_GROUP8, A.FORMAT_SUM_STREAM
FMTS = [G8, SUM, G8 | SUM]


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    A.lib()
    torch.cuda.init()


def _data(dt, n, rng, kind):
    """kind 0: noise; 1: near-Nyquist (alternating sign, slow envelope);
    2: smooth; 3: a mix changing every few blocks."""
    t = np.arange(n)
    if kind == 0:
        v = rng.standard_normal(n)
    elif kind == 1:
        v = (-1.0) ** t * (np.cumsum(rng.standard_normal(n)) * 0.2 + 20) + 0.05 * rng.standard_normal(n)
    elif kind == 2:
        v = np.sin(t * 0.01) * 20 + 0.01 * rng.standard_normal(n)
    else:
        v = np.where((t // 300) % 3 == 0, (-1.0) ** t * 15, np.cos(t * 0.02) * 15)
        v = v + 0.1 * rng.standard_normal(n)
    if dt <= 3:
        info = np.iinfo(NP[dt])
        amp = {1: 5, 2: 1000, 3: 5e7}[dt]
        return np.clip(np.rint(v * amp), info.min, info.max).astype(NP[dt])
    return (v * np.exp(rng.uniform(-5, 5))).astype(NP[dt])


def _bits(a):
    a = np.ascontiguousarray(a)
    return a.view(UINT[O.DTYPE_CODE[a.dtype]])


def _check_roundtrip(x, N, mode, rate, code, fmt, search=0):
    n = x.size
    want = O.encode(x, N, mode, rate[0], rate[1], code, threads=0, search=search, fmt=fmt)
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    got = A.encode(xt, N, mode, rate, code, search=search, fmt=fmt)
    gb = got.cpu().numpy().tobytes()
    assert len(gb) == len(want), (len(gb), len(want))
    if gb != want:
        diff = np.nonzero(np.frombuffer(gb, np.uint8) != np.frombuffer(want, np.uint8))[0]
        raise AssertionError(f"container differs at byte {diff[0]} of {len(want)} ({len(diff)} bytes)")
    assert got[4].item() == 2 and (got[7].item() >> 1) == fmt
    y = A.decode(got, TT[O.DTYPE_CODE[x.dtype]], n).cpu().numpy()
    yo = O.decode(want, x.dtype, n, threads=0)
    np.testing.assert_array_equal(_bits(y), _bits(yo))
    return got, want


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("dt", [1, 2, 3, 4, 5])
def test_formats_all_types_fixed_quality(fmt, dt):
    rng = np.random.default_rng(10 * dt + fmt)
    for N in (64, 136, 256):
        for n in (1, 7, N + 5, 37 * N + 13):
            for kind in range(4):
                x = _data(dt, n, rng, kind)
                for code in (0, 384, int(rng.integers(1, 4095))):
                    _check_roundtrip(x, N, A.FIXED_QUALITY, (1, 1), code, fmt)


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("dt", [2, 3, 4, 5])
@pytest.mark.parametrize("search", [0, 1])
def test_formats_fixed_rate(fmt, dt, search):
    rng = np.random.default_rng(100 + 10 * dt + fmt + 7 * search)
    for N in (64, 256, 1024):
        n = 23 * N + 17
        for kind in range(4):
            x = _data(dt, n, rng, kind)
            for rate in ((2, 1), (4, 1), (6, 1)):
                try:
                    O.encoded_size(x.dtype, n, N, O.MODE_FR, rate[0], rate[1], fmt=fmt)
                except O.OracleError:
                    continue
                _check_roundtrip(x, N, A.FIXED_RATE, rate, 0, fmt, search)


@pytest.mark.parametrize("fmt", FMTS)
def test_formats_large_blocks_and_teams_of_32(fmt):
    rng = np.random.default_rng(7 + fmt)
    for dt, N in ((4, 8192), (2, 16384), (5, 4096)):
        n = 5 * N + 333
        for kind in (1, 3):
            x = _data(dt, n, rng, kind)
            _check_roundtrip(x, N, A.FIXED_QUALITY, (1, 1), 700, fmt)
            _check_roundtrip(x, N, A.FIXED_RATE, (4, 1), 0, fmt, search=kind & 1)


@pytest.mark.parametrize("fmt", FMTS)
def test_formats_block_per_thread_decoder(fmt):
    # 33,000 blocks of 64: the decoder's one-block-per-thread path, and its
    # block ranges; the encoder keeps teams for version 2
    rng = np.random.default_rng(30 + fmt)
    N = 64
    x = _data(4, N * 33000 + 9, rng, 3)
    for mode, rate, code in ((A.FIXED_QUALITY, (1, 1), 1280), (A.FIXED_RATE, (3, 1), 0)):
        got, want = _check_roundtrip(x, N, mode, rate, code, fmt)
        for b0, b1 in ((0, 1), (100, 32700), (32990, 33001)):
            yb = A.decode_blocks(got, torch.float32, x.size, b0, b1, N).cpu().numpy()
            yo = O.decode(want, x.dtype, x.size, threads=0)[b0 * N:min(b1 * N, x.size)]
            np.testing.assert_array_equal(_bits(yb), _bits(yo))


def test_sum_stream_chosen_for_nyquist_data():
    # the alternating block takes S3 (selector 3 in the next packet's header)
    N = 64
    x = (1000 * (-1) ** np.arange(4 * N)).astype(np.int16)
    got, want = _check_roundtrip(x, N, A.FIXED_QUALITY, (1, 1), 0, SUM)
    c = got.cpu().numpy().tobytes()
    offs = struct.unpack_from("<4I", c, 40)
    poff = 40 + 16
    sel = [struct.unpack_from("<I", c, poff + 4 * o)[0] & 3 for o in offs]
    assert sel == [3, 3, 3, 3]
    # the same data without the option: S0
    _, w1 = _check_roundtrip(x, N, A.FIXED_QUALITY, (1, 1), 0, G8)
    offs = struct.unpack_from("<4I", w1, 40)
    assert [struct.unpack_from("<I", w1, poff + 4 * o)[0] & 3 for o in offs] == [0, 0, 0, 0]


def test_sum_selector_corrupt_without_the_flag():
    N = 64
    x = (1000 * (-1) ** np.arange(40 * N)).astype(np.int16)
    for n_blocks in (40, 33000):  # teams, and the block-per-thread decoder
        xx = np.tile(x, n_blocks // 40 + 1)[:n_blocks * N]
        c = bytearray(O.encode(xx, N, O.MODE_FQ, code=0, threads=0, fmt=SUM))
        c[4], c[7] = 1, 1  # a version-1 container: selector 3 is not allowed
        t = torch.from_numpy(np.frombuffer(bytes(c), np.uint8).copy()).cuda()
        y = torch.empty(xx.size, dtype=torch.int16, device="cuda")
        ws = torch.empty(A.decode_workspace_size(), dtype=torch.uint8, device="cuda")
        res = A.new_result("cuda")
        A.decode_into(t, y, ws, res)
        assert A.read_result(res).status == O.ST_CORRUPT
        c[4], c[7] = 2, 1 | (G8 << 1)  # version 2 with groups of 8 but no sum stream
        t = torch.from_numpy(np.frombuffer(bytes(c), np.uint8).copy()).cuda()
        res = A.new_result("cuda")
        A.decode_into(t, y, ws, res)
        assert A.read_result(res).status == O.ST_CORRUPT


def test_format_argument_checks():
    x = torch.zeros(1000, dtype=torch.float32, device="cuda")
    with pytest.raises(A.ApaxError) as e:
        A.encode(x, 68, A.FIXED_QUALITY, (1, 1), 0, fmt=G8)  # no multiple of 8
    assert e.value.status == -2
    A.encode(x, 68, A.FIXED_QUALITY, (1, 1), 0, fmt=SUM)      # groups of 4: fine
    with pytest.raises(A.ApaxError) as e:
        A.encode(x, 64, A.FIXED_QUALITY, (1, 1), 0, fmt=4)
    assert e.value.status == -1


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("dt", [2, 4, 5])
def test_profile_formats(fmt, dt):
    rng = np.random.default_rng(50 + dt + fmt)
    for N, n in ((64, 64 * 40 + 3), (256, 256 * 16 * 5 + 77)):
        x = _data(dt, n, rng, 3)
        cands = [0, 256, 640, 1536, 2100, 3000] if dt != 5 else [0, 128, 1024, 2048]
        po, rec, missed = O.profile(x, N=N, candidates=cands, target=0.999, threads=0, fmt=fmt)
        xt = torch.from_numpy(x).cuda()
        pts, summ = A.profile(xt, N, cands, 0.999, fmt=fmt)
        assert summ.status == 0
        for o, g in zip(po, pts):
            assert (o.code, o.bytes) == (g.code, g.bytes), (o.code, o.bytes, g.bytes)
            for f in ("sx", "sy", "sxx", "sxy", "syy", "sdd", "r"):
                assert struct.pack("<d", getattr(o, f)) == struct.pack("<d", getattr(g, f))
        assert summ.recommended == rec and bool(summ.flags & 1) == missed


def test_profile_formats_large_float32_field():
    # an array the version-1 float32 sweep would take one block per thread:
    # with a format option the team sweep sizes the packets
    x = synth.grf2d(1024, 1024, seed=5).reshape(-1)
    for fmt in FMTS:
        po, rec, missed = O.profile(x, N=64, candidates=list(A.DEFAULT_CANDIDATES), target=0.9999,
                                    threads=0, fmt=fmt)
        pts, summ = A.profile(torch.from_numpy(x).cuda(), 64, list(A.DEFAULT_CANDIDATES), 0.9999,
                              fmt=fmt)
        assert [p.bytes for p in pts] == [p.bytes for p in po]
        assert [p.r for p in pts] == [p.r for p in po]
        assert summ.recommended == rec


def test_batch_formats():
    rng = np.random.default_rng(60)
    arrays, ps = [], []
    for i in range(30):
        dt = int(rng.integers(1, 6))
        fmt = [0, G8, SUM, G8 | SUM][i % 4]
        N = int(rng.choice([64, 256, 1000, 16384]))
        n = int(rng.integers(1, 20000))
        x = _data(dt, n, rng, i % 4)
        if i % 2:
            p = A.params(N, A.FIXED_QUALITY, (1, 1), int(rng.integers(0, 4096)), fmt=fmt)
        else:
            p = A.params(N, A.FIXED_RATE, (4, 1), 0, search=i % 3 == 0, fmt=fmt)
            try:
                A.encoded_size(dt, n, p)
            except A.ApaxError:
                p = A.params(N, A.FIXED_QUALITY, (1, 1), 512, fmt=fmt)
        arrays.append(x)
        ps.append(p)
    want = [O.encode(a, p.block_size, p.mode, p.rate_num, p.rate_den, p.atten_code, threads=0,
                     search=p.search, fmt=p.format) for a, p in zip(arrays, ps)]
    xs = [torch.from_numpy(a).cuda() for a in arrays]
    outs = [torch.zeros(A.encoded_size(A.TORCH_CODE[x.dtype], x.numel(), p), dtype=torch.uint8,
                        device="cuda") for x, p in zip(xs, ps)]
    results = torch.zeros(16 * len(xs), dtype=torch.uint8, device="cuda")
    jobs = A.encode_jobs(xs, ps, outs, results)
    ws = A.aligned_workspace(A.batch_encode_workspace_size(jobs))
    plan = A.EncodeBatch(jobs, ws)
    plan.run()
    torch.cuda.synchronize()
    rs = A.read_results(results, len(want))
    for i, (o, r, w) in enumerate(zip(outs, rs, want)):
        assert r.status == 0 and r.bytes == len(w), (i, r, len(w))
        assert o[:r.bytes].cpu().numpy().tobytes() == w, f"array {i}"
    plan.close()
    # the batched decoder on the version-2 containers
    conts = [torch.from_numpy(np.frombuffer(w, np.uint8).copy()).cuda() for w in want]
    ys = [torch.empty(a.size, dtype=TT[O.DTYPE_CODE[a.dtype]], device="cuda") for a in arrays]
    dres = torch.zeros(16 * len(ys), dtype=torch.uint8, device="cuda")
    djobs = A.decode_jobs(conts, ys, [p.block_size for p in ps], dres)
    dws = A.aligned_workspace(A.batch_decode_workspace_size(djobs))
    dplan = A.Batch(djobs, dws)
    dplan.run()
    torch.cuda.synchronize()
    for i, (r, y, a, w) in enumerate(zip(A.read_results(dres, len(ys)), ys, arrays, want)):
        assert r.status == 0, (i, r)
        np.testing.assert_array_equal(_bits(y.cpu().numpy()), _bits(O.decode(w, a.dtype, a.size)))
    dplan.close()


def test_batch_profile_formats():
    rng = np.random.default_rng(61)
    arrays, Ns, cands, fmts = [], [], [], []
    for i, (dt, n) in enumerate([(4, 5000), (2, 256 * 16 * 3 + 5), (5, 777), (1, 4000), (4, 70000)]):
        arrays.append(_data(dt, n, rng, 3))
        Ns.append([64, 256, 128, 64, 256][i])
        cands.append([0, 128, 1024, 2176, 3000])
        fmts.append(FMTS[i % 3])
    xs = [torch.from_numpy(a).cuda() for a in arrays]
    pts = [torch.zeros(A.POINT_BYTES * len(c), dtype=torch.uint8, device="cuda") for c in cands]
    sums = [torch.zeros(A.SUMMARY_BYTES, dtype=torch.uint8, device="cuda") for _ in cands]
    jobs = A.profile_jobs(xs, Ns, cands, [0.999] * len(xs), pts, sums, fmts)
    ws = A.aligned_workspace(A.batch_profile_workspace_size(jobs))
    plan = A.Batch(jobs, ws)
    plan.run()
    torch.cuda.synchronize()
    for i, a in enumerate(arrays):
        po, rec, missed = O.profile(a, N=Ns[i], candidates=cands[i], target=0.999, fmt=fmts[i])
        got = A.read_points(pts[i], len(cands[i]))
        assert [g.bytes for g in got] == [o.bytes for o in po], i
        assert [g.sdd for g in got] == [o.sdd for o in po], i
        assert A.read_summary(sums[i]).recommended == rec
    plan.close()


@pytest.mark.parametrize("fmt", FMTS)
def test_shards_formats(fmt):
    rng = np.random.default_rng(70 + fmt)
    N = 128
    x = _data(4, N * 500 + 21, rng, 3)
    n, nb = x.size, (x.size + N - 1) // N
    xt = torch.from_numpy(x).cuda()
    for p in (A.params(N, A.FIXED_QUALITY, (1, 1), 1500, fmt=fmt),
              A.params(N, A.FIXED_RATE, (4, 1), 0, fmt=fmt)):
        want = O.encode(x, N, p.mode, p.rate_num, p.rate_den, p.atten_code, threads=0, fmt=fmt)
        ranges = S.block_ranges(nb, 3)
        shards = []
        for b0, b1 in ranges:
            e0, e1 = S.halo_elements(n, N, b0, b1)
            shards.append(A.encode_shard(xt[e0:e1].contiguous(), n, p, b0, b1))
        merged = A.merge_shards(shards, ranges, 4, n, p)
        assert merged.cpu().numpy().tobytes() == want
        host = S.merge_host([c.cpu().numpy().tobytes() for c in shards], ranges, n,
                            p.mode == A.FIXED_QUALITY)
        assert host == want


def test_noalloc_formats():
    rng = np.random.default_rng(80)
    x = _data(2, 64 * 300 + 7, rng, 1)
    xt = torch.from_numpy(x).cuda()
    for fmt in FMTS:
        p = A.params(64, A.FIXED_QUALITY, (1, 1), 256, fmt=fmt)
        out = torch.zeros(A.encoded_size(2, x.size, p), dtype=torch.uint8, device="cuda")
        res = A.new_result("cuda")
        A.encode_noalloc_into(xt, p, out, res)
        r = A.read_result(res)
        assert r.status == 0
        assert out[:r.bytes].cpu().numpy().tobytes() == O.encode(x, 64, O.MODE_FQ, code=256, fmt=fmt)
