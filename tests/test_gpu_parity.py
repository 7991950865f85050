"""GPU parity: the CUDA library against the CPU oracle, through the C ABI.

Bit-exact bar: encoded containers are byte-identical, decoded arrays are
bit-identical, profiler sums and correlations are identical binary64 values.
Sizes span several tiles (16 blocks each) with ragged tails; edge cases cover
empty/one-sample arrays, block sizes at both limits (multi-chunk blocks),
adversarial float values (subnormals, huge exponents, zeros), corrupt
streams, non-finite input and the bounded-wait timeout.
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

NP = {1: np.int8, 2: np.int16, 3: np.int32, 4: np.float32, 5: np.float64}
TT = {1: torch.int8, 2: torch.int16, 3: torch.int32, 4: torch.float32, 5: torch.float64}
UINT = {1: np.uint8, 2: np.uint16, 3: np.uint32, 4: np.uint32, 5: np.uint64}


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    A.lib()
    torch.cuda.init()


def _data(dt, n, rng, kind=0):
    if dt <= 3:
        info = np.iinfo(NP[dt])
        if kind == 0:
            return rng.integers(info.min, info.max, n, endpoint=True).astype(NP[dt])
        t = np.arange(n)
        x = np.sin(t * 0.03) * info.max * 0.6 + rng.normal(0, 3, n)
        return np.clip(np.rint(x), info.min, info.max).astype(NP[dt])
    if kind == 0:
        return (rng.standard_normal(n) * np.exp(rng.uniform(-8, 8, n))).astype(NP[dt])
    if kind == 1:
        return np.cumsum(rng.standard_normal(n)).astype(NP[dt])
    # adversarial: zeros, subnormals, huge values, mixed binades
    fi = np.finfo(NP[dt])
    x = (rng.standard_normal(n) * np.exp(rng.uniform(-80, 80, n))).astype(NP[dt])
    x[::7] = 0
    x[3::11] = fi.smallest_subnormal * rng.integers(1, 9, len(x[3::11]))
    if n > 5:
        x[5] = fi.max
        x[4] = -fi.max / 3
    return x


def _gpu_encode(x, p):
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return A.encode(xt, p.block_size, p.mode, (p.rate_num, p.rate_den), p.atten_code)


def _bits(a):
    a = np.ascontiguousarray(a)
    return a.view(UINT[O.DTYPE_CODE[a.dtype]])


def _roundtrip(x, N, mode, rate, code):
    n = x.size
    want = O.encode(x, N, mode, rate[0], rate[1], code)
    p = A.params(N, mode, rate, code)
    got = _gpu_encode(x, p)
    gb = got.cpu().numpy().tobytes()
    assert len(gb) == len(want), (len(gb), len(want))
    if gb != want:
        diff = np.nonzero(np.frombuffer(gb, np.uint8) != np.frombuffer(want, np.uint8))[0]
        raise AssertionError(f"container differs at byte {diff[0]} of {len(want)} "
                             f"({len(diff)} bytes)")
    ydt = TT[O.DTYPE_CODE[x.dtype]]
    y = A.decode(got, ydt, n).cpu().numpy()
    yo = O.decode(want, x.dtype, n)
    np.testing.assert_array_equal(_bits(y), _bits(yo))
    return got, y


@pytest.mark.parametrize("dt", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("mode", [0, 1])
def test_parity_small_all_types(dt, mode):
    rng = np.random.default_rng(100 * dt + mode)
    N = 256
    for n in (1, 3, N - 1, N, N + 1, 37 * N + 13):
        for kind in (0, 1, 2) if dt >= 4 else (0, 1):
            x = _data(dt, n, rng, kind)
            if mode == 1:
                for code in (0, 300, int(rng.integers(0, 4096)), 2048 + 5, 4095):
                    _roundtrip(x, N, 1, (1, 1), code)
            else:
                for rate in ((4, 1), (2, 1), (6, 1)):
                    try:
                        O.encoded_size(x.dtype, n, N, 0, rate[0], rate[1])
                    except O.OracleError:
                        continue
                    _roundtrip(x, N, 0, rate, 0)


def _roundtrip_predict(x, N, rate):
    n = x.size
    want = O.encode(x, N, O.MODE_FR, rate[0], rate[1], 0, threads=0, search=O.SEARCH_PREDICT)
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    got = A.encode(xt, N, A.FIXED_RATE, rate, 0, search=A.SEARCH_PREDICT)
    gb = got.cpu().numpy().tobytes()
    assert gb == want, (x.dtype, N, rate, n)
    y = A.decode(got, TT[O.DTYPE_CODE[x.dtype]], n).cpu().numpy()
    np.testing.assert_array_equal(_bits(y), _bits(O.decode(want, x.dtype, n)))


@pytest.mark.parametrize("dt", [1, 2, 3, 4, 5])
def test_parity_fixed_rate_predict(dt):
    # the PREDICT search: teams of 32 (small arrays), teams of 8 and block
    # sizes above 1024, all five types, rates that make most blocks search
    rng = np.random.default_rng(90 + dt)
    for N, n in ((256, 256 * 37 + 13), (64, 64 * 5000 + 3), (2048, 2048 * 40 + 7), (1000, 1000 * 9)):
        for kind in (0, 1, 2) if dt >= 4 else (0, 1):
            x = _data(dt, n, rng, kind)
            for rate in ((2, 1), (4, 1), (6, 1), (5, 2)):
                try:
                    O.encoded_size(x.dtype, n, N, 0, rate[0], rate[1])
                except O.OracleError:
                    continue
                _roundtrip_predict(x, N, rate)


def test_parity_fixed_rate_predict_block_per_thread():
    # 40,000 blocks: the one-block-per-thread encoder runs the search
    rng = np.random.default_rng(95)
    for dt in (2, 4):
        x = _data(dt, 256 * 40000 - 5, rng, 1)
        _roundtrip_predict(x, 256, (4, 1))
    x = synth.sensor_trace(64 * 40000, seed=3)
    _roundtrip_predict(x, 64, (4, 1))


@pytest.mark.parametrize("dt", [2, 4, 5])
@pytest.mark.parametrize("N", [64, 68, 1000, 4096, 16384])
def test_parity_block_sizes(dt, N):
    rng = np.random.default_rng(N + dt)
    n = 3 * N + 17
    x = _data(dt, n, rng, 1)
    _roundtrip(x, N, 1, (1, 1), 256)
    _roundtrip(x, N, 1, (1, 1), 0)
    try:
        O.encoded_size(x.dtype, n, N, 0, 4, 1)
        _roundtrip(x, N, 0, (4, 1), 0)
    except O.OracleError:
        pass


@pytest.mark.parametrize("dt", [4, 5])
def test_quantiser_code_classes(dt):
    # every class of attenuation code: k = 0 with m = 0 and m > 0, both ends
    # of m, large k, the zero code, and random codes; wide and narrow blocks
    rng = np.random.default_rng(70 + dt)
    codes = [0, 1, 5, 64, 127, 128, 129, 255, 256, 300, 1000, 2047, 2048, 3000, 3968, 3969,
             4000, 4094, 4095] + [int(c) for c in rng.integers(0, 4096, 24)]
    for kind in (0, 1, 2):
        x = _data(dt, 256 * 6 + 7, rng, kind)
        for code in codes:
            _roundtrip(x, 256, 1, (1, 1), code)


def test_empty_array():
    for dt in (2, 4):
        x = np.zeros(0, dtype=NP[dt])
        want = O.encode(x, 256, 1)
        got = _gpu_encode(x, A.params(256, 1))
        assert got.cpu().numpy().tobytes() == want
        y = A.decode(got, TT[dt], 0)
        assert y.numel() == 0


def test_sensor_trace_full_size_fixed_rate():
    """int16 sensor trace, 262,144 samples, fixed rate 4:1: full parity."""
    x = synth.sensor_trace()
    got, y = _roundtrip(x, 256, 0, (4, 1), 0)
    assert got.numel() == 131112


def test_decode_blocks_random_access():
    rng = np.random.default_rng(5)
    for mode, dt in ((1, 4), (0, 2), (1, 5)):
        x = _data(dt, 256 * 50 + 77, rng, 1)
        c = _gpu_encode(x, A.params(256, mode, (4, 1), 700))
        full = O.decode(c.cpu().numpy().tobytes(), x.dtype, x.size)
        for _ in range(10):
            b0 = int(rng.integers(0, 51))
            b1 = int(rng.integers(b0, 52))
            y = A.decode_blocks(c, TT[dt], x.size, b0, b1, 256).cpu().numpy()
            np.testing.assert_array_equal(_bits(y), _bits(full[b0 * 256:min(b1 * 256, x.size)]))


def test_decode_rejects_mismatch_and_corruption():
    rng = np.random.default_rng(6)
    x = _data(4, 256 * 20 + 5, rng, 1)
    c = _gpu_encode(x, A.params(256, 1, (1, 1), 256))
    _, r = A.decode(c, torch.float64, x.size, check=False)
    assert r.status == -1
    _, r = A.decode(c, torch.float32, x.size + 1, check=False)
    assert r.status == -1
    cb = c.cpu().numpy()
    for trial in range(300):
        b = cb.copy()
        i = int(rng.integers(0, len(b)))
        b[i] ^= np.uint8(1 << int(rng.integers(0, 8)))
        st_o = O.decode_status(b.tobytes(), np.float32, x.size)
        yg, r = A.decode(torch.from_numpy(b).cuda(), torch.float32, x.size, check=False)
        if st_o == 0:
            assert r.status == 0
            yo = O.decode(b.tobytes(), np.float32, x.size)
            np.testing.assert_array_equal(_bits(yg.cpu().numpy()), _bits(yo))
        else:
            assert r.status < 0, (trial, i, st_o)
    # truncation
    for cut in (0, 10, 39, 40, 48, len(cb) // 2, len(cb) - 4):
        _, r = A.decode(c[:cut].contiguous(), torch.float32, x.size, check=False)
        assert r.status < 0


def test_nonfinite_input_reports_status():
    x = np.ones(1000, dtype=np.float32)
    x[700] = np.nan
    r = A.encode_status(torch.from_numpy(x).cuda(), A.params(256, 1))
    assert r.status == -8
    x[700] = np.inf
    r = A.encode_status(torch.from_numpy(x).cuda(), A.params(256, 0, (4, 1)))
    assert r.status == -8


def test_bounded_wait_timeout_then_context_usable():
    rng = np.random.default_rng(7)
    # 64 tiles at any team geometry (a tile holds at most 16 blocks of 256)
    x = torch.from_numpy(_data(4, 256 * 16 * 64, rng, 1)).cuda()
    r = A.encode_test_stall(x, A.params(256, 1, (1, 1), 256), stall_tile=2, spin_cycles=1 << 22)
    assert r.status == -10
    # the context is still usable and correct afterwards
    _roundtrip(x.cpu().numpy(), 256, 1, (1, 1), 256)


# ----------------------------------------------------------------- profiler
def _profile_parity(x, N, cands, target):
    pts_o, rec_o, missed_o = O.profile(x, N=N, candidates=cands, target=target)
    xt = torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).cuda()
    pts, summ = A.profile(xt, N, cands, target)
    assert summ.status == 0
    for po, pg in zip(pts_o, pts):
        assert po.code == pg.code
        assert po.bytes == pg.bytes, (po.code, po.bytes, pg.bytes)
        for f in ("sx", "sy", "sxx", "sxy", "syy", "sdd", "r"):
            a, b = getattr(po, f), getattr(pg, f)
            # identical binary64 values (NaN when sums overflow on both sides)
            assert struct.pack("<d", a) == struct.pack("<d", b), (po.code, f, a, b)
    assert summ.recommended == rec_o and bool(summ.flags & 1) == missed_o
    assert summ.recommended_code == cands[rec_o]
    return pts, summ


@pytest.mark.parametrize("dt", [1, 2, 3, 4, 5])
def test_profile_parity_small(dt):
    rng = np.random.default_rng(dt)
    N = 256
    x = _data(dt, 256 * 37 + 19, rng, 1)
    _profile_parity(x, N, list(A.DEFAULT_CANDIDATES), 0.9999)
    _profile_parity(x, N, [0, 128, 384, 1024, 3968], 0.99999)


@pytest.mark.parametrize("dt", [4, 5])
def test_profile_parity_adversarial_floats(dt):
    rng = np.random.default_rng(40 + dt)
    x = _data(dt, 256 * 9 + 3, rng, 2)
    _profile_parity(x, 256, list(A.DEFAULT_CANDIDATES), 0.9999)
    _profile_parity(x, 64, [0, 512, 3840], 0.9)


@pytest.mark.parametrize("dt", [4, 5])
def test_profile_parity_tiny_values(dt):
    # unit-scale blocks with samples far below the block maximum: below the
    # quantiser's reach at every power-of-two code, at depths both inside and
    # beyond the profiler's fixed-point grids, and subnormals
    rng = np.random.default_rng(60 + dt)
    n = 256 * 40 + 5
    x = rng.standard_normal(n)
    depths = [25, 30, 47, 60, 90, 100, 126, 140]
    for blk in range(0, 40, 3):
        for i, dpt in enumerate(rng.choice(depths, 4)):
            x[256 * blk + 7 * i + 1] = (-1.0) ** i * 2.0 ** -int(dpt) * (1 + rng.random())
    x = x.astype(NP[dt])
    fi = np.finfo(NP[dt])
    x[256 * 5 + 3] = fi.smallest_subnormal * 3
    x[256 * 9 + 100] = -fi.smallest_subnormal
    _profile_parity(x, 256, list(A.DEFAULT_CANDIDATES), 0.9999)
    _profile_parity(x, 1000, [0, 128, 1024, 2944], 0.99)


@pytest.mark.parametrize("dt", [1, 2, 3, 4, 5])
def test_profile_parity_general_codes(dt):
    # attenuations that are not powers of two (m != 0): integers dequantise
    # with the decoder's reciprocal table, floats go through the exact
    # superaccumulator; points must equal the oracle's bit for bit
    rng = np.random.default_rng(80 + dt)
    x = _data(dt, 256 * 21 + 37, rng, 1)
    _profile_parity(x, 256, [0, 1, 130, 701, 1153, 1999, 2900, 4095], 0.9999)
    _profile_parity(x, 64, [5, 256, 300, 1280, 1333], 0.99)
    if dt >= 4:
        xa = _data(dt, 256 * 5 + 3, rng, 2)
        _profile_parity(xa, 256, [64, 1100, 2049], 0.9)


def test_profile_parity_image_field():
    x = synth.grf2d(512, 512, seed=11)
    pts, summ = _profile_parity(x, 256, list(A.DEFAULT_CANDIDATES), 0.9999)
    assert 0 < summ.recommended < 15


def test_profile_parity_field3d():
    x = synth.field3d(32, seed=12)
    _profile_parity(x, 256, list(A.DEFAULT_CANDIDATES), 0.99999)


def test_encode_recommended_matches_host_code():
    x = synth.grf2d(256, 256, seed=13)
    xt = torch.from_numpy(x.reshape(-1)).cuda()
    nc = 16
    ws, pts, summ = A.profile_buffers(xt, 256, nc)
    A.profile_into(xt, 256, list(A.DEFAULT_CANDIDATES), 0.9999, ws, pts, summ)
    p = A.params(256, 1)
    cap = A.encoded_size(4, xt.numel(), p)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    ews = torch.empty(A.workspace_size(4, xt.numel(), p), dtype=torch.uint8, device="cuda")
    res = A.new_result("cuda")
    A.encode_into(xt, p, out, ews, res, summary=summ)
    r = A.read_result(res)
    s = A.read_summary(summ)
    want = O.encode(x, 256, 1, 1, 1, s.recommended_code)
    assert r.status == 0 and out[:r.bytes].cpu().numpy().tobytes() == want


@pytest.mark.parametrize("dt", [2, 4, 5])
def test_profile_from_host_matches_device(dt):
    # the host-input sweep (copy in pieces on a side stream, sweep beside it)
    # gives the device sweep's points and summary byte for byte, and leaves
    # the array on the device
    rng = np.random.default_rng(60 + dt)
    N = 256
    x = _data(dt, 256 * 16 * 37 + 75, rng, 1)  # 37 runs and a ragged tail
    xt = torch.from_numpy(x).cuda()
    nc = 16
    ws, pts, summ = A.profile_buffers(xt, N, nc)
    A.profile_into(xt, N, list(A.DEFAULT_CANDIDATES), 0.9999, ws, pts, summ)
    torch.cuda.synchronize()
    want_p, want_s = pts.cpu().clone(), summ.cpu().clone()
    xh = torch.from_numpy(x).pin_memory()
    for chunks in (1, 3, 8, 64):
        xd = torch.empty_like(xt).fill_(0)
        ws2, pts2, summ2 = A.profile_buffers(xt, N, nc)
        A.profile_from_host_into(xh, xd, N, list(A.DEFAULT_CANDIDATES), 0.9999, ws2, pts2, summ2,
                                 chunks=chunks)
        torch.cuda.synchronize()
        assert torch.equal(pts2.cpu(), want_p) and torch.equal(summ2.cpu(), want_s), chunks
        assert torch.equal(xd.view(torch.uint8), xt.view(torch.uint8)), chunks
    # empty array
    e = torch.empty(0, dtype=xt.dtype)
    ws3, pts3, summ3 = A.profile_buffers(e.cuda(), N, nc)
    A.profile_from_host_into(e.pin_memory(), e.cuda(), N, None, 0.9999, ws3, pts3, summ3)
    torch.cuda.synchronize()
    assert A.read_summary(summ3).status == 0 and A.read_summary(summ3).n == 0


def test_profile_from_host_graph_capture():
    # the host-input sweep (copies, events, the library's sweep streams)
    # captured into a CUDA graph and replayed gives the device sweep's points
    x = synth.grf2d(1024, 1024, seed=22).reshape(-1)
    xt = torch.from_numpy(x).cuda()
    N, nc = 256, 16
    ws, pts, summ = A.profile_buffers(xt, N, nc)
    A.profile_into(xt, N, list(A.DEFAULT_CANDIDATES), 0.9999, ws, pts, summ)
    torch.cuda.synchronize()
    want_p = pts.cpu().clone()
    xh = torch.from_numpy(x).pin_memory()
    xd = torch.zeros_like(xt)
    w2, p2, s2 = A.profile_buffers(xt, N, nc)
    st, cs = torch.cuda.Stream(), torch.cuda.Stream()
    A.profile_from_host_into(xh, xd, N, list(A.DEFAULT_CANDIDATES), 0.9999, w2, p2, s2,
                             stream=st, copy_stream=cs, chunks=8)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st, capture_error_mode="relaxed"):
        A.profile_from_host_into(xh, xd, N, list(A.DEFAULT_CANDIDATES), 0.9999, w2, p2, s2,
                                 stream=st, copy_stream=cs, chunks=8)
    for _ in range(2):
        xd.zero_()
        p2.zero_()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(p2.cpu(), want_p)
        assert torch.equal(xd, xt)


def test_profile_from_host_two_in_flight():
    # two host-input sweeps enqueued back to back on their own streams (they
    # share the library's sweep streams) each give the device sweep's points;
    # a field large enough for the one-block-per-thread device sweep
    x = synth.grf2d(2048, 2048, seed=21).reshape(-1)  # 16,384 blocks
    xt = torch.from_numpy(x).cuda()
    N, nc = 256, 16
    ws, pts, summ = A.profile_buffers(xt, N, nc)
    A.profile_into(xt, N, list(A.DEFAULT_CANDIDATES), 0.9999, ws, pts, summ)
    torch.cuda.synchronize()
    want_p, want_s = pts.cpu().clone(), summ.cpu().clone()
    xh = torch.from_numpy(x).pin_memory()
    slots = []
    for _ in range(2):
        xd = torch.zeros_like(xt)
        b = A.profile_buffers(xt, N, nc)
        slots.append((xd, b, torch.cuda.Stream(), torch.cuda.Stream()))
    # one piece (the whole array, then the one-block-per-thread sweep) and 16
    # pieces (the team sweep on each as it lands)
    for rep, chunks in enumerate((16, 1, 16)):
        for xd, (w2, p2, s2), st, cs in slots:
            A.profile_from_host_into(xh, xd, N, list(A.DEFAULT_CANDIDATES), 0.9999, w2, p2, s2,
                                     stream=st, copy_stream=cs, chunks=chunks)
        torch.cuda.synchronize()
        for xd, (w2, p2, s2), st, cs in slots:
            assert torch.equal(p2.cpu(), want_p) and torch.equal(s2.cpu(), want_s), rep
            assert torch.equal(xd, xt)


@pytest.mark.parametrize("dt", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("N", [128, 200, 512])
def test_large_arrays_block_sizes_decode(dt, N):
    # 32,768+ blocks of 128..512 samples (the block-per-thread decoder):
    # whole arrays (ragged tails, all three streams, both modes) against the
    # oracle, a block range, and corrupt packets
    rng = np.random.default_rng(300 + 7 * dt + N)
    nb = 32768 + 17
    n = nb * N - 3
    x = _data(dt, n, rng, 1)
    if dt >= 4:
        x[: n // 3] = _data(dt, n // 3, rng, 0)  # noise: stream 0 blocks too
    xt = torch.from_numpy(x).cuda()
    ydt = TT[dt]
    for mode, rate, code in ((1, (1, 1), 700), (0, (4, 1), 0)):
        try:
            O.encoded_size(x.dtype, n, N, mode, rate[0], rate[1])
        except O.OracleError:
            continue
        c = A.encode(xt, N, mode, rate, code)
        cb = c.cpu().numpy().tobytes()
        assert cb == O.encode(x, N, mode, rate[0], rate[1], code, threads=0)
        y = A.decode(c, ydt, n)
        yo = O.decode(cb, x.dtype, n, threads=0)
        np.testing.assert_array_equal(_bits(y.cpu().numpy()), _bits(yo))
        part = A.decode_blocks(c, ydt, n, 100, 32700, N)
        assert torch.equal(part.view(torch.uint8), y[100 * N:32700 * N].view(torch.uint8))
        bad = bytearray(cb)
        poff = 40 + (((4 * nb + 7) // 8) * 8 if mode == 1 else 0)
        B_ = 0 if mode == 1 else int(np.frombuffer(cb, np.uint32, 1, 16)[0])
        start = poff + (4 * int(np.frombuffer(cb, np.uint32, 1, 40 + 4 * 20000)[0])
                        if mode == 1 else B_ * 20000)
        bad[start] |= 3  # reserved stream selector
        _, r = A.decode(torch.frombuffer(bad, dtype=torch.uint8).cuda(), ydt, n, check=False)
        assert r.status == -9
        bad = bytearray(cb)
        bad[start + 6] ^= 0xFF  # scrambled tokens: a status or the oracle's values
        st = O.decode_status(bytes(bad), x.dtype, n)
        yb, r = A.decode(torch.frombuffer(bad, dtype=torch.uint8).cuda(), ydt, n, check=False)
        if st == 0:
            assert r.status == 0
        else:
            assert r.status == -9
