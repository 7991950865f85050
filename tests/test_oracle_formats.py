"""Pins of the oracle's second container version: BFPE groups of 8 (Sec. 6
bit packer, "groups of 4 or 8") and the sum stream u_i = q_i + q_{i-1}
(Sec. 6 signal monitor choosing the correlated neighbours; Sec. 5, Fig. 3b:
a signal near the Nyquist frequency alternates in sign, so the sum of
neighbours is small where their difference is large).

* Hand-derived packet sizes of a Nyquist tone (every stream, both group
  sizes) and of a constant block.
* Lossless round trips at code 0 for integers, and the decoded values of a
  lossy code independent of the format (the format only changes how q is
  packed, never q).
* The independent pure-Python codec (tests/pycodec.py) on random tiny
  arrays: both fixed-quality and fixed-rate (BISECT and PREDICT), every
  type, ragged tails.
* Closed-form fixed-rate sizes with the group-of-8 minimum packet.
* Header rules: version 2 exactly when an option is on; selector 3 is
  corrupt without the sum-stream flag; groups of 8 need a block size that
  is a multiple of 8.
* The profiler: the same sums as the version-1 sweep, byte counts equal to
  the Python codec's containers.
"""
import struct

import numpy as np
import pytest

import oracle as O
import pycodec as P

G8, SUM = O.FMT_GROUP8, O.FMT_SUM_STREAM
FMTS = [G8, SUM, G8 | SUM]
TYPES = [np.int8, np.int16, np.int32, np.float32, np.float64]


def _ceil_half(v):
    return (v + 1) // 2


def test_nyquist_tone_packet_bits_by_hand():
    # x_i = 1000 (-1)^i, int16, one block of 64, code 0 (q = x).  Widths
    # (magnitude bits + sign): |1000| -> 11, |2000| -> 12, |4000| -> 13.
    #   S0: every u = +-1000, all exponents 11.
    #   S1: u_0 = 1000, then +-2000: exponents 12 (u_0's group holds 2000s).
    #   S2: u_0 = 1000, u_1 = -2000, then +-4000: exponents 13.
    #   S3: u_0 = 1000, then 0: exponents [11, 0, 0, ...].
    # Tokens: the first exponent absolute (2 nibbles); a run of zero diffs
    # pairs into joint tokens, an odd one left makes a single token; the
    # jump 11 -> 0 is absolute (2 nibbles).
    N, H = 64, 32
    x = (1000 * (-1) ** np.arange(N)).astype(np.int16)
    for gs, fmt in ((4, SUM), (8, G8 | SUM)):
        G = N // gs
        flat = 2 + _ceil_half(G - 1)           # absolute, then G-1 zero diffs
        want = {
            0: H + 4 * flat + gs * G * 11,
            1: H + 4 * flat + gs * G * 12,
            2: H + 4 * flat + gs * G * 13,
            3: H + 4 * (2 + 2 + _ceil_half(G - 2)) + gs * 11,
        }
        for s, bits in want.items():
            assert O.packet_bits(x, N, 0, 0, s, fmt=fmt) == bits, (gs, s)
    assert O.packet_bits(x, N, 0, 0, 3, fmt=SUM) == 120
    assert O.packet_bits(x, N, 0, 0, 3, fmt=G8 | SUM) == 148
    # the decision: the sum stream only when the option is on
    y = np.concatenate([x, x])
    assert O.streams(y, N, 0, 2, fmt=SUM) == [3, 3]
    assert O.streams(y, N, 0, 2, fmt=0) == [0, 0]
    assert O.streams(y, N, 0, 2, fmt=G8) == [0, 0]


def test_constant_block_group8_by_hand():
    # x = 5 (int16): S0 all 4 bits wide; S1 [4, 0, ...]; S2 [4, 0, ...]
    # (u_1 = 0); S3 u_0 = 5 and u_i = 10 (5 bits), so every group of 8,
    # the first included, is 5 wide.  Groups of 8 halve the exponent count.
    N, H = 128, 32
    x = np.full(N, 5, dtype=np.int16)
    G = N // 8
    flat = 2 + _ceil_half(G - 1)
    assert O.packet_bits(x, N, 0, 0, 0, fmt=G8) == H + 4 * flat + 8 * G * 4
    assert O.packet_bits(x, N, 0, 0, 1, fmt=G8) == H + 4 * (2 + 2 + _ceil_half(G - 2)) + 8 * 4
    assert O.packet_bits(x, N, 0, 0, 2, fmt=G8) == H + 4 * (2 + 2 + _ceil_half(G - 2)) + 8 * 4
    assert O.packet_bits(x, N, 0, 0, 3, fmt=G8 | SUM) == H + 4 * flat + 8 * G * 5


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("dt", [np.int8, np.int16, np.int32])
def test_integer_lossless_round_trip(fmt, dt):
    rng = np.random.default_rng(fmt * 10 + np.dtype(dt).itemsize)
    info = np.iinfo(dt)
    for n in (1, 7, 64, 200, 1000):
        for kind in range(3):
            if kind == 0:
                x = rng.integers(info.min, info.max, n, endpoint=True).astype(dt)
            elif kind == 1:  # alternating signs near full scale: the sum stream
                x = ((-1) ** np.arange(n) * rng.integers(info.max // 2, info.max, n)).astype(dt)
            else:
                x = np.cumsum(rng.integers(-3, 4, n)).astype(dt)
            for N in (64, 72, 128):
                c = O.encode(x, N, O.MODE_FQ, code=0, fmt=fmt)
                assert c[4] == 2 and (c[7] >> 1) == fmt
                np.testing.assert_array_equal(O.decode(c, dt, n), x)


@pytest.mark.parametrize("dt", TYPES)
def test_decoded_values_do_not_depend_on_the_format(dt):
    rng = np.random.default_rng(np.dtype(dt).itemsize + 5)
    n = 777
    if np.dtype(dt).kind == "i":
        x = np.cumsum(rng.integers(-50, 51, n)).astype(dt)
    else:
        x = (np.cumsum(rng.standard_normal(n)) * 1e3).astype(dt)
    for code in (0, 300, 1111, 2900):
        y0 = O.decode(O.encode(x, 64, O.MODE_FQ, code=code), dt, n)
        for fmt in FMTS:
            y = O.decode(O.encode(x, 64, O.MODE_FQ, code=code, fmt=fmt), dt, n)
            np.testing.assert_array_equal(y, y0)


def _rand(rng, dt, n, kind):
    if np.dtype(dt).kind == "i":
        info = np.iinfo(dt)
        if kind == 0:
            return rng.integers(info.min, info.max, n, endpoint=True).astype(dt)
        if kind == 1:
            return ((-1) ** np.arange(n) * (np.cumsum(rng.integers(-5, 6, n)) % 60)).astype(dt)
        return (np.cumsum(rng.integers(-5, 6, n)) % 50).astype(dt)
    if kind == 0:
        return (rng.standard_normal(n) * np.exp(rng.uniform(-20, 20, n))).astype(dt)
    if kind == 1:
        return (np.cos(np.arange(n) * 3.0) * 100).astype(dt)  # close to Nyquist
    return np.sin(np.arange(n) * 0.05).astype(dt)


def test_python_codec_crosscheck_formats():
    rng = np.random.default_rng(31)
    done = 0
    while done < 150:
        dt = TYPES[done % 5]
        fmt = FMTS[(done // 5) % 3]
        N = int(rng.choice([64, 72, 128] if fmt & G8 else [64, 68, 128]))
        n = int(rng.integers(1, 3 * N + 7))
        x = _rand(rng, dt, n, done % 3)
        mode = (done // 2) % 2
        search = int(rng.integers(0, 2))
        if mode == O.MODE_FQ:
            code, num, den = int(rng.integers(0, 4096)), 1, 1
        else:
            code = 0
            num, den = [(2, 1), (3, 1), (4, 1), (6, 1)][int(rng.integers(0, 4))]
            try:
                O.encoded_size(dt, n, N, mode, num, den, fmt=fmt)
            except O.OracleError:
                continue
        c = O.encode(x, N, mode, num, den, code, search=search, fmt=fmt)
        assert c == P.encode(x, N, mode, num, den, code, search=search, fmt=fmt), (dt, fmt, N, n)
        if mode == O.MODE_FR:
            assert len(c) == O.encoded_size(dt, n, N, mode, num, den, fmt=fmt)
        O.decode(c, dt, n)
        done += 1


@pytest.mark.parametrize("fmt", [G8, G8 | SUM])
def test_group8_fixed_rate_size_closed_form(fmt):
    # B_j = max(floor(L s den / (4 num)) * 4, minimum packet); the minimum
    # packet is the header, the first absolute token and one joint token per
    # two further groups of 8, padded to 32 bits
    for dt, H in ((np.int16, 32), (np.float32, 48), (np.float64, 48)):
        s = np.dtype(dt).itemsize
        for N in (64, 136, 1024):
            for L in (1, 8, 9, N):
                G = -(-L // 8)
                mp = 4 * -(-(H + 8 + 4 * (G // 2)) // 32)
                assert O.min_packet(dt, N, L, fmt=fmt) == mp
                for num, den in ((2, 1), (4, 1), (12, 1)):
                    assert O.fr_budget(dt, N, L, num, den, fmt=fmt) == max(L * s * den // (4 * num) * 4, mp)


def test_header_rules():
    x = (1000 * (-1) ** np.arange(256)).astype(np.int16)
    c = bytearray(O.encode(x, 64, O.MODE_FQ, code=0, fmt=SUM))
    assert c[4] == 2 and c[7] == 1 | (SUM << 1)
    poff = 40 + 32
    assert struct.unpack_from("<I", c, poff)[0] & 3 == 3   # block 0 on the sum stream
    np.testing.assert_array_equal(O.decode(bytes(c), np.int16, 256), x)
    v1 = bytearray(c)
    v1[4], v1[7] = 1, 1                                      # as a version-1 container
    assert O.decode_status(bytes(v1), np.int16, 256) == O.ST_CORRUPT
    nosum = bytearray(c)
    nosum[7] = 1 | (G8 << 1)                                 # version 2 without the flag
    assert O.decode_status(bytes(nosum), np.int16, 256) == O.ST_CORRUPT
    v2zero = bytearray(O.encode(x, 64, O.MODE_FQ, code=0))
    assert v2zero[4] == 1 and v2zero[7] == 1
    v2zero[4] = 2                                            # version 2, no option
    assert O.decode_status(bytes(v2zero), np.int16, 256) == O.ST_CORRUPT
    bad = bytearray(c)
    bad[7] = 1 | (8 << 1)                                    # an unknown option bit
    assert O.decode_status(bytes(bad), np.int16, 256) == O.ST_CORRUPT
    with pytest.raises(O.OracleError) as e:
        O.encode(x, 68, O.MODE_FQ, fmt=G8)                   # 68 is no multiple of 8
    assert e.value.status == O.ST_BLOCK_SIZE
    with pytest.raises(O.OracleError) as e:
        O.encode(x, 64, O.MODE_FQ, fmt=4)
    assert e.value.status == O.ST_INVALID_ARG


def test_group8_predict_against_the_ladder():
    # PREDICT with groups of 8: the code is the first ladder rung at or
    # above the predicted start whose packet fits, and the start comes from
    # red(k) = 8 sum_g min(e_g, k) (checked through the Python codec)
    rng = np.random.default_rng(40)
    lad = P.ladder()
    for t in range(40):
        dt = [np.int16, np.int32, np.float32, np.float64][t % 4]
        N = 64
        x = _rand(rng, dt, N, t % 3)
        s = t % 4
        size = np.dtype(dt).itemsize
        H = 48 if np.dtype(dt).kind == "f" else 32
        bud = P.budget(N, size, 4, 1, H, 8)
        got = O.fr_code(x, N, 0, s, bud, search=O.SEARCH_PREDICT, fmt=G8 | SUM)
        assert got == P.predict_code(list(x.tolist()), x.dtype, s, bud, 8)
        fits = lambda c: 4 * -(-O.packet_bits(x, N, 0, c, s, fmt=G8 | SUM) // 32) <= bud
        assert fits(got)
        start = P.predict_start(list(x.tolist()), x.dtype, s, bud, 8)
        if start is not None and got > start:
            assert not fits(lad[lad.index(got) - 1])


@pytest.mark.parametrize("fmt", FMTS)
def test_profile_formats(fmt):
    rng = np.random.default_rng(41)
    x = (np.cumsum(rng.standard_normal(1500)) * ((-1) ** np.arange(1500))).astype(np.float32)
    cands = [0, 128, 700, 1536, 3000]
    p0, r0, m0 = O.profile(x, 64, cands, 0.999)
    p1, r1, m1 = O.profile(x, 64, cands, 0.999, fmt=fmt)
    assert (r0, m0) == (r1, m1)
    for a, b, code in zip(p0, p1, cands):
        for f in ("sx", "sy", "sxx", "sxy", "syy", "sdd", "r"):
            assert getattr(a, f) == getattr(b, f)
        assert b.bytes == len(P.encode(x, 64, O.MODE_FQ, 1, 1, code, fmt=fmt))
    pt, rt, mt = O.profile(x, 64, cands, 0.999, threads=3, fmt=fmt)
    assert [p.bytes for p in pt] == [p.bytes for p in p1] and (rt, mt) == (r1, m1)


def test_threaded_encode_formats():
    rng = np.random.default_rng(42)
    x = _rand(rng, np.int16, 5000, 1)
    for fmt in FMTS:
        for mode, num in ((O.MODE_FQ, 1), (O.MODE_FR, 3)):
            a = O.encode(x, 128, mode, num, 1, 77, fmt=fmt)
            assert O.encode(x, 128, mode, num, 1, 77, threads=4, fmt=fmt) == a
            np.testing.assert_array_equal(O.decode(a, np.int16, x.size, threads=3),
                                          O.decode(a, np.int16, x.size))
