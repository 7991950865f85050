"""Independent pure-Python APAX mini-codec for tiny inputs (test helper).

A second, deliberately different implementation of the frozen bitstream
reading, used only to cross-check the C oracle on small random arrays.  It
rounds with exact rationals (``fractions.Fraction``) and assembles packets as
one big Python integer, where the oracle uses integer shifts and a bit
writer.  Paper passages: Sec. 6 (blocks, attenuator, redundancy remover,
one-block-lag stream decision, 4/6-byte headers, BFPE groups of 4 or 8 and
JEE tokens; the sum stream of the second container version) and Sec. 4
(profiler formula).
"""
from __future__ import annotations

import math
import struct
from fractions import Fraction

import numpy as np

INFO = {  # dtype -> (code, bytes, W, Q, header bits)
    np.dtype(np.int8): (1, 1, 8, None, 32),
    np.dtype(np.int16): (2, 2, 16, None, 32),
    np.dtype(np.int32): (3, 4, 32, None, 32),
    np.dtype(np.float32): (4, 4, 32, 23, 48),
    np.dtype(np.float64): (5, 8, 32, 29, 48),
}


def atten(c: int) -> Fraction:
    """a(c) = (256 - m) 2^-(8+k), k = c>>7, m = c&127; a(4095) = 0."""
    if c == 4095:
        return Fraction(0)
    return Fraction(256 - (c & 127), 2 ** (8 + (c >> 7)))


def rne(fr: Fraction) -> int:
    return round(fr)  # Fraction.__round__ rounds half to even


def signed_w(v: int, W: int) -> int:
    v &= (1 << W) - 1
    return v - (1 << W) if v >> (W - 1) else v


def nbits(v: int) -> int:
    if v == 0:
        return 0
    return (v.bit_length() + 1) if v > 0 else ((-v - 1).bit_length() + 1)


def block_exp(vals) -> int:
    m = max((abs(Fraction(float(v))) for v in vals), default=Fraction(0))
    if m == 0:
        return 0
    return math.frexp(float(m))[1]


def quant(x, dt, c, Eb):
    W, Q = INFO[dt][2], INFO[dt][3]
    if Q is None:
        return [rne(Fraction(int(v)) * atten(c)) for v in x]
    return [rne(Fraction(float(v)) * Fraction(2) ** (Q - Eb) * atten(c)) for v in x]


def streams(q, W):
    n = len(q)
    s0 = [signed_w(v, W) for v in q]
    s1 = [signed_w(q[i] - (q[i - 1] if i else 0), W) for i in range(n)]
    s2 = []
    for i in range(n):
        if i == 0:
            v = q[0]
        elif i == 1:
            v = q[1] - q[0]
        else:
            v = q[i] - 2 * q[i - 1] + q[i - 2]
        s2.append(signed_w(v, W))
    s3 = [signed_w(q[i] + (q[i - 1] if i else 0), W) for i in range(n)]
    return [s0, s1, s2, s3]


def exps(u, gs=4):
    out = []
    for g in range(len(u) // gs):
        e = max(nbits(v) for v in u[gs * g:gs * g + gs])
        out.append(32 if e == 31 else e)
    return out


def tokens(e):
    """Greedy JEE token list as nibbles."""
    def absol(v):
        v = min(v, 31)
        return [14 + (v >> 4), v & 15]
    nib = absol(e[0])
    d = [None] + [e[i] - e[i - 1] for i in range(1, len(e))]
    i = 1
    while i < len(e):
        if i + 1 < len(e) and abs(d[i]) <= 1 and abs(d[i + 1]) <= 1:
            nib.append(3 * (d[i] + 1) + (d[i + 1] + 1))
            i += 2
        elif abs(d[i]) <= 2:
            nib.append(11 + d[i])
            i += 1
        else:
            nib += absol(e[i])
            i += 1
    return nib


def pkt_bits(u, H, gs=4):
    e = exps(u, gs)
    return H + 4 * len(tokens(e)) + gs * sum(e)


def build_packet(u, s, c, Eb, H, plen, gs=4):
    e = exps(u, gs)
    val, pos = 0, 0

    def put(v, n):
        nonlocal val, pos
        val |= (v & ((1 << n) - 1)) << pos
        pos += n

    put(s, 2)
    put(c, 12)
    put(plen, 18)
    if H == 48:
        put(Eb & 0xFFFF, 16)
    for t in tokens(e):
        put(t, 4)
    for g, eg in enumerate(e):
        for v in u[gs * g:gs * g + gs]:
            if eg:
                put(v, eg)
    return val.to_bytes(plen, "little")


def _blocks(x, N):
    return [x[j:j + N] for j in range(0, len(x), N)]


def _padded_q(xb, dt, c, Eb, gs=4):
    q = quant(xb, dt, c, Eb)
    G = -(-len(q) // gs)
    return q + [q[-1]] * (gs * G - len(q))


def _best(xb, dt, gs=4, ns=3):
    """Fewest bits at code 0 among the first ns streams (ties to the lower)."""
    W, H = INFO[dt][2], INFO[dt][4]
    Eb = block_exp(xb) if INFO[dt][3] else 0
    q = _padded_q(xb, dt, 0, Eb, gs)
    sizes = [pkt_bits(u, H, gs) for u in streams(q, W)[:ns]]
    return sizes.index(min(sizes))


def minpacket(L, H, gs=4):
    G = -(-L // gs)
    return 4 * -(-(H + 8 + 4 * ((G - 1 + 1) // 2)) // 32)


def budget(L, size, num, den, H, gs=4):
    return max((L * size * den // (4 * num)) * 4, minpacket(L, H, gs))


LADDER_M = [0, 11, 21, 31, 41, 50, 59, 67, 75, 83, 90, 97, 104, 110, 116, 122]


def ladder():
    """Codes 128 k + M[f], k = 0..31, f = 0..15, then 4095, increasing."""
    return sorted({128 * k + m for k in range(32) for m in LADDER_M}) + [4095]


def predict_start(xb, dt, s, bud, gs=4):
    """PREDICT's start code on one block (None when code 0 fits): the excess
    bits over the budget at code 0 against the bits predicted to go at
    attenuation 2^-k, interpolated between two powers of two."""
    W, H = INFO[dt][2], INFO[dt][4]
    Eb = block_exp(xb) if INFO[dt][3] else 0
    b0 = pkt_bits(streams(_padded_q(xb, dt, 0, Eb, gs), W)[s], H, gs)
    if 4 * -(-b0 // 32) <= bud:
        return None
    e = exps(streams(_padded_q(xb, dt, 0, Eb, gs), W)[s], gs)
    D = b0 - 8 * bud
    red = [gs * sum(min(v, k) for v in e) for k in range(32)]
    k1 = next((k for k in range(1, 32) if red[k] >= D), 31)
    num, den = 16 * (D - red[k1 - 1]), red[k1] - red[k1 - 1]
    f = 16 if den == 0 else -(-num // den)
    f = min(max(f, 1), 16)
    return 128 * (k1 - 1) + LADDER_M[f] if f < 16 else 128 * k1


def predict_code(xb, dt, s, bud, gs=4):
    """PREDICT fixed-rate search on one block: code 0 if it fits, else up
    the ladder from the predicted start until the packet fits."""
    W, H = INFO[dt][2], INFO[dt][4]
    Eb = block_exp(xb) if INFO[dt][3] else 0

    def bits_at(cc):
        return pkt_bits(streams(_padded_q(xb, dt, cc, Eb, gs), W)[s], H, gs)

    c = predict_start(xb, dt, s, bud, gs)
    if c is None:
        return 0
    lad = ladder()
    i = lad.index(c)
    while lad[i] < 4095 and 4 * -(-bits_at(lad[i]) // 32) > bud:
        i += 1
    return lad[i]


def encode(x: np.ndarray, N: int, mode: int, num=1, den=1, code=0, search=0, fmt=0) -> bytes:
    """fmt bit 0: groups of 8; bit 1: the sum stream (either makes a
    version-2 container)."""
    dt = x.dtype
    code_dt, size, W, Q, H = INFO[dt]
    gs = 8 if fmt & 1 else 4
    ns = 4 if fmt & 2 else 3
    x = list(x.reshape(-1).tolist())
    n = len(x)
    blocks = _blocks(x, N)
    nb = len(blocks)
    best = [_best(b, dt, gs, ns) for b in blocks]
    packets = []
    B = budget(N, size, num, den, H, gs) if mode == 0 else 0
    for j, xb in enumerate(blocks):
        s = best[0] if j == 0 else best[j - 1]
        Eb = block_exp(xb) if Q else 0
        if mode == 1:
            c = code
            u = streams(_padded_q(xb, dt, c, Eb, gs), W)[s]
            plen = 4 * -(-pkt_bits(u, H, gs) // 32)
        else:
            bud = budget(len(xb), size, num, den, H, gs)
            if search == 1:
                c = predict_code(xb, dt, s, bud, gs)
                u = streams(_padded_q(xb, dt, c, Eb, gs), W)[s]
                packets.append(build_packet(u, s, c, Eb, H, bud, gs))
                continue

            def fits(cc):
                uu = streams(_padded_q(xb, dt, cc, Eb, gs), W)[s]
                return 4 * -(-pkt_bits(uu, H, gs) // 32) <= bud
            if fits(0):
                c = 0
            else:
                lo, hi = 0, 4095
                while hi - lo > 1:
                    mid = (lo + hi) // 2
                    if fits(mid):
                        hi = mid
                    else:
                        lo = mid
                c = hi
            u = streams(_padded_q(xb, dt, c, Eb, gs), W)[s]
            plen = bud
        packets.append(build_packet(u, s, c, Eb, H, plen, gs))
    head = b"APX1" + bytes([2 if fmt else 1, code_dt, mode, (1 if mode == 1 else 0) | (fmt << 1)])
    head += struct.pack("<IHHIQ", N, code if mode == 1 else 0, 0, B, n)
    payload = b"".join(packets)
    head += struct.pack("<Q", len(payload)) + b"\0" * 4
    table = b""
    if mode == 1:
        offs, pos = [], 0
        for p in packets:
            offs.append(pos // 4)
            pos += len(p)
        table = struct.pack(f"<{nb}I", *offs)
        table += b"\0" * ((-len(table)) % 8)
    return head + table + payload


def corr(sxx, sxy, syy):
    if sxx == 0 and syy == 0:
        return 1.0
    if sxx == 0 or syy == 0:
        return 0.0
    return sxy / math.sqrt(sxx * syy)
