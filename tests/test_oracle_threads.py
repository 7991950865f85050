"""The oracle's threaded drivers against its plain sequential calls.

The threaded encode, decode, metrics and profile run the same per-block
routines over contiguous block ranges (Sec. 6: blocks are coded on their
own; the one-block-lag decision reads only the predecessor's samples) and
assemble the ranges in block order, so every container, decoded array and
sum must be identical, byte for byte and bit for bit, for any thread count.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O

DTS = [np.int8, np.int16, np.int32, np.float32, np.float64]


def _sample(dt, n, seed):
    rng = np.random.default_rng(seed)
    walk = np.cumsum(rng.standard_normal(n))
    if np.issubdtype(dt, np.integer):
        lim = np.iinfo(dt).max
        return np.clip(np.round(walk * lim / (8 * (np.abs(walk).max() + 1))), -lim - 1, lim).astype(dt)
    return (walk * 3.7).astype(dt)


@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("threads", [1, 2, 3, 7, 0])
def test_threaded_encode_decode_equal_plain(dt, threads):
    x = _sample(dt, 64 * 37 + 13, seed=5)
    for mode, num, den, code in ((O.MODE_FQ, 1, 1, 0), (O.MODE_FQ, 1, 1, 1100),
                                 (O.MODE_FR, 3, 1, 0), (O.MODE_FR, 2, 1, 0)):
        a = O.encode(x, 64, mode, num, den, code)
        b = O.encode(x, 64, mode, num, den, code, threads=threads)
        assert a == b, (mode, num, code)
        ya = O.decode(a, dt, x.size)
        yb = O.decode(a, dt, x.size, threads=threads)
        assert ya.tobytes() == yb.tobytes()


@pytest.mark.parametrize("threads", [2, 5])
def test_threaded_edge_sizes(threads):
    for n in (0, 1, 63, 64, 65, 64 * 3):
        x = _sample(np.float32, max(n, 1), seed=n)[:n]
        a = O.encode(x, 64, O.MODE_FQ, 1, 1, 512)
        assert a == O.encode(x, 64, O.MODE_FQ, 1, 1, 512, threads=threads)
        assert O.decode(a, np.float32, n, threads=threads).tobytes() == \
            O.decode(a, np.float32, n).tobytes()


def test_threaded_decode_reports_corruption():
    x = _sample(np.int16, 64 * 20, seed=3)
    good = bytearray(O.encode(x, 64, O.MODE_FR, 4, 1, 0))
    poff = 40
    good[poff + 32 * 11] |= 3  # block 11's stream selector: the reserved value
    with pytest.raises(O.OracleError) as e:
        O.decode(bytes(good), np.int16, x.size, threads=4)
    assert e.value.status == O.ST_CORRUPT


@pytest.mark.parametrize("dt", [np.int16, np.float32, np.float64])
def test_threaded_metrics_and_profile_equal_plain(dt):
    x = _sample(dt, 64 * 45 + 7, seed=11)
    y = O.decode(O.encode(x, 64, O.MODE_FQ, 1, 1, 768), dt, x.size)
    assert O.metrics(x, y, 64).tobytes() == O.metrics(x, y, 64, threads=3).tobytes()
    cands = [0, 256, 768, 1280]
    pa, ra, ma = O.profile(x, 64, cands, 0.9999)
    pb, rb, mb = O.profile(x, 64, cands, 0.9999, threads=4)
    assert (ra, ma) == (rb, mb)
    for a, b in zip(pa, pb):
        assert bytes(a) == bytes(b)


def test_thread_count():
    assert O.threads(3) == 3
    assert O.threads(0) >= 1
