"""GPU parity of the profiler's signal-quality metrics (windows 3 and 4 of
Sec. 4) against the oracle (oracle/quality.py).

The 2-sigma S2R margin is an order statistic of per-sample ratios computed
with correctly rounded binary64 operations on both sides: its ratio must be
identical bit for bit, and so its dB value (the same host log10).  The
spectral levels are binary64 FFT sums added in different orders on the two
sides (numpy's FFT and pairwise means against the kernels' radix-2 FFT and
fixed trees): they must agree within 1e-6 dB, far below the levels'
resolution (Table 3 prints 0.1 dB).
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import quality as OQ
from paper_1303_4994_gb300 import apax as A
from paper_1303_4994_gb300 import build as B
from paper_1303_4994_gb300 import synth

pytestmark = pytest.mark.gpu
TOL_DB = 1e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    A.lib()
    torch.cuda.init()


def _check(x, y):
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    qr, db = A.quality(xt, yt)
    want_r = OQ.s2r_margin_ratio(x, y)
    if math.isnan(want_r):
        assert math.isnan(qr.s2r_ratio)
    else:
        assert qr.s2r_ratio == want_r, (qr.s2r_ratio, want_r)
        assert db["s2r_2sigma"] == OQ.ratio_db(want_r)
    m = OQ.spectral_metrics(x, y)
    assert qr.L == m["L"] and qr.segments == m.get("segments", 0)
    if m.get("segments", 0):
        for k in ("peak_x", "floor_x", "peak_y", "floor_y", "peak_d", "floor_d", "mean_d", "dr",
                  "srr", "fft_s2r_margin"):
            a, b = db[k], m[k]
            if math.isinf(b):
                assert a == b, k
            else:
                assert abs(a - b) <= TOL_DB, (k, a, b)
    return db


def test_quality_image_field_recommended_point():
    x = synth.grf2d(1024, 1024, seed=3).reshape(-1)
    c = O.encode(x, 256, O.MODE_FQ, 1, 1, 2048)
    y = O.decode(c, np.float32, x.size)
    db = _check(x, y)
    assert 0 < db["s2r_2sigma"] < 200 and db["dr"] > 0


@pytest.mark.parametrize("dt", [np.int16, np.int32, np.float32, np.float64])
def test_quality_types_and_sizes(dt):
    rng = np.random.default_rng(7)
    for n in (0, 1, 3, 5, 4095, 4096, 4097, 4096 * 3 + 17, 100000):
        if np.dtype(dt).kind == "i":
            x = np.round(np.cumsum(rng.standard_normal(n)) * 50).astype(dt)
            y = (x.astype(np.int64) + rng.integers(-2, 3, n)).astype(dt)
        else:
            x = np.cumsum(rng.standard_normal(n)).astype(dt)
            y = (x + (rng.standard_normal(n) * 1e-4).astype(dt)).astype(dt)
        if n > 10:
            x[::9] = 0
            y[::7] = x[::7]
        _check(x, y)


def test_quality_lossless_and_sensor():
    x = synth.sensor_trace(262144, seed=0)
    _check(x, x.copy())  # residual zero everywhere: margins +inf
    c = O.encode(x, 256, O.MODE_FR, 4, 1, 0)
    _check(x, O.decode(c, np.int16, x.size))
