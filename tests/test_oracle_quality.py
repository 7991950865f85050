"""Pins of the profiler's signal-quality oracle (oracle/quality.py): the
2-sigma S2R margin of window 4 and the spectral levels of window 3 (Sec. 4).

* S2R: against exact rational ratios (Fraction) sorted by brute force on
  small arrays, the 95.5% property, and the zero conventions.
* Spectra: a pure tone's peak at its closed-form level A^2 L / 6 (periodic
  Hann window, power normalised by sum w^2), a white noise floor at its
  variance, a 6.02 dB shift for a doubled signal, SRR - margin = DR, and the
  paper's rsds example (peak 71, floor 26, residual mean 2 dB; Table 3's SDR
  and spectral margin) satisfying the same relations within printed
  rounding.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import quality as Q

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden(name):
    out = {}
    for ln in open(os.path.join(HERE, "golden", name)):
        ln = ln.strip()
        if ln and not ln.startswith("#"):
            k, v = ln.split()
            out[k] = float(v)
    return out


def _exact_ratio(x, y):
    fx, fd = Fraction(float(x)), Fraction(float(x)) - Fraction(float(y))
    if fd == 0:
        return math.inf
    return abs(fx) / abs(fd)


@pytest.mark.parametrize("dt", [np.int16, np.int32, np.float32])
def test_s2r_margin_vs_exact_ratios(dt):
    rng = np.random.default_rng(3)
    for n in (1, 7, 22, 23, 100, 333, 1000):
        if np.dtype(dt).kind == "i":
            x = rng.integers(-3000, 3000, n).astype(dt)
            y = (x.astype(np.int64) + rng.integers(-40, 41, n)).astype(dt)
        else:
            x = rng.standard_normal(n).astype(dt)
            y = (x + (rng.standard_normal(n) * 1e-3).astype(dt)).astype(dt)
        x[::11] = 0
        y[::13] = x[::13]
        ex = sorted((_exact_ratio(a, b) for a, b in zip(x, y)),
                    key=lambda v: (v == math.inf, v))
        k = 45 * n // 1000
        want = ex[k]
        got = Q.s2r_margin_ratio(x, y)
        # the oracle's ratio is the k-th exact ratio rounded once
        assert got == (math.inf if want == math.inf else float(want))
        # at least 95.5% of the samples at or above it
        ge = sum(1 for v in ex if v >= want)
        assert ge >= 0.955 * n


def test_s2r_conventions_and_db():
    x = np.array([0, 0, 5, 5], dtype=np.int32)
    y = np.array([0, 1, 5, 4], dtype=np.int32)
    assert Q.s2r_ratios(x, y).tolist() == [math.inf, 0.0, math.inf, 5.0]
    assert Q.ratio_db(10.0) == 20.0 and Q.ratio_db(0.0) == -math.inf
    assert Q.ratio_db(math.inf) == math.inf
    assert math.isnan(Q.s2r_margin_ratio(x[:0], y[:0]))
    # a uniform residual 1/1000 of the signal: 60 dB
    xs = np.full(1000, 1000, dtype=np.int32)
    assert Q.s2r_margin_db(xs, xs - 1) == pytest.approx(60.0, abs=1e-12)


def test_spectrum_pure_tone_peak():
    L = 4096
    for A, k0 in ((1.0, 100), (3.5, 1000), (0.25, 7)):
        m = np.arange(8 * L)
        x = A * np.cos(2 * np.pi * k0 * m / L)
        P = Q.welch_power(x, L)
        assert int(np.argmax(P)) + 1 == k0
        assert P.max() == pytest.approx(A * A * L / 6.0, rel=1e-12)
        # Hann main lobe: the neighbours hold a quarter of the peak power
        assert P[k0 - 2] == pytest.approx(P.max() / 4, rel=1e-12)


def test_spectrum_white_noise_floor_and_shift():
    rng = np.random.default_rng(4)
    n = 4096 * 400
    x = rng.standard_normal(n) * 2.0
    y = x + rng.standard_normal(n) * 0.01
    m = Q.spectral_metrics(x.astype(np.float32), y.astype(np.float32))
    assert m["L"] == 4096 and m["segments"] == 400
    assert m["floor_x"] == pytest.approx(10 * math.log10(4.0), abs=0.15)
    assert m["floor_d"] == pytest.approx(10 * math.log10(1e-4), abs=0.15)
    assert m["srr"] - m["fft_s2r_margin"] == pytest.approx(m["dr"], abs=1e-12)
    m2 = Q.spectral_metrics(2 * x, 2 * y)
    for key in ("peak_x", "floor_x", "peak_y", "floor_y", "floor_d", "mean_d"):
        assert m2[key] - Q.spectral_metrics(x, y)[key] == pytest.approx(20 * math.log10(2), abs=1e-9)
    # lossless: the residual spectrum is -inf, margins +inf
    m3 = Q.spectral_metrics(x, x)
    assert m3["mean_d"] == -math.inf and m3["fft_s2r_margin"] == math.inf


def test_window3_relations_on_the_paper_example():
    g = _golden("window3_rsds.txt")
    # Sec. 4: DR = peak - floor, margin = floor - residual mean
    assert g["peak_db"] - g["floor_db"] == g["dr_db"]
    assert g["floor_db"] - g["residual_mean_db"] == g["fft_s2r_margin_db"]
    # Table 3 prints the same encoding to 0.1 dB: SDR - margin = DR within
    # the integer rounding of the Sec. 4 levels
    assert abs((g["table3_sdr_db"] - g["table3_spectral_margin_db"]) - g["dr_db"]) <= 1.0
    assert abs(g["table3_spectral_margin_db"] - g["fft_s2r_margin_db"]) <= 0.5
    assert abs(g["table3_sdr_db"] - (g["peak_db"] - g["residual_mean_db"])) <= 1.0
    assert g["table3_s2r_2sigma_db"] == g["s2r_2sigma_db"]


def test_segment_length():
    assert Q.segment_length(10 ** 6) == 4096 and Q.segment_length(4096) == 4096
    assert Q.segment_length(4095) == 2048 and Q.segment_length(5) == 4


def _tables23():
    rows = []
    for ln in open(os.path.join(HERE, "golden", "tables2_3_spectral.txt")):
        ln = ln.strip()
        if ln and not ln.startswith("#"):
            name, *v = ln.split()
            rows.append((name, *map(float, v)))
    return rows


def test_tables2_3_sdr_is_dr_plus_margin():
    # Table 2's DR is its peak minus its floor on every row (within the 0.1 dB
    # rounding of three printed values), and Table 3's SDR equals Table 2's DR
    # plus Table 3's spectral margin on all rows but the first and third 8-bit
    # datasets: the paper's SDR is the oracle's SRR (input peak minus residual
    # mean) and its margin the oracle's floor minus residual mean
    rows = _tables23()
    assert len(rows) == 25
    tol = 0.15 + 1e-9
    for name, pk, fl, dr, sdr, mg in rows:
        assert abs(pk - fl - dr) <= tol, name
    bad = [r[0] for r in rows if abs(r[4] - (r[3] + r[5])) > tol]
    assert bad == ["image1_i8", "oscilloscope_i8"]
    # the oracle's levels obey the same identities exactly on a field whose
    # levels span several tens of dB
    rng = np.random.default_rng(23)
    x = np.cumsum(rng.standard_normal(3 * 4096 + 17))
    y = x + rng.standard_normal(x.size) * 1e-3
    m = Q.spectral_metrics(x, y)
    assert m["dr"] == m["peak_x"] - m["floor_x"]
    assert m["srr"] == pytest.approx(m["dr"] + m["fft_s2r_margin"], abs=1e-9)
