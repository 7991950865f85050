"""CPU oracle of the profiler's signal-quality metrics (test infrastructure
only: the test-suite, the smoke check and the benchmark's CPU baseline use
it; the product library never does).

Sec. 4 of Wegener, arXiv 1303.4994, describes the profiler's windows 2-4
beyond the correlation and the sums:
  * Window 4, the 2-sigma S2R margin: the level M such that 95.5% of the
    decoded samples have residuals at least M dB smaller than the input
    sample (the per-sample signal-to-residual ratio 20 log10(|x|/|d|),
    d = x - y).
  * Window 3, the spectra: the input spectrum's peak and floor (their
    difference is the dynamic range DR), the residual spectrum's mean, the
    FFT S2R margin (input floor minus residual mean) and the SRR (input peak
    minus residual mean); Window 2 also lists the peaks and floors of y and d.

Readings (the paper gives no estimator, FFT length or window):
  * S2R: d = x - y rounded once to binary64 (exact for every type but
    float64); ratio |x|/|d| rounded once; d = 0 gives +inf (also for x = 0),
    x = 0 with d != 0 gives 0.  The margin's ratio is the k-th smallest of
    the n ratios (0-based), k = floor(45 n / 1000): at least 95.5% of the
    samples have a ratio >= it, and it is the largest value with that
    property.  In dB: 20 log10(ratio).
  * Spectra: Welch-Bartlett averaging over the array flattened in C order:
    segments of L = 4096 samples (the largest power of two <= n when
    n < 4096; no spectrum below 4 samples), hop L, full segments only; each segment has its mean removed
    and is multiplied by the periodic Hann window w[m] = (1 - cos(2 pi m / L))/2;
    P[k] = mean over segments of |FFT[k]|^2 / sum(w^2), for bins k = 1..L/2
    (DC left out).  Peak = max P, floor = the lower median (the
    (L/4)-th smallest of the L/2 bins, 1-based), residual mean = the mean of
    10 log10 P_d over the bins; all levels in dB = 10 log10(P).
"""
from __future__ import annotations

import math

import numpy as np

S2R_PERMILLE_BELOW = 45  # 95.5% at or above the margin


def residual(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """d = x - y in binary64 (one rounding)."""
    return np.asarray(x, dtype=np.float64).reshape(-1) - np.asarray(y, dtype=np.float64).reshape(-1)


def s2r_ratios(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Per-sample |x| / |d| (binary64), +inf where d = 0, 0 where x = 0 and
    d != 0."""
    xa = np.abs(np.asarray(x, dtype=np.float64).reshape(-1))
    da = np.abs(residual(x, y))
    with np.errstate(divide="ignore", invalid="ignore"):
        r = xa / da
    r[da == 0] = np.inf
    return r


def s2r_margin_ratio(x: np.ndarray, y: np.ndarray) -> float:
    """The 2-sigma S2R margin as a ratio: the k-th smallest per-sample ratio,
    k = floor(45 n / 1000) (0-based); NaN for an empty array."""
    r = s2r_ratios(x, y)
    n = r.size
    if n == 0:
        return float("nan")
    k = (S2R_PERMILLE_BELOW * n) // 1000
    return float(np.partition(r, k)[k])


def s2r_margin_db(x: np.ndarray, y: np.ndarray) -> float:
    return ratio_db(s2r_margin_ratio(x, y))


def ratio_db(ratio: float) -> float:
    """20 log10 of an amplitude ratio (+inf for inf, -inf for 0)."""
    if math.isnan(ratio):
        return ratio
    if ratio == 0.0:
        return -math.inf
    if math.isinf(ratio):
        return math.inf
    return 20.0 * math.log10(ratio)


def segment_length(n: int) -> int:
    if n >= 4096:
        return 4096
    if n < 2:
        return 0
    return 1 << (n.bit_length() - 1)


def hann(L: int) -> np.ndarray:
    m = np.arange(L, dtype=np.float64)
    return 0.5 - 0.5 * np.cos(2.0 * np.pi * m / L)


def welch_power(v: np.ndarray, L: int) -> np.ndarray:
    """Averaged periodogram of the full segments of v (binary64), bins
    1..L/2."""
    v = np.asarray(v, dtype=np.float64).reshape(-1)
    S = v.size // L
    seg = v[:S * L].reshape(S, L)
    seg = seg - seg.mean(axis=1, keepdims=True)
    w = hann(L)
    X = np.fft.rfft(seg * w, axis=1)
    P = (X.real ** 2 + X.imag ** 2) / np.sum(w * w)
    return P.mean(axis=0)[1:L // 2 + 1]


def _db(p: float) -> float:
    return 10.0 * math.log10(p) if p > 0 else -math.inf


def spectral_metrics(x: np.ndarray, y: np.ndarray) -> dict:
    """Peaks and floors of x, y and d, the residual's mean level, DR, SRR and
    the FFT S2R margin (dB), with the raw powers beside them."""
    n = np.asarray(x).size
    L = segment_length(n)
    if L < 4:  # no spectrum below 4 samples (a segment of 2 has one bin)
        return {"L": 0, "segments": 0}
    xd = np.asarray(x, dtype=np.float64).reshape(-1)
    yd = np.asarray(y, dtype=np.float64).reshape(-1)
    out = {"L": L, "segments": n // L}
    for name, v in (("x", xd), ("y", yd), ("d", residual(x, y))):
        P = welch_power(v, L)
        srt = np.sort(P)
        out[f"peak_{name}_pow"] = float(srt[-1])
        out[f"floor_{name}_pow"] = float(srt[(L // 2 - 1) // 2])
        out[f"peak_{name}"] = _db(out[f"peak_{name}_pow"])
        out[f"floor_{name}"] = _db(out[f"floor_{name}_pow"])
        if name == "d":
            with np.errstate(divide="ignore"):
                out["mean_d"] = float(np.mean(10.0 * np.log10(P)))
    out["dr"] = out["peak_x"] - out["floor_x"]
    out["srr"] = out["peak_x"] - out["mean_d"]
    out["fft_s2r_margin"] = out["floor_x"] - out["mean_d"]
    return out
