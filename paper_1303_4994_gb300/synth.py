"""Seeded synthetic inputs shaped like the paper's sensor, image and
simulation datasets (Sec. 7, Table 2), which are not available here.

This module holds none of the codec's arithmetic: it only draws arrays.
The same bytes feed the CUDA library and the CPU oracle, so generator
rounding differences between machines never reach a parity check.

Recipes (seeded ``numpy.random.default_rng``):
  sensor_trace  int16 1-D trace: 3 sinusoids, frequencies U(0.001, 0.1)
                cycles/sample, phases U(0, 2 pi), amplitudes U(0,1)
                normalised to sum 2^11; plus N(0, 8^2) noise; rounded to
                nearest, clipped to int16.
  grf2d         float32 2-D Gaussian random field with power ~ k^-3: white
                normal -> FFT -> x |k|^(-3/2) (k = 0 zeroed) -> inverse FFT
                -> unit variance; plus white noise of std 1e-3.
  field3d       float64 3-D smooth field with power ~ k^-4, unit variance,
                plus 4 Gaussian blobs of amplitude 10 and std 8 cells at
                centres U(0, n)^3 (not periodic).
"""
from __future__ import annotations

import hashlib

import numpy as np


def sensor_trace(n: int = 262144, seed: int = 0, amp_sum: float = 2.0 ** 11, sigma: float = 8.0,
                 dtype=np.int16) -> np.ndarray:
    rng = np.random.default_rng(seed)
    f = rng.uniform(0.001, 0.1, 3)
    ph = rng.uniform(0.0, 2 * np.pi, 3)
    a = rng.uniform(0.0, 1.0, 3)
    a = a / a.sum() * amp_sum
    t = np.arange(n, dtype=np.float64)
    x = sum(a[i] * np.sin(2 * np.pi * f[i] * t + ph[i]) for i in range(3))
    x = x + rng.normal(0.0, sigma, n)
    info = np.iinfo(dtype)
    return np.clip(np.rint(x), info.min, info.max).astype(dtype)


def _spectral_field(shape, slope: float, rng) -> np.ndarray:
    w = rng.standard_normal(shape)
    F = np.fft.rfftn(w)
    ks = [np.fft.fftfreq(s) for s in shape[:-1]] + [np.fft.rfftfreq(shape[-1])]
    grids = np.meshgrid(*ks, indexing="ij", sparse=True)
    k2 = sum(g * g for g in grids)
    with np.errstate(divide="ignore"):
        amp = np.where(k2 > 0, k2 ** (-slope / 4.0), 0.0)
    f = np.fft.irfftn(F * amp, s=shape, axes=list(range(len(shape))))
    f -= f.mean()
    return f / f.std()


def nyquist_trace(n: int = 262144, seed: int = 0) -> np.ndarray:
    """The sensor trace with its spectrum mirrored to the Nyquist band:
    x_i (-1)^i, tones at 0.5 - f (the data that alternate in sign, where
    neighbouring samples are anti-correlated; Sec. 5 Fig. 3b)."""
    x = sensor_trace(n, seed).astype(np.int32)
    x[1::2] = -x[1::2]
    return np.clip(x, -32768, 32767).astype(np.int16)


def grf2d(h: int = 4096, w: int = 4096, seed: int = 1, slope: float = 3.0,
          noise: float = 1e-3) -> np.ndarray:
    rng = np.random.default_rng(seed)
    f = _spectral_field((h, w), slope, rng)
    f = f + rng.normal(0.0, noise, f.shape)
    return f.astype(np.float32)


def field3d(n: int = 512, seed: int = 2, slope: float = 4.0, blobs: int = 4, amp: float = 10.0,
            width: float = 8.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    f = _spectral_field((n, n, n), slope, rng)
    idx = np.arange(n, dtype=np.float64)
    for _ in range(blobs):
        c = rng.uniform(0.0, n, 3)
        gx, gy, gz = (np.exp(-((idx - c[d]) ** 2) / (2 * width * width)) for d in range(3))
        f += amp * gx[:, None, None] * gy[None, :, None] * gz[None, None, :]
    return f.astype(np.float64)


def digest(x: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(x).tobytes()).hexdigest()[:16]


def sha256(*parts) -> str:
    """SHA-256 of arrays (their bytes, C order) and strings, in order: the
    fingerprint of a workload's generated inputs in the benchmark results."""
    h = hashlib.sha256()
    for x in parts:
        h.update(x.encode() if isinstance(x, str) else np.ascontiguousarray(x).tobytes())
    return h.hexdigest()


# Workloads named by what they are (used by tests and the benchmark).
SENSOR_I16 = dict(name="int16 sensor trace 262144 samples, fixed rate 4:1",
                  n=262144, block_size=256, rate=(4, 1))
IMAGE_F32 = dict(name="float32 4096x4096 k^-3 field, profile 16 codes at r>=0.9999, fixed quality",
                 shape=(4096, 4096), block_size=256, target=0.9999)
FIELD_F64 = dict(name="float64 512^3 k^-4 field with 4 blobs, profile at r>=0.99999, fixed quality",
                 n=512, block_size=256, target=0.99999)


# ---------------------------------------------------------------- many arrays
# Batched workload: `count` arrays with lengths log-uniform over 4 KB..64 MB
# in bytes (rounded down to the element size), element types uniform over
# int16 / int32 / float32 / float64, fixed rates uniform over 2:1, 3:1, 4:1,
# 6:1.  Contents are wrapped slices, at seeded offsets, of one master signal
# per type (the sensor trace for the integers -- int32 with amplitudes
# summing to 2^27 and noise 8 * 2^16 -- the k^-3 field for float32 and the
# k^-4 field for float64), so the whole batch can be built on the device
# from four masters.
BATCH_DTYPES = ("int16", "int32", "float32", "float64")
BATCH_RATES = ((2, 1), (3, 1), (4, 1), (6, 1))


def batch_specs(count: int = 8192, seed: int = 3, lo_bytes: int = 4096,
                hi_bytes: int = 64 << 20):
    """[(dtype name, elements, (num, den), master offset)] of the batch."""
    rng = np.random.default_rng(seed)
    nbytes = np.exp(rng.uniform(np.log(lo_bytes), np.log(hi_bytes), count))
    kinds = rng.integers(0, 4, count)
    rates = rng.integers(0, 4, count)
    offs = rng.integers(0, 1 << 40, count)
    size = {"int16": 2, "int32": 4, "float32": 4, "float64": 8}
    out = []
    for b, k, r, o in zip(nbytes, kinds, rates, offs):
        dt = BATCH_DTYPES[int(k)]
        out.append((dt, int(b) // size[dt], BATCH_RATES[int(r)], int(o)))
    return out


def batch_masters(n16: int = 1 << 25, field3d_n: int = 256):
    """Master signals of the batched and serving workloads."""
    return {
        "int16": sensor_trace(n16, seed=3),
        "int32": sensor_trace(n16 // 2, seed=4, amp_sum=2.0 ** 27, sigma=8.0 * 2 ** 16,
                              dtype=np.int32),
        "float32": grf2d(4096, 4096, seed=1).reshape(-1),
        "float64": field3d(field3d_n, seed=2).reshape(-1),
    }


# ---------------------------------------------------------------- request trace
def serving_trace(seconds: float = 60.0, rate: float = 2000.0, seed: int = 4,
                  lo_bytes: int = 64 << 10, hi_bytes: int = 256 << 20):
    """Poisson arrivals: [(t, op 'encode'|'decode', 'float32'|'int16', bytes,
    pool offset)] with payload sizes log-uniform over lo..hi bytes."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            break
        op = "encode" if rng.random() < 0.5 else "decode"
        dt = "float32" if rng.random() < 0.5 else "int16"
        nb = int(np.exp(rng.uniform(np.log(lo_bytes), np.log(hi_bytes))))
        out.append((t, op, dt, nb, int(rng.integers(0, 1 << 40))))
    return out
