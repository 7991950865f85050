"""CPU oracle of the APAX codec (test infrastructure only).

Plain, slow ctypes wrapper around ``apax_oracle.c``, a scalar restatement of
the APAX encoder, decoder and profiler of Wegener, arXiv 1303.4994 (Sec. 4
profiler, Sec. 5 signal characteristics, Sec. 6 encoder block diagram and
bit packer).  Only the test-suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the product library
never does.  It shares no code with the CUDA path.

Functions whose results the paper pins only through our own readings are
listed in the module docstring of ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "apax_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

DTYPES = {1: np.int8, 2: np.int16, 3: np.int32, 4: np.float32, 5: np.float64}
DTYPE_CODE = {np.dtype(v): k for k, v in DTYPES.items()}
MODE_FR, MODE_FQ = 0, 1

ST_OK, ST_INVALID_ARG, ST_BLOCK_SIZE, ST_DTYPE, ST_RATE = 0, -1, -2, -3, -4
ST_CAPACITY, ST_TOO_LARGE, ST_NONFINITE, ST_CORRUPT = -5, -6, -8, -9


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FP contraction, so binary64 metric
    arithmetic is exactly the IEEE operations written in the source)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call([
            "gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class Point(ctypes.Structure):
    _fields_ = [("code", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("bytes", ctypes.c_uint64),
                ("sx", ctypes.c_double), ("sy", ctypes.c_double),
                ("sxx", ctypes.c_double), ("sxy", ctypes.c_double),
                ("syy", ctypes.c_double), ("sdd", ctypes.c_double),
                ("r", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        u64, i32, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
        u32, p64 = ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64)
        _lib.oracle_encoded_size.argtypes = [i32, u64, u32, i32, i32, u32, u32, i32, p64]
        _lib.oracle_encode.argtypes = [vp, i32, u64, u32, i32, u32, u32, i32, vp, u64, p64]
        _lib.oracle_encode_s.argtypes = [vp, i32, u64, u32, i32, i32, u32, u32, i32, i32, vp, u64,
                                         p64]
        _lib.oracle_decode.argtypes = [vp, u64, vp, i32, u64]
        _lib.oracle_metrics.argtypes = [vp, vp, i32, u64, u32, vp]
        _lib.oracle_block_sums.argtypes = [vp, vp, i32, u64, u32, u64, u64, vp]
        _lib.oracle_corr.argtypes = [ctypes.c_double] * 3
        _lib.oracle_corr.restype = ctypes.c_double
        _lib.oracle_profile.argtypes = [vp, i32, u64, u32, i32, vp, i32, ctypes.c_double, vp,
                                        ctypes.POINTER(ctypes.c_int)]
        _lib.oracle_bits.argtypes = [ctypes.c_int32]
        _lib.oracle_recip.argtypes = [i32]
        _lib.oracle_recip.restype = ctypes.c_int64
        _lib.oracle_rne_shift.argtypes = [ctypes.c_int64, i32]
        _lib.oracle_rne_shift.restype = ctypes.c_int64
        _lib.oracle_jee_encode.argtypes = [vp, i32, vp]
        _lib.oracle_jee_decode.argtypes = [vp, i32, i32, vp]
        _lib.oracle_quantise.argtypes = [vp, i32, u64, i32, i32]
        _lib.oracle_quantise.restype = ctypes.c_int32
        _lib.oracle_dequantise.argtypes = [ctypes.c_int32, i32, i32, i32, vp]
        _lib.oracle_block_exponent.argtypes = [vp, i32, u64, i32, ctypes.POINTER(ctypes.c_int)]
        _lib.oracle_packet_bits.argtypes = [vp, i32, u64, u32, i32, u64, i32, i32, p64]
        _lib.oracle_streams.argtypes = [vp, i32, u64, u32, i32, u64, u64, vp]
        _lib.oracle_fr_code.argtypes = [vp, i32, u64, u32, i32, u64, i32, u64, i32,
                                        ctypes.POINTER(ctypes.c_int)]
        _lib.oracle_encode_blocks.argtypes = [vp, i32, u64, u32, i32, i32, u32, u32, i32, i32,
                                              u64, u64, vp, u64, vp]
        _lib.oracle_fr_budget.argtypes = [i32, u32, i32, i32, u32, u32, p64]
        _lib.oracle_min_packet.argtypes = [i32, u32, i32, i32, p64]
        _lib.oracle_derived.argtypes = [vp, u64, vp]
        _lib.oracle_threads.argtypes = [i32]
        _lib.oracle_encode_mt.argtypes = [vp, i32, u64, u32, i32, i32, u32, u32, i32, i32, vp,
                                          u64, p64, i32]
        _lib.oracle_decode_mt.argtypes = [vp, u64, vp, i32, u64, i32]
        _lib.oracle_metrics_mt.argtypes = [vp, vp, i32, u64, u32, vp, i32]
        _lib.oracle_profile_mt.argtypes = [vp, i32, u64, u32, i32, vp, i32, ctypes.c_double, vp,
                                           ctypes.POINTER(ctypes.c_int), i32]
    return _lib


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: oracle status {status}")
        self.status = status


def _code(x: np.ndarray) -> int:
    return DTYPE_CODE[x.dtype]


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# format options (container version 2): BFPE groups of 8, the sum stream
FMT_GROUP8, FMT_SUM_STREAM = 1, 2


def encoded_size(dtype, n: int, N: int = 256, mode: int = MODE_FQ, num: int = 1,
                 den: int = 1, code: int = 0, fmt: int = 0) -> int:
    out = ctypes.c_uint64()
    st = lib().oracle_encoded_size(DTYPE_CODE[np.dtype(dtype)], n, N, fmt, mode, num, den, code,
                                   ctypes.byref(out))
    if st:
        raise OracleError(st, "encoded_size")
    return out.value


def threads(t: int = 0) -> int:
    """Threads the threaded drivers use for `t` (0: one per online core)."""
    return lib().oracle_threads(t)


SEARCH_BISECT, SEARCH_PREDICT = 0, 1


def encode(x: np.ndarray, N: int = 256, mode: int = MODE_FQ, num: int = 1, den: int = 1,
           code: int = 0, threads: int | None = None, search: int = SEARCH_BISECT,
           fmt: int = 0) -> bytes:
    """Encode a C-contiguous array; returns the container bytes.  threads:
    None runs the plain sequential encoder; an int runs the same per-block
    code on that many threads over block ranges (0 = all cores).  search:
    the fixed-rate search policy (BISECT or PREDICT).  fmt: format options
    (FMT_GROUP8 | FMT_SUM_STREAM; 0 writes a version-1 container)."""
    x = np.ascontiguousarray(x).reshape(-1)
    cap = encoded_size(x.dtype, x.size, N, mode, num, den, code, fmt)
    buf = np.zeros(cap, dtype=np.uint8)
    out = ctypes.c_uint64()
    if threads is None:
        st = lib().oracle_encode_s(_ptr(x), _code(x), x.size, N, fmt, mode, num, den, code,
                                   search, _ptr(buf), cap, ctypes.byref(out))
    else:
        st = lib().oracle_encode_mt(_ptr(x), _code(x), x.size, N, fmt, mode, num, den, code,
                                    search, _ptr(buf), cap, ctypes.byref(out), threads)
    if st:
        raise OracleError(st, "encode")
    return buf[:out.value].tobytes()


def decode(stream: bytes, dtype, n: int, threads: int | None = None) -> np.ndarray:
    """Decode a container (threads as for encode)."""
    s = np.frombuffer(stream, dtype=np.uint8)
    y = np.zeros(max(n, 1), dtype=dtype)
    if threads is None:
        st = lib().oracle_decode(_ptr(s), s.size, _ptr(y), DTYPE_CODE[np.dtype(dtype)], n)
    else:
        st = lib().oracle_decode_mt(_ptr(s), s.size, _ptr(y), DTYPE_CODE[np.dtype(dtype)], n,
                                    threads)
    if st:
        raise OracleError(st, "decode")
    return y[:n]


def decode_status(stream: bytes, dtype, n: int) -> int:
    s = np.frombuffer(stream, dtype=np.uint8).copy()
    y = np.zeros(max(n, 1), dtype=dtype)
    return lib().oracle_decode(_ptr(s), s.size, _ptr(y), DTYPE_CODE[np.dtype(dtype)], n)


def metrics(x: np.ndarray, y: np.ndarray, N: int = 256, threads: int | None = None) -> np.ndarray:
    """[sum x, sum y, sum x^2, sum xy, sum y^2, sum d^2] (binary64)."""
    x = np.ascontiguousarray(x).reshape(-1)
    y = np.ascontiguousarray(y).reshape(-1)
    out = np.zeros(6, dtype=np.float64)
    if threads is None:
        st = lib().oracle_metrics(_ptr(x), _ptr(y), _code(x), x.size, N, _ptr(out))
    else:
        st = lib().oracle_metrics_mt(_ptr(x), _ptr(y), _code(x), x.size, N, _ptr(out), threads)
    if st:
        raise OracleError(st, "metrics")
    return out


def block_sums(x: np.ndarray, y: np.ndarray, N: int, b0: int, b1: int) -> np.ndarray:
    x = np.ascontiguousarray(x).reshape(-1)
    y = np.ascontiguousarray(y).reshape(-1)
    out = np.zeros((b1 - b0, 6), dtype=np.float64)
    st = lib().oracle_block_sums(_ptr(x), _ptr(y), _code(x), x.size, N, b0, b1, _ptr(out))
    if st:
        raise OracleError(st, "block_sums")
    return out


DERIVED = ("r", "r_centred", "snr_db", "rms_pct", "rms_db", "mean_x", "mean_y", "mean_d",
           "std_x", "std_y", "std_d")


def derived(sums, n: int) -> dict:
    s = np.asarray(sums, dtype=np.float64)
    out = np.zeros(len(DERIVED), dtype=np.float64)
    lib().oracle_derived(_ptr(s), n, _ptr(out))
    return dict(zip(DERIVED, out.tolist()))


def corr(sxx: float, sxy: float, syy: float) -> float:
    return lib().oracle_corr(sxx, sxy, syy)


DEFAULT_CANDIDATES = tuple(256 * i for i in range(16))


def profile(x: np.ndarray, N: int = 256, candidates=DEFAULT_CANDIDATES, target: float = 0.99999,
            threads: int | None = None, fmt: int = 0):
    """Returns (points, recommended_index, target_missed); threads and fmt
    as for encode."""
    x = np.ascontiguousarray(x).reshape(-1)
    c = np.asarray(candidates, dtype=np.uint16)
    pts = (Point * len(c))()
    rec = ctypes.c_int()
    if threads is None:
        st = lib().oracle_profile(_ptr(x), _code(x), x.size, N, fmt, _ptr(c), len(c), target,
                                  pts, ctypes.byref(rec))
    else:
        st = lib().oracle_profile_mt(_ptr(x), _code(x), x.size, N, fmt, _ptr(c), len(c), target,
                                     pts, ctypes.byref(rec), threads)
    if st < 0:
        raise OracleError(st, "profile")
    return list(pts), rec.value, st == 1


def bits(v: int) -> int:
    return lib().oracle_bits(v)


def recip(m: int) -> int:
    return lib().oracle_recip(m)


def rne_shift(t: int, s: int) -> int:
    return lib().oracle_rne_shift(t, s)


def jee_encode(exps) -> list:
    e = np.asarray(exps, dtype=np.int32)
    nib = np.zeros(2 * len(e) + 2, dtype=np.uint8)
    t = lib().oracle_jee_encode(_ptr(e), len(e), _ptr(nib))
    return nib[:t].tolist()


def jee_decode(nibbles, G: int):
    """Returns (exponents, nibbles consumed) or (None, -1) for a malformed stream."""
    nib = np.asarray(nibbles, dtype=np.uint8)
    e = np.zeros(max(G, 1), dtype=np.int32)
    t = lib().oracle_jee_decode(_ptr(nib), len(nib), G, _ptr(e))
    if t < 0:
        return None, -1
    return e[:G].tolist(), t


def quantise(x: np.ndarray, i: int, code: int, Eb: int = 0) -> int:
    x = np.ascontiguousarray(x)
    return lib().oracle_quantise(_ptr(x), _code(x), i, code, Eb)


def dequantise(q: int, dtype, code: int, Eb: int = 0):
    y = np.zeros(1, dtype=dtype)
    st = lib().oracle_dequantise(q, DTYPE_CODE[np.dtype(dtype)], code, Eb, _ptr(y))
    if st:
        raise OracleError(st, "dequantise")
    return y[0]


def block_exponent(x: np.ndarray, off: int, L: int) -> int:
    x = np.ascontiguousarray(x)
    e = ctypes.c_int()
    st = lib().oracle_block_exponent(_ptr(x), _code(x), off, L, ctypes.byref(e))
    if st:
        raise OracleError(st, "block_exponent")
    return e.value


def packet_bits(x: np.ndarray, N: int, j: int, code: int, s: int, fmt: int = 0) -> int:
    x = np.ascontiguousarray(x).reshape(-1)
    out = ctypes.c_uint64()
    st = lib().oracle_packet_bits(_ptr(x), _code(x), x.size, N, fmt, j, code, s,
                                  ctypes.byref(out))
    if st:
        raise OracleError(st, "packet_bits")
    return out.value


def streams(x: np.ndarray, N: int, b0: int, b1: int, fmt: int = 0) -> list:
    x = np.ascontiguousarray(x).reshape(-1)
    out = np.zeros(b1 - b0, dtype=np.int32)
    st = lib().oracle_streams(_ptr(x), _code(x), x.size, N, fmt, b0, b1, _ptr(out))
    if st:
        raise OracleError(st, "streams")
    return out.tolist()


def fr_code(x: np.ndarray, N: int, j: int, s: int, budget: int, search: int = SEARCH_BISECT,
            fmt: int = 0) -> int:
    x = np.ascontiguousarray(x).reshape(-1)
    out = ctypes.c_int()
    st = lib().oracle_fr_code(_ptr(x), _code(x), x.size, N, fmt, j, s, budget, search,
                              ctypes.byref(out))
    if st:
        raise OracleError(st, "fr_code")
    return out.value


def fr_budget(dtype, N: int, L: int, num: int, den: int, fmt: int = 0) -> int:
    out = ctypes.c_uint64()
    st = lib().oracle_fr_budget(DTYPE_CODE[np.dtype(dtype)], N, fmt, L, num, den,
                                ctypes.byref(out))
    if st:
        raise OracleError(st, "fr_budget")
    return out.value


def min_packet(dtype, N: int, L: int, fmt: int = 0) -> int:
    out = ctypes.c_uint64()
    st = lib().oracle_min_packet(DTYPE_CODE[np.dtype(dtype)], N, fmt, L, ctypes.byref(out))
    if st:
        raise OracleError(st, "min_packet")
    return out.value


def encode_blocks(x: np.ndarray, N: int, mode: int, num: int, den: int, code: int, b0: int,
                  b1: int, search: int = SEARCH_BISECT, fmt: int = 0):
    """Packets of blocks [b0, b1) as a list of bytes objects."""
    x = np.ascontiguousarray(x).reshape(-1)
    maxp = 4 * ((48 + 8 * (N // 4) + 32 * N + 31) // 32)
    cap = maxp * (b1 - b0)
    buf = np.zeros(cap, dtype=np.uint8)
    lens = np.zeros(b1 - b0, dtype=np.uint64)
    st = lib().oracle_encode_blocks(_ptr(x), _code(x), x.size, N, fmt, mode, num, den, code,
                                    search, b0, b1, _ptr(buf), cap, _ptr(lens))
    if st:
        raise OracleError(st, "encode_blocks")
    out, pos = [], 0
    for L in lens.tolist():
        out.append(buf[pos:pos + L].tobytes())
        pos += L
    return out
