"""C-ABI checks that need no GPU: the library builds, loads and exports every
function include/apax.h declares; host-side sizes and argument checks agree
with the oracle's closed forms."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1303_4994_gb300 import apax as A
from paper_1303_4994_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return A.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "apax.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(apax_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(A.EXPORTS)
    assert "sm_103a" in A.build_info()


NP = {1: np.int8, 2: np.int16, 3: np.int32, 4: np.float32, 5: np.float64}


@pytest.mark.parametrize("dt", [1, 2, 3, 4, 5])
def test_encoded_size_matches_oracle(lib, dt):
    rng = np.random.default_rng(dt)
    for _ in range(60):
        N = int(rng.choice([64, 68, 256, 1000, 4096, 16384]))
        n = int(rng.integers(0, 5 * N))
        mode = int(rng.integers(0, 2))
        num, den = [(2, 1), (3, 1), (4, 1), (6, 1), (5, 2), (1, 2)][int(rng.integers(0, 6))]
        p = A.params(N, mode, (num, den), 0)
        try:
            want = O.encoded_size(NP[dt], n, N, mode, num, den, 0)
        except O.OracleError as e:
            with pytest.raises(A.ApaxError) as g:
                A.encoded_size(dt, n, p)
            assert g.value.status == e.status
            continue
        assert A.encoded_size(dt, n, p) == want


def test_argument_errors(lib):
    for N in (0, 60, 63, 66, 16388):
        with pytest.raises(A.ApaxError) as e:
            A.encoded_size(2, 100, A.params(N))
        assert e.value.status == -2
    with pytest.raises(A.ApaxError) as e:
        A.encoded_size(9, 100, A.params(256))
    assert e.value.status == -3
    with pytest.raises(A.ApaxError) as e:  # 64:1 on int8 is below the all-zero packet
        A.encoded_size(1, 1000, A.params(256, A.FIXED_RATE, (64, 1)))
    assert e.value.status == -4
    with pytest.raises(A.ApaxError) as e:
        A.encoded_size(4, 1000, A.params(256, A.FIXED_QUALITY, (1, 1), 5000))
    assert e.value.status == -1
    with pytest.raises(A.ApaxError) as e:  # no third fixed-rate search policy
        A.encoded_size(2, 1000, A.params(256, A.FIXED_RATE, (4, 1), 0, search=2))
    assert e.value.status == -1
    assert A.encoded_size(2, 1000, A.params(256, A.FIXED_RATE, (4, 1), 0, A.SEARCH_PREDICT)) == \
        A.encoded_size(2, 1000, A.params(256, A.FIXED_RATE, (4, 1), 0, A.SEARCH_BISECT))
    assert lib.apax_status_string(-9) == b"corrupt stream"
    # fixed-rate size of the int16 sensor workload at 4:1
    assert A.encoded_size(2, 262144, A.params(256, A.FIXED_RATE, (4, 1))) == 131112


def test_derived_metrics_match_oracle(lib):
    rng = np.random.default_rng(3)
    for _ in range(200):
        s = rng.standard_normal(6) * 10 ** rng.uniform(-3, 3, 6)
        s[2] = abs(s[2]); s[4] = abs(s[4]); s[5] = abs(s[5])
        if rng.random() < 0.2:
            s[5] = 0.0
        n = int(rng.integers(1, 10 ** 6))
        p = A.Point(0, 0, 0, *s.tolist(), 0.0)
        got = A.derived(p, n)
        want = O.derived(s, n)
        for k in want:
            assert got[k] == want[k] or (np.isnan(got[k]) and np.isnan(want[k])), k


def test_profile_argument_checks(lib):
    out = ctypes.c_uint64()
    assert lib.apax_profile_workspace_size(4, 1000, 256, 16, ctypes.byref(out)) == 0
    assert out.value > 0
    assert lib.apax_profile_workspace_size(4, 1000, 256, 33, ctypes.byref(out)) == -1


def test_workspace_follows_team_geometry(lib):
    # fixed quality keeps one look-back word per tile: tiles of 4 blocks
    # (teams of 32) up to 4096 blocks, of 16 blocks (teams of 8) above;
    # fixed rate needs only the 64-byte head
    out = ctypes.c_uint64()
    for nb in (1, 5, 1024, 4095, 4096, 4097, 65536):
        n = nb * 256 - 3
        p = A.params(256, A.FIXED_QUALITY, (1, 1), 0)
        assert lib.apax_workspace_size(4, n, ctypes.byref(p), ctypes.byref(out)) == 0
        per = 4 if nb <= 4096 else 16
        assert out.value == 64 + 8 * ((nb + per - 1) // per), nb
        p = A.params(256, A.FIXED_RATE, (4, 1), 0)
        assert lib.apax_workspace_size(4, n, ctypes.byref(p), ctypes.byref(out)) == 0
        assert out.value == 64, nb


def test_profile_from_host_argument_checks(lib):
    # every check returns before any CUDA call (the pointers are never
    # dereferenced on these paths)
    ws_need = ctypes.c_uint64()
    assert lib.apax_profile_workspace_size(4, 100000, 256, 16, ctypes.byref(ws_need)) == 0
    xh, xd, ws, pts, summ = 0x100000, 0x200000, 0x300000, 0x400000, 0x500000
    s1, s2 = 0x1000, 0x2000

    def call(**kw):
        a = dict(x_host=xh, x_dev=xd, dtype=4, n=100000, N=256, chunks=8, ws=ws,
                 wsb=ws_need.value, s=s1, cs=s2)
        a.update(kw)
        return lib.apax_profile_from_host(a["x_host"], a["x_dev"], a["dtype"], a["n"], a["N"], None,
                                          16, 0.9999, a["chunks"], a["ws"], a["wsb"], pts, summ,
                                          a["s"], a["cs"])
    assert call(N=66) == -2                # block size not a multiple of 4
    assert call(dtype=9) == -3             # unknown type
    assert call(x_host=0) == -1            # no input
    assert call(chunks=0) == -1 and call(chunks=65) == -1
    assert call(cs=s1) == -1               # copy stream must differ from the stream
    assert call(ws=0) == -1 and call(ws=ws + 8) == -1  # missing or misaligned workspace
    assert call(wsb=ws_need.value - 8) == -5


def _job(dt=4, n=1000, p=None, x=0x10000, out=0x20000, cap=1 << 20, res=0x30000):
    p = p or A.params(256, A.FIXED_QUALITY, (1, 1), 0)
    return A.EncodeJob(x, dt, 0, n, p, None, out, cap, res)


def _batch_ws(jobs):
    arr = (A.EncodeJob * len(jobs))(*jobs)
    out = ctypes.c_uint64()
    st = A.lib().apax_batch_encode_workspace_size(arr, len(jobs), ctypes.byref(out))
    return st, out.value


def test_batch_argument_checks(lib):
    # host-side validation of every job, with apax_encode's rules
    st, ws = _batch_ws([_job(), _job(dt=2, n=0), _job(dt=5, n=77777)])
    assert st == 0 and ws > 0 and ws % 256 == 0
    assert _batch_ws([_job(p=A.params(66, 1))])[0] == -2
    assert _batch_ws([_job(), _job(dt=9)])[0] == -3
    assert _batch_ws([_job(p=A.params(256, A.FIXED_RATE, (1000, 1)))])[0] == -4
    assert _batch_ws([_job(cap=40)])[0] == -5
    assert _batch_ws([_job(res=0)])[0] == -1
    assert _batch_ws([_job(x=0x10002)])[0] == -1   # misaligned float32 input
    arr = (A.EncodeJob * 1)(_job())
    out = ctypes.c_uint64()
    assert A.lib().apax_batch_encode_workspace_size(arr, 0, ctypes.byref(out)) == -1
    # fixed-rate jobs need no look-back words; fixed-quality ones grow with tiles
    fr = _batch_ws([_job(n=1 << 20, p=A.params(256, A.FIXED_RATE, (4, 1)), cap=1 << 22)])[1]
    fq = _batch_ws([_job(n=1 << 20, cap=1 << 23)])[1]
    assert fq > fr


def test_copy_container_argument_checks(lib):
    # host-side checks of apax_copy_container (nothing is launched): null or
    # misaligned pointers and overlapping source and destination are refused,
    # an empty destination is a no-op
    f = lib.apax_copy_container
    src, res, dst = 0x10000, 0x20000, 0x40000
    assert f(None, res, dst, 64, None) == -1
    assert f(src, None, dst, 64, None) == -1
    assert f(src, res, None, 64, None) == -1
    assert f(src + 2, res, dst, 64, None) == -1   # source not 4-byte aligned
    assert f(src, res, dst + 1, 64, None) == -1   # destination not 4-byte aligned
    assert f(src, res + 4, dst, 64, None) == -1   # result not 8-byte aligned
    assert f(src, res, src + 32, 64, None) == -1  # destination inside the source span
    assert f(src + 32, res, src, 64, None) == -1  # and the other way round
    assert f(src, res, dst, 0, None) == 0         # nothing to copy
