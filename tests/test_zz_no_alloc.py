"""apax_encode_noalloc: the encode entry point for callers that cannot
allocate device memory (it keeps its scratch in the library's fixed device
array instead of a caller workspace).

Checked through the C ABI against apax_encode on the same inputs, byte for
byte (the codec's tolerance is exact equality), on two calls in a row, so a
second call that reused stale scratch contents from the first would show.
This file sorts last so that a failure here never hides the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1303_4994_gb300 import apax as A
from paper_1303_4994_gb300 import build as B
from paper_1303_4994_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    B.build()
    return A.lib()


def _reference(x, p):
    dc = A.TORCH_CODE[x.dtype]
    cap = A.encoded_size(dc, x.numel(), p)
    out = torch.zeros(cap, dtype=torch.uint8, device=x.device)
    ws = torch.empty(A.workspace_size(dc, x.numel(), p), dtype=torch.uint8, device=x.device)
    res = A.new_result(x.device)
    A.encode_into(x, p, out, ws, res)
    r = A.read_result(res)
    assert r.status == 0
    return out[:r.bytes].cpu().numpy().tobytes()


def _noalloc(lib, x, p):
    dc = A.TORCH_CODE[x.dtype]
    cap = A.encoded_size(dc, x.numel(), p)
    out = torch.full((cap,), 0xA5, dtype=torch.uint8, device=x.device)
    res = A.new_result(x.device)
    st = lib.apax_encode_noalloc(x.data_ptr(), dc, x.numel(), ctypes.byref(p), out.data_ptr(),
                                 cap, res.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0
    r = A.read_result(res)
    assert r.status == 0
    return out[:r.bytes].cpu().numpy().tobytes()


def test_noalloc_matches_encode_twice(lib):
    cases = [
        (torch.from_numpy(synth.grf2d(512, 512, seed=31).reshape(-1)).cuda(),
         A.params(256, A.FIXED_QUALITY, (1, 1), 2048)),
        (torch.from_numpy(synth.sensor_trace(50000, seed=32)).cuda(),
         A.params(256, A.FIXED_RATE, (4, 1), 0)),
        (torch.from_numpy(synth.grf2d(300, 301, seed=33).astype(np.float64).reshape(-1)).cuda(),
         A.params(1000, A.FIXED_QUALITY, (1, 1), 300)),
    ]
    for x, p in cases:
        want = _reference(x, p)
        first = _noalloc(lib, x, p)
        second = _noalloc(lib, x, p)
        assert first == want
        assert second == want
        y = A.decode(torch.frombuffer(bytearray(second), dtype=torch.uint8).cuda(), x.dtype,
                     x.numel())
        assert y.numel() == x.numel()


def test_noalloc_rejects_more_tiles_than_its_array(lib):
    # the smallest fixed-quality float32 encode (whole 256-sample blocks)
    # whose tile table no longer fits the fixed array: refused on the host
    p = A.params(256, A.FIXED_QUALITY, (1, 1), 0)

    def need(blocks):
        return A.workspace_size(A.F32, 256 * blocks, p)

    lo, hi = 1, 2
    while need(hi) <= A.NOALLOC_SCRATCH_BYTES:
        lo, hi = hi, 2 * hi
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if need(mid) <= A.NOALLOC_SCRATCH_BYTES:
            lo = mid
        else:
            hi = mid
    n = 256 * hi
    assert need(hi) > A.NOALLOC_SCRATCH_BYTES >= need(lo)
    x = torch.zeros(n, dtype=torch.float32, device="cuda")
    cap = A.encoded_size(A.F32, n, p)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    res = A.new_result("cuda")
    st = lib.apax_encode_noalloc(x.data_ptr(), A.F32, n, ctypes.byref(p), out.data_ptr(), cap,
                                 res.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == -5
    del x, out
    torch.cuda.empty_cache()
