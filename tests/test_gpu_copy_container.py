"""apax_copy_container: a container moved out of device memory with its size
read on the device, to pinned host memory (written over the host link) or
to device memory, on a stream that waits for the encode by an event."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1303_4994_gb300 import apax as A
from paper_1303_4994_gb300 import build as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    A.lib()
    torch.cuda.init()


def _encoded(n, code, seed):
    x = np.cumsum(np.random.default_rng(seed).standard_normal(n)).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    p = A.params(256, A.FIXED_QUALITY, (1, 1), code)
    out = torch.zeros(A.encoded_size(A.F32, n, p), dtype=torch.uint8, device="cuda")
    ws = torch.empty(A.workspace_size(A.F32, n, p), dtype=torch.uint8, device="cuda")
    res = A.new_result("cuda")
    return x, xt, p, out, ws, res


@pytest.mark.parametrize("n", [1, 1000, 256 * 5000 + 3])
def test_copy_to_pinned_host_beside_the_decode(n):
    x, xt, p, out, ws, res = _encoded(n, 1536, n)
    side = torch.cuda.Stream()
    done = torch.cuda.Event()
    host = torch.full((out.numel(),), 0xA5, dtype=torch.uint8).pin_memory()
    for rep in range(2):  # the second call overwrites the first's bytes
        host.fill_(0xA5 if rep == 0 else 0x3C)
        A.encode_into(xt, p, out, ws, res)
        done.record()
        side.wait_event(done)
        A.copy_container_into(out, res, host, side)
        y = A.decode(out, torch.float32, n)  # on the current stream, beside the copy
        torch.cuda.synchronize()
        r = A.read_result(res)
        want = O.encode(x, 256, O.MODE_FQ, 1, 1, 1536, threads=0)
        assert r.bytes == len(want)
        assert host[:r.bytes].numpy().tobytes() == want
        assert bool((host[r.bytes:] == (0xA5 if rep == 0 else 0x3C)).all())  # nothing past the size
        assert torch.equal(y.view(torch.int32).cpu(),
                           torch.from_numpy(O.decode(want, np.float32, n)).view(torch.int32))


def test_copy_capacity_alignment_and_device_target():
    x, xt, p, out, ws, res = _encoded(256 * 40 + 17, 700, 5)
    A.encode_into(xt, p, out, ws, res)
    torch.cuda.synchronize()
    nb = A.read_result(res).bytes
    dev = torch.zeros(nb + 64, dtype=torch.uint8, device="cuda")
    A.copy_container_into(out, res, dev)
    short = torch.zeros(100, dtype=torch.uint8, device="cuda")
    A.copy_container_into(out, res, short)  # truncated to the capacity
    torch.cuda.synchronize()
    assert torch.equal(dev[:nb], out[:nb]) and bool((dev[nb:] == 0).all())
    assert torch.equal(short, out[:100])
    with pytest.raises(A.ApaxError) as e:
        A.copy_container_into(out, res, dev[1:])  # not 4-byte aligned
    assert e.value.status == -1
    with pytest.raises(A.ApaxError) as e:
        A.copy_container_into(out, res, out[4:])  # overlaps the source
    assert e.value.status == -1
