"""Request server with continuous batching, through the C ABI: every
request's output is identical to the single-array call on the same input,
whether it runs alone or in a mix of encodes and decodes of mixed sizes and
types; a small arena throttles admission without losing or corrupting
requests; the arena's bytes in use never exceed its size."""
import time

import numpy as np
import pytest
import torch

import oracle as O
from paper_1303_4994_gb300 import apax as A
from paper_1303_4994_gb300 import build as B
from paper_1303_4994_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    A.lib()
    torch.cuda.init()


def _requests(seed, count):
    """(op, array, params, container-for-decode) tuples: float32 fields at a
    fixed quality and int16 traces at a fixed rate, as in the serving mix."""
    rng = np.random.default_rng(seed)
    field = synth.grf2d(512, 512, seed=seed).reshape(-1)
    out = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(16384), np.log(200000))))
        if rng.random() < 0.5:
            off = int(rng.integers(0, field.size))
            x = np.resize(np.roll(field, -off), n).astype(np.float32)
            p = A.params(256, A.FIXED_QUALITY, (1, 1), 2048)
        else:
            x = synth.sensor_trace(n, seed=int(rng.integers(0, 1 << 30)))
            p = A.params(256, A.FIXED_RATE, (4, 1), 0)
        op = A.OP_ENCODE if rng.random() < 0.5 else A.OP_DECODE
        c = None
        if op == A.OP_DECODE:
            c = O.encode(x, 256, p.mode, p.rate_num, p.rate_den, p.atten_code)
        out.append((op, x, p, c))
    return out


def _alone(op, x, p, c):
    xt = torch.from_numpy(x).cuda()
    if op == A.OP_ENCODE:
        return A.encode(xt, 256, p.mode, (p.rate_num, p.rate_den), p.atten_code).cpu().numpy()
    ct = torch.from_numpy(np.frombuffer(c, np.uint8).copy()).cuda()
    return A.decode(ct, xt.dtype, x.size).cpu().numpy().view(np.uint8)


def _run_server(reqs, arena_bytes, slots=4, max_batch=64, stagger=0.0):
    arena = A.aligned_workspace(arena_bytes)
    srv = A.Server(arena, slots=slots, max_batch=max_batch)
    inputs = {}
    for i, (op, x, p, c) in enumerate(reqs):
        xt = torch.from_numpy(x).cuda()
        if op == A.OP_ENCODE:
            inputs[i] = (xt,)
        else:
            inputs[i] = (torch.from_numpy(np.frombuffer(c, np.uint8).copy()).cuda(), xt)
    torch.cuda.synchronize()
    got = {}
    peak = 0
    pending = list(range(len(reqs)))
    t_end = time.time() + 120
    while len(got) < len(reqs):
        assert time.time() < t_end, "server made no progress"
        # submit a few at a time so that requests arrive while others run
        for _ in range(3):
            if pending:
                i = pending.pop(0)
                op, x, p, c = reqs[i]
                if op == A.OP_ENCODE:
                    srv.submit_encode(i, inputs[i][0], p)
                else:
                    srv.submit_decode(i, inputs[i][0], inputs[i][1].dtype, x.size, 256)
        for comp in srv.poll():
            op, x, p, c = reqs[comp.id]
            assert comp.status == 0, (comp.id, comp.status)
            nb = comp.bytes if op == A.OP_ENCODE else x.size * x.itemsize
            got[comp.id] = srv.output(comp, nb).cpu().numpy().copy()
            assert comp.t_arrival <= comp.t_submit + 1e-9 <= comp.t_launch + 1e-6 <= comp.t_done + 1e-6
            srv.release(comp.out)
        st = srv.stats()
        peak = max(peak, st["arena_used"])
        assert st["arena_used"] <= arena_bytes
        if stagger:
            time.sleep(stagger)
    st = srv.stats()
    srv.close()
    return got, st, peak


def test_server_mix_equals_alone():
    reqs = _requests(1, 40)
    got, st, peak = _run_server(reqs, 1 << 30)
    assert st["completed"] == len(reqs) and st["arena_used"] == 0
    assert st["steps"] < len(reqs)  # requests were batched together
    for i, (op, x, p, c) in enumerate(reqs):
        want = _alone(op, x, p, c)
        if op == A.OP_ENCODE:
            assert got[i].tobytes() == want.tobytes(), i
            assert want.tobytes() == O.encode(x, 256, p.mode, p.rate_num, p.rate_den, p.atten_code)
        else:
            assert got[i].tobytes() == want.tobytes(), i
            assert want.tobytes() == O.decode(c, x.dtype, x.size).tobytes(), i


def test_server_small_arena_throttles_admission():
    reqs = _requests(2, 24)
    biggest = max(x.size * x.itemsize for _, x, _, _ in reqs)
    cap = 3 * biggest + (1 << 20)  # a few requests at a time
    got, st, peak = _run_server(reqs, cap, slots=2, max_batch=8)
    assert st["completed"] == len(reqs) and peak <= cap
    for i, (op, x, p, c) in enumerate(reqs):
        assert got[i].tobytes() == _alone(op, x, p, c).tobytes(), i
        if op == A.OP_DECODE:
            assert got[i].tobytes() == O.decode(c, x.dtype, x.size).tobytes(), i


def test_server_rejects_bad_requests_at_submit():
    arena = A.aligned_workspace(1 << 20)
    srv = A.Server(arena, slots=1, max_batch=4)
    x = torch.zeros(1000, dtype=torch.float32, device="cuda")
    with pytest.raises(A.ApaxError) as e:
        srv.submit_encode(0, x, A.params(66, A.FIXED_QUALITY))
    assert e.value.status == -2
    big = torch.zeros(1 << 20, dtype=torch.float32, device="cuda")
    with pytest.raises(A.ApaxError) as e:
        srv.submit_encode(1, big, A.params(256, A.FIXED_QUALITY))
    assert e.value.status == -5  # can never fit the arena
    srv.close()
