"""Batched codec (many arrays per launch) against the CPU oracle, through
the C ABI: every container of a mixed batch is byte-identical to the
oracle's encoding of that array, on repeated runs, under every geometry
the tuner may pick, and when the run is captured in a CUDA graph and
replayed."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1303_4994_gb300 import apax as A
from paper_1303_4994_gb300 import build as B
from paper_1303_4994_gb300 import synth

pytestmark = pytest.mark.gpu

NP = {1: np.int8, 2: np.int16, 3: np.int32, 4: np.float32, 5: np.float64}


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    A.lib()
    torch.cuda.init()


def _array(rng, dt, n):
    if dt <= 3:
        info = np.iinfo(NP[dt])
        t = np.arange(n)
        x = np.sin(t * rng.uniform(0.001, 0.1)) * info.max * 0.5 + rng.normal(0, 4, n)
        return np.clip(np.rint(x), info.min, info.max).astype(NP[dt])
    return np.cumsum(rng.standard_normal(n) * np.exp(rng.uniform(-3, 3))).astype(NP[dt])


def _mixed_batch(seed, count, big_blocks=False):
    rng = np.random.default_rng(seed)
    arrays, ps = [], []
    sizes = [0, 1, 3, 255, 256, 257, 4096 + 17, 3 * 4096, 20000]
    for i in range(count):
        dt = int(rng.integers(1, 6))
        n = int(sizes[i % len(sizes)] if i < len(sizes) else rng.integers(1, 40000))
        N = int(rng.choice([64, 256, 1000] + ([16384] if big_blocks else [])))
        if rng.random() < 0.5:
            rate = [(2, 1), (3, 1), (4, 1), (6, 1)][int(rng.integers(0, 4))]
            p = A.params(N, A.FIXED_RATE, rate, 0)
            try:
                A.encoded_size(dt, max(n, 1), p)
            except A.ApaxError:
                p = A.params(N, A.FIXED_QUALITY, (1, 1), int(rng.integers(0, 4096)))
        else:
            p = A.params(N, A.FIXED_QUALITY, (1, 1), int(rng.choice([0, 256, 777, 2048, 4095])))
        if p.mode == A.FIXED_RATE and i % 3 == 0:
            p.search = A.SEARCH_PREDICT  # both fixed-rate policies in one batch
        arrays.append(_array(rng, dt, n))
        ps.append(p)
    return arrays, ps


def _setup(arrays, ps):
    xs = [torch.from_numpy(a).cuda() for a in arrays]
    outs = [torch.full((A.encoded_size(A.TORCH_CODE[x.dtype], x.numel(), p),), 0x5A,
                       dtype=torch.uint8, device="cuda") for x, p in zip(xs, ps)]
    results = torch.zeros(16 * len(xs), dtype=torch.uint8, device="cuda")
    jobs = A.encode_jobs(xs, ps, outs, results)
    ws = torch.empty(A.batch_encode_workspace_size(jobs) + 256, dtype=torch.uint8, device="cuda")
    off = (-ws.data_ptr()) % 256
    ws = ws[off:]
    return xs, outs, results, jobs, ws


def _want(arrays, ps):
    return [O.encode(a, p.block_size, p.mode, p.rate_num, p.rate_den, p.atten_code,
                     search=p.search) for a, p in zip(arrays, ps)]


def _check(outs, results, want):
    rs = A.read_results(results, len(want))
    for i, (o, r, w) in enumerate(zip(outs, rs, want)):
        assert r.status == 0, (i, r)
        assert r.bytes == len(w), (i, r.bytes, len(w))
        got = o[:r.bytes].cpu().numpy().tobytes()
        assert got == w, f"array {i}: container differs"


def test_batch_encode_matches_oracle_repeated_and_all_geometries():
    arrays, ps = _mixed_batch(1, 48)
    want = _want(arrays, ps)
    xs, outs, results, jobs, ws = _setup(arrays, ps)
    plan = A.EncodeBatch(jobs, ws)
    for _ in range(2):
        results.zero_()
        plan.run()
        torch.cuda.synchronize()
        _check(outs, results, want)
    for cfg in [(64, 1), (64, 3), (128, 1), (128, 2), (128, 0)]:
        plan.config = cfg
        results.zero_()
        plan.run()
        torch.cuda.synchronize()
        _check(outs, results, want)
    plan.tune(reps=1)
    threads, ctas = plan.config
    assert threads in (64, 128) and ctas >= 1
    results.zero_()
    plan.run()
    torch.cuda.synchronize()
    _check(outs, results, want)
    plan.close()


def test_batch_encode_large_blocks_use_warp_teams():
    arrays, ps = _mixed_batch(2, 12, big_blocks=True)
    ps[0] = A.params(16384, A.FIXED_QUALITY, (1, 1), 300)
    arrays[0] = _array(np.random.default_rng(9), 4, 3 * 16384 + 5)
    want = _want(arrays, ps)
    xs, outs, results, jobs, ws = _setup(arrays, ps)
    plan = A.EncodeBatch(jobs, ws)
    plan.run()
    torch.cuda.synchronize()
    _check(outs, results, want)
    for cfg in [(32, 1), (64, 2)]:
        try:
            plan.config = cfg
        except A.ApaxError:
            continue
        results.zero_()
        plan.run()
        torch.cuda.synchronize()
        _check(outs, results, want)


def test_batch_encode_graph_replay_and_device_code():
    x = synth.grf2d(256, 256, seed=21).reshape(-1)
    xt = torch.from_numpy(x).cuda()
    nc = 16
    pws, pts, summ = A.profile_buffers(xt, 256, nc)
    A.profile_into(xt, 256, list(A.DEFAULT_CANDIDATES), 0.9999, pws, pts, summ)
    torch.cuda.synchronize()
    code = A.read_summary(summ).recommended_code
    rng = np.random.default_rng(3)
    arrays = [x, _array(rng, 2, 50000), _array(rng, 5, 7777)]
    ps = [A.params(256, A.FIXED_QUALITY, (1, 1), 0), A.params(256, A.FIXED_RATE, (4, 1), 0),
          A.params(256, A.FIXED_QUALITY, (1, 1), 512)]
    want = _want(arrays, ps)
    want[0] = O.encode(x, 256, 1, 1, 1, code)
    xs = [torch.from_numpy(a).cuda() for a in arrays]
    outs = [torch.zeros(A.encoded_size(A.TORCH_CODE[t.dtype], t.numel(), p), dtype=torch.uint8,
                        device="cuda") for t, p in zip(xs, ps)]
    results = torch.zeros(16 * 3, dtype=torch.uint8, device="cuda")
    # array 0 takes its code from the profile summary on the device
    code_dev = summ[8:12].view(torch.int32)
    jobs = A.encode_jobs(xs, ps, outs, results, code_devs=[code_dev, None, None])
    ws = torch.empty(A.batch_encode_workspace_size(jobs) + 256, dtype=torch.uint8, device="cuda")
    ws = ws[(-ws.data_ptr()) % 256:]
    plan = A.EncodeBatch(jobs, ws)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.run(s)  # warm-up outside the capture
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(s)
    for o in outs:
        o.zero_()
    results.zero_()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    _check(outs, results, want)


UINT = {1: np.uint8, 2: np.uint16, 3: np.uint32, 4: np.uint32, 5: np.uint64}


def _decode_batch(containers, arrays, ps, block_sizes=None):
    ys = [torch.full((a.size,), 7, dtype=torch.from_numpy(a[:0]).dtype, device="cuda")
          for a in arrays]
    results = torch.zeros(16 * len(ys), dtype=torch.uint8, device="cuda")
    bs = block_sizes or [p.block_size for p in ps]
    jobs = A.decode_jobs(containers, ys, bs, results)
    ws = A.aligned_workspace(A.batch_decode_workspace_size(jobs))
    return ys, results, A.Batch(jobs, ws)


@pytest.mark.parametrize("big", [False, True])
def test_batch_decode_matches_oracle(big):
    arrays, ps = _mixed_batch(5 + big, 40, big_blocks=big)
    want = _want(arrays, ps)
    containers = [torch.from_numpy(np.frombuffer(w, dtype=np.uint8).copy()).cuda() for w in want]
    ys, results, plan = _decode_batch(containers, arrays, ps)
    for cfg in [None, (64, 1), (128, 2)] if not big else [None, (32, 2), (128, 1)]:
        if cfg is not None:
            plan.config = cfg
        results.zero_()
        for y in ys:
            y.fill_(7)
        plan.run()
        torch.cuda.synchronize()
        rs = A.read_results(results, len(ys))
        for i, (a, w, y, r) in enumerate(zip(arrays, want, ys, rs)):
            assert r.status == 0 and r.bytes == a.size, (i, r)
            yo = O.decode(w, a.dtype, a.size)
            np.testing.assert_array_equal(y.cpu().numpy().view(UINT[A.TORCH_CODE[y.dtype]]),
                                          yo.view(UINT[A.TORCH_CODE[y.dtype]]))
    plan.tune(reps=1)
    plan.close()


def test_batch_decode_reports_per_container_errors():
    arrays, ps = _mixed_batch(8, 10)
    want = _want(arrays, ps)
    containers = [torch.from_numpy(np.frombuffer(w, dtype=np.uint8).copy()).cuda() for w in want]
    bs = [p.block_size for p in ps]
    bad = 6  # declared block size differs from the container's
    bs[bad] = 128 if bs[bad] != 128 else 64
    containers[7] = containers[7][:20].contiguous()  # truncated header
    ys, results, plan = _decode_batch(containers, arrays, ps, block_sizes=bs)
    plan.run()
    torch.cuda.synchronize()
    rs = A.read_results(results, len(ys))
    for i, (a, w, y, r) in enumerate(zip(arrays, want, ys, rs)):
        if i == bad:
            assert r.status == -9
        elif i == 7:
            assert r.status == -9
        else:
            assert r.status == 0, (i, r)
            yo = O.decode(w, a.dtype, a.size)
            np.testing.assert_array_equal(y.cpu().numpy().view(UINT[A.TORCH_CODE[y.dtype]]),
                                          yo.view(UINT[A.TORCH_CODE[y.dtype]]))


def test_batch_profile_matches_oracle():
    import struct
    rng = np.random.default_rng(11)
    arrays, Ns, cands, targets = [], [], [], []
    specs = [(4, 0), (2, 1), (5, 300), (4, 256 * 16 * 3 + 5), (1, 4000), (3, 9000),
             (4, 70000), (5, 33333), (2, 256 * 16)]
    for dt, n in specs:
        arrays.append(_array(rng, dt, n))
        Ns.append(int(rng.choice([64, 256, 1000])))
        k = int(rng.integers(1, 17))
        cands.append(sorted(set(int(c) * 128 for c in rng.choice(32, k, replace=False))))
        targets.append(float(rng.choice([0.9, 0.999, 0.99999])))
    xs = [torch.from_numpy(a).cuda() for a in arrays]
    pts = [torch.zeros(A.POINT_BYTES * len(c), dtype=torch.uint8, device="cuda") for c in cands]
    sums = [torch.zeros(A.SUMMARY_BYTES, dtype=torch.uint8, device="cuda") for _ in cands]
    jobs = A.profile_jobs(xs, Ns, cands, targets, pts, sums)
    ws = A.aligned_workspace(A.batch_profile_workspace_size(jobs))
    plan = A.Batch(jobs, ws)
    for rep in range(2):
        for p in pts + sums:
            p.zero_()
        plan.run()
        torch.cuda.synchronize()
        for i, a in enumerate(arrays):
            po, rec, missed = O.profile(a, N=Ns[i], candidates=cands[i], target=targets[i])
            got = A.read_points(pts[i], len(cands[i]))
            sm = A.read_summary(sums[i])
            assert sm.status == 0 and sm.n == a.size
            for o, g in zip(po, got):
                assert o.code == g.code and o.bytes == g.bytes, (i, o.code, o.bytes, g.bytes)
                for f in ("sx", "sy", "sxx", "sxy", "syy", "sdd", "r"):
                    assert struct.pack("<d", getattr(o, f)) == struct.pack("<d", getattr(g, f)), \
                        (i, f, getattr(o, f), getattr(g, f))
            assert sm.recommended == rec and bool(sm.flags & 1) == missed
        if rep == 0:
            plan.tune(reps=1)
