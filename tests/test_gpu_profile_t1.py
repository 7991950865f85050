"""GPU parity of the one-block-per-thread float32 profiler sweep.

Arrays of at least 16,384 blocks of at most 256 float32 samples, swept with
code 0 first and power-of-two attenuations after it, take the sweep that
gives each thread one block; blocks it does not cover exactly hand their
run (16 blocks) to the team sweep.  Every point (bytes, the six sums, r)
must equal the oracle's bit for bit: default ladders, candidate counts that
fill one, two or three walks, block sizes 64..256, ragged tails, samples far
below the block maximum, extreme block exponents, a non-finite sample (the
status), and decisions that cross CTA and run boundaries.
"""
import struct

import numpy as np
import pytest
import torch

import oracle as O
from paper_1303_4994_gb300 import apax as A
from paper_1303_4994_gb300 import build as B
from paper_1303_4994_gb300 import synth

pytestmark = pytest.mark.gpu

MIN_BLOCKS = 16384


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    A.lib()
    torch.cuda.init()


def _check(x, N, cands, target=0.9999):
    pts_o, rec_o, missed_o = O.profile(x, N=N, candidates=cands, target=target, threads=0)
    xt = torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).cuda()
    pts, summ = A.profile(xt, N, cands, target)
    assert summ.status == 0
    for po, pg in zip(pts_o, pts):
        assert (po.code, po.bytes) == (pg.code, pg.bytes), (po.code, po.bytes, pg.bytes)
        for f in ("sx", "sy", "sxx", "sxy", "syy", "sdd", "r"):
            a, b = getattr(po, f), getattr(pg, f)
            assert struct.pack("<d", a) == struct.pack("<d", b), (po.code, f, a, b)
    assert summ.recommended == rec_o and bool(summ.flags & 1) == missed_o


def _walk(n, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return (np.cumsum(rng.standard_normal(n)) * scale).astype(np.float32)


@pytest.mark.parametrize("N", [64, 128, 200, 256])
def test_t1_default_ladder_block_sizes(N):
    x = _walk(N * MIN_BLOCKS + 5 * N, seed=N)
    _check(x, N, list(A.DEFAULT_CANDIDATES))


@pytest.mark.parametrize("cands", [
    [0],                                    # code 0 only
    [0, 128],                               # one walked code, taken in the code-0 pass
    [0] + [128 * k for k in range(1, 6)],   # one full walk of 5
    [0] + [128 * k for k in range(1, 7)],   # 5, and the sixth in the code-0 pass
    [0] + [128 * k for k in range(1, 10)],  # 5 + 4
    [0] + [128 * k for k in range(1, 32)],  # 5 + 5 + 5 + 5 + 3, and k = 24..31 all zero
    [0, 384, 1024, 2048, 3968],
])
def test_t1_candidate_counts(cands):
    x = _walk(64 * MIN_BLOCKS + 333, seed=len(cands))
    _check(x, 64, cands)


def test_t1_error_sum_at_its_bound():
    # blocks of +-(2^23 - 1) (block exponent 23, X = x): at k = 1 every sample
    # has q = RNE(X / 2) on a tie, so (q0 - 2 q) q = -2^22 and a block's
    # 32-bit error sum reaches -2^30; the other codes and blocks of a walk
    # (k up to 22) around them
    rng = np.random.default_rng(41)
    N = 256
    x = _walk(N * MIN_BLOCKS + 3 * N, seed=41, scale=1000.0)
    m = np.float32(2 ** 23 - 1)
    for b in range(0, MIN_BLOCKS, 97):
        x[b * N:(b + 1) * N] = np.where(rng.random(N) < 0.5, m, -m)
    cands = [0, 128] + [256 * k for k in range(1, 12)]
    _check(x, N, cands)


def test_t1_image_field_full_ladder():
    x = synth.grf2d(1024, 1024, seed=5).reshape(-1)  # 16,384 blocks of 64
    _check(x, 64, list(A.DEFAULT_CANDIDATES))


def test_t1_exceptional_blocks_fall_back():
    # tiny samples (below 2^(Eb-24)), a subnormal block, huge and tiny block
    # exponents, exact zeros and a zero block, spread over runs and CTA edges
    N = 64
    nb = MIN_BLOCKS + 37
    x = _walk(N * nb - 11, seed=77)
    rng = np.random.default_rng(78)
    for b in rng.choice(nb - 1, 200, replace=False):
        x[N * b + int(rng.integers(0, N))] *= np.float32(2.0 ** -int(rng.integers(20, 60)))
    x[N * 64:N * 65] = 0.0                        # an all-zero block (Eb = 0)
    x[N * 127:N * 128] *= np.float32(2.0 ** -120)  # block exponent near -120
    x[N * 128:N * 129] = np.float32(1e-44)        # subnormal block
    x[N * 255:N * 256] *= np.float32(2.0 ** 90)   # Eb + k beyond 127 at large k
    x[N * 1023 + 5] = 0.0
    x[N * 4096:N * 4100] *= np.float32(2.0 ** -82)  # just below the sweep's exponent range
    x[N * 300 + 7] *= np.float32(2.0 ** -100)     # deeper than the side sums' grid
    x[N * 301 + 9] = np.float32(3e-45)            # a subnormal in a unit-scale block
    x[-3] *= np.float32(2.0 ** -40)               # a tiny sample in the ragged last block
    _check(x, N, list(A.DEFAULT_CANDIDATES))
    _check(x, N, [0, 128, 1024, 2048, 3968])


def test_t1_tiny_samples_field():
    # the image field with many samples far below their block's maximum
    # (the side sums), at block size 256 and a ragged tail
    x = synth.grf2d(2048, 2056, seed=6).reshape(-1)[:256 * MIN_BLOCKS + 99].copy()
    rng = np.random.default_rng(81)
    idx = rng.choice(x.size, 5000, replace=False)
    x[idx] *= np.float32(2.0) ** -rng.integers(24, 80, idx.size).astype(np.float32)
    _check(x, 256, list(A.DEFAULT_CANDIDATES))


def test_t1_stream_decisions_cross_boundaries():
    # blocks alternate between noise (stream 0), a walk (1) and a parabola (2)
    # so that the decision taken from the predecessor changes at run and CTA
    # boundaries (64 blocks per CTA)
    N = 64
    nb = MIN_BLOCKS + 100
    rng = np.random.default_rng(79)
    x = np.empty(N * nb, dtype=np.float32)
    t = np.arange(N, dtype=np.float64)
    for b in range(nb):
        kind = (b * 7 + b // 16) % 3
        if kind == 0:
            v = rng.standard_normal(N)
        elif kind == 1:
            v = np.cumsum(rng.standard_normal(N))
        else:
            v = 0.01 * (t - rng.uniform(0, N)) ** 2 + rng.standard_normal(N) * 1e-3
        x[N * b:N * (b + 1)] = v
    _check(x, N, list(A.DEFAULT_CANDIDATES))


def test_t1_nonfinite_sets_status():
    x = _walk(64 * MIN_BLOCKS, seed=80)
    x[64 * 999 + 3] = np.inf
    xt = torch.from_numpy(x).cuda()
    _, summ = A.profile(xt, 64, list(A.DEFAULT_CANDIDATES), 0.9999)
    assert summ.status == -8
