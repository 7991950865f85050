"""The bench's host-side pieces on CPU: the ncu figures it reads from the
committed summary, the input fingerprints, and the oracle's encode/decode
timing helper (its codec round trip must be exact on the sample)."""
import numpy as np

import bench
import oracle as O
from paper_1303_4994_gb300 import synth


def test_profile_figures_parse():
    # the dominant kernel's DRAM bytes per launch and its ncu fractions
    t = bench._traffic("profile")
    assert isinstance(t, int) and 67_108_864 <= t < 2 * 67_108_864  # about one read of 64 MiB
    for f in (bench._issue_active("profile"), bench._fma_heavy("profile")):
        assert isinstance(f, float) and 0.0 < f < 1.0
    assert bench._traffic("no_such_kernel") is None and bench._issue_active("encode") is None


def test_fingerprints():
    a = np.arange(1000, dtype=np.int16)
    b = a.copy()
    b[7] += 1
    assert synth.sha256(a) == synth.sha256(a.copy())
    assert synth.sha256(a) != synth.sha256(b)
    assert synth.sha256(a) != synth.sha256(a, "job table")
    assert synth.sha256(a)[:16] == synth.digest(a)
    assert len(synth.sha256(a)) == 64


def test_oracle_codec_timing_helper():
    O.build()
    x = synth.sensor_trace(256 * 64, seed=0)
    r = bench.oracle_codec(x, 0, 4, 1, 0, "a 16,384-sample trace")
    for side in ("all_cores", "one_core"):
        assert r[side]["encode"] > 0 and r[side]["decode"] > 0
    assert r["one_core"]["cores"] == 1 and r["all_cores"]["cores"] >= 1
    assert r["kind"] == "oracle" and r["unit"] == "GB/s"
    # what it timed is the oracle's own round trip: fixed rate 4:1 is a
    # quarter of the bytes plus the 40-byte header
    c = O.encode(x, 256, O.MODE_FR, 4, 1, 0, threads=0)
    assert len(c) == 40 + x.nbytes // 4
    y = O.decode(c, np.int16, x.size, threads=0)
    assert y.shape == x.shape
