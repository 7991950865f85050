"""The batched workload at its full size against the oracle: all 8,192
arrays (4 KB..64 MB, int16/int32/float32/float64, fixed rates 2:1..6:1,
56.6 GB) encoded and decoded by one persistent launch each; every array
must finish with status 0, and a seeded subset of 64 arrays (the oracle
cannot code 56.6 GB in a test's time) must be byte-identical containers
and bit-identical decoded arrays to the oracle's."""
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


def _slice(master, off, n):
    """n samples of the master signal from offset off, wrapping around."""
    M = master.numel()
    pos, parts, need = off % M, [], n
    while need > 0:
        take = min(need, M - pos)
        parts.append(master[pos:pos + take])
        need -= take
        pos = 0
    return torch.cat(parts) if len(parts) > 1 else parts[0].clone()


def test_batched_config_full_size():
    specs = synth.batch_specs(8192)
    masters = {k: torch.from_numpy(v).cuda() for k, v in synth.batch_masters().items()}
    xs = [_slice(masters[dt], off, n) for dt, n, _, off in specs]
    ps = [A.params(256, A.FIXED_RATE, rate, 0) for _, _, rate, _ in specs]
    total = sum(x.numel() * x.element_size() for x in xs)
    assert 56e9 < total < 57e9
    outs = [torch.empty(A.encoded_size(A.TORCH_CODE[x.dtype], x.numel(), p), dtype=torch.uint8,
                        device="cuda") for x, p in zip(xs, ps)]
    k = len(xs)
    res = torch.zeros(16 * k, dtype=torch.uint8, device="cuda")
    ejobs = A.encode_jobs(xs, ps, outs, res)
    eplan = A.Batch(ejobs, A.aligned_workspace(A.batch_encode_workspace_size(ejobs)))
    eplan.run()
    torch.cuda.synchronize()
    st = A.read_results(res, k)
    assert all(r.status == 0 for r in st)
    assert all(r.bytes == o.numel() for r, o in zip(st, outs))  # fixed rate: the exact size
    ys = [torch.empty_like(x) for x in xs]
    dres = torch.zeros(16 * k, dtype=torch.uint8, device="cuda")
    djobs = A.decode_jobs(outs, ys, [256] * k, dres)
    dplan = A.Batch(djobs, A.aligned_workspace(A.batch_decode_workspace_size(djobs)))
    dplan.run()
    torch.cuda.synchronize()
    assert all(r.status == 0 for r in A.read_results(dres, k))
    rng = np.random.default_rng(12)
    for i in sorted(rng.choice(k, 64, replace=False).tolist()):
        x = xs[i].cpu().numpy()
        p = ps[i]
        want = O.encode(x, 256, O.MODE_FR, p.rate_num, p.rate_den, 0, threads=0)
        assert outs[i].cpu().numpy().tobytes() == want, i
        yo = O.decode(want, x.dtype, x.size, threads=0)
        assert ys[i].cpu().numpy().tobytes() == yo.tobytes(), i
    eplan.close()
    dplan.close()
    del xs, ys, outs, masters
    torch.cuda.empty_cache()
