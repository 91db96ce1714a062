"""The bench step itself against the oracle: the dense 128^3 box (32^3 blocks,
Gaussian blobs, seed 1) as one lgf_batch_apply of G_L and E(0.05), E(0.5),
E(2.0) on a non-default stream, i.e. captured into a CUDA graph with the
Poisson part and the three integrating factors on concurrent branches, then
replayed.  Poisson output: 512 sampled targets; integrating factors: every
point against the untruncated oracle.  FP32, 1e-5 relative."""
import numpy as np
import pytest
import torch

import lgf_inputs as li
import paper_1604_01814_gb300 as lgf
from conftest import rel_linf

pytestmark = pytest.mark.gpu
ALPHAS = (0.05, 0.5, 2.0)


def test_bench_step_batch_graph_against_oracle(ctx32, oracle):
    p = li.dense_blobs(n=128, b=32, seed=1)
    f = torch.tensor(p.f.reshape(-1), dtype=torch.float32, device="cuda")
    outs = [torch.full_like(f, float("nan")) for _ in range(1 + len(ALPHAS))]
    batch = [dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=outs[0], op=lgf.LGF_OP_POISSON)]
    batch += [dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=o, op=lgf.LGF_OP_INTFACTOR, alpha=a)
              for a, o in zip(ALPHAS, outs[1:])]
    s = torch.cuda.Stream()
    for _ in range(2):   # capture, then replay of the captured graph
        for o in outs:
            o.fill_(float("nan"))
        with torch.cuda.stream(s):
            ctx32.batch_apply(batch, stream=s)
        s.synchronize()
    got = [o.cpu().numpy().astype(np.float64) for o in outs]
    rng = np.random.default_rng(101)
    idx = rng.choice(got[0].size, size=512, replace=False)
    pts = oracle.block_points(p.b, p.tgt)[idx]
    ref = oracle.poisson_direct(p.b, p.src, p.f[0, 0], pts, R=64)
    assert rel_linf(got[0][idx], ref) < 1e-5
    for a, g in zip(ALPHAS, got[1:]):
        ref_e = oracle.intfactor_blocks(a, p.b, p.src, p.f[0, 0], p.tgt).reshape(-1)
        assert rel_linf(g, ref_e) < 1e-5, a
