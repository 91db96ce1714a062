"""Context caches on the GPU, through lgf_ctx_stats.

- Scratch growth drops every captured batch graph: a batch captured with
  small scratch, a larger single apply that reallocates the scratch, then the
  same batch again (same tensors, so the same key): the graph is captured
  afresh instead of replaying freed addresses, and the result matches the
  oracle (the FP64 direct sum of Sec. 2.2, Eq. dpoisson_conv).
- Bounded plan caches: with max_plans = 4, a sequence of applies on changing
  block sets keeps at most 4 plans per kind, evicts the rest, and every result
  still matches the oracle.
Each test uses a fresh context, so the session contexts' caches are untouched.
"""
import numpy as np
import pytest
import torch

import lgf_inputs as li
import paper_1604_01814_gb300 as lgf
from conftest import build_lib, rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture()
def fresh_ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_lib()
    c = lgf.Context("f64")
    c.table_build(48)
    yield c
    c.close()


def _oracle_poisson(oracle, p, c=0):
    pts = oracle.block_points(p.b, p.tgt)
    return oracle.poisson_direct(p.b, p.src, p.f[0, c], pts, R=64)


def test_scratch_growth_drops_captured_graphs(fresh_ctx, oracle):
    ctx = fresh_ctx
    small = li.random_sparse(61, b=8, nsrc=3, ntgt=4, extent=(3, 2, 2))
    f = torch.tensor(small.f.reshape(-1), dtype=torch.float64, device="cuda")
    u = torch.full((small.tgt.shape[0] * small.b ** 3,), float("nan"), dtype=torch.float64, device="cuda")
    batch = [dict(b=small.b, src=small.src, tgt=small.tgt, f=f, u=u, op=lgf.LGF_OP_POISSON)]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx.batch_apply(batch, stream=s)
    s.synchronize()
    ref = _oracle_poisson(oracle, small)
    assert rel_linf(u.cpu().numpy(), ref) < 1e-12
    st0 = ctx.stats()
    assert st0["graphs_cached"] == 1
    # a much larger single apply on branch 0's scratch: the buffers grow
    big = li.uniform_box(16, (4, 4, 3), seed=62)
    fb = torch.tensor(big.f.reshape(-1), dtype=torch.float64, device="cuda")
    ub = torch.empty_like(fb)
    ctx.poisson_apply(big.b, big.src, big.tgt, fb, ub)
    torch.cuda.synchronize()
    st1 = ctx.stats()
    assert st1["scratch_reallocs"] > st0["scratch_reallocs"]
    assert st1["scratch_bytes"] > st0["scratch_bytes"]
    assert st1["graphs_cached"] == 0, "scratch growth must drop the graphs captured with the old buffers"
    assert st1["generation"] > st0["generation"]
    # the same batch again: recaptured with the new buffers, result unchanged
    u.fill_(float("nan"))
    with torch.cuda.stream(s):
        ctx.batch_apply(batch, stream=s)
    s.synchronize()
    assert ctx.stats()["graphs_cached"] == 1
    assert rel_linf(u.cpu().numpy(), ref) < 1e-12
    # and replayed once more from the cache
    u.fill_(float("nan"))
    with torch.cuda.stream(s):
        ctx.batch_apply(batch, stream=s)
    s.synchronize()
    assert rel_linf(u.cpu().numpy(), ref) < 1e-12


def test_plan_caches_are_bounded(fresh_ctx, oracle):
    ctx = fresh_ctx
    ctx.cache_limits(max_plans=4, max_spectra=3)
    for k in range(7):
        p = li.random_sparse(70 + k, b=8, nsrc=2 + k % 3, ntgt=3, extent=(3 + k % 2, 2, 2))
        f = torch.tensor(p.f.reshape(-1), dtype=torch.float64, device="cuda")
        u = torch.full((p.tgt.shape[0] * p.b ** 3,), float("nan"), dtype=torch.float64, device="cuda")
        v = torch.full_like(u, float("nan"))
        ctx.poisson_apply(p.b, p.src, p.tgt, f, u)
        ctx.intfactor_apply(0.3, p.b, p.src, p.tgt, f, v)
        torch.cuda.synchronize()
        st = ctx.stats()
        assert st["poisson_plans"] <= 4 and st["intfactor_plans"] <= 4 and st["spectra"] <= 3
        assert rel_linf(u.cpu().numpy(), _oracle_poisson(oracle, p)) < 1e-12
        refv = oracle.intfactor_blocks(0.3, p.b, p.src, p.f[0, 0], p.tgt).reshape(-1)
        assert rel_linf(v.cpu().numpy(), refv) < 1e-12
    assert ctx.stats()["evictions"] > 0


def test_batch_larger_than_the_plan_bound_keeps_its_plans(fresh_ctx, oracle):
    """One call needing more plans than the bound: none of them is evicted
    before the call returns (the entries of the running call are pinned)."""
    ctx = fresh_ctx
    ctx.cache_limits(max_plans=2)
    probs = [li.random_sparse(80 + k, b=8, nsrc=2, ntgt=2 + k, extent=(3, 2, 2)) for k in range(5)]
    batch = []
    for p in probs:
        f = torch.tensor(p.f.reshape(-1), dtype=torch.float64, device="cuda")
        u = torch.full((p.tgt.shape[0] * p.b ** 3,), float("nan"), dtype=torch.float64, device="cuda")
        batch.append(dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=u, op=lgf.LGF_OP_POISSON))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx.batch_apply(batch, stream=s)
    s.synchronize()
    assert ctx.stats()["poisson_plans"] == 5
    for p, q in zip(probs, batch):
        assert rel_linf(q["u"].cpu().numpy(), _oracle_poisson(oracle, p)) < 1e-12
