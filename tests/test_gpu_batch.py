"""Batched applies (one CUDA graph) against the single-problem applies."""
import numpy as np
import pytest
import torch

import lgf_inputs as li
import paper_1604_01814_gb300 as lgf

pytestmark = pytest.mark.gpu


def make_problems(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        b = (8, 16)[i % 2]
        p = li.random_sparse(seed * 100 + i, b=b, nsrc=int(rng.integers(1, 6)), ntgt=int(rng.integers(1, 7)),
                             extent=(3, 3, 2), ncomp=int(rng.integers(1, 4)))
        out.append(p)
    return out


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_batch_equals_single_applies(prec, ctx32, ctx64):
    ctx = ctx32 if prec == "f32" else ctx64
    probs = make_problems(7, seed=1)
    ops = [lgf.LGF_OP_POISSON, lgf.LGF_OP_INTFACTOR, lgf.LGF_OP_POISSON_THEN_INTFACTOR]
    batch, ref = [], []
    for i, p in enumerate(probs):
        f = torch.tensor(p.f.reshape(-1), dtype=ctx.dtype, device="cuda")
        n_out = p.ncomp * p.tgt.shape[0] * p.b ** 3
        u = torch.full((n_out,), float("nan"), dtype=ctx.dtype, device="cuda")
        op = ops[i % 3]
        batch.append(dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=u, ncomp=p.ncomp, nrhs=1, op=op, alpha=0.2 + 0.1 * i,
                          dx=1.0))
        r = torch.empty_like(u)
        if op == lgf.LGF_OP_POISSON:
            ctx.poisson_apply(p.b, p.src, p.tgt, f, r, ncomp=p.ncomp)
        elif op == lgf.LGF_OP_INTFACTOR:
            ctx.intfactor_apply(0.2 + 0.1 * i, p.b, p.src, p.tgt, f, r, ncomp=p.ncomp)
        else:
            tmp = torch.empty_like(r)
            ctx.poisson_apply(p.b, p.src, p.tgt, f, tmp, ncomp=p.ncomp)
            ctx.intfactor_apply(0.2 + 0.1 * i, p.b, p.tgt, p.tgt, tmp, r, ncomp=p.ncomp)
        ref.append(r)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx.batch_apply(batch, stream=s)
    s.synchronize()
    for q, r in zip(batch, ref):
        assert torch.equal(q["u"], r)
    # replay of the captured graph: same results
    for q in batch:
        q["u"].fill_(float("nan"))
    with torch.cuda.stream(s):
        ctx.batch_apply(batch, stream=s)
    s.synchronize()
    for q, r in zip(batch, ref):
        assert torch.equal(q["u"], r)


def test_batch_on_default_stream_runs_without_graph(ctx32):
    probs = make_problems(3, seed=2)
    batch, ref = [], []
    for p in probs:
        f = torch.tensor(p.f.reshape(-1), dtype=torch.float32, device="cuda")
        u = torch.empty(p.ncomp * p.tgt.shape[0] * p.b ** 3, dtype=torch.float32, device="cuda")
        batch.append(dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=u, ncomp=p.ncomp))
        r = torch.empty_like(u)
        ctx32.poisson_apply(p.b, p.src, p.tgt, f, r, ncomp=p.ncomp)
        ref.append(r)
    ctx32.batch_apply(batch, stream=0)
    torch.cuda.synchronize()
    for q, r in zip(batch, ref):
        assert torch.equal(q["u"], r)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_grouped_integrating_factors_equal_single_applies(prec, ctx32, ctx64):
    """Integrating factors on the same block sets run as one grouped launch
    per pass; each result equals its single apply bit for bit."""
    ctx = ctx32 if prec == "f32" else ctx64
    p = li.random_sparse(31, b=16, nsrc=5, ntgt=6, extent=(3, 3, 2), ncomp=2)
    alphas = [0.05, 0.3, 0.5, 1.0, 2.0, 0.01, 0.7, 1.5, 0.2, 0.4]   # more than 8: two launches per pass
    rng = np.random.default_rng(9)
    batch, ref = [], []
    for a in alphas:
        f = torch.tensor(rng.uniform(-1, 1, p.f.size), dtype=ctx.dtype, device="cuda")
        u = torch.full((p.ncomp * p.tgt.shape[0] * p.b ** 3,), float("nan"), dtype=ctx.dtype, device="cuda")
        batch.append(dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=u, ncomp=p.ncomp, op=lgf.LGF_OP_INTFACTOR, alpha=a))
        r = torch.empty_like(u)
        ctx.intfactor_apply(a, p.b, p.src, p.tgt, f, r, ncomp=p.ncomp)
        ref.append(r)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx.batch_apply(batch, stream=s)
    s.synchronize()
    for q, r in zip(batch, ref):
        assert torch.equal(q["u"], r)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_branches_and_shared_dependent_groups(prec, ctx32, ctx64):
    """A batch whose Poisson parts spread over concurrent branches while an
    integrating-factor group shared by several Poisson-then-E problems runs
    after the join: every result equals its single applies bit for bit, with
    the graph, on replay, and with profiling on (serial, no graph)."""
    ctx = ctx32 if prec == "f32" else ctx64
    shared = li.random_sparse(41, b=16, nsrc=4, ntgt=5, extent=(3, 3, 2), ncomp=1)
    others = make_problems(5, seed=4)
    rng = np.random.default_rng(5)
    batch, ref = [], []

    def add(p, op, alpha):
        f = torch.tensor(rng.uniform(-1, 1, p.f.size), dtype=ctx.dtype, device="cuda")
        u = torch.full((p.ncomp * p.tgt.shape[0] * p.b ** 3,), float("nan"), dtype=ctx.dtype, device="cuda")
        batch.append(dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=u, ncomp=p.ncomp, op=op, alpha=alpha, dx=0.5))
        r = torch.empty_like(u)
        if op == lgf.LGF_OP_POISSON:
            ctx.poisson_apply(p.b, p.src, p.tgt, f, r, ncomp=p.ncomp, dx=0.5)
        elif op == lgf.LGF_OP_INTFACTOR:
            ctx.intfactor_apply(alpha, p.b, p.src, p.tgt, f, r, ncomp=p.ncomp)
        else:
            tmp = torch.empty_like(r)
            ctx.poisson_apply(p.b, p.src, p.tgt, f, tmp, ncomp=p.ncomp, dx=0.5)
            ctx.intfactor_apply(alpha, p.b, p.tgt, p.tgt, tmp, r, ncomp=p.ncomp)
        ref.append(r)

    for a in (0.1, 0.6, 1.3):
        add(shared, lgf.LGF_OP_POISSON_THEN_INTFACTOR, a)
    for i, p in enumerate(others):
        add(p, (lgf.LGF_OP_POISSON, lgf.LGF_OP_INTFACTOR, lgf.LGF_OP_POISSON_THEN_INTFACTOR)[i % 3], 0.25 + 0.2 * i)
    s = torch.cuda.Stream()
    for _ in range(2):   # capture, then replay
        for q in batch:
            q["u"].fill_(float("nan"))
        with torch.cuda.stream(s):
            ctx.batch_apply(batch, stream=s)
        s.synchronize()
        for q, r in zip(batch, ref):
            assert torch.equal(q["u"], r)
    ctx.profile_enable(True)
    try:
        for q in batch:
            q["u"].fill_(float("nan"))
        with torch.cuda.stream(s):
            ctx.batch_apply(batch, stream=s)
        s.synchronize()
        for q, r in zip(batch, ref):
            assert torch.equal(q["u"], r)
    finally:
        ctx.profile_enable(False)
