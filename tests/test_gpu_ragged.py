"""The ragged batch mode: the Poisson parts of all problems of a batch run
together, one launch per pass and transform length, each CTA finding its
problem in the job table of its launch.

- bit for bit equal to the single applies (FP32 and FP64), over a mix of
  block edges, transform lengths, both shifted windows, every operation, a
  problem without source blocks and one without target blocks, direct and
  through the captured graph;
- more problems of one transform length (and one integrating-factor group)
  than one launch's table holds; an integrating factor whose radius needs
  the generic passes inside the ragged mode;
- against the oracle: the FP64 direct sum (Sec. 2.2, Eq. dpoisson_conv) and
  E(alpha) of the oracle's Poisson result (App. A, Eq. lgf_intfac);
- the same batch with per-problem launches (the other mode);
- the autotuner's report names the mode.
"""
import numpy as np
import pytest
import torch

import lgf_inputs as li
import paper_1604_01814_gb300 as lgf
from conftest import build_lib, rel_linf

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def rag_ctx():
    """Contexts per (precision, mode): the ragged mode and per-problem launches."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_lib()
    ctxs = {}
    flags = {"ragged": lgf._binding.LGF_FLAG_BATCH_RAGGED, "per_problem": lgf._binding.LGF_FLAG_BATCH_PER_PROBLEM}
    for prec in ("f32", "f64"):
        for mode, fl in flags.items():
            c = lgf.Context(prec, flags=fl)
            c.table_build(48)
            ctxs[prec, mode] = c
            if mode == "ragged":
                ctxs[prec] = c
    yield ctxs
    for k, c in ctxs.items():
        if isinstance(k, tuple):
            c.close()


def _problem(seed, b, src, tgt, ncomp):
    rng = np.random.default_rng(seed)
    src = np.asarray(src, np.int32).reshape(-1, 3)
    tgt = np.asarray(tgt, np.int32).reshape(-1, 3)
    f = rng.uniform(-1.0, 1.0, size=(1, ncomp, src.shape[0], b ** 3))
    return li.Problem("ragged", b, src, tgt, f)


def mixed_problems():
    """Block edges 8 and 16, several lengths per axis, a small source with a
    long target along x and along y (the shifted windows), an empty source
    set and an empty target set."""
    out = [li.random_sparse(500 + i, b=(8, 16)[i % 2], nsrc=1 + i % 4, ntgt=2 + i % 5,
                            extent=(2 + i % 3, 2 + (i // 2) % 3, 1 + i % 2), ncomp=1 + i % 3) for i in range(9)]
    out.append(_problem(1, 8, [[0, 0, 0]], li.box_blocks(7, 1, 1), 2))   # long target along x
    out.append(_problem(2, 8, [[0, 0, 0]], li.box_blocks(1, 7, 1), 1))   # long target along y
    out.append(_problem(3, 16, np.zeros((0, 3)), li.box_blocks(2, 1, 1), 1))
    out.append(_problem(4, 16, li.box_blocks(1, 2, 1), np.zeros((0, 3)), 1))
    return out


def _single(ctx, p, op, alpha, f):
    n_out = p.ncomp * p.tgt.shape[0] * p.b ** 3
    r = torch.empty(n_out, dtype=ctx.dtype, device="cuda")
    if n_out == 0:
        return r
    if op == lgf.LGF_OP_POISSON:
        ctx.poisson_apply(p.b, p.src, p.tgt, f, r, ncomp=p.ncomp)
    elif op == lgf.LGF_OP_INTFACTOR:
        ctx.intfactor_apply(alpha, p.b, p.src, p.tgt, f, r, ncomp=p.ncomp)
    elif op == lgf.LGF_OP_KINV:
        ctx.kinv_apply(alpha, p.b, p.src, p.tgt, f, r, ncomp=p.ncomp)
    else:
        tmp = torch.empty_like(r)
        ctx.poisson_apply(p.b, p.src, p.tgt, f, tmp, ncomp=p.ncomp)
        ctx.intfactor_apply(alpha, p.b, p.tgt, p.tgt, tmp, r, ncomp=p.ncomp)
    return r


def _batch_and_refs(ctx, probs, ops, alphas=None):
    batch, ref = [], []
    for i, (p, op) in enumerate(zip(probs, ops)):
        alpha = alphas[i] if alphas else 0.15 + 0.05 * (i % 4)
        nin = max(1, p.ncomp * p.src.shape[0] * p.b ** 3)
        f = torch.zeros(nin, dtype=ctx.dtype, device="cuda")
        if p.src.shape[0]:
            f.copy_(torch.tensor(p.f.reshape(-1), dtype=ctx.dtype))
        u = torch.full((max(1, p.ncomp * p.tgt.shape[0] * p.b ** 3),), float("nan"), dtype=ctx.dtype,
                       device="cuda")
        batch.append(dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=u, ncomp=p.ncomp, nrhs=1, op=op, alpha=alpha, dx=1.0))
        ref.append(_single(ctx, p, op, alpha, f))
    return batch, ref


def _check_equal(batch, ref):
    for q, r in zip(batch, ref):
        n = r.numel()
        assert torch.equal(q["u"][:n], r)


@pytest.mark.parametrize("mode", ["ragged", "per_problem"])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_ragged_batch_equals_single_applies(prec, mode, rag_ctx):
    ctx = rag_ctx[prec, mode]
    probs = mixed_problems()
    cycle = [lgf.LGF_OP_POISSON, lgf.LGF_OP_POISSON_THEN_INTFACTOR, lgf.LGF_OP_KINV, lgf.LGF_OP_INTFACTOR]
    ops = [cycle[i % 4] for i in range(len(probs))]
    ops[9] = ops[10] = lgf.LGF_OP_POISSON_THEN_INTFACTOR
    # alpha 9 needs a stencil radius beyond the register windows: that group
    # runs through the generic passes inside the ragged mode
    alphas = [9.0 if i == 7 else 0.15 + 0.05 * (i % 4) for i in range(len(probs))]
    batch, ref = _batch_and_refs(ctx, probs, ops, alphas)
    s = torch.cuda.Stream()
    for _ in range(2):   # capture, then replay of the graph
        for q in batch:
            q["u"].fill_(float("nan"))
        with torch.cuda.stream(s):
            ctx.batch_apply(batch, stream=s)
        s.synchronize()
        _check_equal(batch, ref)
    assert ctx.tune_report()["last_ragged"] == (mode == "ragged")
    # direct launches on the legacy stream
    for q in batch:
        q["u"].fill_(float("nan"))
    ctx.batch_apply(batch, stream=0)
    torch.cuda.synchronize()
    _check_equal(batch, ref)


def test_ragged_more_jobs_than_one_table(rag_ctx):
    """70 problems of one geometry: one transform-length group and one
    integrating-factor group, two launches per pass."""
    ctx = rag_ctx["f32"]
    base = li.random_sparse(77, b=8, nsrc=3, ntgt=4, extent=(3, 2, 2))
    probs = []
    for i in range(70):
        rng = np.random.default_rng(1000 + i)
        probs.append(li.Problem("same", base.b, base.src, base.tgt,
                                rng.uniform(-1.0, 1.0, size=(1, 1, base.src.shape[0], base.b ** 3))))
    ops = [lgf.LGF_OP_POISSON, lgf.LGF_OP_POISSON_THEN_INTFACTOR] * 35
    batch, ref = _batch_and_refs(ctx, probs, ops, [0.3] * 70)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx.batch_apply(batch, stream=s)
    s.synchronize()
    _check_equal(batch, ref)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_ragged_batch_against_oracle(prec, rag_ctx, oracle):
    ctx = rag_ctx[prec]
    probs = [li.random_sparse(600 + i, b=8, nsrc=2 + i, ntgt=3 + i, extent=(3, 2 + i % 2, 2)) for i in range(4)]
    probs.append(_problem(5, 8, [[0, 0, 0]], li.box_blocks(6, 1, 1), 1))
    ops = [lgf.LGF_OP_POISSON, lgf.LGF_OP_POISSON_THEN_INTFACTOR] * 2 + [lgf.LGF_OP_POISSON]
    alpha = 0.25
    batch = []
    for p, op in zip(probs, ops):
        f = torch.tensor(p.f.reshape(-1), dtype=ctx.dtype, device="cuda")
        u = torch.empty(p.tgt.shape[0] * p.b ** 3, dtype=ctx.dtype, device="cuda")
        batch.append(dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=u, ncomp=1, op=op, alpha=alpha))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx.batch_apply(batch, stream=s)
    s.synchronize()
    for p, op, q in zip(probs, ops, batch):
        pts = oracle.block_points(p.b, p.tgt)
        ref = oracle.poisson_direct(p.b, p.src, p.f[0, 0], pts, R=64)
        if op == lgf.LGF_OP_POISSON_THEN_INTFACTOR:
            ref = oracle.intfactor_blocks(alpha, p.b, p.tgt, ref.reshape(-1, p.b ** 3), p.tgt).reshape(-1)
        assert rel_linf(q["u"].cpu().numpy(), ref) < TOL[prec]


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_ragged_random_batches_equal_per_problem(seed, rag_ctx):
    """Seeded random batches (block edges 8 and 16, uneven sets, every
    operation, several fields and right-hand sides): the ragged mode equals
    per-problem launches bit for bit."""
    rng = np.random.default_rng(seed)
    probs, ops, alphas, nrhs = [], [], [], []
    for i in range(24):
        b = int(rng.choice([8, 16]))
        ext = tuple(int(v) for v in rng.integers(1, 5, size=3))
        nsrc = int(rng.integers(1, 1 + min(6, ext[0] * ext[1] * ext[2])))
        ntgt = int(rng.integers(1, 1 + min(7, ext[0] * ext[1] * ext[2])))
        r = int(rng.integers(1, 3))
        p = li.random_sparse(seed * 1000 + i, b=b, nsrc=nsrc, ntgt=ntgt, extent=ext, nrhs=r,
                             ncomp=int(rng.choice([1, 3])))
        probs.append(p)
        nrhs.append(r)
        ops.append(int(rng.choice([lgf.LGF_OP_POISSON, lgf.LGF_OP_POISSON_THEN_INTFACTOR, lgf.LGF_OP_KINV,
                                   lgf.LGF_OP_INTFACTOR])))
        alphas.append(float(rng.choice([0.05, 0.25, 1.0])))
    outs = {}
    for mode in ("ragged", "per_problem"):
        ctx = rag_ctx["f32", mode]
        batch = []
        for p, op, a in zip(probs, ops, alphas):
            f = torch.tensor(p.f.reshape(-1), dtype=torch.float32, device="cuda")
            u = torch.full((p.nrhs * p.ncomp * p.tgt.shape[0] * p.b ** 3,), float("nan"), device="cuda")
            batch.append(dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=u, ncomp=p.ncomp, nrhs=p.nrhs, op=op, alpha=a,
                              dx=1.0))
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            ctx.batch_apply(batch, stream=s)
        s.synchronize()
        outs[mode] = [q["u"].cpu() for q in batch]
    for a, b in zip(outs["ragged"], outs["per_problem"]):
        assert torch.equal(a, b)
        assert not torch.isnan(a).any()
