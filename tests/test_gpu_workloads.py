"""Parity on the paper-shaped workloads at full size, on sampled targets.

- 64 uneven flat-plate problems (16^3 blocks, N_b log-uniform in [8, 1200],
  3 components) through one lgf_batch_apply, FP32, 8 random targets per
  problem and component against the oracle; G_L followed by E(0.25) equal to
  the single applies bit for bit.
- the 512 x 256 x 256 wake domain (32^3 blocks, 3 components x 4 right-hand
  sides), FP32, 6 random targets per field against the oracle.
"""
import functools

import numpy as np
import pytest
import torch

import lgf_inputs as li
import paper_1604_01814_gb300 as lgf
pytestmark = pytest.mark.gpu


def rel_sampled(got_s, ref_s, field_max):
    """max |got - ref| over the sampled targets, relative to the field's
    largest |u| (a sample far from the sources sees a much smaller |u| than
    the field, while FP32 transform error scales with the field)."""
    return float(np.abs(np.asarray(got_s, np.float64) - ref_s).max() / max(np.abs(ref_s).max(), field_max))


@functools.lru_cache(maxsize=1)
def plates():
    return li.plate_batch()


def test_plate_batch_poisson_sampled(ctx32, oracle):
    probs = plates()
    batch = []
    for p in probs:
        f = torch.tensor(p.f.reshape(-1), dtype=torch.float32, device="cuda")
        u = torch.full((p.ncomp * p.tgt.shape[0] * p.b ** 3,), float("nan"), device="cuda")
        batch.append(dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=u, ncomp=p.ncomp, op=lgf.LGF_OP_POISSON))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx32.batch_apply(batch, stream=s)
    s.synchronize()
    rng = np.random.default_rng(33)
    worst = 0.0
    for p, q in zip(probs, batch):
        got = q["u"].cpu().numpy().reshape(p.ncomp, -1)
        assert not np.isnan(got).any()
        pts_all = oracle.block_points(p.b, p.tgt)
        idx = rng.choice(pts_all.shape[0], size=8, replace=False)
        for c in range(p.ncomp):
            ref = oracle.poisson_direct(p.b, p.src, p.f[0, c], pts_all[idx], R=64)
            worst = max(worst, rel_sampled(got[c, idx], ref, float(np.abs(got[c]).max())))
    assert worst < 1e-5


def test_plate_batch_poisson_then_intfactor_equals_single_applies(ctx32):
    probs = plates()[:12]
    batch, ref = [], []
    for p in probs:
        f = torch.tensor(p.f.reshape(-1), dtype=torch.float32, device="cuda")
        n = p.ncomp * p.tgt.shape[0] * p.b ** 3
        u = torch.full((n,), float("nan"), device="cuda")
        batch.append(dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=u, ncomp=p.ncomp,
                          op=lgf.LGF_OP_POISSON_THEN_INTFACTOR, alpha=0.25))
        tmp = torch.empty(n, device="cuda")
        r = torch.empty(n, device="cuda")
        ctx32.poisson_apply(p.b, p.src, p.tgt, f, tmp, ncomp=p.ncomp)
        ctx32.intfactor_apply(0.25, p.b, p.tgt, p.tgt, tmp, r, ncomp=p.ncomp)
        ref.append(r)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx32.batch_apply(batch, stream=s)
    s.synchronize()
    for q, r in zip(batch, ref):
        assert torch.equal(q["u"], r)


def test_wake_domain_sampled(ctx32, oracle):
    p = li.wake_domain()
    f = torch.tensor(p.f.reshape(-1), dtype=torch.float32, device="cuda")
    u = torch.full_like(f, float("nan"))
    ctx32.poisson_apply(p.b, p.src, p.tgt, f, u, ncomp=p.ncomp, nrhs=p.nrhs)
    torch.cuda.synchronize()
    got = u.cpu().numpy().reshape(p.nrhs, p.ncomp, -1)
    del f, u
    pts_all = oracle.block_points(p.b, p.tgt)
    rng = np.random.default_rng(44)
    for r in range(p.nrhs):
        for c in range(p.ncomp):
            idx = rng.choice(pts_all.shape[0], size=6, replace=False)
            ref = oracle.poisson_direct(p.b, p.src, p.f[r, c], pts_all[idx], R=64)
            assert rel_sampled(got[r, c, idx], ref, float(np.abs(got[r, c]).max())) < 1e-5, (r, c)
