"""K(alpha)^{-1} = [E(-alpha) L]^{-1} through G_K(alpha) (App. A, Eq. lgf_iflap)
on the GPU against the CPU oracle.

Tolerances as for the Poisson apply: 1e-12 (FP64) and 1e-5 (FP32) relative
L-infinity; the G_K table itself to 1e-13 relative."""
import numpy as np
import pytest
import torch

import lgf_inputs as li
import paper_1604_01814_gb300 as lgf
from conftest import rel_linf

pytestmark = pytest.mark.gpu
TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.mark.parametrize("alpha", [0.05, 0.5, 1.0, 2.5])
def test_gk_table_matches_oracle(alpha, ctx64, oracle):
    offs = [(0, 0, 0), (1, 0, 0), (0, -1, 0), (2, 1, 0), (3, -2, 1), (7, 7, 7), (12, 0, 5), (-20, 3, 9),
            (40, 2, 1), (47, 47, 1), (60, 10, 0), (100, -3, 8)]
    got = ctx64.kinv_lookup(alpha, torch.tensor(offs, dtype=torch.int32)).cpu().numpy()
    ref = oracle.gk(np.array(offs), alpha, R=64)
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-13


def test_gk_alpha_zero_is_gl(ctx64):
    offs = torch.tensor([(0, 0, 0), (3, 2, 1), (30, 0, 1), (90, 9, 9)], dtype=torch.int32)
    a = ctx64.kinv_lookup(0.0, offs)
    b = ctx64.table_lookup(offs)
    assert torch.equal(a, b)


def run_kinv(ctx, alpha, p, dx=1.0):
    f = torch.tensor(p.f.reshape(-1), dtype=ctx.dtype, device="cuda")
    u = torch.full((p.nrhs * p.ncomp * p.tgt.shape[0] * p.b ** 3,), float("nan"), dtype=ctx.dtype, device="cuda")
    ctx.kinv_apply(alpha, p.b, p.src, p.tgt, f, u, ncomp=p.ncomp, nrhs=p.nrhs, dx=dx)
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.float64).reshape(p.nrhs, p.ncomp, -1)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("alpha,seed,b,ns,nt,ext", [(0.25, 1, 8, 5, 7, (4, 3, 3)), (1.0, 2, 16, 3, 4, (3, 2, 2)),
                                                   (0.5, 3, 4, 9, 6, (5, 4, 3))])
def test_kinv_apply_every_point(prec, alpha, seed, b, ns, nt, ext, ctx64, ctx32, oracle):
    ctx = ctx64 if prec == "f64" else ctx32
    p = li.random_sparse(seed, b=b, nsrc=ns, ntgt=nt, extent=ext, ncomp=2)
    got = run_kinv(ctx, alpha, p, dx=0.5)
    pts = oracle.block_points(p.b, p.tgt)
    ref = np.stack([[oracle.kinv_direct(alpha, p.b, p.src, p.f[r, c], pts, dx=0.5, R=64)
                     for c in range(p.ncomp)] for r in range(p.nrhs)])
    assert rel_linf(got, ref) < TOL[prec]


def test_kinv_alpha_zero_equals_poisson(ctx32):
    p = li.random_sparse(5, b=8, nsrc=4, ntgt=5, extent=(3, 3, 2))
    f = torch.tensor(p.f.reshape(-1), dtype=torch.float32, device="cuda")
    u1 = torch.empty(p.tgt.shape[0] * p.b ** 3, dtype=torch.float32, device="cuda")
    u2 = torch.empty_like(u1)
    ctx32.kinv_apply(0.0, p.b, p.src, p.tgt, f, u1)
    ctx32.poisson_apply(p.b, p.src, p.tgt, f, u2)
    torch.cuda.synchronize()
    assert torch.equal(u1, u2)


def test_kinv_is_lgf_after_integrating_factor(ctx64):
    """K(alpha)^{-1} f = L^{-1} (E(alpha) f) on the unbounded lattice (the
    symbols multiply: e^{alpha sigma} / sigma).  E(alpha) f spreads past the
    source blocks, so the two-step route carries E onto the source set grown
    by one block ring, where E(alpha) is below 1e-13 beyond (alpha = 0.3,
    b = 16)."""
    alpha, b = 0.3, 16
    src = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 1]], dtype=np.int32)
    tgt = np.array([[2, 1, 0], [0, 0, 0], [-1, 2, 1]], dtype=np.int32)
    rng = np.random.default_rng(7)
    f = torch.tensor(rng.uniform(-1, 1, src.shape[0] * b ** 3), dtype=torch.float64, device="cuda")
    grown = sorted({tuple(c + d) for c in src for d in np.array(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1],
                                                                          indexing="ij")).reshape(3, -1).T})
    grown = np.array(grown, dtype=np.int32)
    ef = torch.empty(grown.shape[0] * b ** 3, dtype=torch.float64, device="cuda")
    ctx64.intfactor_apply(alpha, b, src, grown, f, ef)
    u2 = torch.empty(tgt.shape[0] * b ** 3, dtype=torch.float64, device="cuda")
    ctx64.poisson_apply(b, grown, tgt, ef, u2)
    u1 = torch.empty_like(u2)
    ctx64.kinv_apply(alpha, b, src, tgt, f, u1)
    torch.cuda.synchronize()
    u1, u2 = u1.cpu().numpy(), u2.cpu().numpy()
    assert np.max(np.abs(u1 - u2)) / np.max(np.abs(u2)) < 1e-11


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_kinv_in_batch_equals_single(prec, ctx32, ctx64):
    ctx = ctx32 if prec == "f32" else ctx64
    rng = np.random.default_rng(3)
    batch, ref = [], []
    for i, a in enumerate((0.2, 0.7, 0.0)):
        p = li.random_sparse(20 + i, b=8, nsrc=3, ntgt=4, extent=(3, 2, 2))
        f = torch.tensor(rng.uniform(-1, 1, p.f.size), dtype=ctx.dtype, device="cuda")
        u = torch.full((p.tgt.shape[0] * p.b ** 3,), float("nan"), dtype=ctx.dtype, device="cuda")
        batch.append(dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=u, op=lgf.LGF_OP_KINV, alpha=a, dx=0.25))
        r = torch.empty_like(u)
        ctx.kinv_apply(a, p.b, p.src, p.tgt, f, r, dx=0.25)
        ref.append(r)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx.batch_apply(batch, stream=s)
    s.synchronize()
    for q, r in zip(batch, ref):
        assert torch.equal(q["u"], r)


def test_kinv_rejects_bad_alpha(ctx32):
    offs = torch.tensor([(0, 0, 0)], dtype=torch.int32)
    with pytest.raises(lgf.LgfError) as e:
        ctx32.kinv_lookup(-1.0, offs)
    assert e.value.status == 1   # LGF_EINVAL
    # R(alpha) far from negligible on the outer shell of the table: refused
    with pytest.raises(lgf.LgfError) as e:
        ctx32.kinv_lookup(60.0, offs)
    assert e.value.status == 5   # LGF_EUNSUPPORTED
