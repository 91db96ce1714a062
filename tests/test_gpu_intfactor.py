"""Integrating factor E(alpha) on the GPU against the CPU oracle (untruncated sums)."""
import numpy as np
import pytest
import torch

import lgf_inputs as li
from conftest import rel_linf

pytestmark = pytest.mark.gpu
TOL = {"f64": 1e-12, "f32": 1e-5}


def run_intf(ctx, p, alpha, src=None, f=None):
    src = p.src if src is None else src
    f = p.f if f is None else f
    dt = ctx.dtype
    ft = torch.tensor(f.reshape(-1), dtype=dt, device="cuda")
    u = torch.full((p.nrhs * p.ncomp * p.tgt.shape[0] * p.b ** 3,), float("nan"), dtype=dt, device="cuda")
    ctx.intfactor_apply(alpha, p.b, src, p.tgt, ft, u, ncomp=p.ncomp, nrhs=p.nrhs)
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.float64).reshape(p.nrhs, p.ncomp, -1)


def oracle_intf(oracle, p, alpha):
    out = np.empty((p.nrhs, p.ncomp, p.tgt.shape[0] * p.b ** 3))
    for r in range(p.nrhs):
        for c in range(p.ncomp):
            out[r, c] = oracle.intfactor_blocks(alpha, p.b, p.src, p.f[r, c], p.tgt).reshape(-1)
    return out


def test_box32_fp64(ctx64, oracle):
    p = li.plain_box32()
    got = run_intf(ctx64, p, 0.1)
    assert rel_linf(got, oracle_intf(oracle, p, 0.1)) < TOL["f64"]


@pytest.mark.parametrize("alpha", [0.05, 0.5, 2.0])
def test_dense128_fp32(ctx32, oracle, alpha):
    p = li.dense_blobs(b=32)
    got = run_intf(ctx32, p, alpha)
    assert rel_linf(got, oracle_intf(oracle, p, alpha)) < TOL["f32"]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("alpha", [0.0, 0.1, 1.0, 3.0])
@pytest.mark.parametrize("seed,b", [(1, 8), (2, 16), (3, 4)])
def test_random_sparse(ctx64, ctx32, oracle, prec, alpha, seed, b):
    ctx = ctx64 if prec == "f64" else ctx32
    p = li.random_sparse(seed, b=b, nsrc=6, ntgt=6, extent=(4, 3, 3), ncomp=2)
    got = run_intf(ctx, p, alpha)
    ref = oracle_intf(oracle, p, alpha)
    if np.abs(ref).max() == 0:
        assert np.abs(got).max() == 0
    else:
        assert rel_linf(got, ref) < TOL[prec]


def test_alpha_zero_is_identity_on_shared_blocks(ctx64):
    b = 8
    src = np.array([[0, 0, 0], [1, 0, 0]], dtype=np.int32)
    tgt = np.array([[1, 0, 0], [5, 5, 5]], dtype=np.int32)
    f = torch.randn(2 * b ** 3, dtype=torch.float64, device="cuda")
    u = torch.empty(2 * b ** 3, dtype=torch.float64, device="cuda")
    ctx64.intfactor_apply(0.0, b, src, tgt, f, u)
    torch.cuda.synchronize()
    assert torch.equal(u[:b ** 3], f[b ** 3:])
    assert torch.all(u[b ** 3:] == 0)


def test_semigroup_on_gpu(ctx64):
    """E(a) E(b) f = E(a+b) f on a padded box (sources far from the edge)."""
    b = 8
    box = li.box_blocks(8, 8, 8)
    # sources at least 24 points from the box edge: what E(0.3) sends outside
    # the box (and E(0.45) would have brought back) is below 1e-25
    inner = np.array([c for c in box.tolist() if all(3 <= v <= 4 for v in c)], dtype=np.int32)
    rng = np.random.default_rng(3)
    f = torch.tensor(rng.uniform(-1, 1, inner.shape[0] * b ** 3), device="cuda")
    u1 = torch.empty(box.shape[0] * b ** 3, dtype=torch.float64, device="cuda")
    u2 = torch.empty_like(u1)
    u3 = torch.empty_like(u1)
    ctx64.intfactor_apply(0.3, b, inner, box, f, u1)
    ctx64.intfactor_apply(0.45, b, box, box, u1, u2)
    ctx64.intfactor_apply(0.75, b, inner, box, f, u3)
    torch.cuda.synchronize()
    assert torch.max(torch.abs(u2 - u3)).item() < 1e-12 * torch.max(torch.abs(u3)).item()


def test_invalid_alpha(ctx32):
    import paper_1604_01814_gb300 as lgf
    b = 8
    f = torch.ones(b ** 3, device="cuda")
    u = torch.empty(b ** 3, device="cuda")
    with pytest.raises(lgf.LgfError) as e:
        ctx32.intfactor_apply(-0.1, b, [[0, 0, 0]], [[0, 0, 0]], f, u)
    assert e.value.status == 1
    with pytest.raises(lgf.LgfError) as e:
        ctx32.intfactor_apply(float("nan"), b, [[0, 0, 0]], [[0, 0, 0]], f, u)
    assert e.value.status == 1


def _window_class(R):
    return next((c for c in (4, 8, 12, 16) if R <= c), 0)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("b,seed", [(32, 13), (16, 12)])
def test_every_window_class_single_and_paired_blocks(ctx32, ctx64, oracle, prec, b, seed):
    """The fused x+y kernel in each radius class (4, 8, 12, 16) on target sets
    that hold both y-adjacent block pairs and lone blocks, every point against
    the oracle.  FP32 runs the packed FP32x2 stencils (x stencil on
    interleaved row pairs), FP64 the scalar ones."""
    ctx = ctx64 if prec == "f64" else ctx32
    p = li.random_sparse(seed, b=b, nsrc=5, ntgt=7, extent=(3, 3, 2), ncomp=2)
    tgt = {tuple(t) for t in p.tgt.tolist()}
    paired = any((x, y + 1, z) in tgt for x, y, z in tgt)
    lone = any((x, y + 1, z) not in tgt and (x, y - 1, z) not in tgt for x, y, z in tgt)
    assert paired and lone
    seen = set()
    # one alpha per class at the context's truncation tolerance (1e-7 FP32, 1e-13 FP64)
    alphas = (0.02, 0.3, 1.0, 2.0) if prec == "f32" else (1e-4, 0.05, 0.25, 0.75)
    for alpha in alphas:
        R, _ = ctx.intfactor_weights(alpha)
        seen.add(_window_class(R))
        got = run_intf(ctx, p, alpha)
        assert rel_linf(got, oracle_intf(oracle, p, alpha)) < TOL[prec], (alpha, R)
    assert seen == {4, 8, 12, 16}
