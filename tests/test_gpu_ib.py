"""Immersed-boundary regularisation R and interpolation I (Sec. 2.1) on the
GPU against the CPU oracle: 1e-13 relative for FP64, 1e-6 for FP32 (each value
is a sum of at most 27 products per marker)."""
import numpy as np
import pytest
import torch

import lgf_inputs as li
from conftest import rel_linf

pytestmark = pytest.mark.gpu
TOL = {"f64": 1e-13, "f32": 1e-6}


def _case(seed, nm, b=8):
    rng = np.random.default_rng(seed)
    X = li.icosphere_markers(3)[:nm] * 9.0 + np.array([3.3, -2.1, 0.7])     # markers on a sphere, cell units
    blocks = li.blocks_touched(b, X)
    # drop one block so that some support points fall outside the set
    return rng, X, blocks[1:]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_ib_spread_every_point(prec, ctx64, ctx32, oracle):
    ctx = ctx64 if prec == "f64" else ctx32
    rng, X, blocks = _case(1, 200)
    b, nrhs, dx = 8, 2, 0.4
    g = rng.normal(size=(nrhs, 3, X.shape[0]))
    f = torch.full((nrhs * 3 * blocks.shape[0] * b ** 3,), float("nan"), dtype=ctx.dtype, device="cuda")
    Xt = torch.tensor(X, dtype=torch.float64, device="cuda")
    ctx.ib_spread(b, blocks, Xt, torch.tensor(g.reshape(-1), dtype=ctx.dtype, device="cuda"), f, nrhs=nrhs, dx=dx)
    torch.cuda.synchronize()
    got = f.cpu().numpy().astype(np.float64).reshape(nrhs, 3, blocks.shape[0], b ** 3)
    ref = oracle.ib_spread(b, blocks, X, g, dx)
    assert rel_linf(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_ib_interp_every_marker(prec, ctx64, ctx32, oracle):
    ctx = ctx64 if prec == "f64" else ctx32
    rng, X, blocks = _case(2, 320)
    b, nrhs = 8, 2
    v = rng.uniform(-1, 1, size=(nrhs, 3, blocks.shape[0], b ** 3))
    U = torch.full((nrhs * 3 * X.shape[0],), float("nan"), dtype=ctx.dtype, device="cuda")
    Xt = torch.tensor(X, dtype=torch.float64, device="cuda")
    ctx.ib_interp(b, blocks, Xt, torch.tensor(v.reshape(-1), dtype=ctx.dtype, device="cuda"), U, nrhs=nrhs)
    torch.cuda.synchronize()
    got = U.cpu().numpy().astype(np.float64).reshape(nrhs, 3, X.shape[0])
    ref = oracle.ib_interp(b, blocks, X, v)
    assert rel_linf(got, ref) < TOL[prec]


def test_ib_interp_is_scaled_adjoint_on_gpu(ctx64):
    """<R g, v> dx^3 = <g, I v> with both operators from the library."""
    rng, X, blocks = _case(3, 160)
    b, dx = 8, 0.7
    g = torch.tensor(rng.normal(size=3 * X.shape[0]), dtype=torch.float64, device="cuda")
    v = torch.tensor(rng.normal(size=3 * blocks.shape[0] * b ** 3), dtype=torch.float64, device="cuda")
    Xt = torch.tensor(X, dtype=torch.float64, device="cuda")
    f = torch.empty_like(v)
    U = torch.empty_like(g)
    ctx64.ib_spread(b, blocks, Xt, g, f, dx=dx)
    ctx64.ib_interp(b, blocks, Xt, v, U)
    lhs = float((f * v).sum()) * dx ** 3
    rhs = float((g * U).sum())
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def test_ib_empty_and_outside_cases(ctx32):
    b = 8
    blocks = np.array([[0, 0, 0]], dtype=np.int32)
    f = torch.full((3 * b ** 3,), 1.0, dtype=torch.float32, device="cuda")
    X0 = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    ctx32.ib_spread(b, blocks, X0, torch.zeros(0, dtype=torch.float32, device="cuda"), f)
    torch.cuda.synchronize()
    assert float(f.abs().max()) == 0.0      # no markers: zero field
    # a marker whose support lies entirely outside the set interpolates to zero
    Xf = torch.tensor([[50.0, 50.0, 50.0]], dtype=torch.float64, device="cuda")
    U = torch.full((3,), 7.0, dtype=torch.float32, device="cuda")
    ctx32.ib_interp(b, blocks, Xf, torch.ones(3 * b ** 3, dtype=torch.float32, device="cuda"), U)
    torch.cuda.synchronize()
    assert float(U.abs().max()) == 0.0
