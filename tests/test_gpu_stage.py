"""The nested-projection stage (Sec. 3.1, Eq. nested_proj: ip -> f -> pc -> vc)
on the GPU against the oracle's composition of the same steps, element by
element: u on every face of D, d_hat on every cell of D, f_hat at every
marker.  FP64 at 1e-12 and FP32 at 1e-5 relative L-infinity.

With W1 = C^-1 (the oracle's force Schur complement of Eq. force_schur) the
GPU's u also meets the no-slip row I^i u = u_Gamma at the markers."""
import numpy as np
import pytest
import torch

import lgf_inputs as li
from conftest import rel_linf

pytestmark = pytest.mark.gpu
TOL = {"f64": 1e-12, "f32": 1e-5}


def _case(nm, move, seed):
    rng = np.random.default_rng(seed)
    b = 8
    D = li.box_blocks(4, 3, 3)
    c = np.array([16.0, 12.0, 12.0])
    ang = np.linspace(0, 2 * np.pi, nm, endpoint=False)
    X = c + np.stack([3.5 * np.cos(ang), 3.0 * np.sin(ang), 1.2 * np.cos(3 * ang)], axis=1)
    Xp = X + move * np.array([1.0, -0.5, 0.25])
    r = rng.uniform(-1, 1, size=(3, D.shape[0], b ** 3))
    ub = rng.normal(size=(3, nm))
    return b, D, X, Xp, r, ub


def _run(ctx, b, D, X, Xp, r, ub, W1, W2, alpha, dx):
    dt = ctx.dtype
    dev = "cuda"
    nD = D.shape[0]
    rt = torch.tensor(r.reshape(-1), dtype=dt, device=dev)
    u = torch.full((3 * nD * b ** 3,), float("nan"), dtype=dt, device=dev)
    d = torch.full((nD * b ** 3,), float("nan"), dtype=dt, device=dev)
    kw = {}
    f = None
    if X.shape[0]:
        f = torch.full((3 * X.shape[0],), float("nan"), dtype=dt, device=dev)
        kw = dict(X_prev=torch.tensor(Xp, dtype=torch.float64, device=dev),
                  X=torch.tensor(X, dtype=torch.float64, device=dev),
                  ub=torch.tensor(ub.reshape(-1), dtype=dt, device=dev),
                  W1=torch.tensor(W1, dtype=dt, device=dev),
                  W2=None if W2 is None else torch.tensor(W2, dtype=dt, device=dev), f=f)
    ctx.nested_projection_stage(b, D, rt, u, alpha=alpha, dx=dx, d=d, **kw)
    torch.cuda.synchronize()
    return (u.cpu().numpy().reshape(3, nD, -1), d.cpu().numpy().reshape(nD, -1),
            None if f is None else f.cpu().numpy().reshape(3, -1))


def test_stage_fp64_no_slip_with_exact_schur_inverse(ctx64, oracle):
    b, D, X, Xp, r, ub = _case(8, 0.0, 11)
    alpha, dx = 0.15, 0.5
    C = oracle.force_schur(b, D, Xp, X, alpha, dx, R=64)
    W1, W2 = np.linalg.inv(C), np.eye(C.shape[0])
    u, d, f = _run(ctx64, b, D, X, Xp, r, ub, W1, W2, alpha, dx)
    ur, dr, fr = oracle.nested_projection_stage(b, D, r, Xp, X, ub, W1, W2, alpha=alpha, dx=dx, R=64)
    assert rel_linf(u, ur) < TOL["f64"]
    assert rel_linf(d, dr) < TOL["f64"]
    assert rel_linf(f, fr) < TOL["f64"]
    U = oracle.ib_interp(b, D, X, u[None].astype(np.float64))[0]
    assert np.abs(U - ub).max() < 1e-9 * np.abs(ub).max()


@pytest.mark.parametrize("prec,move,nm", [("f64", 0.3, 6), ("f32", 0.0, 8), ("f32", 0.3, 6), ("f64", 0.0, 0)])
def test_stage_matches_oracle(prec, move, nm, ctx64, ctx32, oracle):
    ctx = ctx64 if prec == "f64" else ctx32
    b, D, X, Xp, r, ub = _case(nm, move, 12 + nm)
    alpha, dx = 0.25, 1.0
    W1 = np.random.default_rng(3).normal(size=(3 * nm, 3 * nm)) * 0.2
    W2 = None if move == 0.0 else np.random.default_rng(4).normal(size=(3 * nm, 3 * nm)) * 0.2
    u, d, f = _run(ctx, b, D, X, Xp, r, ub, W1, W2, alpha, dx)
    ur, dr, fr = oracle.nested_projection_stage(b, D, r, Xp, X, ub, W1, W2, alpha=alpha, dx=dx, R=64)
    assert not np.isnan(u).any() and not np.isnan(d).any()
    assert rel_linf(u, ur) < TOL[prec]
    assert rel_linf(d, dr) < TOL[prec]
    if nm:
        assert rel_linf(f, fr) < TOL[prec]


def test_stage_empty_flow_set(ctx64):
    f = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    X = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    ub = torch.zeros(6, dtype=torch.float64, device="cuda")
    W = torch.zeros((6, 6), dtype=torch.float64, device="cuda")
    ctx64.nested_projection_stage(8, np.zeros((0, 3), np.int32), None, None, X_prev=X, X=X, ub=ub, W1=W, f=f)
    torch.cuda.synchronize()
    assert torch.equal(f, torch.zeros_like(f))
