"""Staggered curl C, its adjoint and the velocity refresh (Sec. 4.1, Eq.
vel_refresh) on the GPU against the CPU oracle.

The stencils are integer combinations of the inputs, so FP64 results match
the oracle to rounding (1e-14 relative); the refresh carries the Poisson
apply's tolerances (1e-12 FP64, 1e-5 FP32)."""
import numpy as np
import pytest
import torch

import lgf_inputs as li
from conftest import rel_linf

pytestmark = pytest.mark.gpu
TOL = {"f64": 1e-12, "f32": 1e-5}


def _sets(seed, b, ns, nt, ext):
    p = li.random_sparse(seed, b=b, nsrc=ns, ntgt=nt, extent=ext)
    return p.src, p.tgt


def oracle_stencil(oracle, b, src, vals, tgt, adjoint, dx):
    """C or C^dagger of a block-set field (zero outside src), restricted to tgt."""
    src = np.asarray(src, dtype=np.int64)
    tgt = np.asarray(tgt, dtype=np.int64)
    allc = np.concatenate([src, tgt])
    lo = allc.min(axis=0) - 1
    hi = allc.max(axis=0) + 2
    shape = tuple(int(v) for v in ((hi - lo) * b)[::-1])
    box = np.stack([oracle.blocks_to_box(b, src, vals[k], lo, shape)[0] for k in range(3)])
    out = oracle.curl_adj_box(box, dx) if adjoint else oracle.curl_box(box, dx)
    return np.stack([oracle.box_to_blocks(b, tgt, out[k], lo) for k in range(3)])


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("seed,b,ns,nt,ext", [(1, 8, 6, 7, (3, 3, 2)), (2, 4, 9, 9, (4, 3, 3)),
                                            (3, 16, 3, 4, (2, 2, 2)), (4, 32, 2, 2, (2, 1, 1))])
def test_curl_and_adjoint_every_point(prec, adjoint, seed, b, ns, nt, ext, ctx64, ctx32, oracle):
    ctx = ctx64 if prec == "f64" else ctx32
    src, tgt = _sets(seed, b, ns, nt, ext)
    rng = np.random.default_rng(seed)
    nrhs = 2
    vals = rng.uniform(-1, 1, size=(nrhs, 3, src.shape[0], b ** 3))
    a = torch.tensor(vals.reshape(-1), dtype=ctx.dtype, device="cuda")
    out = torch.full((nrhs * 3 * tgt.shape[0] * b ** 3,), float("nan"), dtype=ctx.dtype, device="cuda")
    (ctx.curl_adjoint if adjoint else ctx.curl)(b, src, tgt, a, out, nrhs=nrhs, dx=0.5)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64).reshape(nrhs, 3, tgt.shape[0], b ** 3)
    for r in range(nrhs):
        ref = oracle_stencil(oracle, b, src, vals[r], tgt, adjoint, 0.5)
        assert rel_linf(got[r], ref) < (1e-14 if prec == "f64" else 1e-6)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_velocity_refresh_every_point(prec, ctx64, ctx32, oracle):
    ctx = ctx64 if prec == "f64" else ctx32
    b = 8
    src = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 0, 1]], dtype=np.int32)
    tgt = np.array([[1, 0, 0], [2, 0, 0], [0, 1, 1], [-1, 0, 0]], dtype=np.int32)
    rng = np.random.default_rng(11)
    u = rng.uniform(-1, 1, size=(3, src.shape[0], b ** 3))
    ut = torch.tensor(u.reshape(-1), dtype=ctx.dtype, device="cuda")
    out = torch.full((3 * tgt.shape[0] * b ** 3,), float("nan"), dtype=ctx.dtype, device="cuda")
    ctx.velocity_refresh(b, src, tgt, ut, out, dx=0.25)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64).reshape(3, tgt.shape[0], b ** 3)
    ref = oracle.velocity_refresh(b, src, u, tgt, dx=0.25, R=64)
    assert rel_linf(got, ref) < TOL[prec]


def test_velocity_refresh_keeps_divergence_free_field(ctx64, oracle):
    """u = C^dagger psi with its vorticity inside the source blocks comes back
    unchanged, on the source blocks and beyond them (zero there)."""
    b = 16
    src = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], dtype=np.int32)
    rng = np.random.default_rng(12)
    psi = np.zeros((3, b, 2 * b, 2 * b))
    psi[:, 4:12, 4:28, 4:28] = rng.uniform(-1, 1, size=(3, 8, 24, 24))
    ubox = oracle.curl_adj_box(psi)
    lo = np.zeros(3, dtype=np.int64)
    u = np.stack([oracle.box_to_blocks(b, src, ubox[k], lo) for k in range(3)])
    tgt = np.array([[0, 0, 0], [1, 1, 0], [2, 0, 0], [0, 0, -1]], dtype=np.int32)
    ut = torch.tensor(u.reshape(-1), dtype=torch.float64, device="cuda")
    out = torch.empty(3 * tgt.shape[0] * b ** 3, dtype=torch.float64, device="cuda")
    ctx64.velocity_refresh(b, src, tgt, ut, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(3, tgt.shape[0], b ** 3)
    ref = np.zeros_like(got)
    ref[:, 0] = u[:, 0]
    ref[:, 1] = u[:, 3]
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(u))


def test_velocity_refresh_multiple_rhs_equal_single(ctx32):
    b = 8
    src = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.int32)
    tgt = np.array([[0, 0, 0], [1, 1, 0]], dtype=np.int32)
    rng = np.random.default_rng(13)
    u = torch.tensor(rng.uniform(-1, 1, 2 * 3 * src.shape[0] * b ** 3), dtype=torch.float32, device="cuda")
    both = torch.empty(2 * 3 * tgt.shape[0] * b ** 3, dtype=torch.float32, device="cuda")
    ctx32.velocity_refresh(b, src, tgt, u, both, nrhs=2)
    n_in, n_out = 3 * src.shape[0] * b ** 3, 3 * tgt.shape[0] * b ** 3
    for r in range(2):
        one = torch.empty(n_out, dtype=torch.float32, device="cuda")
        ctx32.velocity_refresh(b, src, tgt, u[r * n_in:(r + 1) * n_in].contiguous(), one)
        torch.cuda.synchronize()
        assert torch.equal(one, both[r * n_out:(r + 1) * n_out])
