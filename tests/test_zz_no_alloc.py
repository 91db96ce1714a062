"""The allocation-free integrating factor gives what the context-based apply gives.

lgf_intfactor_apply_noalloc serves callers that must not allocate device
memory while they run (their device memory is reserved up front by another
allocator, where a cudaMalloc could fail or stall the device); its scratch is a
fixed __device__ array shared by every call.  Two calls in a row must each
match lgf_intfactor_apply, so that whatever the first call leaves in the shared
array cannot leak into the second; both are also checked against the oracle
(the untruncated E(alpha) of Sec. 2.3 and App. A, Eq. lgf_intfac), so that a
mistake both GPU paths share would still fail.  Collected last on purpose
(file name).
"""
import numpy as np
import pytest
import torch

import lgf_inputs as li
from conftest import rel_linf

pytestmark = pytest.mark.gpu
TOL = {"f64": 1e-12, "f32": 1e-5}


def _apply_both(ctx, prec, p, alpha):
    import paper_1604_01814_gb300 as lgf
    f = torch.tensor(p.f.reshape(-1), dtype=ctx.dtype, device="cuda")
    n_out = p.nrhs * p.ncomp * p.tgt.shape[0] * p.b ** 3
    ref = torch.full((n_out,), float("nan"), dtype=ctx.dtype, device="cuda")
    got = torch.full((n_out,), float("nan"), dtype=ctx.dtype, device="cuda")
    ctx.intfactor_apply(alpha, p.b, p.src, p.tgt, f, ref, ncomp=p.ncomp, nrhs=p.nrhs)
    lgf.lgf_intfactor_apply_noalloc(prec, alpha, p.b, p.src, p.tgt, f, got, ncomp=p.ncomp, nrhs=p.nrhs)
    torch.cuda.synchronize()
    return got.cpu().numpy(), ref.cpu().numpy()


def _oracle(oracle, p, alpha):
    """E(alpha) f on the target blocks, every field, FP64, untruncated."""
    out = [oracle.intfactor_blocks(alpha, p.b, p.src, p.f[r, c], p.tgt).reshape(-1)
           for r in range(p.nrhs) for c in range(p.ncomp)]
    return np.concatenate(out)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_noalloc_matches_context_apply_on_two_calls_in_a_row(prec, ctx64, ctx32, oracle):
    ctx = ctx64 if prec == "f64" else ctx32
    first = li.random_sparse(21, b=16, nsrc=6, ntgt=8, extent=(4, 3, 3), ncomp=2)
    second = li.random_sparse(22, b=8, nsrc=9, ntgt=5, extent=(5, 4, 3), nrhs=2)
    for p, alpha in ((first, 0.5), (second, 2.0)):
        got, ref = _apply_both(ctx, prec, p, alpha)
        assert not np.isnan(got).any()
        assert rel_linf(got, ref) < TOL[prec]
        exact = _oracle(oracle, p, alpha)
        assert rel_linf(got, exact) < TOL[prec]
        assert rel_linf(ref, exact) < TOL[prec]


def test_noalloc_rejects_sizes_beyond_its_limits():
    import paper_1604_01814_gb300 as lgf
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    b = 32
    src = li.box_blocks(2, 1, 1)
    tgt = np.array([[100, 0, 0]], dtype=np.int32)          # 100 blocks apart: beyond the 64-block box
    f = torch.zeros(2 * b ** 3, device="cuda")
    u = torch.zeros(b ** 3, device="cuda")
    with pytest.raises(lgf.LgfError) as e:
        lgf.lgf_intfactor_apply_noalloc("f32", 0.5, b, src, tgt, f, u)
    assert e.value.status == 5 and "64 blocks" in str(e.value)
    big = li.box_blocks(16, 16, 5)                          # 1280 blocks > 1024
    f = torch.zeros(big.shape[0] * 8 ** 3, device="cuda")
    with pytest.raises(lgf.LgfError) as e:
        lgf.lgf_intfactor_apply_noalloc("f32", 0.5, 8, big, big, f, f.clone())
    assert e.value.status == 5
