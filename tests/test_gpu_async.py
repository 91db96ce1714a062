"""Bulk asynchronous staging of the integrating factor's z pass and the
bounded device-side waits.

- With LGF_FLAG_BULK_STAGING the z pass stages its slabs with cp.async.bulk
  copies on mbarriers (double-buffered, persistent); without it, with
  per-thread 16-byte loads.  Both give the oracle's E(alpha) f (Sec. 2.3
  footnote; App. A, Eq. lgf_intfac) on every point, and no wait runs out
  (the device error word stays 0).
- Fields that are not 16-byte aligned are refused before any launch.
- The timeout path: a CTA waiting on an mbarrier that no copy completes gives
  up after its limit and sets the error word; lgf_device_status reports
  LGF_ETIMEOUT once, and the context keeps working.  Nothing traps or faults.
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
def bulk_ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_lib()
    ctxs = {p: lgf.Context(p, flags=lgf._binding.LGF_FLAG_BULK_STAGING) for p in ("f32", "f64")}
    for c in ctxs.values():
        c.table_build(48)
    yield ctxs
    for c in ctxs.values():
        c.close()


def _e_problem(ctx, seed):
    p = li.random_sparse(seed, b=16, nsrc=6, ntgt=7, extent=(3, 3, 3), ncomp=2)
    f = torch.tensor(p.f.reshape(-1), dtype=ctx.dtype, device="cuda")
    u = torch.full((p.ncomp * p.tgt.shape[0] * p.b ** 3,), float("nan"), dtype=ctx.dtype, device="cuda")
    return p, f, u


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("staging", ["bulk", "loads"])
def test_z_pass_staging_matches_oracle(prec, staging, bulk_ctx, ctx32, ctx64, oracle):
    ctx = bulk_ctx[prec] if staging == "bulk" else (ctx64 if prec == "f64" else ctx32)
    p, f, u = _e_problem(ctx, 91)
    for alpha in (0.5, 2.0):
        u.fill_(float("nan"))
        ctx.intfactor_apply(alpha, p.b, p.src, p.tgt, f, u, ncomp=p.ncomp)
        assert ctx.device_status() == 0
        ref = np.concatenate([oracle.intfactor_blocks(alpha, p.b, p.src, p.f[0, c], p.tgt).reshape(-1)
                              for c in range(p.ncomp)])
        assert rel_linf(u.cpu().numpy(), ref) < TOL[prec]


def test_misaligned_fields_are_refused(ctx32):
    p, f, u = _e_problem(ctx32, 93)
    store = torch.zeros(f.numel() + 1, dtype=torch.float32, device="cuda")
    fo = store[1:]                                           # 4 bytes off a 16-byte boundary
    with pytest.raises(lgf.LgfError) as e:
        ctx32.intfactor_apply(0.5, p.b, p.src, p.tgt, fo, u, ncomp=p.ncomp)
    assert e.value.status == lgf._binding.LGF_EINVAL and "aligned" in str(e.value)
    assert ctx32.device_status() == 0


def test_wait_that_runs_out_sets_the_error_word(ctx32, oracle):
    ctx32.wait_selftest(cycles=2_000_000)                    # about a millisecond
    with pytest.raises(lgf.LgfError) as e:
        ctx32.device_status()
    assert e.value.status == lgf._binding.LGF_ETIMEOUT
    assert ctx32.device_status() == 0                        # cleared once reported
    # the context keeps working
    p = li.random_sparse(92, b=8, nsrc=3, ntgt=4, extent=(3, 2, 2))
    f = torch.tensor(p.f.reshape(-1), dtype=torch.float32, device="cuda")
    u = torch.empty(p.tgt.shape[0] * p.b ** 3, dtype=torch.float32, device="cuda")
    ctx32.intfactor_apply(0.25, p.b, p.src, p.tgt, f, u)
    assert ctx32.device_status() == 0
    ref = oracle.intfactor_blocks(0.25, p.b, p.src, p.f[0, 0], p.tgt).reshape(-1)
    assert rel_linf(u.cpu().numpy(), ref) < TOL["f32"]
