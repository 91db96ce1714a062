"""Diagnostics of the library: the a-posteriori error estimate of a Poisson
result, and the saved G_L table.

- lgf_poisson_error_estimate forms the exact sum of Sec. 2.2, Eq.
  dpoisson_conv, in FP64 on the GPU at sampled targets: its estimate agrees
  with the error the oracle measures at every target (within a factor that
  sampling explains), stays under the 1e-5 / 1e-12 bars for correct results,
  and catches a result that is off by 1e-3.
- lgf_table_save / lgf_table_load: a loaded table gives the built table's
  values bit for bit and the same applies; a corrupted file is refused.
"""
import numpy as np
import pytest
import torch

import lgf_inputs as li
import paper_1604_01814_gb300 as lgf
from conftest import build_lib, rel_linf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_error_estimate_tracks_the_oracle(prec, ctx32, ctx64, oracle):
    ctx = ctx64 if prec == "f64" else ctx32
    p = li.random_sparse(51, b=8, nsrc=5, ntgt=6, extent=(4, 3, 3), ncomp=2)
    f = torch.tensor(p.f.reshape(-1), dtype=ctx.dtype, device="cuda")
    u = torch.empty(p.ncomp * p.tgt.shape[0] * p.b ** 3, dtype=ctx.dtype, device="cuda")
    ctx.poisson_apply(p.b, p.src, p.tgt, f, u, ncomp=p.ncomp)
    est = ctx.poisson_error_estimate(p.b, p.src, p.tgt, f, u, ncomp=p.ncomp, nsample=256)
    pts = oracle.block_points(p.b, p.tgt)
    ref = oracle.poisson_direct_multi(p.b, p.src, p.f[0], pts, R=64)
    true = max(rel_linf(u.cpu().numpy().reshape(p.ncomp, -1)[c], ref[c]) for c in range(p.ncomp))
    bar = 1e-5 if prec == "f32" else 1e-12
    assert est < bar and true < bar
    assert est <= 1.5 * true + 1e-15              # a sample cannot see more than every point does
    if prec == "f32":
        assert est > true / 30                    # and sees the same rounding level
    u.mul_(1.001)
    assert ctx.poisson_error_estimate(p.b, p.src, p.tgt, f, u, ncomp=p.ncomp, nsample=64) > 5e-4


def test_table_save_and_load(tmp_path, ctx64):
    path = str(tmp_path / "gl.tab")
    ctx64.table_save(path)
    c2 = lgf.Context("f64")
    c2.table_load(path)
    r, mm = c2.table_info()
    assert (r, mm) == ctx64.table_info()
    off = torch.tensor(np.random.default_rng(3).integers(-70, 70, size=(500, 3)), dtype=torch.int32)
    assert torch.equal(c2.table_lookup(off), ctx64.table_lookup(off))
    p = li.random_sparse(52, b=8, nsrc=3, ntgt=3, extent=(3, 2, 2))
    f = torch.tensor(p.f.reshape(-1), dtype=torch.float64, device="cuda")
    u1 = torch.empty(p.tgt.shape[0] * p.b ** 3, dtype=torch.float64, device="cuda")
    u2 = torch.empty_like(u1)
    ctx64.poisson_apply(p.b, p.src, p.tgt, f, u1)
    c2.poisson_apply(p.b, p.src, p.tgt, f, u2)
    assert torch.equal(u1, u2)
    raw = bytearray(open(path, "rb").read())
    raw[100] ^= 0x40                                  # one flipped bit in the values
    open(path, "wb").write(bytes(raw))
    with pytest.raises(lgf.LgfError) as e:
        c2.table_load(path)
    assert e.value.status == lgf._binding.LGF_EINVAL
    c2.close()
