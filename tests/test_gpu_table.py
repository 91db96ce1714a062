"""GPU G_L table (FP64 quadrature + far-field expansion) against the CPU oracle."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_table_matches_oracle_quadrature(ctx64, oracle):
    R = 48
    radius, mismatch = ctx64.table_info()
    assert radius == R
    ref = oracle.lgf_table(R)
    offs = []
    for a in range(R + 1):
        for b in range(a + 1):
            for c in range(b + 1):
                offs.append((a, b, c))
    offs = torch.tensor(offs, dtype=torch.int32)
    got = ctx64.table_lookup(offs).cpu().numpy()
    rel = np.abs(got - ref) / np.abs(ref)
    assert rel.max() < 1e-13, rel.max()
    # near/far matching on the outer shell (expansion error at |n| ~ 45..48)
    assert mismatch < 1e-10


def test_lookup_signs_and_permutations(ctx64, oracle):
    offs = torch.tensor([(3, -2, 1), (-2, 1, -3), (1, 3, 2), (0, 0, 0), (-47, 5, 0)], dtype=torch.int32)
    got = ctx64.table_lookup(offs).cpu().numpy()
    assert np.all(got[:3] == got[0])
    assert abs(got[3] - oracle.lgf_quad(0, 0, 0)) < 1e-15
    assert abs(got[4] - oracle.lgf_quad(47, 5, 0)) < 1e-15


def test_lookup_beyond_table_uses_expansion(ctx64, oracle):
    offs = [(49, 0, 0), (60, 31, 7), (200, 1, 1), (1000, 700, 300), (49, 49, 49)]
    got = ctx64.table_lookup(torch.tensor(offs, dtype=torch.int32)).cpu().numpy()
    for n, g in zip(offs, got):
        ref = oracle.lgf_asym(*n, order=7)
        assert abs(g - ref) <= 1e-14 * abs(ref), n
    # and the expansion is the Green's function there (quadrature overlap)
    for n in [(49, 0, 0), (60, 31, 7)]:
        q = oracle.lgf_quad(*n)
        g = ctx64.table_lookup(torch.tensor([n], dtype=torch.int32)).item()
        assert abs(g - q) / abs(q) < 1e-11


def test_intfactor_weights_match_oracle(ctx64, oracle):
    for alpha in (0.0, 0.05, 0.1, 0.25, 0.5, 1.0, 2.0):
        R, w = ctx64.intfactor_weights(alpha)
        ref = oracle.intfactor_weights(alpha, R + 1)
        assert np.allclose(w.cpu().numpy(), ref[:R + 1], rtol=1e-13, atol=1e-300)
        if alpha > 0:
            # truncation rule: w_R < tol/8 w_0 <= w_{R-1}  (tol = 1e-13 for FP64 contexts)
            assert ref[R] < 1e-13 / 8 * ref[0] <= ref[R - 1]
        else:
            assert R == 0
