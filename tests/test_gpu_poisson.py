"""LGF Poisson apply on the GPU against the CPU oracle (direct summation).

Tolerances (relative L-infinity over every compared value): 1e-12 for FP64
contexts and 1e-5 for FP32 contexts."""
import numpy as np
import pytest
import torch

import lgf_inputs as li
from conftest import rel_linf

pytestmark = pytest.mark.gpu
TOL = {"f64": 1e-12, "f32": 1e-5}


def run_poisson(ctx, p, dx=1.0):
    dt = ctx.dtype
    f = torch.tensor(p.f.reshape(-1), dtype=dt, device="cuda")
    u = torch.full((p.nrhs * p.ncomp * p.tgt.shape[0] * p.b ** 3,), float("nan"), dtype=dt, device="cuda")
    ctx.poisson_apply(p.b, p.src, p.tgt, f, u, ncomp=p.ncomp, nrhs=p.nrhs, dx=dx)
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.float64).reshape(p.nrhs, p.ncomp, p.tgt.shape[0] * p.b ** 3)


def oracle_fields(oracle, p, pts_idx=None, dx=1.0, f=None):
    f = p.f if f is None else f
    pts = oracle.block_points(p.b, p.tgt)
    if pts_idx is not None:
        pts = pts[pts_idx]
    out = np.empty((p.nrhs, p.ncomp, pts.shape[0]))
    for r in range(p.nrhs):
        for c in range(p.ncomp):
            out[r, c] = oracle.poisson_direct(p.b, p.src, f[r, c], pts, dx=dx, R=64)
    return out


def test_box32_fp64_every_point(ctx64, oracle):
    """32^3 box, f ~ U[-1,1] (seed 0), all 32768 targets, FP64."""
    p = li.plain_box32()
    got = run_poisson(ctx64, p)
    ref = oracle_fields(oracle, p)
    assert rel_linf(got, ref) < TOL["f64"]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("seed,b,ns,nt,ext", [(1, 8, 5, 7, (4, 3, 3)), (2, 16, 3, 4, (3, 2, 2)),
                                            (3, 4, 9, 6, (5, 4, 3)), (4, 32, 1, 2, (2, 1, 1))])
def test_random_sparse_sets_every_point(prec, seed, b, ns, nt, ext, ctx64, ctx32, oracle):
    """Ragged block sets, source and target sets disjoint or overlapping."""
    ctx = ctx64 if prec == "f64" else ctx32
    p = li.random_sparse(seed, b=b, nsrc=ns, ntgt=nt, extent=ext)
    got = run_poisson(ctx, p)
    ref = oracle_fields(oracle, p)
    assert rel_linf(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_multiple_components_and_rhs(prec, ctx64, ctx32, oracle):
    ctx = ctx64 if prec == "f64" else ctx32
    p = li.random_sparse(11, b=8, nsrc=4, ntgt=5, extent=(3, 3, 2), nrhs=2, ncomp=3)
    got = run_poisson(ctx, p, dx=0.5)
    ref = oracle_fields(oracle, p, dx=0.5)
    for r in range(2):
        for c in range(3):
            assert rel_linf(got[r, c], ref[r, c]) < TOL[prec]


def test_dense128_fp32_sampled(ctx32, oracle):
    """128^3 dense box of Gaussian blobs (seed 1), FP32, 512 random targets."""
    p = li.dense_blobs()
    got = run_poisson(ctx32, p)
    rng = np.random.default_rng(101)
    idx = rng.choice(p.tgt.shape[0] * p.b ** 3, size=512, replace=False)
    ref = oracle_fields(oracle, p, pts_idx=idx)
    assert rel_linf(got[0, 0, idx], ref[0, 0]) < TOL["f32"]


def test_dense128_fp64_residual(ctx64):
    """FP64 apply on the 128^3 box satisfies L u = f (lgf_residual, FP64)."""
    p = li.dense_blobs(b=16)
    dt = torch.float64
    f = torch.tensor(p.f.reshape(-1), dtype=dt, device="cuda")
    u = torch.empty_like(f)
    ctx64.poisson_apply(p.b, p.src, p.tgt, f, u)
    r, rmax, fmax = ctx64.residual(p.b, p.tgt, u, f)
    assert rmax < 1e-11 * fmax
    # every interior point was checked: the residual field is zero only on the boundary
    assert torch.count_nonzero(r).item() > 0.9 * (126 ** 3)


def test_sphere_fp32_sampled(ctx32, oracle):
    """Sphere + wake block set (b=16), 3-component IB-like sources, 256 targets."""
    p = li.sphere_ib()
    got = run_poisson(ctx32, p)
    rng = np.random.default_rng(5)
    idx = rng.choice(p.tgt.shape[0] * p.b ** 3, size=256, replace=False)
    ref = oracle_fields(oracle, p, pts_idx=idx)
    for c in range(3):
        assert rel_linf(got[0, c, idx], ref[0, c]) < TOL["f32"]


def test_point_source_reproduces_table(ctx64):
    b = 8
    f = torch.zeros(b ** 3, dtype=torch.float64, device="cuda")
    f[(2 * b + 3) * b + 1] = 1.0                       # point (1, 3, 2)
    tgt = np.array([[0, 0, 0], [3, -1, 2], [-2, 0, 0]], dtype=np.int32)
    u = torch.empty(3 * b ** 3, dtype=torch.float64, device="cuda")
    ctx64.poisson_apply(b, [[0, 0, 0]], tgt, f, u)
    pts = li.block_point_coords(b, tgt).reshape(-1, 3)
    offs = torch.tensor(pts - np.array([1, 3, 2]), dtype=torch.int32)
    g = ctx64.table_lookup(offs)
    assert torch.max(torch.abs(u - g)).item() < 1e-13 * torch.max(torch.abs(g)).item()


def test_empty_sets(ctx32):
    b = 8
    u = torch.full((2 * b ** 3,), 7.0, device="cuda")
    ctx32.poisson_apply(b, np.zeros((0, 3)), [[0, 0, 0], [1, 0, 0]], None, u)
    torch.cuda.synchronize()
    assert torch.all(u == 0)
    f = torch.ones(b ** 3, device="cuda")
    ctx32.poisson_apply(b, [[0, 0, 0]], np.zeros((0, 3)), f, None)


def test_invalid_arguments(ctx32):
    import paper_1604_01814_gb300 as lgf
    b = 8
    f = torch.ones(b ** 3, device="cuda")
    u = torch.empty(b ** 3, device="cuda")
    with pytest.raises(lgf.LgfError) as e:
        ctx32.poisson_apply(b, [[0, 0, 0], [0, 0, 0]], [[0, 0, 0]], torch.ones(2 * b ** 3, device="cuda"), u)
    assert e.value.status == 1
    with pytest.raises(lgf.LgfError) as e:
        ctx32.poisson_apply(b, [[0, 0, 0]], [[0, 0, 0]], f, u, dx=-1.0)
    assert e.value.status == 1
    with pytest.raises(lgf.LgfError) as e:
        ctx32.poisson_apply(b, [[0, 0, 0]], [[300, 0, 0]], f, u)   # union spans > 2048 points
    assert e.value.status == 5
    with pytest.raises(ValueError):
        ctx32.poisson_apply(b, [[0, 0, 0]], [[0, 0, 0]], f.double(), u)


def _box_lengths(p):
    """Transform lengths the library's plan picks for this problem (smallest of
    2^k, 3*2^k, 5*2^k in 32..4096 at or above 2L - 1 per axis)."""
    sizes = (32, 64, 80, 96, 128, 160, 192, 256, 320, 384, 512, 640, 768, 1024, 1280, 1536, 2048, 2560, 3072, 4096)
    allc = np.concatenate([p.src, p.tgt])
    L = (allc.max(0) - allc.min(0) + 1) * p.b
    return [next(m for m in sizes if m >= 2 * l - 1) for l in L]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("b,ext,lengths", [(16, (3, 2, 5), (96, 64, 160)), (8, (5, 3, 1), (80, 64, 32)),
                                           (16, (6, 3, 2), (192, 96, 64)), (16, (2, 5, 3), (64, 160, 96))])
def test_mixed_radix_lengths_every_point(prec, b, ext, lengths, ctx64, ctx32, oracle):
    """Sparse block sets spanning boxes whose transform lengths include
    3 * 2^k or 5 * 2^k (radix-12 or radix-20 last stage) on every axis
    position: every target point against the oracle."""
    ctx = ctx64 if prec == "f64" else ctx32
    ex, ey, ez = ext
    src = np.array([[0, 0, 0], [ex - 1, ey - 1, ez - 1], [ex // 2, 0, ez - 1]], dtype=np.int32)
    tgt = np.array([[ex - 1, 0, 0], [0, ey - 1, ez - 1], [ex // 2, ey - 1, 0]], dtype=np.int32)
    rng = np.random.default_rng(7)
    p = li.Problem("mixed", b, src, tgt, rng.uniform(-1, 1, size=(1, 1, src.shape[0], b ** 3)))
    assert tuple(_box_lengths(p)) == lengths
    got = run_poisson(ctx, p)
    ref = oracle_fields(oracle, p)
    assert rel_linf(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("src,tgt,lengths", [
    ([[0, 0, 0], [5, 0, 1], [2, 4, 0], [11, 1, 1]], [[0, 0, 0], [6, 1, 1], [11, 0, 0], [3, 1, 1]], (768, 320, 128)),
    ([[0, 0, 0], [9, 5, 1], [4, 2, 0]], [[9, 0, 0], [0, 5, 1], [5, 3, 1]], (640, 384, 128))])
def test_mixed_radix_long_lengths_sampled(prec, src, tgt, lengths, ctx64, ctx32, oracle):
    """Lengths 320 to 768 (three-stage plans with a radix-12 or radix-20 last
    stage) on sparse sets; 400 sampled targets against the oracle."""
    ctx = ctx64 if prec == "f64" else ctx32
    b = 32
    src = np.array(src, dtype=np.int32)
    tgt = np.array(tgt, dtype=np.int32)
    rng = np.random.default_rng(8)
    f = rng.uniform(-1, 1, size=(1, 1, src.shape[0], b ** 3))
    p = li.Problem("sparse", b, src, tgt, f)
    assert tuple(_box_lengths(p)) == lengths
    got = run_poisson(ctx, p).reshape(-1)
    pts = oracle.block_points(b, tgt)
    idx = rng.choice(pts.shape[0], size=400, replace=False)
    ref = oracle.poisson_direct(b, src, f[0, 0], pts[idx], R=64)
    assert rel_linf(got[idx], ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("nbx,length", [(20, 1280), (24, 1536), (40, 2560), (48, 3072), (64, 4096)])
def test_longest_lengths_sampled(prec, nbx, length, ctx64, ctx32, oracle):
    """The long plans up to the largest supported length (4096, a union box of
    2048 points along x): two source blocks at the ends of a thin box, 300
    sampled targets against the oracle."""
    ctx = ctx64 if prec == "f64" else ctx32
    b = 32
    src = np.array([[0, 0, 0], [nbx - 1, 0, 0]], dtype=np.int32)
    tgt = np.array([[nbx // 2, 0, 0], [nbx - 1, 0, 0], [1, 0, 0]], dtype=np.int32)
    rng = np.random.default_rng(nbx)
    f = rng.uniform(-1, 1, size=(1, 1, src.shape[0], b ** 3))
    p = li.Problem("thin", b, src, tgt, f)
    assert tuple(_box_lengths(p)) == (length, 64, 64)
    got = run_poisson(ctx, p).reshape(-1)
    pts = oracle.block_points(b, tgt)
    idx = rng.choice(pts.shape[0], size=300, replace=False)
    ref = oracle.poisson_direct(b, src, f[0, 0], pts[idx], R=64)
    assert rel_linf(got[idx], ref) < TOL[prec]


def _line_problem(seed, b, src_x, tgt_x, yz=((0, 0), (0, 1)), ncomp=1, nrhs=1):
    """Blocks along x: sources at src_x (y, z from yz[0]), targets at tgt_x (y, z
    from yz[1] and its neighbour row), f ~ U[-1, 1]."""
    rng = np.random.default_rng(seed)
    src = np.array([[x, yz[0][0], yz[0][1]] for x in src_x], dtype=np.int32)
    tgt = np.array([[x, yz[1][0] + dy, yz[1][1]] for x in tgt_x for dy in (0, 1)], dtype=np.int32)
    f = rng.uniform(-1, 1, size=(nrhs, ncomp, src.shape[0], b ** 3))
    return li.Problem("line", b, src, tgt, f)


def _transposed(p):
    """The same problem with x and y exchanged (a wake along y)."""
    sw = lambda c: np.ascontiguousarray(c[:, [1, 0, 2]])
    b = p.b
    f = p.f.reshape(p.nrhs, p.ncomp, -1, b, b, b).transpose(0, 1, 2, 3, 5, 4).reshape(p.f.shape)
    return li.Problem(p.name + "_yx", b, sw(p.src), sw(p.tgt), np.ascontiguousarray(f))


def _blob_problem(seed, b, src, tgt):
    rng = np.random.default_rng(seed)
    src = np.array(src, dtype=np.int32)
    tgt = np.array(tgt, dtype=np.int32)
    return li.Problem("blob", b, src, tgt, rng.uniform(-1, 1, size=(1, 1, src.shape[0], b ** 3)))


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("case", ["body_and_wake", "source_after_target", "far_apart", "long_source",
                                  "wake_along_y", "wake_along_x_and_y"])
def test_shifted_window_every_point(prec, case, ctx64, ctx32, oracle):
    """Source and target extents that differ along x or y: the plan embeds
    that axis with the shifted window (M >= Ls + Lt - 1, complex spectrum;
    no symmetry in ky for y) where that is shorter than the even one, with
    targets past M/2 (every output of that axis's inverse stage formed); a
    long source keeps the even embedding."""
    ctx = ctx64 if prec == "f64" else ctx32
    b = 8
    cases = {"body_and_wake": lambda: _line_problem(21, b, [0, 1], range(-1, 11), ncomp=2),
             "source_after_target": lambda: _line_problem(22, b, [10, 11], range(0, 10), yz=((1, 0), (0, 0))),
             "far_apart": lambda: _line_problem(23, b, [0], range(6, 10), nrhs=2),
             "long_source": lambda: _line_problem(24, b, range(0, 6), [3], yz=((0, 0), (0, 0))),
             "wake_along_y": lambda: _transposed(_line_problem(25, b, [0, 1], range(-1, 11), ncomp=2)),
             "wake_along_x_and_y": lambda: _blob_problem(26, b, [[0, 0, 0], [1, 0, 0]],
                                                         [[x, y, 0] for x in range(-1, 9) for y in range(-1, 7)])}
    p = cases[case]()
    got = run_poisson(ctx, p)
    ref = oracle_fields(oracle, p)
    assert rel_linf(got, ref) < TOL[prec]
