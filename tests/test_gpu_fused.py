"""The fused y+x inverse (one thread-block cluster per target plane, the
plane's rows in distributed shared memory) against the two separate passes
and the oracle.

Each case is run in two contexts that read their plan choice from a tuning
file: the same embedding and lengths, the inverse fused in one and apart in
the other.  The outputs must agree bit for bit (the fused kernel runs the same
line arithmetic), the fused one must be reported as such, and it must match
the FP64 direct sum (Sec. 2.2, Eq. dpoisson_conv) on sampled targets.  The
cases cover the four lengths along y the fused kernel exists for, clusters of
one, two and four CTAs, targets past half the length along x and y (the
full-output stages), planes and row blocks without targets, and several
fields.
"""
import numpy as np
import pytest
import torch

import lgf_inputs as li
import paper_1604_01814_gb300 as lgf
from conftest import build_lib, rel_linf

pytestmark = pytest.mark.gpu


def _key(p, nf):
    s, t = p.src, p.tgt
    nbs = s.max(0) - s.min(0) + 1
    nbt = t.max(0) - t.min(0) + 1
    off = t.min(0) - s.min(0)
    j = lambda v: ",".join(str(int(x)) for x in v)
    return f"P f32 b{p.b} s{j(nbs)} t{j(nbt)} o{j(off)} nf{nf}"


def _case(seed, b, src, tgt, ncomp=1):
    rng = np.random.default_rng(seed)
    src = np.asarray(src, np.int32).reshape(-1, 3)
    tgt = np.asarray(tgt, np.int32).reshape(-1, 3)
    return li.Problem("fused", b, src, tgt, rng.uniform(-1.0, 1.0, size=(1, ncomp, src.shape[0], b ** 3)))


def cases():
    out = []
    # My = 64 (union extent 32 along y), a long x extent: cluster of 2 or 4
    out.append(("y64_long_x", "x0 y0", _case(1, 16, li.box_blocks(2, 1, 1), li.box_blocks(20, 2, 2), 2)))
    # My = 80 (b = 8, five blocks along y), two fields
    out.append(("y80", "x0 y0", _case(2, 8, li.box_blocks(2, 2, 1), li.box_blocks(3, 5, 2), 2)))
    # My = 96: targets only in some planes and row blocks (sparse target set)
    t = np.array([[0, 0, 0], [2, 2, 0], [1, 0, 2], [3, 1, 3]], np.int32)
    out.append(("y96_sparse", "x0 y0", _case(3, 16, [[0, 0, 0], [1, 2, 1]], t)))
    # My = 128 (b = 16, four blocks along y), shifted x window: targets past half along x
    out.append(("y128_shift_x", "x1 y0", _case(4, 16, [[0, 0, 0]], li.box_blocks(6, 4, 1))))
    # shifted y window (length 64 or 80 along y): targets past half along y
    out.append(("shift_y", "x0 y1", _case(5, 8, [[0, 0, 0]], li.box_blocks(1, 7, 2))))
    return out


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_lib()


@pytest.mark.parametrize("name,xy,p", cases(), ids=[c[0] for c in cases()])
def test_fused_inverse_equals_separate_passes(name, xy, p, built, tmp_path, oracle):
    nf = p.ncomp
    outs, reps = {}, {}
    for fuse in (1, 0):
        path = tmp_path / f"tune_{fuse}.txt"
        path.write_text(f"{_key(p, nf)} -> {xy} bx0 by0 bz0 z0 f{fuse}\n")
        ctx = lgf.Context("f32")
        ctx.table_build(48)
        ctx.autotune(lgf.LGF_TUNE_CACHED, str(path))
        f = torch.tensor(p.f.reshape(-1), dtype=torch.float32, device="cuda")
        u = torch.full((nf * p.tgt.shape[0] * p.b ** 3,), float("nan"), device="cuda")
        ctx.poisson_apply(p.b, p.src, p.tgt, f, u, ncomp=nf)
        torch.cuda.synchronize()
        outs[fuse] = u.cpu()
        reps[fuse] = ctx.tune_report()
        ctx.close()
    assert reps[1]["plans_from_cache"] == 1 and reps[0]["plans_from_cache"] == 1
    assert reps[1]["fused_inverse"] == 1 and reps[0]["fused_inverse"] == 0
    assert torch.equal(outs[1], outs[0])
    # against the oracle on sampled targets, every field
    pts_all = oracle.block_points(p.b, p.tgt)
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(pts_all.shape[0], size=min(384, pts_all.shape[0]), replace=False))
    got = outs[1].numpy().reshape(nf, -1)
    for c in range(nf):
        ref = oracle.poisson_direct(p.b, p.src, p.f[0, c], pts_all[idx], R=64)
        assert rel_linf(got[c, idx], ref) < 1e-5


def test_fused_inverse_in_ragged_batches(built, tmp_path):
    """Several problems whose plans take the fused inverse (different lengths
    along x and y, so several fused launches of different cluster sizes, and
    one problem whose length along y has no fused kernel) in one ragged
    batch: equal bit for bit to the same batch with every inverse apart."""
    probs = [c[2] for c in cases()]
    probs.append(_case(9, 16, [[0, 0, 0]], li.box_blocks(2, 10, 1)))   # 160+ along y: never fused
    outs, reps = {}, {}
    for fuse in (1, 0):
        path = tmp_path / f"tune_{fuse}.txt"
        path.write_text("".join(f"{_key(p, p.ncomp)} -> x0 y0 bx0 by0 bz0 z0 f{fuse}\n" for p in probs))
        ctx = lgf.Context("f32", flags=lgf._binding.LGF_FLAG_BATCH_RAGGED)
        ctx.table_build(48)
        ctx.autotune(lgf.LGF_TUNE_CACHED, str(path))
        batch = []
        for p in probs:
            f = torch.tensor(p.f.reshape(-1), dtype=torch.float32, device="cuda")
            u = torch.full((p.ncomp * p.tgt.shape[0] * p.b ** 3,), float("nan"), device="cuda")
            batch.append(dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=u, ncomp=p.ncomp, op=lgf.LGF_OP_POISSON))
        s = torch.cuda.Stream()
        for _ in range(2):   # capture, then replay
            with torch.cuda.stream(s):
                ctx.batch_apply(batch, stream=s)
            s.synchronize()
        outs[fuse] = [q["u"].cpu() for q in batch]
        reps[fuse] = ctx.tune_report()
        ctx.close()
    assert reps[1]["last_ragged"] == 1 and reps[1]["fused_inverse"] == len(probs) - 1
    assert reps[0]["fused_inverse"] == 0
    for a, b in zip(outs[1], outs[0]):
        assert torch.equal(a, b) and not torch.isnan(a).any()
