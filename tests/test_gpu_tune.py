"""The autotuner (lgf_autotune): tuned plans keep parity with the oracle, the
choices persist to a file and a later context reuses them without timing,
and a batch's branch count is chosen once per shape.

Parity is the oracle's direct sum (Sec. 2.2, Eq. dpoisson_conv): FP64 at
1e-12 and FP32 at 1e-5 relative L-infinity, every target point."""
import numpy as np
import pytest
import torch

import lgf_inputs as li
import paper_1604_01814_gb300 as lgf
from conftest import build_lib, rel_linf

pytestmark = pytest.mark.gpu
TOL = {"f64": 1e-12, "f32": 1e-5}


def _fresh(prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_lib()
    c = lgf.Context(prec)
    c.table_build(48)
    return c


def _wake_problem(seed, b=8):
    """A small body and a long wake: several geometries are worth timing."""
    rng = np.random.default_rng(seed)
    src = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.int32)
    tgt = np.array([[x, y, 0] for x in range(-1, 9) for y in range(-1, 3)], dtype=np.int32)
    return li.Problem("wake", b, src, tgt, rng.uniform(-1, 1, size=(1, 2, src.shape[0], b ** 3)))


def _apply(ctx, p):
    f = torch.tensor(p.f.reshape(-1), dtype=ctx.dtype, device="cuda")
    u = torch.full((p.ncomp * p.tgt.shape[0] * p.b ** 3,), float("nan"), dtype=ctx.dtype, device="cuda")
    ctx.poisson_apply(p.b, p.src, p.tgt, f, u, ncomp=p.ncomp)
    torch.cuda.synchronize()
    return u.cpu().numpy().reshape(p.ncomp, -1)


def _oracle(oracle, p):
    return oracle.poisson_direct_multi(p.b, p.src, p.f[0], oracle.block_points(p.b, p.tgt), R=64)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_tuned_plan_parity_and_persistence(prec, oracle, tmp_path):
    path = str(tmp_path / "tune.txt")
    p = _wake_problem(31)
    ref = _oracle(oracle, p)
    c1 = _fresh(prec)
    c1.autotune(lgf.LGF_TUNE_ON, path)
    got = _apply(c1, p)
    assert rel_linf(got, ref) < TOL[prec]
    r1 = c1.tune_report()
    assert r1["plans_tuned"] == 1 and r1["candidates_timed"] >= 3 and r1["tune_ms"] > 0
    text = open(path).read()
    assert text.count(" -> ") == 1 and text.startswith("P " + prec)
    # the same plan again in this context: no second tuning
    _apply(c1, p)
    assert c1.tune_report()["candidates_timed"] == r1["candidates_timed"]
    c1.close()
    # a new context reads the file: same choice, nothing timed
    c2 = _fresh(prec)
    c2.autotune(lgf.LGF_TUNE_CACHED, path)
    got2 = _apply(c2, p)
    r2 = c2.tune_report()
    assert r2["plans_from_cache"] == 1 and r2["candidates_timed"] == 0
    for k in ("shifted_x", "shifted_y", "longer_x", "longer_y", "longer_z", "z_variant"):
        assert r2[k] == r1[k], k
    assert rel_linf(got2, ref) < TOL[prec]
    c2.close()


def test_batch_branch_count_tuned_once_per_shape(oracle, tmp_path):
    path = str(tmp_path / "tune.txt")
    probs = [li.random_sparse(40 + k, b=8, nsrc=3, ntgt=4 + k, extent=(4, 3, 2), ncomp=2) for k in range(5)]
    c = _fresh("f32")
    c.autotune(lgf.LGF_TUNE_ON, path)
    batch = []
    for p in probs:
        f = torch.tensor(p.f.reshape(-1), dtype=torch.float32, device="cuda")
        u = torch.full((p.ncomp * p.tgt.shape[0] * p.b ** 3,), float("nan"), device="cuda")
        batch.append(dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=u, ncomp=p.ncomp, op=lgf.LGF_OP_POISSON))
    s = torch.cuda.Stream()
    for _ in range(2):
        with torch.cuda.stream(s):
            c.batch_apply(batch, stream=s)
        s.synchronize()
    r = c.tune_report()
    assert r["batches_tuned"] == 1 and r["last_branches"] in (1, 2, 4, 8) and r["plans_tuned"] == len(probs)
    assert any(l.startswith("B f32 ") for l in open(path).read().splitlines())
    for p, q in zip(probs, batch):
        assert rel_linf(q["u"].cpu().numpy().reshape(p.ncomp, -1), _oracle(oracle, p)) < TOL["f32"]
    c.close()


@pytest.mark.parametrize("mode", ["rg4", "nb2"])
def test_batch_execution_read_back_from_file(mode, oracle, tmp_path):
    """A batch shape's persisted execution (the ragged mode on 4 branches, or
    per-problem launches on 2) is taken from the file by a new context, which
    times nothing, reports the mode and matches the oracle."""
    path = tmp_path / "tune.txt"
    probs = [li.random_sparse(60 + k, b=8, nsrc=2, ntgt=3 + k, extent=(3, 3, 2), ncomp=1) for k in range(4)]

    def run(ctx):
        batch = []
        for p in probs:
            f = torch.tensor(p.f.reshape(-1), dtype=torch.float32, device="cuda")
            u = torch.full((p.tgt.shape[0] * p.b ** 3,), float("nan"), device="cuda")
            batch.append(dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=u, ncomp=1, op=lgf.LGF_OP_POISSON))
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            ctx.batch_apply(batch, stream=s)
        s.synchronize()
        return batch

    # a tuned context writes the batch key; its value is then replaced by `mode`
    c1 = _fresh("f32")
    c1.autotune(lgf.LGF_TUNE_ON, str(path))
    run(c1)
    c1.close()
    lines = path.read_text().splitlines()
    key = next(l.split(" -> ")[0] for l in lines if l.startswith("B f32 "))
    path.write_text("\n".join(lines) + f"\n{key} -> {mode}\n")
    c2 = _fresh("f32")
    c2.autotune(lgf.LGF_TUNE_CACHED, str(path))
    batch = run(c2)
    r = c2.tune_report()
    assert r["candidates_timed"] == 0 and r["batches_tuned"] == 0
    assert r["last_ragged"] == (mode == "rg4") and r["last_branches"] == int(mode[2:])
    for p, q in zip(probs, batch):
        assert rel_linf(q["u"].cpu().numpy(), _oracle(oracle, p).reshape(-1)) < TOL["f32"]
    c2.close()
