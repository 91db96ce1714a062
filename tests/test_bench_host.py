"""Host-side logic of bench.py on the CPU: the multi-rank timing reduction
(gloo, world size 2), the split of a batch's problems across ranks, the
reference arm's JSON line and the clock parsing."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist = bench.dist_init(world, "gloo")
    local_ms = 1.0 + rank            # rank 1 is the slowest replica
    ms = bench.reduce_max(local_ms, dist)
    dist.barrier()
    q.put((rank, ms, bench.job_throughput(1000.0, ms, world)))
    dist.destroy_process_group()


def test_two_rank_timing_uses_the_slowest_replica():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == 2.0                                   # max over ranks
        assert value == pytest.approx(2 * 1000.0 / 2e-3)  # whole-job points / s


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_init(1, "gloo") is None
    assert bench.reduce_max(3.5, None) == 3.5
    assert bench.job_throughput(2e6, 1.0, 1) == pytest.approx(2e9)


def test_clock_sampler_parses_reasons():
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)

    class P:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c.proc = P()
    c.lines = ["1965, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Active",
               "2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage"]
    r = c.stop()
    assert r["sm_mhz"] == pytest.approx(2017.5) and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]


def test_reference_arm_prints_one_json_line():
    env = dict(os.environ, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--ref-points", "4"], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "points/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["metric"].startswith("active lattice points/sec")


def test_reference_arm_other_ranks_do_no_work():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        workload, ref_points, warmup, steps = "dense128", 4, 3, 1

    assert bench.run_reference(A, rank=1, world=2) is None


def _plate_like_costs(n=64, seed=3):
    """Poisson costs shaped like the plate batch: block counts log-uniform in
    [8, 1200], transform volume of a box twice the blocks' extent."""
    import numpy as np
    rng = np.random.default_rng(seed)
    nb = np.exp(rng.uniform(np.log(8), np.log(1200), size=n))
    return [float(v) for v in 3 * (2 * 16 * np.cbrt(nb)) ** 3]


def test_shard_covers_the_batch_once_and_balances():
    sys.path.insert(0, ROOT)
    import bench
    costs = _plate_like_costs()
    assert bench.shard(costs, 1, 0) == list(range(len(costs)))
    for world in (2, 3, 4, 8):
        parts = [bench.shard(costs, world, r) for r in range(world)]
        assert sorted(i for p in parts for i in p) == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) <= sum(costs) / world + max(costs)     # the longest-first greedy bound
        assert max(loads) < 1.05 * sum(costs) / world            # and close to even on this batch


def _shard_rank(rank, world, port, costs, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist = bench.dist_init(world, "gloo")
    mine = bench.shard(costs, world, rank)
    seen = [None] * world
    dist.all_gather_object(seen, mine)      # the test's own check: the split itself needs no exchange
    q.put((rank, mine, seen))
    dist.destroy_process_group()


def test_two_ranks_split_the_batch_alike():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    costs = _plate_like_costs()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, mine0, seen0), (r1, mine1, seen1) = out
    assert seen0 == seen1 == [mine0, mine1]
    assert not set(mine0) & set(mine1)
    assert sorted(mine0 + mine1) == list(range(len(costs)))
