#!/usr/bin/env python
"""Benchmark of the LGF Poisson apply (+ integrating factors) on one GB300.

Workload (default "dense128"): the dense 128^3 lattice box of Liska &
Colonius-style smooth sources (8 Gaussian blobs, sigma = 6 cells, seed 1), FP32,
32^3 blocks.  One step = one lgf_batch_apply call (one CUDA graph) holding the
whole hot path for that input: the G_L Poisson apply u = G_L * f and the
integrating factors E(0.05) f, E(0.5) f, E(2.0) f.  The metric counts the
Poisson apply's active target lattice points (2,097,152 per step) over the
whole step's time, so the integrating factors only lower the reported value.
The kernel spectra and the G_L table are pre-processing (built before timing,
once per simulation as in App. A).

Timing: W untimed warm-up steps; then K steps, each bracketed by CUDA events
on the launch stream, with a 512 MiB buffer written between steps (L2 flush,
the 8 MiB input is smaller than L2); barrier + synchronize around the timed
region; max over ranks.  Multi-GPU runs (torchrun) of the dense box are
independent replicas (the problem does not shard): value = ranks x points /
max time.  The plate batch (--workload plates64) splits its independent
problems across the ranks instead: value = the batch's points / max time.

Other JSON keys: roofline of the dominant kernel (algorithmic bytes per
launch / CUDA-event launch time, against MEASURED_PEAKS.json), e2e (the same
metric with the host->device copy of f from pinned memory and the
device->host copy of all outputs inside the timed region), cpu_baseline (the
CPU oracle on a bounded sample, with its error against the GPU result) and the
SM clocks sampled during the timed region.

`--impl reference` times the CPU oracle (direct summation) as the reference
arm on the same workload, one bounded sample of target points per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 512 << 20


# ----------------------------------------------------------------------------
# distributed plumbing (replicas; a batch of independent problems is split)
# ----------------------------------------------------------------------------
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def dist_init(world: int, backend: str):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend)
    return dist if world > 1 else None


def reduce_max(value: float, dist) -> float:
    """Largest value over ranks (the slowest replica sets the job time)."""
    if dist is None:
        return value
    import torch
    dev = "cuda" if (torch.cuda.is_available() and dist.get_backend() == "nccl") else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(points_per_step: float, ms_per_step_max: float, world: int) -> float:
    """Whole-job points per second: every replica processes the same work."""
    return world * points_per_step / (ms_per_step_max * 1e-3)


def shard(costs, world: int, rank: int) -> list:
    """Independent problems of a batch split across ranks, longest first onto
    the least loaded rank (ties to the lower index): the indices this rank
    runs.  Every rank computes the same split from the same costs, so no
    collective is needed; the ranks' problem lists are disjoint and cover the
    batch."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    owner = [0] * len(costs)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += costs[i]
    return [i for i in range(len(costs)) if owner[i] == rank]


def poisson_cost(p) -> float:
    """Work estimate of one problem's Poisson part: transform-box volume times
    fields (the batch scheduler's own measure)."""
    M, _, _ = geometry(p)
    return float(M[0]) * M[1] * M[2] * p.nrhs * p.ncomp


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------
ALPHAS = (0.05, 0.5, 2.0)


def make_workload(name: str):
    import lgf_inputs as li
    if name == "dense128":
        p = li.dense_blobs(n=128, b=32, seed=1)
        desc = {"workload": "dense 128^3 box, 8 Gaussian blobs (sigma 6, seed 1), 32^3 blocks, FP32; "
                            "G_L apply + E(0.05), E(0.5), E(2.0) per step",
                "lattice": [128, 128, 128], "block": 32, "blocks": int(p.src.shape[0]), "fields": 1,
                "alphas": list(ALPHAS)}
        return p, desc
    raise ValueError(f"unknown workload {name}")


# transform lengths of the library's plans: 2^k, 3 * 2^k and 5 * 2^k from 32 to 4096
FFT_SIZES = (32, 64, 80, 96, 128, 160, 192, 256, 320, 384, 512, 640, 768, 1024, 1280, 1536, 2048, 2560, 3072, 4096)


def geometry(p):
    """Transform-box geometry of the Poisson plan (mirrors the library's plan)."""
    b = p.b
    allc = np.concatenate([p.src, p.tgt])
    lo, hi = allc.min(0), allc.max(0)
    L = (hi - lo + 1) * b
    M = [next(m for m in FFT_SIZES if m >= 2 * l - 1) for l in L]
    Ls = [int(v) for v in (p.src.max(0) - p.src.min(0) + 1) * b]
    Lt = [int(v) for v in (p.tgt.max(0) - p.tgt.min(0) + 1) * b]
    return [int(m) for m in M], Ls, Lt


def algorithmic_bytes_per_step(p, nfields: int, n_intf: int) -> dict:
    """Compulsory bytes per step of each kernel (FP32): every input element
    read once, every output element written once.  n_intf integrating factors
    on the dense box share each pass's launches (grouped jobs)."""
    M, Ls, Lt = geometry(p)
    K = M[0] // 2 + 1
    c8 = 8  # complex64
    b3 = p.b ** 3
    nsrc, ntgt = int(p.src.shape[0]), int(p.tgt.shape[0])
    spec = (M[2] // 2 + 1) * (M[1] // 2 + 1) * K * 4
    by = {
        "poisson_x_forward": nfields * (nsrc * b3 * 4 + Ls[2] * Ls[1] * K * c8),
        "poisson_y_forward": nfields * (Ls[2] * Ls[1] * K * c8 + Ls[2] * M[1] * K * c8),
        "poisson_z_convolve": nfields * (Ls[2] * M[1] * K * c8 + Lt[2] * M[1] * K * c8) + spec,
        "poisson_y_inverse": nfields * (Lt[2] * M[1] * K * c8 + Lt[2] * Lt[1] * K * c8),
        "poisson_x_inverse": nfields * (Lt[2] * Lt[1] * K * c8 + ntgt * b3 * 4),
    }
    # integrating-factor passes on a dense box: every pass reads and writes the box once per apply
    for ax in ("x", "y", "z", "xy"):
        by[f"intfactor_pass_{ax}"] = n_intf * nfields * 2 * ntgt * b3 * 4
    return by


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1604_01814_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh")):
            h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    k = d.get("kernels", {}).get(kernel)
    return None if k is None else float(k["dram_bytes_per_launch"])


def measured_peaks():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ----------------------------------------------------------------------------
def oracle_sample(p, npts: int, seed: int = 101):
    from oracle import oracle
    rng = np.random.default_rng(seed)
    ntot = p.tgt.shape[0] * p.b ** 3
    idx = np.sort(rng.choice(ntot, size=npts, replace=False))
    pts = oracle.block_points(p.b, p.tgt)[idx]
    oracle.lgf_table(64)   # table build is pre-processing, outside the timing
    t0 = time.perf_counter()
    ref = oracle.poisson_direct(p.b, p.src, p.f[0, 0], pts, R=64)
    dt = time.perf_counter() - t0
    return idx, ref, dt, oracle.num_threads()


def run_reference(args, rank, world):
    if rank != 0:
        return None
    p, desc = make_workload(args.workload)
    npts = args.ref_points
    times = []
    for k in range(args.warmup + args.steps):
        _, _, dt, cores = oracle_sample(p, npts, seed=1000 + k)
        if k >= args.warmup:
            times.append(dt)
    ms = 1e3 * float(np.mean(times))
    value = npts / (ms * 1e-3)
    sample = f"{npts} random target points of the Poisson apply per step (direct summation over all sources)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": desc,
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


METRIC = "active lattice points/sec for LGF Poisson apply at rel err 1e-5; % HBM roofline"


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def run_ours(args, rank, world, dist):
    import torch
    import paper_1604_01814_gb300 as lgf

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    p, desc = make_workload(args.workload)
    ctx = lgf.Context("f32", device=dev.index)
    ctx.table_build(48)
    f_host = torch.tensor(p.f.reshape(-1), dtype=torch.float32).pin_memory()
    f = f_host.to(dev)
    n_out = p.tgt.shape[0] * p.b ** 3
    u = torch.empty(n_out, dtype=torch.float32, device=dev)
    vs = [torch.empty(n_out, dtype=torch.float32, device=dev) for _ in ALPHAS]
    batch = [dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=u, op=lgf.LGF_OP_POISSON, dx=1.0)]
    batch += [dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=v, op=lgf.LGF_OP_INTFACTOR, alpha=a)
              for a, v in zip(ALPHAS, vs)]
    s = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    points = float(n_out)   # Poisson target points per step (one field)

    with torch.cuda.stream(s):
        for _ in range(max(3, args.warmup)):
            ctx.batch_apply(batch, stream=s)
    s.synchronize()

    # ---- timed region (device time, CUDA events on the launch stream) ----
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(dev.index)
    clk.start()
    time.sleep(0.3)
    with torch.cuda.stream(s):
        for a, b in evs:
            flush.zero_()
            a.record(s)
            ctx.batch_apply(batch, stream=s)
            b.record(s)
    s.synchronize()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop()
    ms_local = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    ms = reduce_max(ms_local, dist)
    value = job_throughput(points, ms, world)

    # ---- per-kernel times (events around every launch, direct launches) ----
    ctx.profile_enable(True)
    with torch.cuda.stream(s):
        for _ in range(args.steps):
            flush.zero_()
            ctx.batch_apply(batch, stream=s)
    stats = ctx.profile_read()
    ctx.profile_enable(False)
    launches_per_step = sum(n for n, _ in stats.values()) / args.steps
    alg_step = algorithmic_bytes_per_step(p, 1, len(ALPHAS))
    # bytes per launch = bytes per step / launches per step
    alg = {k: alg_step[k] * args.steps / n for k, (n, _) in stats.items() if k in alg_step}
    dom = max(stats, key=lambda k: stats[k][1])
    dom_ms = stats[dom][1] / stats[dom][0]
    peak, peak_kind = measured_peaks()
    achieved = alg[dom] / (dom_ms * 1e-3) / 1e9
    kernels = {k: {"launches_per_step": n / args.steps, "ms_per_launch": t / n,
                   "share": t / sum(v[1] for v in stats.values()),
                   "alg_bytes_per_launch": int(alg[k]) if k in alg else None,
                   "alg_GBps": (alg[k] / (t / n * 1e-3) / 1e9) if k in alg else None}
               for k, (n, t) in stats.items()}

    # ---- end to end: pinned host input -> apply -> outputs back to host ----
    # A streaming pipeline with two device buffer sets: the host->device copy
    # of step k+1 and the device->host copy of step k-1 run on their own
    # streams while step k computes.  Every step still copies its whole input
    # from pinned host memory and all four output fields back to pinned host
    # memory; the time is first copy-in start to last copy-out end over K steps.
    n_out_fields = 1 + len(ALPHAS)
    sets = []
    for j in range(2):
        fj = torch.empty_like(f)
        oj = [torch.empty(n_out, dtype=torch.float32, device=dev) for _ in range(n_out_fields)]
        bj = [dict(b=p.b, src=p.src, tgt=p.tgt, f=fj, u=oj[0], op=lgf.LGF_OP_POISSON, dx=1.0)]
        bj += [dict(b=p.b, src=p.src, tgt=p.tgt, f=fj, u=o, op=lgf.LGF_OP_INTFACTOR, alpha=a)
               for a, o in zip(ALPHAS, oj[1:])]
        hj = [torch.empty(n_out, dtype=torch.float32).pin_memory() for _ in range(n_out_fields)]
        sets.append((fj, oj, bj, hj))
    s_in = torch.cuda.Stream(device=dev)
    s_out = torch.cuda.Stream(device=dev)

    def pipeline(nsteps, t0=None, t1=None):
        comp = [torch.cuda.Event() for _ in range(nsteps)]
        d2h = [torch.cuda.Event() for _ in range(nsteps)]
        if t0 is not None:
            t0.record(s_in)
        for k in range(nsteps):
            fj, oj, bj, hj = sets[k % 2]
            if k >= 2:
                s_in.wait_event(comp[k - 2])          # step k-2 no longer reads f_j
            with torch.cuda.stream(s_in):
                fj.copy_(f_host, non_blocking=True)
            h2d = torch.cuda.Event()
            h2d.record(s_in)
            s.wait_event(h2d)
            if k >= 2:
                s.wait_event(d2h[k - 2])              # step k-2's outputs are on the host
            ctx.batch_apply(bj, stream=s)
            comp[k].record(s)
            s_out.wait_event(comp[k])
            with torch.cuda.stream(s_out):
                for o, d in zip(hj, oj):
                    o.copy_(d, non_blocking=True)
            d2h[k].record(s_out)
        if t1 is not None:
            t1.record(s_out)
        torch.cuda.synchronize()

    pipeline(4)                                        # warm-up (captures both graphs)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    pipeline(args.steps, e0, e1)
    e2e_ms = reduce_max(e0.elapsed_time(e1) / args.steps, dist)
    e2e = {"value": job_throughput(points, e2e_ms, world), "unit": "points/s",
           "h2d_bytes_per_step": int(f.numel() * 4), "d2h_bytes_per_step": int(n_out * 4 * n_out_fields),
           "ms_per_step": e2e_ms,
           "how": "two buffer sets; copy-in of step k+1 and copy-out of step k-1 overlap step k; "
                  "no L2 flush (every input is re-copied from the host)"}
    # the end-to-end results must be the device-timed results
    for o, d in zip(sets[(args.steps - 1) % 2][3], [u] + vs):
        assert torch.equal(o, d.cpu()), "end-to-end output differs from the device-timed output"

    # ---- the plain FP64 single-problem form on the same GPU ----
    # Separate lgf_poisson_apply / lgf_intfactor_apply calls in an FP64 context
    # (no batch, no graph, no concurrent branch), timed like the main loop.
    fp64 = None
    if not args.no_fp64:
        ctx64 = lgf.Context("f64", device=dev.index)
        ctx64.table_build(48)
        f64 = f.double()
        u64 = torch.empty(n_out, dtype=torch.float64, device=dev)
        v64 = [torch.empty_like(u64) for _ in ALPHAS]

        def plain64():
            ctx64.poisson_apply(p.b, p.src, p.tgt, f64, u64, stream=s)
            for a, v in zip(ALPHAS, v64):
                ctx64.intfactor_apply(a, p.b, p.src, p.tgt, f64, v, stream=s)

        with torch.cuda.stream(s):
            for _ in range(3):
                plain64()
        s.synchronize()
        ev64 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
        with torch.cuda.stream(s):
            for a, b in ev64:
                flush.zero_()
                a.record(s)
                plain64()
                b.record(s)
        s.synchronize()
        ms64 = reduce_max(float(np.mean([a.elapsed_time(b) for a, b in ev64])), dist)
        errs = [float((x.double() - y).abs().max() / y.abs().max()) for x, y in zip([u] + vs, [u64] + v64)]
        fp64 = {"ms_per_step": ms64, "value": job_throughput(points, ms64, world), "unit": "points/s",
                "speedup_of_fp32_batched": ms64 / ms, "fp32_vs_fp64_rel_err": max(errs),
                "how": "FP64 context, one lgf_poisson_apply and three lgf_intfactor_apply calls per step "
                       "(tol 1e-13), no batch or graph; the FP32 batched outputs agree with it to "
                       "fp32_vs_fp64_rel_err (both within the 1e-5 bar)"}
        ctx64.close()

    line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(desc, l2="flushed between timed steps (512 MiB write); input 8 MiB < L2",
                           parallelism="replicas" if world > 1 else "single GPU",
                           kernels=kernels),
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "alg_bytes_per_launch": int(alg[dom]), "ms_per_launch": dom_ms,
                         "traffic": load_traffic(dom)},
            "e2e": e2e, "gpu_launches": int(round(launches_per_step * args.steps)),
            "clocks": clocks}
    if fp64 is not None:
        line["fp64_plain"] = fp64
    # ---- CPU baseline: the oracle on a bounded sample, and the GPU error there ----
    if rank == 0 and not args.no_cpu:
        idx, ref, dt, cores = oracle_sample(p, args.cpu_points)
        got = u.cpu().numpy().astype(np.float64)[idx]
        err = float(np.abs(got - ref).max() / np.abs(ref).max())
        line["cpu_baseline"] = {"value": args.cpu_points / dt, "unit": "points/s", "cores": cores, "kind": "oracle",
                                "sample": f"{args.cpu_points} random target points of the Poisson apply "
                                          f"(direct summation over all 2^21 sources), {dt:.1f} s"}
        line["rel_err_vs_oracle"] = err
    ctx.close()
    return line


def run_ncu_case(args):
    """The bench step (one lgf_batch_apply on the legacy stream) run `--steps`
    times untimed: the small, short case that ncu captures."""
    import torch
    import lgf_inputs as li
    import paper_1604_01814_gb300 as lgf
    ctx = lgf.Context("f32")
    ctx.table_build(48)
    if args.workload == "wake512":
        # one right-hand side (3 fields, about 3 GB on the device): the wake
        # domain's transform shape at a size a full capture handles
        p = li.wake_domain(nrhs=1)
        f = torch.tensor(p.f.reshape(-1), dtype=torch.float32, device="cuda")
        outs = [torch.empty(f.numel(), dtype=torch.float32, device="cuda")]
        batch = [dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=outs[0], ncomp=3, nrhs=1, op=lgf.LGF_OP_POISSON)]
    else:
        p, _ = make_workload(args.workload)
        f = torch.tensor(p.f.reshape(-1), dtype=torch.float32, device="cuda")
        outs = [torch.empty_like(f) for _ in range(1 + len(ALPHAS))]
        batch = [dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=outs[0], op=lgf.LGF_OP_POISSON)]
        batch += [dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=o, op=lgf.LGF_OP_INTFACTOR, alpha=a)
                  for a, o in zip(ALPHAS, outs[1:])]
    for _ in range(args.steps):
        ctx.batch_apply(batch, stream=0)
    torch.cuda.synchronize()
    print("ncu case done:", [float(o.abs().max()) for o in outs], flush=True)
    ctx.close()


EXTRA = {
    "wake512": "512x256x256 wake domain, 32^3 blocks (384 active), curl-of-blobs source, 3 components x 4 "
               "RK right-hand sides (12 fields), FP32; one G_L apply of all fields per step",
    "plates64": "64 flat-plate problems, 16^3 blocks, N_b log-uniform in [8, 1200], 3 components, FP32; "
                "one lgf_batch_apply of G_L then E(0.25) for every problem per step",
    "refresh_sphere": "velocity refresh u <- -C^dagger L^{-1} C u (Eq. vel_refresh) on the sphere-plus-wake "
                      "active set (16^3 blocks), u = curl of a Gaussian-blob vector potential, FP32; one refresh "
                      "per step",
    "ib_sphere": "immersed-boundary regularisation R then interpolation I (Sec. 2.1) of 5120 icosphere markers "
                 "(radius 20 cells) on the 32 blocks of 16^3 their three-point support touches, 3 components, "
                 "FP32; throughput in marker-components per second",
    "kinv_sphere": "K(0.25)^{-1} on the surface blocks of the icosphere (5120 markers, radius 20 cells, 16^3 "
                   "blocks, source = target = the blocks the 3-point delta touches), 3 components, FP32; one "
                   "G_K(0.25) apply per step",
}


def run_extra(args, rank, world, dist):
    """The larger paper-shaped workloads (working sets far above L2) and the
    rows beyond the Poisson/integrating-factor path: their own JSON line with
    throughput and per-kernel algorithmic GB/s.  Not the bench line: the bench
    workload is the dense 128^3 box."""
    import torch
    import lgf_inputs as li
    import paper_1604_01814_gb300 as lgf

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    probs = []
    if args.workload == "wake512":
        probs = [(li.wake_domain(), lgf.LGF_OP_POISSON, 0.0)]
    elif args.workload == "plates64":
        probs = [(q, lgf.LGF_OP_POISSON_THEN_INTFACTOR, 0.25) for q in li.plate_batch()]
        points_all = float(sum(q.nrhs * q.ncomp * q.tgt.shape[0] * q.b ** 3 for q, _, _ in probs))
        if world > 1:   # independent problems: each rank runs its share, no data-path collective
            probs = [probs[i] for i in shard([poisson_cost(q) for q, _, _ in probs], world, rank)]
    elif args.workload == "kinv_sphere":
        q = li.sphere_ib()
        q = li.Problem("sphere_surface", q.b, q.src, q.src.copy(), q.f, alphas=(0.25,))
        probs = [(q, lgf.LGF_OP_KINV, 0.25)]
    elif args.workload not in ("refresh_sphere", "ib_sphere"):
        raise ValueError(f"unknown workload {args.workload}")
    ctx = lgf.Context("f32", device=dev.index)
    ctx.table_build(48)
    batch, points = [], 0.0
    alg_step = {}
    s = torch.cuda.Stream(device=dev)
    if args.workload == "refresh_sphere":
        q = li.sphere_ib()
        cells = q.tgt
        u = li.curl_blob_field(q.b, cells, centres=np.array([[-30.0, 0.0, 0.0], [40.0, 10.0, -5.0]]),
                               amps=np.array([[0.0, 0.0, 1.0], [0.5, -1.0, 0.0]]), sigma=8.0)
        ut = torch.tensor(u.reshape(-1), dtype=torch.float32, device=dev)
        uo = torch.empty_like(ut)
        ncell = cells.shape[0] * q.b ** 3
        points = float(3 * ncell)
        # the Poisson part maps the cells to the cells and their +x, +y, +z neighbour blocks
        grown = set(map(tuple, cells.tolist()))
        for e in np.eye(3, dtype=np.int64):
            grown |= set(map(tuple, (cells + e).tolist()))
        grown = np.array(sorted(grown), dtype=np.int32)
        pg = li.Problem("refresh", q.b, cells, grown, np.zeros((1, 3, cells.shape[0], 1)))
        alg_step = algorithmic_bytes_per_step(pg, 3, 0)
        alg_step["curl"] = 2 * 3 * 4 * ncell
        alg_step["curl_adjoint"] = 2 * 3 * 4 * ncell

        def step():
            ctx.velocity_refresh(q.b, cells, cells, ut, uo, stream=s)
    elif args.workload == "ib_sphere":
        q = li.sphere_ib()
        Xm = torch.tensor(li.icosphere_markers(5) * 20.0, dtype=torch.float64, device=dev)   # as in sphere_ib
        nm = Xm.shape[0]
        gm = torch.tensor(np.random.default_rng(2).normal(size=3 * nm), dtype=torch.float32, device=dev)
        fm = torch.empty(3 * q.src.shape[0] * q.b ** 3, dtype=torch.float32, device=dev)
        Um = torch.empty_like(gm)
        points = float(3 * nm)
        # marker values and positions read, the field written (spread) or the 27 support values read (interp)
        alg_step = {"ib_spread": 4 * 3 * nm + 24 * nm + 4 * fm.numel(), "ib_interp": 4 * 3 * nm * 28 + 24 * nm}

        def step():
            ctx.ib_spread(q.b, q.src, Xm, gm, fm, stream=s)
            ctx.ib_interp(q.b, q.src, Xm, fm, Um, stream=s)
    else:
        for p, op, a in probs:
            nf = p.nrhs * p.ncomp
            f = torch.tensor(p.f.reshape(-1), dtype=torch.float32, device=dev)
            u = torch.empty(nf * p.tgt.shape[0] * p.b ** 3, dtype=torch.float32, device=dev)
            batch.append(dict(b=p.b, src=p.src, tgt=p.tgt, f=f, u=u, ncomp=p.ncomp, nrhs=p.nrhs, op=op, alpha=a))
            points += float(u.numel())
            n_intf = 1 if op in (lgf.LGF_OP_INTFACTOR, lgf.LGF_OP_POISSON_THEN_INTFACTOR) else 0
            for k, v in algorithmic_bytes_per_step(p, nf, n_intf).items():
                alg_step[k] = alg_step.get(k, 0) + v

        def step():
            ctx.batch_apply(batch, stream=s)
    with torch.cuda.stream(s):
        for _ in range(max(3, args.warmup)):
            step()
    s.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(dev.index)
    clk.start()
    with torch.cuda.stream(s):
        for a, b in evs:
            a.record(s)
            step()
            b.record(s)
    s.synchronize()
    clocks = clk.stop()
    ms = reduce_max(float(np.mean([a.elapsed_time(b) for a, b in evs])), dist)
    ctx.profile_enable(True)
    with torch.cuda.stream(s):
        for _ in range(args.steps):
            step()
    stats = ctx.profile_read()
    ctx.profile_enable(False)
    tot = sum(t for _, t in stats.values())
    kernels = {}
    for k, (n, t) in stats.items():
        per_launch = alg_step.get(k, 0) * args.steps / n if k in alg_step else None
        kernels[k] = {"launches_per_step": n / args.steps, "ms_per_launch": t / n, "share": t / tot,
                      "alg_GBps": per_launch / (t / n * 1e-3) / 1e9 if per_launch else None}
    peak, peak_kind = measured_peaks()
    dom = max(stats, key=lambda k: stats[k][1]) if stats else None   # (a rank may hold no problem)
    sharded = args.workload == "plates64" and world > 1
    value = points_all / (ms * 1e-3) if sharded else job_throughput(points, ms, world)
    line = {"workload": args.workload, "config": EXTRA[args.workload], "metric": METRIC,
            "value": value, "unit": "points/s", "ms_per_step": ms,
            "points_per_step": points_all if sharded else points, "steps": args.steps, "n_gpus": world,
            "dtype": "f32",
            "parallelism": ("problems sharded across ranks, longest first" if sharded else
                            "replicas" if world > 1 else "single GPU"),
            "scaling": "strong" if sharded else "weak",
            "l2": "no flush: the working set of every pass exceeds the 129 MB L2",
            "kernels": kernels, "dominant": dom,
            "dominant_hbm_frac": (kernels[dom]["alg_GBps"] / peak) if dom and kernels[dom]["alg_GBps"] else None,
            "peak_GBps": peak, "peak_kind": peak_kind, "clocks": clocks,
            "note": "integrating-factor bytes counted as read + write of the target set per pass"}
    ctx.close()
    return line


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dense128")
    ap.add_argument("--cpu-points", type=int, default=3072)
    ap.add_argument("--ref-points", type=int, default=1024)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--ncu-case", action="store_true", help="run the step --steps times untimed (for ncu)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, _ = dist_env()
    if args.ncu_case:
        run_ncu_case(args)
        return
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        import torch
        dist = dist_init(world, "nccl" if torch.cuda.is_available() else "gloo")
        if args.workload in EXTRA:
            line = run_extra(args, rank, world, dist)
        else:
            line = run_ours(args, rank, world, dist)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
