#!/usr/bin/env python
"""Benchmark of the LGF Poisson apply (+ integrating factor) on one GB300.

Workload (default "plates64"): 64 independent block-adaptive flat-plate
problems (16^3 blocks, active block counts log-uniform in [8, 1200], 3
components, FP32, seed 3), the batched form of Liska & Colonius's plate runs.
One step = one lgf_batch_apply call (one CUDA graph) that applies G_L and then
E(0.25) to every problem.  The metric counts the Poisson apply's active
target points (target lattice point x component) of all 64 problems over the
whole step's time, so the integrating factors only lower the reported value.
Kernel spectra and the G_L table are pre-processing (built before timing, once
per simulation as in App. A).  Other workloads: dense128 (the 128^3 box of
Gaussian blobs, G_L + three E(alpha)), wake512 (512x256x256 wake domain, 12
fields), and the extra lines of EXTRA.

Timing: W untimed warm-up steps and a >= 1 s untimed soak with the clock
sampler running; then K steps, each bracketed by CUDA events on the launch
stream; barrier + synchronize around the timed region; max over ranks.  The
plate batch's working set exceeds L2, so no flush is needed; dense128 writes
a 512 MiB buffer between steps.  Under torchrun the plate batch's problems are
split across ranks (longest first; value = the batch's points / the slowest
rank's time); other workloads run as replicas.

Other JSON keys: roofline of the Poisson apply (8 B per target point over the
summed time of its five pass kernels, against MEASURED_PEAKS.json; with the
ncu DRAM bytes of those kernels when profiles/ holds a capture of the current
sources), roofline_step (8 B per point of every apply over the step time),
roofline_dominant_kernel, e2e (host->device copies of every input and
device->host copies of every output inside the timed region), cpu_baseline
(the CPU oracle on a bounded sample), rel_err_vs_oracle, fp64_plain (the FP64
single-problem form at the same truncation tolerance), clocks.

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
# workloads: one step = one lgf_batch_apply
# ----------------------------------------------------------------------------
METRIC = "active lattice points/sec for LGF Poisson apply at rel err 1e-5; % HBM roofline"
DENSE_ALPHAS = (0.05, 0.5, 2.0)
PLATE_ALPHA = 0.25


class Workload:
    """The batch of one step.  entries: dicts (p=Problem, op, alpha); several
    entries may share one source field (same `fkey`)."""

    def __init__(self, name, entries, desc):
        self.name = name
        self.entries = entries
        self.desc = desc

    @property
    def poisson_entries(self):
        return [e for e in self.entries if e["op"] in (0, 2, 3)]

    def points(self):
        """Poisson target points per step (one point = target lattice point x
        component x right-hand side)."""
        return float(sum(e["p"].tgt.shape[0] * e["p"].b ** 3 * e["p"].ncomp * e["p"].nrhs
                         for e in self.poisson_entries))

    def intf_points(self):
        return float(sum(e["p"].tgt.shape[0] * e["p"].b ** 3 * e["p"].ncomp * e["p"].nrhs
                         for e in self.entries if e["op"] in (1, 2)))


def make_workload(name: str) -> Workload:
    import lgf_inputs as li
    if name == "plates64":
        probs = li.plate_batch()
        ents = [dict(p=q, op=2, alpha=PLATE_ALPHA, fkey=i) for i, q in enumerate(probs)]
        desc = {"workload": "64 independent flat-plate problems (16^3 blocks, N_b log-uniform in [8, 1200], "
                            "AR 1/2/4, 30 deg, seed 3), 3 components, FP32; one lgf_batch_apply of G_L then "
                            "E(0.25) for every problem per step (one CUDA graph)",
                "problems": 64, "block": 16, "fields_per_problem": 3,
                "target_blocks": int(sum(q.tgt.shape[0] for q in probs)),
                "source_blocks": int(sum(q.src.shape[0] for q in probs)), "alpha": PLATE_ALPHA}
        return Workload(name, ents, desc)
    if name == "dense128":
        p = li.dense_blobs(n=128, b=32, seed=1)
        ents = [dict(p=p, op=0, alpha=0.0, fkey=0)] + [dict(p=p, op=1, alpha=a, fkey=0) for a in DENSE_ALPHAS]
        desc = {"workload": "dense 128^3 box, 8 Gaussian blobs (sigma 6, seed 1), 32^3 blocks, FP32; "
                            "G_L apply + E(0.05), E(0.5), E(2.0) per step",
                "lattice": [128, 128, 128], "block": 32, "blocks": int(p.src.shape[0]), "fields": 1,
                "alphas": list(DENSE_ALPHAS)}
        return Workload(name, ents, desc)
    if name == "sphere":
        p = li.sphere_ib()
        ents = [dict(p=p, op=0, alpha=0.0, fkey=0)]
        desc = {"workload": "block-adaptive sphere: 556 blocks of 16^3 (ball of 4 block radii and a wake cylinder), "
                            "sources spread from 5120 icosphere markers (radius 20 cells, N(0,1) forces, seed 2) on "
                            "the 32 blocks they touch, 3 components, FP32; one G_L apply per step",
                "block": 16, "target_blocks": int(p.tgt.shape[0]), "source_blocks": int(p.src.shape[0]),
                "fields": 3}
        return Workload(name, ents, desc)
    if name == "wake512":
        p = li.wake_domain()
        ents = [dict(p=p, op=0, alpha=0.0, fkey=0)]
        desc = {"workload": "512x256x256 wake domain, 32^3 blocks (384 active), curl-of-blobs source, "
                            "3 components x 4 RK right-hand sides (12 fields), FP32; one G_L apply of all fields "
                            "per step", "lattice": [512, 256, 256], "block": 32, "blocks": int(p.src.shape[0]),
                "fields": 12}
        return Workload(name, ents, desc)
    raise ValueError(f"unknown workload {name}")


# transform lengths of the library's plans: 2^k, 3 * 2^k and 5 * 2^k from 32 to 4096
FFT_SIZES = (32, 64, 80, 96, 128, 160, 192, 256, 320, 384, 512, 640, 768, 1024, 1280, 1536, 2048, 2560, 3072, 4096)


def geometry(p):
    """Transform-box geometry of the Poisson plan (mirrors the library's
    default plan: even embedding, M >= 2L - 1 on the union extent L, except
    along x and y where the shifted window M >= Ls + Lt - 1 is shorter and
    Ls <= M/2)."""
    b = p.b
    allc = np.concatenate([p.src, p.tgt])
    lo, hi = allc.min(0), allc.max(0)
    L = (hi - lo + 1) * b
    nxt = lambda n: next(m for m in FFT_SIZES if m >= n)
    M = [nxt(2 * l - 1) for l in L]
    Ls = [int(v) for v in (p.src.max(0) - p.src.min(0) + 1) * b]
    Lt = [int(v) for v in (p.tgt.max(0) - p.tgt.min(0) + 1) * b]
    for d in (0, 1):
        Ma = nxt(Ls[d] + Lt[d] - 1)
        if Ma < M[d] and 2 * Ls[d] <= Ma:
            M[d] = Ma
    return [int(m) for m in M], Ls, Lt


def pass_io_bytes(p, nfields: int) -> dict:
    """Bytes each Poisson pass reads and writes by this design (FP32): its
    input and output arrays once, intermediates included.  A diagnostic of the
    design, not the algorithmic cost of the apply (8 B per target point)."""
    M, Ls, Lt = geometry(p)
    K = M[0] // 2 + 1
    c8 = 8
    b3 = p.b ** 3
    nsrc, ntgt = int(p.src.shape[0]), int(p.tgt.shape[0])
    spec = (M[2] // 2 + 1) * (M[1] // 2 + 1) * K * 4
    return {
        "poisson_x_forward": nfields * (nsrc * b3 * 4 + Ls[2] * Ls[1] * K * c8),
        "poisson_y_forward": nfields * (Ls[2] * Ls[1] * K * c8 + Ls[2] * M[1] * K * c8),
        "poisson_z_convolve": nfields * (Ls[2] * M[1] * K * c8 + Lt[2] * M[1] * K * c8) + spec,
        "poisson_y_inverse": nfields * (Lt[2] * M[1] * K * c8 + Lt[2] * Lt[1] * K * c8),
        "poisson_x_inverse": nfields * (Lt[2] * Lt[1] * K * c8 + ntgt * b3 * 4),
        # the y and x inverses fused (one cluster per target plane): B in, u out
        "poisson_yx_inverse": nfields * (Lt[2] * M[1] * K * c8 + ntgt * b3 * 4),
    }


def z_pass_flops(p, nfields: int) -> float:
    """FP32 flops of the z pass by the standard 5 N log2 N count per complex
    transform of length N (forward and inverse along z for every (kx, ky)
    column, times the 2-flop real spectral multiply per bin)."""
    M, _, _ = geometry(p)
    K = M[0] // 2 + 1
    cols = K * M[1] * nfields
    return float(cols * (2 * 5 * M[2] * math.log2(M[2]) + 2 * M[2]))


POISSON_PASSES = ("poisson_x_forward", "poisson_y_forward", "poisson_z_convolve", "poisson_y_inverse",
                  "poisson_x_inverse", "poisson_yx_inverse")
INTF_PASSES = ("intfactor_pass_xy", "intfactor_pass_z", "intfactor_pass_x", "intfactor_pass_y")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1604_01814_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(workload: str):
    """DRAM bytes per step of each kernel role from the committed ncu summary
    of this workload, if it was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"ncu_traffic_{workload}.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    return {k: float(v["dram_bytes_per_step"]) for k, v in d.get("kernels", {}).items()}


def measured_peaks():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


# FP32 ALU peak of the z pass's roofline: 152 SMs x 128 FP32 lanes x 2 flops
# (one FMA) x 2.07 GHz, the nominal unit count and maximum SM clock.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


# ----------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ----------------------------------------------------------------------------
def oracle_sample(w: Workload, per_problem: int, seed: int = 101):
    """The oracle's direct sum (single-field form, as it stands) at a bounded
    random sample of Poisson targets: per_problem points of every Poisson
    entry, every field.  Returns (samples, seconds, threads) with samples a
    list of (entry index, field, point indices, values)."""
    from oracle import oracle
    rng = np.random.default_rng(seed)
    oracle.lgf_table(64)   # the table build is pre-processing, outside the timing
    out, dt = [], 0.0
    for k, e in enumerate(w.entries):
        if e["op"] not in (0, 2):
            continue
        p = e["p"]
        ntot = p.tgt.shape[0] * p.b ** 3
        idx = np.sort(rng.choice(ntot, size=min(per_problem, ntot), replace=False))
        pts = oracle.block_points(p.b, p.tgt)[idx]
        for r in range(p.nrhs):
            for c in range(p.ncomp):
                t0 = time.perf_counter()
                ref = oracle.poisson_direct(p.b, p.src, p.f[r, c], pts, R=64)
                dt += time.perf_counter() - t0
                out.append((k, r * p.ncomp + c, idx, ref))
    return out, dt, oracle.num_threads()


REF_SAMPLE = {"plates64": 16, "dense128": 1024, "wake512": 2, "sphere": 256}      # reference arm, per problem and field
CPU_SAMPLE = {"plates64": 768, "dense128": 3072, "wake512": 16, "sphere": 1024}    # cpu_baseline and the error check


def run_reference(args, rank, world):
    if rank != 0:
        return None
    w = make_workload(args.workload)
    per = args.ref_points if args.ref_points > 0 else REF_SAMPLE[args.workload]
    times, npts = [], 0
    for k in range(args.warmup + args.steps):
        samples, dt, cores = oracle_sample(w, per, seed=1000 + k)
        if k >= args.warmup:
            times.append(dt)
            npts = sum(len(s[2]) for s in samples)
    ms = 1e3 * float(np.mean(times))
    value = npts / (ms * 1e-3)
    sample = (f"{per} random Poisson targets per problem and field ({npts} target points per step), direct "
              f"summation over all sources")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": w.desc,
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def build_batch(lgf, w: Workload, dev, dtype, f_of=None, u_of=None, only_poisson=False):
    """Device tensors and the batch list.  f_of / u_of override the tensors."""
    import torch
    fs, batch, outs = {}, [], []
    for k, e in enumerate(w.entries):
        p = e["p"]
        if only_poisson and e["op"] not in (0, 2):
            continue
        if e["fkey"] not in fs:
            fs[e["fkey"]] = (f_of(k) if f_of else
                             torch.tensor(p.f.reshape(-1), dtype=dtype).to(dev))
        n_out = p.nrhs * p.ncomp * p.tgt.shape[0] * p.b ** 3
        u = u_of(k) if u_of else torch.empty(n_out, dtype=dtype, device=dev)
        op = 0 if (only_poisson and e["op"] == 2) else e["op"]
        batch.append(dict(b=p.b, src=p.src, tgt=p.tgt, f=fs[e["fkey"]], u=u, ncomp=p.ncomp, nrhs=p.nrhs,
                          op=op, alpha=e["alpha"], dx=1.0))
        outs.append(u)
    return fs, batch, outs


def timed_steps(step, s, nsteps, flush=None):
    """Per-step CUDA-event times (ms) on stream s."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
    with torch.cuda.stream(s):
        for a, b in evs:
            if flush is not None:
                flush.zero_()
            a.record(s)
            step()
            b.record(s)
    s.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def run_ours(args, rank, world, dist):
    import torch
    import paper_1604_01814_gb300 as lgf

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w = make_workload(args.workload)
    points_all = w.points()
    sharded = w.name == "plates64" and world > 1
    if sharded:   # independent problems: each rank runs its share, no data-path collective
        costs = [float(np.prod(geometry(e["p"])[0])) * e["p"].ncomp * e["p"].nrhs for e in w.entries]
        mine = shard(costs, world, rank)
        w = Workload(w.name, [w.entries[i] for i in mine], w.desc)
    ctx = lgf.Context("f32", device=dev.index)
    ctx.table_build(48)
    # the autotuner picks each plan's geometry and the batch's branch count in
    # the first warm-up step (persisted to $LGF_TUNE_CACHE when set)
    if not args.no_tune:
        ctx.autotune(lgf.LGF_TUNE_ON)
    fs, batch, outs = build_batch(lgf, w, dev, torch.float32)
    s = torch.cuda.Stream(device=dev)
    small = w.name in ("dense128", "sphere")   # working sets that L2 could hold
    l2_note = ("flushed between timed steps (512 MiB write)" if small else
               "not flushed: every step's working set (inputs, intermediates, outputs) exceeds the 129 MB L2")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev) if small else None

    def step():
        ctx.batch_apply(batch, stream=s)

    t_tune = time.perf_counter()
    with torch.cuda.stream(s):
        step()
    s.synchronize()
    t_tune = time.perf_counter() - t_tune
    with torch.cuda.stream(s):
        for _ in range(max(3, args.warmup) - 1):
            step()
    s.synchronize()
    tuning = dict(ctx.tune_report(), first_step_s=t_tune, mode="off" if args.no_tune else "on")

    # ---- soak: >= 1 s of steps with the clock sampler running, untimed ----
    clk = ClockSampler(dev.index)
    clk.start()
    t_end = time.perf_counter() + 1.0
    with torch.cuda.stream(s):
        while time.perf_counter() < t_end:
            step()
            s.synchronize()
    # ---- timed region (device time, CUDA events on the launch stream) ----
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms_steps = timed_steps(step, s, args.steps, flush)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop()
    ms_local = float(np.mean(ms_steps))
    ms = reduce_max(ms_local, dist)
    value = points_all / (ms * 1e-3) if sharded else job_throughput(w.points(), ms, world)

    # ---- per-kernel times (events around every launch, direct launches) ----
    ctx.profile_enable(True)
    nprof = max(3, min(args.steps, 10))
    with torch.cuda.stream(s):
        for _ in range(nprof):
            if flush is not None:
                flush.zero_()
            step()
    stats = ctx.profile_read()
    ctx.profile_enable(False)
    launches_per_step = sum(n for n, _ in stats.values()) / nprof
    tot_ms = sum(t for _, t in stats.values())
    io = {}
    for e in w.entries:
        if e["op"] in (0, 2):
            for k, v in pass_io_bytes(e["p"], e["p"].ncomp * e["p"].nrhs).items():
                io[k] = io.get(k, 0) + v
    kernels = {k: {"launches_per_step": n / nprof, "ms_per_step": t / nprof, "ms_per_launch": t / n,
                   "share": t / tot_ms,
                   "pass_io_GBps": (io[k] / (t / nprof * 1e-3) / 1e9) if k in io else None}
               for k, (n, t) in stats.items()}
    peak, peak_kind = measured_peaks()
    # roofline of the Poisson apply: 8 B per target point
    # (4 B read of f + 4 B write of u, FP32) over the summed time of its five
    # pass kernels per step
    pois_ms = sum(stats[k][1] for k in POISSON_PASSES if k in stats) / nprof
    pois_bytes = 8.0 * w.points()
    traffic = load_traffic(w.name)
    pois_traffic = (sum(traffic.get(k, 0.0) for k in POISSON_PASSES) if traffic else None)
    roofline = {"bound": "hbm", "kernel": "poisson apply (its five pass kernels)",
                "achieved": pois_bytes / (pois_ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                "frac": pois_bytes / (pois_ms * 1e-3) / 1e9 / peak, "peak_kind": peak_kind,
                "traffic": pois_traffic, "alg_bytes_per_step": pois_bytes, "ms_per_step": pois_ms,
                "alg_bytes_per_unit": 8, "unit_def": "target lattice point x component x rhs (FP32)",
                "dram_frac": (pois_traffic / (pois_ms * 1e-3) / 1e9 / peak) if pois_traffic else None}
    step_bytes = 8.0 * (w.points() + w.intf_points())
    roofline_step = {"bound": "hbm", "achieved": step_bytes / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": step_bytes / (ms * 1e-3) / 1e9 / peak,
                     "alg_bytes_per_step": step_bytes,
                     "how": "8 B per target point of every Poisson and integrating-factor apply over the "
                            "step's CUDA-event time"}
    dom = max(stats, key=lambda k: stats[k][1])
    roofline_dom = {"kernel": dom, "share": stats[dom][1] / tot_ms}
    if dom == "poisson_z_convolve":
        fl = sum(z_pass_flops(e["p"], e["p"].ncomp * e["p"].nrhs) for e in w.entries if e["op"] in (0, 2))
        t = stats[dom][1] / nprof * 1e-3
        roofline_dom.update({"bound": "alu", "achieved": fl / t / 1e12, "peak": FP32_PEAK_TFLOPS,
                             "unit": "TFLOP/s", "frac": fl / t / 1e12 / FP32_PEAK_TFLOPS,
                             "how": "5 N log2 N flops per complex transform, forward and inverse per column, "
                                    "against 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"})

    # ---- error against the oracle: the Poisson part of the same step ----
    # (the bench step writes E(0.25) G_L f; the Poisson values are taken from a
    # Poisson-only batch of the same inputs in the same context)
    samples, cpu_dt, cores = (None, None, None)
    rel_err = None
    if rank == 0 and not args.no_cpu:
        per = args.cpu_points if args.cpu_points > 0 else CPU_SAMPLE[w.name]
        samples, cpu_dt, cores = oracle_sample(w, per)
        fsp, bp, outp = build_batch(lgf, w, dev, torch.float32, f_of=None, only_poisson=True)
        with torch.cuda.stream(s):
            ctx.batch_apply(bp, stream=s)
        s.synchronize()
        pois_idx = [k for k, e in enumerate(w.entries) if e["op"] in (0, 2)]
        errs = []
        for k, fld, idx, ref in samples:
            p = w.entries[k]["p"]
            got = outp[pois_idx.index(k)].view(p.nrhs * p.ncomp, -1)[fld].cpu().numpy().astype(np.float64)[idx]
            errs.append((np.abs(got - ref).max(), np.abs(ref).max()))
        # per field: max |err| over its samples / max |ref| over its samples
        rel_err = float(max(a / b for a, b in errs if b > 0))
        # the library's own a-posteriori estimate (FP64 direct sums on the GPU)
        lib_est = 0.0
        for e, q in zip([e for e in w.entries if e["op"] in (0, 2)], bp):
            p = e["p"]
            lib_est = max(lib_est, ctx.poisson_error_estimate(p.b, p.src, p.tgt, q["f"], q["u"], ncomp=p.ncomp,
                                                              nrhs=p.nrhs, nsample=16))
        del fsp, bp, outp
        npts = sum(len(x[2]) for x in samples)

    # ---- end to end: pinned host inputs -> apply -> all outputs to host ----
    # Two device buffer sets; the host->device copy of step k+1 and the
    # device->host copy of step k-1 run on their own streams while step k
    # computes.  Every step copies every problem's input from pinned host
    # memory and every output field back to pinned host memory.
    host_f = {}
    for e in w.entries:
        if e["fkey"] not in host_f:
            host_f[e["fkey"]] = torch.tensor(e["p"].f.reshape(-1), dtype=torch.float32).pin_memory()
    sets = []
    for j in range(2):
        fj, bj, oj = build_batch(lgf, w, dev, torch.float32)
        hj = [torch.empty(o.numel(), dtype=torch.float32).pin_memory() for o in oj]
        sets.append((fj, oj, bj, hj))
    h2d_bytes = int(sum(t.numel() * 4 for t in host_f.values()))
    d2h_bytes = int(sum(o.numel() * 4 for o in outs))
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
                for key, t in fj.items():
                    t.copy_(host_f[key], non_blocking=True)
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
    e2e = {"value": (points_all / (e2e_ms * 1e-3) if sharded else job_throughput(w.points(), e2e_ms, world)),
           "unit": "points/s", "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": d2h_bytes,
           "ms_per_step": e2e_ms,
           "how": "two buffer sets; copy-in of step k+1 and copy-out of step k-1 overlap step k; "
                  "every input re-copied from pinned host memory and every output copied back each step"}
    # the end-to-end results must be the device-timed results
    last = sets[(args.steps - 1) % 2][3]
    for o, d in zip(last, outs):
        assert torch.equal(o, d.cpu()), "end-to-end output differs from the device-timed output"
    del sets

    # ---- the plain FP64 single-problem form on the same GPU, equal accuracy ----
    # Both contexts truncate E at the same tol (1e-7, which keeps E within the
    # 1e-5 bar); FP64 applies one problem per call (lgf_poisson_apply then
    # lgf_intfactor_apply), no batch, no graph, no concurrent branch.
    fp64 = None
    if not args.no_fp64:
        ctx64 = lgf.Context("f64", tol=1e-7, device=dev.index)
        ctx64.table_build(48)
        f64 = {k: t.double() for k, t in fs.items()}
        o64 = [torch.empty_like(o, dtype=torch.float64) for o in outs]
        tmp64 = [torch.empty_like(o, dtype=torch.float64) if e["op"] == 2 else None
                 for e, o in zip(w.entries, outs)]

        def plain64():
            for e, o, t in zip(w.entries, o64, tmp64):
                p = e["p"]
                f = f64[e["fkey"]]
                if e["op"] == 0:
                    ctx64.poisson_apply(p.b, p.src, p.tgt, f, o, ncomp=p.ncomp, nrhs=p.nrhs, stream=s)
                elif e["op"] == 1:
                    ctx64.intfactor_apply(e["alpha"], p.b, p.src, p.tgt, f, o, ncomp=p.ncomp, nrhs=p.nrhs,
                                          stream=s)
                else:
                    ctx64.poisson_apply(p.b, p.src, p.tgt, f, t, ncomp=p.ncomp, nrhs=p.nrhs, stream=s)
                    ctx64.intfactor_apply(e["alpha"], p.b, p.tgt, p.tgt, t, o, ncomp=p.ncomp, nrhs=p.nrhs,
                                          stream=s)

        with torch.cuda.stream(s):
            for _ in range(3):
                plain64()
        s.synchronize()
        n64 = max(3, min(args.steps, 10))
        ms64 = reduce_max(float(np.mean(timed_steps(plain64, s, n64, flush))), dist)
        errs = [float((x.double() - y).abs().max() / y.abs().max()) for x, y in zip(outs, o64)]
        fp64 = {"ms_per_step": ms64, "steps": n64, "value": job_throughput(w.points(), ms64, world),
                "unit": "points/s", "speedup_of_fp32_batched": ms64 / ms, "fp32_vs_fp64_rel_err": max(errs),
                "tol": 1e-7,
                "how": "FP64 context with the FP32 context's E truncation (tol 1e-7), one Poisson and one "
                       "integrating-factor call per problem per step, no batch or graph; the FP32 batched "
                       "outputs agree with it to fp32_vs_fp64_rel_err"}
        ctx64.close()
        del f64, o64, tmp64

    line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(w.desc, l2=l2_note,
                           parallelism=("problems sharded across ranks, longest first" if sharded else
                                        "replicas" if world > 1 else "single GPU"),
                           points_per_step=points_all, kernels=kernels, tuning=tuning),
            "roofline": roofline, "roofline_step": roofline_step, "roofline_dominant_kernel": roofline_dom,
            "e2e": e2e, "gpu_launches": int(round(launches_per_step * args.steps)),
            "launches_per_step": launches_per_step, "clocks": clocks,
            "timed_region_s": float(sum(ms_steps)) * 1e-3}
    if fp64 is not None:
        line["fp64_plain"] = fp64
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = {"value": npts / cpu_dt, "unit": "points/s", "cores": cores, "kind": "oracle",
                                "sample": f"{per} random Poisson targets per problem and field "
                                          f"({npts} target points; direct summation over every source), "
                                          f"{cpu_dt:.1f} s"}
        line["rel_err_vs_oracle"] = rel_err
        line["rel_err_how"] = ("Poisson apply of the same inputs in the same context, at the cpu_baseline "
                               "sample: per field max |gpu - oracle| / max |oracle|")
        line["rel_err_estimate_lib"] = lib_est
    ctx.close()
    return line


def run_ncu_case(args):
    """The bench step (one lgf_batch_apply on the legacy stream: direct
    launches) run `--steps` times untimed: the case that ncu captures."""
    import torch
    import paper_1604_01814_gb300 as lgf
    ctx = lgf.Context("f32")
    ctx.table_build(48)
    # with $LGF_TUNE_CACHE set (a file a tuned bench run wrote), the captured
    # plans take the tuned geometry without timing anything
    if os.environ.get("LGF_TUNE_CACHE"):
        ctx.autotune(lgf.LGF_TUNE_CACHED)
    if args.workload == "wake512":
        # one right-hand side (3 fields, about 3 GB on the device): the wake
        # domain's transform shape at a size a full capture handles
        import lgf_inputs as li
        p = li.wake_domain(nrhs=1)
        w = Workload("wake512", [dict(p=p, op=0, alpha=0.0, fkey=0)], {})
    else:
        w = make_workload(args.workload)
    _, batch, outs = build_batch(lgf, w, torch.device("cuda"), torch.float32)
    for _ in range(args.steps):
        ctx.batch_apply(batch, stream=0)
    torch.cuda.synchronize()
    print("ncu case done:", len(batch), "problems, max |u|", max(float(o.abs().max()) for o in outs), flush=True)
    ctx.close()


EXTRA = {
    "refresh_sphere": "velocity refresh u <- -C^dagger L^{-1} C u (Eq. vel_refresh) on the sphere-plus-wake "
                      "active set (16^3 blocks), u = curl of a Gaussian-blob vector potential, FP32; one refresh "
                      "per step",
    "ib_sphere": "immersed-boundary regularisation R then interpolation I (Sec. 2.1) of 5120 icosphere markers "
                 "(radius 20 cells) on the 32 blocks of 16^3 their three-point support touches, 3 components, "
                 "FP32; throughput in marker-components per second",
    "stage_sphere": "one IF-HERK stage solve by the nested projection (Eq. nested_proj: ip, f, pc, vc) on the "
                    "sphere-plus-wake active set (556 blocks of 16^3), 5120 icosphere markers (radius 20 cells), "
                    "FP32, random r, a dense 15360 x 15360 factor W (C^-1 = W^T W; random values, timing only), "
                    "alpha 0.05; throughput in face points (3 per cell) per second",
    "kinv_sphere": "K(0.25)^{-1} on the surface blocks of the icosphere (5120 markers, radius 20 cells, 16^3 "
                   "blocks, source = target = the blocks the 3-point delta touches), 3 components, FP32; one "
                   "G_K(0.25) apply per step",
}


def run_extra(args, rank, world, dist):
    """The rows beyond the Poisson/integrating-factor path: their own JSON
    line with throughput and per-kernel times.  Not the bench line."""
    import torch
    import lgf_inputs as li
    import paper_1604_01814_gb300 as lgf

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    ctx = lgf.Context("f32", device=dev.index)
    ctx.table_build(48)
    s = torch.cuda.Stream(device=dev)
    if args.workload == "refresh_sphere":
        q = li.sphere_ib()
        cells = q.tgt
        u = li.curl_blob_field(q.b, cells, centres=np.array([[-30.0, 0.0, 0.0], [40.0, 10.0, -5.0]]),
                               amps=np.array([[0.0, 0.0, 1.0], [0.5, -1.0, 0.0]]), sigma=8.0)
        ut = torch.tensor(u.reshape(-1), dtype=torch.float32, device=dev)
        uo = torch.empty_like(ut)
        points = float(3 * cells.shape[0] * q.b ** 3)

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

        def step():
            ctx.ib_spread(q.b, q.src, Xm, gm, fm, stream=s)
            ctx.ib_interp(q.b, q.src, Xm, fm, Um, stream=s)
    elif args.workload == "stage_sphere":
        q = li.sphere_ib()
        D = q.tgt
        Xm = torch.tensor(li.icosphere_markers(5) * 20.0, dtype=torch.float64, device=dev)
        nm = Xm.shape[0]
        rng = np.random.default_rng(5)
        r = torch.tensor(rng.uniform(-1, 1, size=3 * D.shape[0] * q.b ** 3), dtype=torch.float32, device=dev)
        u = torch.empty_like(r)
        dcell = torch.empty(D.shape[0] * q.b ** 3, dtype=torch.float32, device=dev)
        ub = torch.zeros(3 * nm, dtype=torch.float32, device=dev)
        fm = torch.empty(3 * nm, dtype=torch.float32, device=dev)
        W = torch.randn(3 * nm, 3 * nm, device=dev, generator=torch.Generator(device=dev).manual_seed(5)) * 1e-3
        points = float(r.numel())

        def step():
            ctx.nested_projection_stage(q.b, D, r, u, X_prev=Xm, X=Xm, ub=ub, W1=W, alpha=0.05, d=dcell, f=fm,
                                        stream=s)
    elif args.workload == "kinv_sphere":
        q = li.sphere_ib()
        f = torch.tensor(q.f.reshape(-1), dtype=torch.float32, device=dev)
        u = torch.empty_like(f)
        batch = [dict(b=q.b, src=q.src, tgt=q.src, f=f, u=u, ncomp=3, nrhs=1, op=lgf.LGF_OP_KINV, alpha=0.25)]
        points = float(u.numel())

        def step():
            ctx.batch_apply(batch, stream=s)
    else:
        raise ValueError(f"unknown workload {args.workload}")
    with torch.cuda.stream(s):
        for _ in range(max(3, args.warmup)):
            step()
    s.synchronize()
    clk = ClockSampler(dev.index)
    clk.start()
    ms_steps = timed_steps(step, s, args.steps)
    clocks = clk.stop()
    ms = reduce_max(float(np.mean(ms_steps)), dist)
    ctx.profile_enable(True)
    with torch.cuda.stream(s):
        for _ in range(args.steps):
            step()
    stats = ctx.profile_read()
    ctx.profile_enable(False)
    tot = sum(t for _, t in stats.values())
    kernels = {k: {"launches_per_step": n / args.steps, "ms_per_launch": t / n, "share": t / tot}
               for k, (n, t) in stats.items()}
    line = {"workload": args.workload, "config": EXTRA[args.workload], "metric": METRIC,
            "value": job_throughput(points, ms, world), "unit": "points/s", "ms_per_step": ms,
            "points_per_step": points, "steps": args.steps, "n_gpus": world, "dtype": "f32",
            "parallelism": "replicas" if world > 1 else "single GPU", "scaling": "weak",
            "kernels": kernels, "clocks": clocks}
    ctx.close()
    return line


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=150)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plates64",
                    help="plates64 (default, the bench line), dense128, wake512, sphere; or " + ", ".join(EXTRA))
    ap.add_argument("--cpu-points", type=int, default=0,
                    help="oracle sample per problem and field for cpu_baseline and the error check (0: default)")
    ap.add_argument("--ref-points", type=int, default=0, help="reference arm sample per problem (0: default)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-tune", action="store_true", help="library defaults instead of the autotuner's choices")
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
