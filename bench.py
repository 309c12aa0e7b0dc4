"""Benchmark: joined-chain spin-flip attempts/s of the multicanonical weight
iteration (Sec. 2 algorithm + Sec. 3.1 update) on one GB300.

One step = one weight iteration of the whole hot path on the headline
workload (L = 32, 16384 chains, 1e5 sweeps per chain, random start, seed 2):
generation of every chain (Sec. 2 step 2), the joint by detailed balance
(steps 3-5, speculation + resolution + segmented scan), the weight update
(Eq. new_weight).  value = samples kept in the joined chain per second of
device time (CUDA events on the job's stream).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (under torch.distributed.run): every rank runs an independent job
(seed + rank) -- replicas, nothing exchanged on the data path; value = all
ranks' kept samples over the slowest rank's time.  --impl reference times the
CPU oracle, on bounded samples of the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_0812_2964_gb300.workloads import WORKLOADS, workload as workload_by_name  # noqa: E402

METRIC = "joined-chain spin-flip attempts/s"
UNIT = "attempts/s"
WORKLOAD = "L32_p16384"
# Integer operations one single-spin-flip attempt needs: Philox4x32-10
# amortised over its 4 words (10 rounds x (2 multiplies + 2 three-input
# XORs) / 4 = 10), aligned-neighbour count (4 compares + 3 adds = 7),
# threshold index + load (2), compare (1), flip + level update (2),
# histogram update (3).
ALG_OPS_PER_ATTEMPT = 25
SMS, SUBPARTITIONS, LANES = 152, 4, 32
L2_FLUSH_BYTES = 256 << 20
ORACLE_SAMPLE = dict(chains=128, sweeps=400)    # bounded CPU sample of the workload


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _traffic_record():
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index: int):
        self.index, self.proc, self.lines = index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=lambda: self.lines.extend(
            ln.strip() for ln in self.proc.stdout), daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(self.REASONS, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def aggregate(kept_per_rank, seconds_per_rank):
    """Whole-job throughput: kept samples of all ranks over the slowest rank."""
    t = max(seconds_per_rank)
    return (float(sum(kept_per_rank)) / t if t > 0 else 0.0), t


def gather_max_sum(dist, world, kept, seconds, device):
    """All ranks' (kept, seconds) -> (sum kept, max seconds), on the host side
    of the run; used only for timing, never on the data path."""
    if world == 1:
        return kept, seconds
    import torch
    t = torch.tensor([float(kept), float(seconds)], dtype=torch.float64, device=device)
    out = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(out, t)
    ks = [float(o[0]) for o in out]
    ss = [float(o[1]) for o in out]
    return sum(ks), max(ss)


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(seconds_budget: float, L: int, seed: int, start: int):
    """Kept samples per second of the plain oracle (generation + serial joint
    + weight update) on a bounded sample of the workload, all host cores."""
    import oracle

    cores = os.cpu_count() or 1
    p, S = ORACLE_SAMPLE["chains"], ORACLE_SAMPLE["sweeps"]
    job = oracle.Job(L, p, seed, start)
    kept, iters = 0, 0
    t0 = time.perf_counter()
    while True:
        kept += job.iteration(S, 0, cores)
        iters += 1
        el = time.perf_counter() - t0
        if el >= seconds_budget:
            break
    return {"value": kept / el, "unit": UNIT, "cores": cores, "per_core": kept / el / cores, "kind": "oracle",
            "sample": f"L={L}, {p} chains x {S} sweeps per iteration, {iters} weight iterations "
                      f"from the workload's seed ({el:.1f} s)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = WORKLOADS[WORKLOAD]
    import oracle

    cores = os.cpu_count() or 1
    p, S = ORACLE_SAMPLE["chains"], ORACLE_SAMPLE["sweeps"]
    job = oracle.Job(w.L, p, w.seed, w.start)
    for _ in range(args.warmup):
        job.iteration(S, 0, cores)
    kept = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        kept += job.iteration(S, 0, cores)
    el = time.perf_counter() - t0
    value = kept / el
    sample = (f"L={w.L}, {p} chains x {S} sweeps per step (the workload has {w.chains} chains x "
              f"{w.sweeps} sweeps), weight iterations {args.warmup + 1}..{args.warmup + args.steps}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "L": w.L, "chains": p,
                                            "sweeps_per_iteration": S, "seed": w.seed},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "per_core": value / cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def timed_iterations(torch, job, stream, S, steps, flush):
    """`steps` weight iterations of one job (round of S sweeps, joint, weight
    update, L2 flush), timed with CUDA events on the job's stream: total
    seconds, mean milliseconds per phase, generation milliseconds per step."""
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    # per step: events before generation, the joint, the weight update and the L2 flush
    marks = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for i in range(steps):
            e = marks[i]
            e[0].record(stream)
            job.run_sweeps(S)              # generation kernel (+ round-start copy)
            e[1].record(stream)
            job.join(want_length=False)    # joint: search, resolution, correction, scan
            e[2].record(stream)
            job.update_weights()           # Eq. (new_weight) + threshold table
            e[3].record(stream)
            flush.fill_(1)                 # L2 flushed between timed steps
            e[4].record(stream)
        ev1.record(stream)
    torch.cuda.synchronize()
    gen_ms = [e[0].elapsed_time(e[1]) for e in marks]
    phases = {name: statistics.mean(e[a].elapsed_time(e[a + 1]) for e in marks)
              for a, name in enumerate(("gen_ms", "joint_ms", "update_ms", "l2_flush_ms"))}
    phases["joint_ms_max"] = max(e[1].elapsed_time(e[2]) for e in marks)
    return ev0.elapsed_time(ev1) / 1e3, phases, gen_ms


def alu_roofline(p, S, N, gen_ms):
    """Algorithmic integer operations of one generation launch per second of
    its mean CUDA-event time, against the integer-issue peak."""
    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz") or 2070.0)
    peak_ops = SMS * SUBPARTITIONS * LANES * sm_max * 1e6
    achieved = p * S * N * ALG_OPS_PER_ATTEMPT / (statistics.mean(gen_ms) / 1e3)
    return {"bound": "alu", "achieved": achieved / 1e9, "peak": peak_ops / 1e9, "unit": "Gop/s",
            "frac": achieved / peak_ops, "kernel_ms": statistics.mean(gen_ms), "ops_per_attempt": ALG_OPS_PER_ATTEMPT,
            "peak_source": f"{SMS} SMs x {SUBPARTITIONS} sub-partitions x {LANES} lanes x "
                           f"{sm_max:.0f} MHz (sm_max_mhz of MEASURED_PEAKS.json)"}


# reduced sizes of the other workloads measured beside the headline (one line)
SUB = dict(L64_sweeps=2000, L128_sweeps=400, job_steps=3, job_warmup=3,
           batch_sweeps=5000, batch_steps=2, batch_warmup=1,
           serving_jobs=60, serving_rate=20.0, serving_sweeps=20, serving_slots=16)


def job_record(torch, mc, device, workload, S, steps, warmup):
    """One job of `workload` at S sweeps per iteration (the workload's L, chains,
    seed and start), device-timed like the headline."""
    w = WORKLOADS[workload]
    t_wall = time.perf_counter()
    stream = torch.cuda.Stream(device=device)
    job = mc.Job(w.L, w.chains, w.seed, w.start)
    job.set_stream(stream.cuda_stream)
    job.set_trace(True)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=device)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            job.run_sweeps(S)
            job.join(want_length=False)
            job.update_weights()
    torch.cuda.synchronize()
    kept0 = job.info()["total_joined"]
    el, phases, gen_ms = timed_iterations(torch, job, stream, S, steps, flush)
    info = job.info()
    kept = info["total_joined"] - kept0
    M = S * w.N
    rec = {"metric": METRIC, "value": kept / el, "unit": UNIT,
           "config": {"workload": workload, "L": w.L, "chains": w.chains, "sweeps_per_iteration": S,
                      "sweeps_of_the_workload": w.sweeps, "seed": w.seed,
                      "weight_iterations_timed": f"{warmup + 1}..{warmup + steps}",
                      "launch": {"placement": ["registers", "shared", "global"][info["placement"]],
                                 "chains_per_warp": info["chains_per_warp"],
                                 "warps_per_block": info["warps_per_block"]}},
           "ms_per_step": 1e3 * el / steps, "kept_fraction": kept / (steps * w.chains * M),
           "raw_attempts_per_s": steps * w.chains * M / el, "phases": phases,
           "roofline": alu_roofline(w.chains, S, w.N, gen_ms),
           "timing": "CUDA events on the job's stream"}
    job.close()
    rec["wall_s"] = time.perf_counter() - t_wall
    return rec


def batch_record(torch, mc, S, steps, warmup, tune, rank=0):
    """The uneven batch run three ways on the same chains; kept samples/s of each."""
    from paper_0812_2964_gb300.workloads import BATCH_GROUPS

    modes = {0: "one launch per job", 1: "one fused launch", 2: "fused launch, CUDA graph"}
    out = {}
    t_wall = time.perf_counter()
    for mode in (0, 1, 2):
        jobs = [mc.Job(L, p, seed + rank, 1) for (L, p, seed) in BATCH_GROUPS]
        for j in jobs:
            j.set_trace(True)
            if tune:
                j.autotune(probe_sweeps=max(1, min(S, 2_000_000 // j.N)))
        if mode > 0:
            # shapes of the fused launch from the autotuner (whole-batch probes)
            mc.mc_batch_autotune(jobs, max(1, min(S, 100)))
        mc.mc_batch_run(jobs, warmup, S, mode)
        torch.cuda.synchronize()
        kept0 = sum(j.info()["total_joined"] for j in jobs)
        l0 = mc.mc_kernel_launches()
        t0 = time.perf_counter()
        mc.mc_batch_run(jobs, steps, S, mode)   # synchronises
        el = time.perf_counter() - t0
        launches = mc.mc_kernel_launches() - l0
        kept = sum(j.info()["total_joined"] for j in jobs) - kept0
        attempts = sum(j.p * S * j.N for j in jobs) * steps
        shapes = ([list(mc.mc_batch_shape(j)[:3]) for j in jobs] if mode > 0 else
                  [[j.info()[k] for k in ("placement", "chains_per_warp", "warps_per_block")] for j in jobs])
        out[mode] = {"mode": modes[mode], "value": kept / el, "seconds": el, "kept": kept,
                     "raw_attempts_per_s": attempts / el, "gpu_launches": launches, "shapes": shapes}
        for j in jobs:
            j.close()
    return {"metric": METRIC, "value": out[2]["value"], "unit": UNIT,
            "config": {"workload": "batch_uneven", "groups": [list(g) for g in BATCH_GROUPS],
                       "sweeps_per_iteration": S, "iterations_timed": steps,
                       "fused_shapes": "mc_batch_autotune (whole-batch probes of min(S, 100) sweeps)",
                       "per_job_shapes": "mc_autotune" if tune else "library default",
                       "timing": "host wall clock around the synchronising call"},
            "modes": out, "fused_vs_per_job": out[1]["value"] / out[0]["value"],
            "graph_vs_per_job": out[2]["value"] / out[0]["value"], "wall_s": time.perf_counter() - t_wall}


def serving_record(mc, n_jobs, rate, S, slots, rank=0):
    """A Poisson stream of weight-estimation jobs submitted at their arrival
    times to the continuous-batching server (40 GB budget)."""
    from paper_0812_2964_gb300.workloads import serving_stream

    t_wall = time.perf_counter()
    stream = serving_stream(n_jobs, rate=rate, sweeps=S)
    budget = 40 << 30
    with mc.Server(budget, slots) as srv:     # warm-up: one small job of every size
        for i, L in enumerate((16, 32, 48, 64, 96, 128)):
            srv.wait(srv.submit(L, 256, 99 + i, 2, S))
    l0 = mc.mc_kernel_launches()
    with mc.Server(budget, slots) as srv:
        ids = []
        t_base = srv.clock()
        for job in stream:
            delay = t_base + job.arrival - srv.clock()
            if delay > 0:
                time.sleep(delay)
            ids.append(srv.submit(job.L, job.chains, job.seed + rank, job.iterations, job.sweeps))
        res = [srv.wait(j) for j in ids]
        info = srv.info()
    launches = mc.mc_kernel_launches() - l0
    st = [r[1] for r in res]
    lat = np.array([s["t_done"] - s["t_submit"] for s in st])
    qwait = np.array([s["t_admit"] - s["t_submit"] for s in st])
    span = max(s["t_done"] for s in st) - min(s["t_submit"] for s in st)
    joined = sum(s["joined"] for s in st)
    attempts = sum(s["attempts"] for s in st)
    offered = attempts / max(1e-9, stream[-1].arrival - stream[0].arrival)
    d2h = sum((j.L * j.L + 1) * 8 for j in stream)
    return {"metric": METRIC, "value": joined / span, "unit": UNIT,
            "config": {"workload": "serving", "jobs": len(stream), "rate_jobs_per_s": rate, "arrival_seed": 5,
                       "sizes": [16, 32, 48, 64, 96, 128], "chains": "256..4096 step 256",
                       "iterations": "20..60", "sweeps_per_iteration": S, "budget_bytes": budget, "slots": slots,
                       "step": "one job (arrival to W ready)"},
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "mean": float(lat.mean()), "max": float(lat.max())},
            "queue_wait_s": {"p50": float(np.percentile(qwait, 50)), "p99": float(np.percentile(qwait, 99))},
            "makespan_s": span, "jobs_per_s": len(stream) / span,
            "raw_attempts_per_s": attempts / span, "offered_attempts_per_s": offered,
            "utilisation_proxy": offered / (attempts / span),
            "server": {k: info[k] for k in ("peak_active", "peak_bytes", "admitted", "completed")},
            "d2h_bytes_per_job": d2h / len(stream), "gpu_launches": launches,
            "wall_s": time.perf_counter() - t_wall}


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_0812_2964_gb300 as mc

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    mc.build()
    w = workload_by_name(args.workload)
    S = args.sweeps or w.sweeps
    p, N = w.chains, w.N
    M = S * N
    stream = torch.cuda.Stream(device=device)
    job = mc.Job(w.L, p, w.seed + rank, w.start)
    job.set_stream(stream.cuda_stream)
    job.set_trace(True)
    if args.join_order:
        job.set_join_order(args.join_order)
    if args.tune:
        job.autotune(probe_sweeps=max(1, min(S, 4_000_000 // N)))
    if args.segment_samples:
        job.set_segment_samples(args.segment_samples)
    if args.shape:
        job.set_launch_shape(*(int(v) for v in args.shape.split(",")))
    if args.round_record >= 0:
        job.set_round_record(args.round_record)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=device)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            job.run_sweeps(S)
            job.join(want_length=False)
            job.update_weights()
            flush.fill_(1)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    kept0 = job.info()["total_joined"]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    launches0 = mc.mc_kernel_launches()
    elapsed, phases, gen_ms = timed_iterations(torch, job, stream, S, args.steps, flush)
    launches = mc.mc_kernel_launches() - launches0
    clk = clocks.stop()
    kept = job.info()["total_joined"] - kept0
    info = job.info()
    if world > 1:
        dist.barrier()
    kept_all, t_max = gather_max_sum(dist, world, kept, elapsed, device)
    value = kept_all / t_max

    # ---- end to end through the public API, host buffers (pinned), per step:
    # spins + weights in, run + join + histogram + update, weights + spins out
    e2e_steps = max(1, args.e2e_steps)
    nwords = p * w.L * ((w.L + 31) // 32)
    spins_h = torch.empty(nwords, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    W_h = torch.empty(N + 1, dtype=torch.float64, pin_memory=True).numpy()
    hist_h = torch.empty(N + 1, dtype=torch.int64, pin_memory=True).numpy()
    mc.mc_get_spins(job.h, spins_h)
    mc.mc_get_weights(job.h, W_h)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e2e_kept = 0
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        mc.mc_set_spins(job.h, spins_h)
        mc.mc_set_weights(job.h, W_h)
        mc.mc_run_sweeps(job.h, S)
        e2e_kept += mc.mc_join(job.h, True)
        mc.mc_histogram(job.h, hist_h)
        mc.mc_update_weights(job.h)
        mc.mc_get_weights(job.h, W_h)
        mc.mc_get_spins(job.h, spins_h)
    e2e_el = time.perf_counter() - t0
    e2e_all, e2e_t = gather_max_sum(dist, world, e2e_kept, e2e_el, device)
    h2d = nwords * 4 + (N + 1) * 8
    d2h = 8 + (N + 1) * 8 + (N + 1) * 8 + nwords * 4

    if rank != 0:
        dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel (generation)
    roof = alu_roofline(p, S, N, gen_ms)
    tr = _traffic_record()
    same_kernel = tr.get("workload") == args.workload and tr.get("kernel_rev") == mc.KERNEL_REV
    traffic = None
    if same_kernel and tr.get("bytes_per_launch") and tr.get("sweeps"):
        # captured on a shorter launch of the same kernel and scaled to this
        # one: the trace grows with the sweeps, the rest is per launch
        per_sweep = tr.get("bytes_per_sweep", 0)
        traffic = tr["bytes_per_launch"] + per_sweep * (S - tr["sweeps"])
    # issue-slot use of the same kernel revision measured by ncu on the capture
    # case named in the source (a shorter launch of the same workload)
    issue = tr.get("issue_active_pct") if same_kernel else None

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(args.cpu_seconds, w.L, w.seed, w.start)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": args.workload, "L": w.L, "chains": p, "sweeps_per_iteration": S,
                   "start": "random" if w.start else "all up", "seed": w.seed,
                   "weight_iterations_timed": f"{args.warmup + 1}..{args.warmup + args.steps}",
                   "l2": "flushed between steps (256 MB write)", "trace": "int32 per sweep",
                   "launch": {"placement": ["registers", "shared", "global"][info["placement"]],
                              "chains_per_warp": info["chains_per_warp"],
                              "warps_per_block": info["warps_per_block"]},
                   "parallelism": f"replicas x{world}",
                   "join_order": ["chain index", "ascending final energy"][args.join_order]},
        "phases": phases,
        "kept_fraction": kept / (args.steps * p * M),
        "raw_attempts_per_s": args.steps * p * M * world / t_max,
        "roofline": {**roof, "traffic": traffic,
                     "kernel": "gen_kernel (lattice rows in %s)" % ["registers", "shared memory", "global memory"][info["placement"]],
                     "measured_issue_active": (issue / 100.0) if issue is not None else None,
                     "measured_issue_lane_weighted": (issue / 100.0 * tr.get("lanes_active", 32) / 32)
                     if issue is not None else None,
                     "measured_issue_source": tr.get("issue_active_source") if issue is not None else None,
                     "traffic_source": tr.get("traffic_source") if traffic is not None else None},
        "e2e": {"value": e2e_all / e2e_t, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps},
        "gpu_launches": launches,
        "clocks": clk,
        "last_joint": {k: info[k] for k in ("last_joined", "last_rejected", "last_mismatch",
                                            "last_passes", "last_searched", "segments", "segment_sweeps")},
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if world == 1 and not args.no_subrecords and args.workload == WORKLOAD:
        # the rest of the metric, at reduced sizes named in each record's config
        del job, flush
        torch.cuda.empty_cache()
        line["subrecords"] = {
            "L64_p4096": job_record(torch, mc, device, "L64_p4096", SUB["L64_sweeps"], SUB["job_steps"],
                                    SUB["job_warmup"]),
            "L128_p1024": job_record(torch, mc, device, "L128_p1024", SUB["L128_sweeps"], SUB["job_steps"],
                                     SUB["job_warmup"]),
            "batch_uneven": batch_record(torch, mc, SUB["batch_sweeps"], SUB["batch_steps"], SUB["batch_warmup"],
                                         args.tune),
            "serving": serving_record(mc, SUB["serving_jobs"], SUB["serving_rate"], SUB["serving_sweeps"],
                                      SUB["serving_slots"]),
        }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """The uneven batch: L in {16, 24, 32, 48, 64} with 8192/4096/4096/2048/1024
    chains, every weight iteration run three ways -- one generation launch per
    job, one fused launch, the fused loop as a CUDA graph -- on the same
    chains (identical results); value = the graph form's kept samples/s."""
    import torch

    import paper_0812_2964_gb300 as mc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    mc.build()
    S = args.sweeps or 50_000
    clocks = ClockSampler(local)
    clocks.start()
    rec = batch_record(torch, mc, S, args.steps, args.warmup, args.tune, rank)
    clk = clocks.stop()
    best = rec["modes"][2]
    line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * best["seconds"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": rec["config"], "modes": rec["modes"], "fused_vs_per_job": rec["fused_vs_per_job"],
            "graph_vs_per_job": rec["graph_vs_per_job"], "clocks": clk, "gpu_launches": best["gpu_launches"]}
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args):
    """Serving: a Poisson stream of weight-estimation jobs (L in {16, ..., 128},
    256-4096 chains, 20-60 iterations) submitted at their arrival times to
    the continuous-batching server (40 GB budget); value = kept samples of
    all jobs / makespan (first arrival to last completion); p50/p99 of the
    job latency (arrival to W ready)."""
    import torch

    import paper_0812_2964_gb300 as mc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    mc.build()
    S = args.sweeps or 20
    clocks = ClockSampler(local)
    clocks.start()
    rec = serving_record(mc, args.jobs, args.rate, S, args.slots, rank)
    clk = clocks.stop()
    n = rec["config"]["jobs"]
    line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world, "steps": n,
            "warmup": 6, "ms_per_step": 1e3 * rec["makespan_s"] / n, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": rec["config"],
            "latency_s": rec["latency_s"], "queue_wait_s": rec["queue_wait_s"],
            "raw_attempts_per_s": rec["raw_attempts_per_s"], "offered_attempts_per_s": rec["offered_attempts_per_s"],
            "utilisation_proxy": rec["utilisation_proxy"], "server": rec["server"],
            "e2e": {"value": rec["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": rec["d2h_bytes_per_job"],
                    "note": "host-timed from submission to collection; each job's input is its spec"},
            "gpu_launches": rec["gpu_launches"], "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_fig2(args):
    """The Fig. 2 experiment shape (Sec. 5): L = 20, p = 32 short chains, the
    weight iteration run twice -- chains joined by detailed balance
    (mc_join) and simply concatenated (mc_join_naive) -- each iteration
    collecting M_total samples in rounds of M_node attempts per chain; then
    E/N by Eq. (reweighting2) against the exact finite-lattice values.
    M_node = 100 attempts (a quarter sweep: mc_run_attempts)."""
    import torch

    import paper_0812_2964_gb300 as mc

    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from exact import exact_thermo

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    mc.build()
    L, p, M_node = 20, 32, args.mnode
    N = L * L
    M_total = args.mtotal
    iters = args.iters
    betas = [0.1, 0.2, 0.3, 0.35, 0.4, 0.4406867935097715, 0.5, 0.6, 0.8, 1.0]
    exact = [exact_thermo(L, b)[0] / N for b in betas]
    out = {}
    for name, naive in (("detailed balance", False), ("no detailed balance", True)):
        job = mc.Job(L, p, 10 + rank, 1)
        rounds = 0
        t0 = time.perf_counter()
        for _ in range(iters):
            got = 0
            while got < M_total:
                job.run_attempts(M_node)
                got += job.join_naive() if naive else job.join()
                rounds += 1
            job.update_weights()
        el = time.perf_counter() - t0
        E = job.thermo(betas)[:, 0] / N
        dev = [float(e - x) for e, x in zip(E, exact)]
        out[name] = {"E_per_site": [float(e) for e in E], "deviation": dev,
                     "max_abs_dev_beta_le_0.44": max(abs(d) for b, d in zip(betas, dev) if b <= 0.45),
                     "max_abs_dev_beta_gt_0.44": max(abs(d) for b, d in zip(betas, dev) if b > 0.45),
                     "rounds": rounds, "seconds": el, "ms_per_round": 1e3 * el / max(1, rounds),
                     "kept_fraction": iters * M_total / max(1, rounds * p * M_node)}
        job.close()
    line = {"metric": "fig2: E/N deviation from the exact L=20 values", "unit": "energy per site",
            "value": out["detailed balance"]["max_abs_dev_beta_le_0.44"], "higher_is_better": False,
            "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "fig2", "L": L, "chains": p, "M_node_attempts": M_node, "M_total": M_total,
                       "iterations": iters, "betas": betas},
            "exact_E_per_site": exact, "runs": out}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_fig1(args):
    """The Fig. 1 comparison (Sec. 5) at the paper's lattice size and number
    of weight iterations: L = 100, I = 1300 iterations of the weight
    recursion from W = 0, each from rounds of `sweeps` sweeps on every chain
    joined by detailed balance; then E/N, C/N, F/N and S/N by Eq.
    (reweighting2) against the exact finite-lattice values (Ferdinand and
    Fisher; Kaufman's partition function).  Defaults: the paper's Table 1
    run (workload L100_p32: 32 chains of 313 sweeps, seed 9), rounds repeated
    until M_total = 1e8 samples are kept before each update (step 6;
    `--mtotal 0`: one round per iteration).  The loop stops early, at a
    whole iteration, once `time_limit` seconds have passed."""
    import torch

    import paper_0812_2964_gb300 as mc

    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from exact import exact_thermo

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    mc.build()
    w = WORKLOADS["L100_p32"]
    L = w.L
    N = L * L
    p = args.chains or w.chains
    S = args.sweeps or w.sweeps
    iters = args.iters or w.iterations
    betas = [0.1, 0.2, 0.3, 0.4, 0.42, 0.4406867935097715, 0.46, 0.5, 0.6, 0.8, 1.0]
    job = mc.Job(L, p, w.seed + rank, w.start)
    kept = rounds = done = 0
    t0 = time.perf_counter()
    while done < iters and time.perf_counter() - t0 < args.time_limit:
        if args.mtotal > 0:
            j, r = job.iteration(S, args.mtotal)
            kept += j
            rounds += r
        else:
            job.run_sweeps(S)
            kept += job.join()
            job.update_weights()
            rounds += 1
        done += 1
    job.sync()
    el = time.perf_counter() - t0
    got = job.thermo(betas)
    visited = int(np.count_nonzero(job.visited))
    job.close()
    rows = []
    for b, g in zip(betas, got):
        ex = exact_thermo(L, b)
        rows.append({"beta": b, "E": float(g[0]) / N, "C": float(g[1]) / N, "F": float(g[2]) / N,
                     "S": float(g[3]) / N, "E_exact": ex[0] / N, "C_exact": ex[1] / N, "F_exact": ex[2] / N,
                     "S_exact": ex[3] / N})
    dev = {q: max(abs(r[q] - r[q + "_exact"]) for r in rows) for q in ("E", "C", "F", "S")}
    line = {"metric": "fig1: largest deviation of E/N, C/N, F/N, S/N from the exact L=100 values",
            "unit": "per site", "value": max(dev["E"], dev["F"], dev["S"]), "higher_is_better": False,
            "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "fig1", "L": L, "chains": p, "sweeps_per_iteration": S,
                       "samples_per_round": p * S * N, "M_total": args.mtotal, "iterations": done,
                       "iterations_asked": iters, "rounds": rounds,
                       "seed": w.seed + rank, "start": "random" if w.start else "all up", "betas": betas},
            "max_abs_dev": dev, "levels_visited": visited, "levels": N + 1,
            "kept_fraction": kept / max(1, rounds * p * S * N), "seconds": el,
            "ms_per_iteration": 1e3 * el / max(1, done), "rows": rows}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="L32_p16384 (default), L64_p4096, L128_p1024, L8_p64, batch_uneven, serving, fig1, fig2, "
                         "or L<L>_p<chains> (one job of that size, 20 sweeps a round)")
    ap.add_argument("--shape", default="", help="launch shape placement,chains_per_warp,warps_per_block "
                                                "(0 registers, 1 shared memory, 2 global memory)")
    ap.add_argument("--round-record", type=int, default=-1,
                    help="largest round (samples) whose levels are recorded for the joint (0: none; "
                         "default: the library's); a short profiling run of the headline kernel uses 0, "
                         "as the full-size round is too large to record")
    ap.add_argument("--sweeps", type=int, default=0, help="override sweeps per iteration")
    ap.add_argument("--tune", action="store_true", help="pick the launch shape with mc_autotune first")
    ap.add_argument("--segment-samples", type=int, default=0,
                    help="target length of the joint's checkpoint segments (0: the library's default)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-subrecords", action="store_true",
                    help="skip the reduced-size L=64, L=128, batch and serving records of the default run")
    ap.add_argument("--jobs", type=int, default=400, help="serving: jobs in the arrival stream")
    ap.add_argument("--rate", type=float, default=20.0, help="serving: mean arrivals per second")
    ap.add_argument("--slots", type=int, default=16,
                    help="serving: server slots (16 hold the GPU's capacity; more resident jobs only "
                         "lengthen each job)")
    ap.add_argument("--join-order", type=int, default=0,
                    help="0: chains joined in index order; 1: by ascending final energy (end of Sec. 2)")
    ap.add_argument("--mtotal", type=int, default=100_000_000,
                    help="fig1, fig2: kept samples per weight iteration (M_total; fig1: 0 = one round)")
    ap.add_argument("--iters", type=int, default=0, help="fig1, fig2: weight iterations (default 1300, 20)")
    ap.add_argument("--chains", type=int, default=0, help="fig1: chains (default 32, the paper's)")
    ap.add_argument("--time-limit", type=float, default=600.0,
                    help="fig1: stop after the iteration that passes this many seconds")
    ap.add_argument("--mnode", type=int, default=100, help="fig2: attempts per chain per round (M_node)")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch_uneven":
        return run_batch(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "fig2":
        args.iters = args.iters or 20
        return run_fig2(args)
    if args.workload == "fig1":
        return run_fig1(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
