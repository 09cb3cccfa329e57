#!/usr/bin/env python3
"""Throughput of exact chromosome decodes in the GPU hybrid GA on the dynamic rescheduling
workload (predictive-reactive complete rescheduling, Sec. 4.1 of arXiv 1903.10741).

One step = one whole rescheduling job: 50 initial jobs, 5 stages of U{2..4} identical
machines, int32 processing times U{1..99}, powers U{5..30}, peak 55 % of the all-on
power; the GA (population 1024 in islands of 64, tournament 2, crossover 0.8, mutation
0.1, ring migration every 10) runs 500 generations on the initial problem and again after
each of three events at t = 100, 250, 400 that freeze the executed plan and add 10 jobs.
Every generation decodes the whole population exactly; the metric counts those decodes.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  ``--impl reference`` times the single-threaded CPU
oracle on a bounded sample of the same job.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1903_10741_gb300 import workloads as wl  # noqa: E402

METRIC = "exact chromosome decodes/sec"
UNIT = "decodes/s"
P, ISLAND, TOUR_K, PC, PM, MIGRATE, SEED = 1024, 64, 2, (4, 5), (1, 10), 10, 1
WORKLOAD = ("dynamic rescheduling, plain GA: 50 initial jobs, 5 stages x U{2..4} identical machines, "
            "p U{1..99}, q U{5..30} kW, peak 55% of all-on power; events at t=100,250,400 adding 10 jobs "
            "(due = arrival + U[1.2,2.0] x work); complete reschedule at each event; population 1024 "
            "(16 islands of 64), tournament 2, pc 0.8, pm 0.1, migration every 10; 500 generations per solve")
# Algorithmic work of one exact decode on this job (python -m oracle.work_per_decode
# --generations 500 --every 50, the oracle's own GA trajectory of this job): per-instant
# power checks (Eq. 7) over every machine of the op's stage plus profile updates (Eq. 8),
# 53232 / 62226 / 68630 / 75374 for the four solves, mean 64865.5; and the stage-by-stage
# sort, sum over stages of n_s ceil(log2 n_s) compares: 1500 / 1710 / 2126 / 2409, mean 1936.25.
SLOTS_PER_DECODE = 64865.5
SORT_PER_DECODE = 1936.25
# DRAM bytes (read + write) of one generation-kernel launch from the ncu capture of the
# current kernel (dram__bytes_read.sum + dram__bytes_write.sum, initial solve); None once
# the kernel changes until it is captured again.
TRAFFIC_BYTES = 440320


def work_per_decode() -> float:
    return SLOTS_PER_DECODE + SORT_PER_DECODE


def alu_peak_tops(sms: int, mhz: float) -> float:
    """INT32 issue ceiling: SMs x 4 schedulers x 32 lanes x clock, in 10^12 lane-ops/s."""
    return sms * 128 * mhz * 1e6 / 1e12


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.dev), "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) < 9:
                        continue
                    try:
                        sm.append(float(parts[1]))
                        smax.append(float(parts[2]))
                        power.append(float(parts[3]))
                    except ValueError:
                        continue
                    for nm, v in zip(names, parts[5:9]):
                        if v.lower() == "active":
                            reasons.add(nm)
            os.unlink(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ----------------------------------------------------------------------------- helpers
def aggregate(dist, decodes: float, seconds: float, device=None):
    """Whole-job throughput over ranks: all ranks' decodes / the slowest rank's time."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return decodes, seconds
    import torch
    t = torch.tensor([decodes, seconds], dtype=torch.float64, device=device)
    tot = t.clone()
    dist.all_reduce(tot[0:1], op=dist.ReduceOp.SUM)
    dist.all_reduce(tot[1:2], op=dist.ReduceOp.MAX)
    return float(tot[0]), float(tot[1])


def input_bytes(dyn) -> int:
    pr = dyn.problem
    b = sum(np.asarray(a, np.int32).nbytes for a in (pr.o, pr.p, pr.q, pr.R, pr.D))
    for _, arr in dyn.events:
        b += sum(np.asarray(a, np.int32).nbytes for a in (arr.p, arr.R, arr.D))
    return b


def run_job(ffs, inst, dyn, generations: int, stream, profile, out_stats: dict):
    """Initial solve + one solve per event on `inst`; returns exact decodes performed.
    profile: 0 untimed graph replays, 1 eager launches with the fused kernel timed, 2 graph
    replays each timed (see ga_set_profiling)."""
    decodes = 0
    d2h = 0
    for solve in range(len(dyn.events) + 1):
        pop = ffs.Population(inst, P=P, island=ISLAND, tour_k=TOUR_K, pc=PC, pm=PM, migrate_every=MIGRATE,
                             seed=SEED, instance_id=solve, stream=stream)
        if profile:
            pop.set_profiling(int(profile))
        res = pop.run(generations)
        if profile:
            ms, n = pop.profile()
            out_stats["kernel_ms"] = out_stats.get("kernel_ms", 0.0) + ms
            out_stats["kernel_launches"] = out_stats.get("kernel_launches", 0) + n
        out_stats.setdefault("best_obj", []).append(res["obj"])
        d2h += res["S"].nbytes + res["M"].nbytes + 20
        decodes += P * (generations + 1) + 1
        pop.close()
        if solve < len(dyn.events):
            t_now, arr = dyn.events[solve]
            inst.reschedule(arr, t_now)
    out_stats["d2h"] = d2h
    return decodes


# ----------------------------------------------------------------------------- ours
def bench_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1903_10741_gb300 import ffs

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    ffs.lib()
    stream = torch.cuda.current_stream(dev)
    dyn = wl.dynamic_medium(1)
    G = args.generations
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    # warm-up (untimed)
    for _ in range(args.warmup):
        run_job(ffs, ffs.Instance(dyn.problem), dyn, G, stream, args.eager, {})
    insts = [ffs.Instance(dyn.problem) for _ in range(args.steps)]  # inputs resident before timing
    for inst in insts:
        inst.decode(torch.ones((1, inst.K), dtype=torch.int16, device=dev) *
                    torch.arange(1, inst.K + 1, dtype=torch.int16, device=dev))  # upload tables
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = ffs.kernel_launches()
    stats, total_ms, decodes = {}, 0.0, 0
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        decodes += run_job(ffs, insts[k], dyn, G, stream, args.eager, stats)
        e.record(stream)
        e.synchronize()
        total_ms += s.elapsed_time(e)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    launches = ffs.kernel_launches() - launches0
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    tot_decodes, max_s = aggregate(dist if world > 1 else None, float(decodes), total_ms / 1e3, dev)

    # Roofline passes: the same job again, (a) in the timed run's own launch mode -- graph
    # replays of 8 chained generations, each replay bracketed by CUDA events on the
    # population's stream -- and (b) with every generation launched directly and the fused
    # kernel alone bracketed (no overlap between generations).
    def timed_pass(mode, jobs):
        st_, ms_, dec_ = {}, 0.0, 0
        for k in range(jobs):
            flush.fill_(float(k))
            inst = ffs.Instance(dyn.problem)
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            dec_ += run_job(ffs, inst, dyn, G, stream, mode, st_)
            e.record(stream)
            e.synchronize()
            ms_ += s.elapsed_time(e)
            inst.close()
        return st_, ms_, dec_
    prof, prof_ms, prof_dec = timed_pass(2, args.steps)
    eager, eager_ms, eager_dec = timed_pass(1, min(args.steps, 3))

    # end to end through the public API: host arrays in, host schedules out, per step
    e2e_s, e2e_dec, e2e_stats = 0.0, 0, {}
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        inst = ffs.Instance(dyn.problem)
        e2e_dec += run_job(ffs, inst, dyn, G, stream, args.eager, e2e_stats)
        torch.cuda.synchronize()
        e2e_s += time.perf_counter() - t0
        inst.close()
    e2e_tot, e2e_max = aggregate(dist if world > 1 else None, float(e2e_dec), e2e_s, dev)

    avg_launch_s = prof["kernel_ms"] / prof["kernel_launches"] / 1e3   # per generation, graph mode
    eager_launch_s = eager["kernel_ms"] / eager["kernel_launches"] / 1e3
    achieved = work_per_decode() * P / avg_launch_s / 1e12
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
    alu_peak = alu_peak_tops(sms, mhz)
    line = {
        "metric": METRIC, "value": tot_decodes / max_s, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_s * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "generations_per_solve": G, "solves_per_step": len(dyn.events) + 1,
                   "decodes_per_step": decodes // args.steps, "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "wall_s": t_wall, "best_objectives_last_step": stats["best_obj"][-(len(dyn.events) + 1):],
                   "launch": "eager" if args.eager else ("captured CUDA graphs of 8 generations, each generation launched as a "
                                                         "programmatic dependent of the one before"),
                   "profiled_pass_value": prof_dec / (prof_ms / 1e3),
                   "eager_pass_value": eager_dec / (eager_ms / 1e3)},
        "e2e": {"value": e2e_tot / e2e_max, "unit": UNIT, "h2d_bytes_per_step": input_bytes(dyn),
                "d2h_bytes_per_step": e2e_stats["d2h"]},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": "fused selection/crossover/mutation/decode generation kernel",
                     "achieved": achieved, "peak": alu_peak, "unit": "Tops/s", "frac": achieved / alu_peak,
                     "peak_basis": f"{sms} SMs x 4 schedulers x 32 INT32 lanes x {mhz:.0f} MHz (median sampled SM "
                                   "clock in the timed region), derived",
                     "traffic": TRAFFIC_BYTES, "avg_launch_us": avg_launch_s * 1e6,
                     "timing": f"CUDA events around each graph replay (8 chained generations, the timed run's launch "
                               f"mode) in a pass of {args.steps} jobs: {prof['kernel_launches']} generations",
                     "eager_kernel_us": eager_launch_s * 1e6,
                     "eager_timing": f"CUDA events around the fused kernel alone, each generation launched directly, "
                                     f"{eager['kernel_launches']} launches",
                     "work_per_launch": f"{work_per_decode():.0f} INT32 ops/decode ({SLOTS_PER_DECODE:.0f} power-slot "
                                        f"checks and updates + {SORT_PER_DECODE:.0f} sort compares) x {P} decodes"},
        "clocks": clk,
    }
    if rank == 0 and not args.no_tto:
        # the metric's second half: time-to-objective of the surrogate-assisted GA against
        # the plain GA on the surrogate workload (200 jobs x 8 stages, population 4096)
        line["time_to_objective"] = time_to_objective(ffs, torch, stream)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        if args.cpu_all_cores:
            line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- batched
BATCH_WORKLOAD = ("batched: 256 independent rescheduling instances (jobs U{20..200}, stages U{3..8}, machines "
                  "U{1..6}, p U{1..99}, q U{5..30} kW, peak U{40..70}% of all-on power), each frozen at 30% of a "
                  "seeded plan's makespan with 10% new jobs; population 512 (islands of 64), one persistent "
                  "graph-captured launch per run, mapping from the autotuner")


def batched_instances(ffs, torch, count):
    """Rescheduling snapshots of the batched workload, built with the library's decoder."""
    insts = []
    for it in wl.batched(count, seed=1):
        inst = ffs.Instance(it.problem)
        y = np.random.default_rng(it.plan_seed).permutation(inst.K).astype(np.int16) + 1
        yd = torch.from_numpy(y[None, :]).cuda()
        sch = inst.decode(yd, schedule=True)
        cm = int(inst.decode(yd)["cmax"][0])
        inst.commit(sch["S"][0].cpu().numpy(), sch["M"][0].cpu().numpy())
        t_now = it.rs_permille * cm // 1000
        inst.reschedule(wl.random_arrivals(np.random.default_rng(it.arrival_seed), it.arrivals_n,
                                           it.problem.g, t_now, 99), t_now)
        insts.append(inst)
    return insts


def bench_batched(args):
    import torch

    from paper_1903_10741_gb300 import ffs

    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    count, G = args.batch_count, args.generations
    insts = batched_instances(ffs, torch, count)
    t0 = time.perf_counter()
    batch = ffs.Batch(insts, P=512, island=64, tour_k=2, pc=PC, pm=PM, migrate_every=MIGRATE, seed=SEED,
                      stream=stream)
    create_s = time.perf_counter() - t0
    if args.batch_mapping:
        w, sm, cl = (int(v) for v in args.batch_mapping.split(","))
        batch.set_config(w, sm, cl)
        chosen = batch.config()
    else:
        chosen = batch.tune(args.tune_generations)
    for _ in range(args.warmup):
        batch.run(args.tune_generations)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = ffs.kernel_launches()
    total_ms = 0.0
    for k in range(args.steps):
        flush.fill_(float(k))
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        batch.run(G)
        e.record(stream)
        e.synchronize()
        total_ms += s.elapsed_time(e)
    launches = ffs.kernel_launches() - launches0
    clk = clocks.stop()
    decodes = count * 512 * G * args.steps
    kinfo = [i.info() for i in insts]
    avg_launch_s = total_ms / args.steps / 1e3
    alu_peak = alu_peak_tops(torch.cuda.get_device_properties(local).multi_processor_count,
                             clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0)
    achieved = BATCH_SLOTS_PER_DECODE * count * 512 * G / avg_launch_s / 1e12 if BATCH_SLOTS_PER_DECODE else None
    line = {
        "metric": METRIC, "value": decodes / (total_ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "instances": count, "generations_per_step": G,
                   "genes": [min(k["n_genes"] for k in kinfo), max(k["n_genes"] for k in kinfo)],
                   "tuned_mapping": chosen, "create_and_generation0_s": create_s,
                   "l2": "flushed between steps (256 MiB write)"},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": "persistent batched GA kernel", "achieved": achieved,
                     "peak": alu_peak, "unit": "Tops/s",
                     "frac": achieved / alu_peak if achieved else None, "traffic": None,
                     "avg_launch_us": avg_launch_s * 1e6,
                     "work_per_launch": f"{BATCH_SLOTS_PER_DECODE} slot checks/decode x {count * 512 * G} decodes"},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- surrogate
SUR_WORKLOAD = ("surrogate-assisted GA: 200 jobs, 8 stages, machines U{2..6}, p U{1..99}, q U{5..50} kW, peak 50%; "
                "population 4096 (64 islands of 64), tournament 2, pc 0.8, pm 0.1, migration every 10; the plain GA "
                "runs 1000 generations and its final best total tardiness is the target; each surrogate arm "
                "over-generates F candidates per slot, scores them with the BF16 MLP (256-256-1, trained online by Adam "
                "on the kept children's exact decodes) and decodes exactly only the kept ones; time-to-objective = wall "
                "seconds until the arm's best total tardiness is within 0.5% of the target (checked every 20 generations)")
# Surrogate arms: the configuration as stated (8x over-generation, the top 12.5% of each island's
# pool decoded exactly), the same rule with parent copies kept at the plain GA's rate and only
# offspring ranked, the best per-slot screening found earlier, and -- as a diagnostic, not a
# surrogate -- the stated rule ranked by exact objectives (every candidate decoded), which
# bounds what the rule itself can give.  cap: generations as a multiple of the plain run's.
SUR_ARMS = {
    "island_top_12.5pct_of_8x": dict(oversample=8, keep=1, screen=1.0, train_steps=1, lr=1e-3, pretrain_steps=50,
                                     cap=1.0),
    "island_top_offspring_12.5pct_of_8x": dict(oversample=8, keep=2, screen=1.0, train_steps=1, lr=1e-3,
                                               pretrain_steps=50, cap=1.0),
    "slot_screen_F2_p0.5": dict(oversample=2, keep=0, screen=0.5, train_steps=2, lr=1e-3, pretrain_steps=50, cap=2.0),
    "diagnostic_exact_scores_island_top_12.5pct_of_8x": dict(oversample=8, keep=1, screen=1.0, train_steps=0, lr=1e-3,
                                                             pretrain_steps=0, cap=1.0, exact=True),
}


def time_to_objective(ffs, torch, stream, G=1000, chunk=20, cap_factor=2.0, arms=None, profile_gens=20):
    """Plain GA vs surrogate-assisted arms on the surrogate workload: the plain GA's final
    best total tardiness after G generations is the target; each arm's wall time and
    generations until its best is within 0.5 % of it; both at equal generation counts; and
    the per-generation time split of each arm (profiled eager pass of profile_gens)."""
    arms = SUR_ARMS if arms is None else arms
    prob = wl.surrogate_large(1)
    Ps = 4096
    kw = dict(P=Ps, island=64, tour_k=TOUR_K, pc=PC, pm=PM, migrate_every=MIGRATE, seed=SEED, stream=stream)
    ffs.Population(ffs.Instance(prob), **kw).run(2, want_schedule=False)  # kernels loaded, limits set

    def run_arm(arm, cap, target):
        inst = ffs.Instance(prob)
        pop = ffs.Population(inst, **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if arm is not None:
            sur = ffs.Surrogate(inst, max_batch=Ps, seed=SEED)
            if arm.get("exact"):
                sur.score_exactly(True)
            pop.attach_surrogate(sur, oversample=arm["oversample"], lr=arm["lr"], train_steps=arm["train_steps"],
                                 screen=arm["screen"], pretrain_steps=arm["pretrain_steps"], keep=arm["keep"])
        curve, reached = [], None
        for g in range(0, cap, chunk):
            n = min(chunk, cap - g)
            r = pop.run(n, want_schedule=False)
            el = time.perf_counter() - t0
            curve.append((g + n, round(el, 4), r["tard"], r["obj"]))
            if target is not None and reached is None and r["tard"] <= target * 1.005:
                reached = (g + n, el)
                break
        return curve, reached

    def split(arm, gens):
        inst = ffs.Instance(prob)
        pop = ffs.Population(inst, **kw)
        if arm is not None:
            sur = ffs.Surrogate(inst, max_batch=Ps, seed=SEED)
            if arm.get("exact"):
                sur.score_exactly(True)
            pop.attach_surrogate(sur, oversample=arm["oversample"], lr=arm["lr"], train_steps=arm["train_steps"],
                                 screen=arm["screen"], pretrain_steps=0, keep=arm["keep"])
        pop.set_profiling(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pop.run(gens, want_schedule=False)
        wall = (time.perf_counter() - t0) / gens * 1e3
        if arm is None:
            ms, n = pop.profile()
            return {"exact_decode": ms / n, "wall_ms_per_generation": wall}
        ph = pop.profile_phases()
        out = {k: v / gens for k, v in ph.items()}
        out["wall_ms_per_generation"] = wall
        return out

    plain, _ = run_arm(None, G, None)
    target = plain[-1][2]
    plain_hit = next(c for c in plain if c[2] <= target * 1.005)
    rec = {"workload": SUR_WORKLOAD, "target_total_tardiness": target, "tolerance": 0.005,
           "plain": {"generations": G, "wall_s": plain[-1][1], "generations_to_target": plain_hit[0],
                     "time_to_target_s": plain_hit[1], "final_objective": plain[-1][3],
                     "ms_per_generation": plain[-1][1] / G * 1e3, "curve": plain[::5]}}
    plain_at = {c[0]: c[2] for c in plain}
    best = None
    for name, arm in arms.items():
        curve, reached = run_arm(arm, int(arm.get("cap", cap_factor) * G), target)
        same = [(c[0], c[2], plain_at[c[0]]) for c in curve if c[0] in plain_at]
        rec[name] = {"config": arm, "reached": reached is not None,
                     "generations_to_target": reached[0] if reached else None,
                     "time_to_target_s": reached[1] if reached else None,
                     "generations_run": curve[-1][0], "wall_s": curve[-1][1],
                     "ms_per_generation": curve[-1][1] / curve[-1][0] * 1e3,
                     "speedup_vs_plain_time_to_target": (plain_hit[1] / reached[1]) if reached else None,
                     "tardiness_at_equal_generations": same[::5] + ([same[-1]] if same else []),
                     "curve": curve[::5]}
        if reached and not arm.get("exact") and (best is None or reached[1] < rec[best]["time_to_target_s"]):
            best = name
    if profile_gens:
        rec["time_split_ms_per_generation"] = {"plain": split(None, profile_gens)}
        for name, arm in arms.items():
            rec["time_split_ms_per_generation"][name] = split(arm, profile_gens)
    rec["target_met_by"] = [n for n in arms if rec[n]["reached"] and rec[n]["time_to_target_s"] < plain_hit[1]
                            and not arms[n].get("exact")]
    rec["fastest_surrogate_arm"] = best
    return rec


def bench_surrogate(args):
    import torch

    from paper_1903_10741_gb300 import ffs

    torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
    stream = torch.cuda.current_stream()
    G = args.generations
    arms = SUR_ARMS
    if args.sur_arm:  # a single arm given on the command line
        arms = {"custom": dict(oversample=args.oversample, keep=args.keep, screen=args.screen,
                               train_steps=args.train_steps, lr=args.lr, pretrain_steps=args.pretrain_steps)}
    rec = time_to_objective(ffs, torch, stream, G=G, chunk=args.chunk,
                            cap_factor=(args.surrogate_cap / G) if args.surrogate_cap else 2.0, arms=arms)
    fastest = rec["fastest_surrogate_arm"]
    line = {
        "metric": "time-to-objective, surrogate vs plain GA", "unit": "s", "higher_is_better": False,
        "value": rec[fastest]["time_to_target_s"] if fastest else None, "n_gpus": 1,
        "dtype": "int32 decode / bf16 surrogate", "data": "synthetic",
        "config": {"workload": SUR_WORKLOAD, "generations_plain": G, "chunk": args.chunk},
        "time_to_objective": rec,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- static instance
STATIC_WORKLOAD = ("static instance: 10 jobs, 3 stages with [2,3,2] identical machines, p U{1..20}, q U{1..10}, "
                   "peak 60% of all-on power, releases 0; population 64 (one island), tournament 2, pc 0.8, pm 0.1; "
                   "100 generations per step")


def bench_static(args):
    import torch

    from paper_1903_10741_gb300 import ffs

    torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
    stream = torch.cuda.current_stream()
    prob = wl.static_small(1)
    G, Ps = args.generations, 64
    kw = dict(P=Ps, island=64, tour_k=TOUR_K, pc=PC, pm=PM, migrate_every=MIGRATE, seed=SEED, stream=stream)
    for _ in range(args.warmup):
        ffs.Population(ffs.Instance(prob), **kw).run(G, want_schedule=False)
    total_ms, res = 0.0, None
    for _ in range(args.steps):
        inst = ffs.Instance(prob)
        pop = ffs.Population(inst, **kw)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        res = pop.run(G, want_schedule=False)
        e.record(stream)
        e.synchronize()
        total_ms += s.elapsed_time(e)
    line = {
        "metric": METRIC, "value": Ps * G * args.steps / (total_ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": STATIC_WORKLOAD, "generations_per_step": G, "best_objective": res["obj"],
                   "timing": "CUDA events around ga_run (the GA wall time of one run)"},
    }
    if not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        ga = oracle.GA(oracle.Instance(prob), P=Ps, island=64, tour_k=TOUR_K, pc=PC, pm=PM, migrate_every=MIGRATE,
                       seed=SEED).init().step(G)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": Ps * (G + 1) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"the whole oracle GA run ({G} generations) in {dt:.3f} s",
                                "best_objective": int(ga.bobj.min())}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- insertion placement
INS_WORKLOAD = ("idle-gap insertion placement vs Alg. 2's append placement on the dynamic rescheduling job "
                "(50 initial jobs, 5 stages x U{2..4} machines, events at t=100,250,400 adding 10 jobs; population "
                "1024, 500 generations per solve, stage-by-stage order, earliest machine)")


def bench_insert(args):
    import torch

    from paper_1903_10741_gb300 import ffs

    torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
    stream = torch.cuda.current_stream()
    dyn = wl.dynamic_medium(1)
    G = args.generations
    out = {}
    for name, mach in (("insert", ffs.MACH_EARLIEST | ffs.PLACE_INSERT), ("append", ffs.MACH_EARLIEST)):
        for rep in range(args.warmup + args.steps):
            inst = ffs.Instance(dyn.problem)
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            objs, decodes = [], 0
            for solve in range(len(dyn.events) + 1):
                pop = ffs.Population(inst, P=P, island=ISLAND, tour_k=TOUR_K, pc=PC, pm=PM, migrate_every=MIGRATE,
                                     seed=SEED, instance_id=solve, mach_mode=mach, stream=stream)
                objs.append(pop.run(G, want_schedule=False)["obj"])
                decodes += P * (G + 1) + 1
                if solve < len(dyn.events):
                    inst.reschedule(dyn.events[solve][1], dyn.events[solve][0])
            e.record(stream)
            e.synchronize()
            if rep >= args.warmup:
                out.setdefault(name, []).append((decodes / (s.elapsed_time(e) / 1e3), objs))
    v = float(np.mean([d for d, _ in out["insert"]]))
    line = {
        "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": INS_WORKLOAD, "generations_per_solve": G,
                   "append_decodes_per_s": float(np.mean([d for d, _ in out["append"]])),
                   "best_objectives_insert": out["insert"][-1][1], "best_objectives_append": out["append"][-1][1],
                   "timing": "CUDA events around each whole job, instance creation and commits included"},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- unrelated machines
UNREL_WORKLOAD = ("unrelated parallel machines (Table 2: P_jsm, Q_jsm per job and machine), earliest-completion "
                  "machine choice: 50 jobs, 5 stages x U{2..4} machines, P_jsm U{1..99}, Q_jsm U{5..30}, peak 55% "
                  "of the sum of each machine's largest power; population 1024 (16 islands of 64), tournament 2, "
                  "pc 0.8, pm 0.1; G generations of one solve per step")


def bench_unrelated(args):
    import torch

    from paper_1903_10741_gb300 import ffs

    torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
    stream = torch.cuda.current_stream()
    prob = wl.unrelated_instance(np.random.default_rng(1), 50, 5, 2, 4, 99, 5, 30, 55)
    G = args.generations
    kw = dict(P=P, island=ISLAND, tour_k=TOUR_K, pc=PC, pm=PM, migrate_every=MIGRATE, seed=SEED, stream=stream)
    for _ in range(args.warmup):
        ffs.Population(ffs.Instance(prob), **kw).run(5, want_schedule=False)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    clocks = ClockSampler(_env_int("LOCAL_RANK", 0))
    clocks.start()
    launches0 = ffs.kernel_launches()
    total_ms, best = 0.0, []
    for k in range(args.steps):
        inst = ffs.Instance(prob)
        pop = ffs.Population(inst, **kw)
        flush.fill_(float(k))
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        r = pop.run(G, want_schedule=False)
        e.record(stream)
        e.synchronize()
        total_ms += s.elapsed_time(e)
        best.append(r["obj"])
    launches = ffs.kernel_launches() - launches0
    clk = clocks.stop()
    decodes = P * G * args.steps
    line = {
        "metric": METRIC, "value": decodes / (total_ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": UNREL_WORKLOAD, "generations_per_step": G, "genes": int(inst.K),
                   "best_objectives": best, "l2": "flushed between steps (256 MiB write)",
                   "timing": "CUDA events around ga_run (its final best-schedule decode included)"},
        "gpu_launches": launches, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- static vs reactive
SVR_WORKLOAD = ("reactive vs traditional static rescheduling (Sec. 5.3, Table 10 analogue): the Test 3 setting of "
                "Sec. 5 and Table 5 -- 10 jobs, 3 stages x 2 identical machines, p U[1,5], unit power, peak 4, "
                "R U[0,Pbar], D = R + Pbar(1+U[0,2]), times on a 1/100 grid; a plan optimised by G generations is "
                "interrupted at RS = ratio x its makespan by round(ratio x 10) new jobs (R = RS + U[0,Pbar]); each "
                "arm then runs G generations; population 4096 (islands of 64), tournament 2, pc 0.9, pm 0.1; "
                "objective (Eq. 1) averaged over the seeds")


def bench_static_vs_reactive(args):
    import torch

    from paper_1903_10741_gb300 import ffs

    torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
    G, Ps = args.generations, 4096
    kw = dict(P=Ps, island=ISLAND, tour_k=TOUR_K, pc=(9, 10), pm=(1, 10), migrate_every=MIGRATE, seed=SEED)
    rows, decodes = [], 0
    t0 = time.perf_counter()
    for ratio in (20, 40, 60, 80):
        obj = {"static": [], "reactive": [], "reactive_warm": []}
        for seed in range(1, args.svr_seeds + 1):
            prob = wl.table5_instance(10, 3, 2, 4, seed=seed)
            for arm in obj:
                inst = ffs.Instance(prob)
                plan = ffs.Population(inst, **kw, instance_id=0)
                r0 = plan.run(G)  # the original plan, committed
                rs = ratio * r0["cmax"] // 100
                arr = wl.table5_arrivals(np.random.default_rng(1000 * ratio + seed), (ratio * prob.N + 50) // 100,
                                         prob.g, rs)
                inst.reschedule(arr, rs, static=arm == "static")
                pop = ffs.Population(inst, **kw, instance_id=1, prev=plan if arm == "reactive_warm" else None)
                obj[arm].append(pop.run(G)["obj"])
                decodes += 2 * (Ps * (G + 1) + 1)
        m = {k: float(np.mean(v)) for k, v in obj.items()}
        rows.append({"ratio_pct": ratio, **m, "static_over_reactive": m["static"] / m["reactive"],
                     "static_over_reactive_warm": m["static"] / m["reactive_warm"]})
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    line = {
        "metric": "objective ratio, traditional static / predictive-reactive (Table 10 analogue)",
        "value": rows[0]["static_over_reactive_warm"], "unit": "ratio at RS = 20% of the makespan, warm reactive",
        "higher_is_better": True, "n_gpus": 1, "dtype": "int32", "data": "synthetic",
        "config": {"workload": SVR_WORKLOAD, "generations": G, "seeds": args.svr_seeds, "rows": rows,
                   "arms": "static: plan kept, new jobs appended (ffs_reschedule_static); reactive: complete "
                           "rescheduling from a random population (the paper's); reactive_warm: complete "
                           "rescheduling from the plan's population carried over (ga_population_create_warm)",
                   "paper_table10_improvement": {"20": 2.28, "40": 1.50, "60": 1.17, "80": 1.01},
                   "note": "paper values are for its own instance (K40 runs); shown for the trend only"},
        "decodes_per_s": decodes / wall, "wall_s": wall,
    }
    print(json.dumps(line), flush=True)


# Slot checks per decode of the batched workload, measured by the oracle (python -m
# oracle.work_per_decode --workload batched --samples 8): mean over the 256 rescheduling
# snapshots of 8 uniformly random chromosomes each (min 6038, max 392743 per instance).
BATCH_SLOTS_PER_DECODE = 112338.4


# ----------------------------------------------------------------------------- service
SVC_WORKLOAD = ("rescheduling service: 16 instances (N U{50..500}, g U{5..10}, machines U{2..8}, p U{1..199}, "
                "q U{5..30} kW, peak U{40..70}%); requests arrive as a Poisson process (50/s), each for a uniform "
                "instance: its first request solves it at t=0, later ones advance its clock by U{5..15}% of its "
                "stage load and bring U{5..50} jobs; population 2048 (islands of 64) warm-started from the "
                "instance's last population, 200 generations per request")


def run_service(ffs, work, G, ga_kw, max_active, memory_gb, local):
    """Submits `work`'s requests at their arrival times to a fresh service over fresh
    instances, waits for all of them; returns latency percentiles and throughput."""
    insts = [ffs.Instance(p) for p in work.problems]
    svc = ffs.Service(max_active=max_active, memory_bytes=int(memory_gb * (1 << 30)), **ga_kw)
    launches0 = ffs.kernel_launches()
    t0 = time.perf_counter()
    tickets = []
    for r in work.requests:
        dt = t0 + r.at - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        tickets.append(svc.submit(insts[r.instance], r.arrivals, r.t_now, G))
    infos = [svc.wait(t) for t in tickets]
    wall = time.perf_counter() - t0
    stats = svc.stats()
    svc.close()
    lat = sorted((i["done_ns"] - i["submit_ns"]) / 1e6 for i in infos)
    queue = sorted((i["admit_ns"] - i["submit_ns"]) / 1e6 for i in infos)
    run = sorted((i["done_ns"] - i["admit_ns"]) / 1e6 for i in infos)

    def pct(v, q):
        return v[min(len(v) - 1, int(round(q / 100 * (len(v) - 1))))]

    P_ = ga_kw["P"]
    return {"requests": len(infos), "genes": [min(i.K for i in insts), max(i.K for i in insts)],
            "arrival_window_s": work.requests[-1].at,
            "offered_rate_per_s": len(infos) / max(work.requests[-1].at, 1e-9), "wall_s": wall,
            "requests_per_s": len(infos) / wall,
            "decodes": sum(P_ * (i["generations"] + 1) + 1 for i in infos),
            "p50_latency_ms": pct(lat, 50), "p99_latency_ms": pct(lat, 99),
            "p50_queue_ms": pct(queue, 50), "p99_queue_ms": pct(queue, 99),
            "p50_run_ms": pct(run, 50), "p99_run_ms": pct(run, 99),
            "warm_starts": sum(i["warm"] for i in infos), "peak_memory_bytes": stats["peak_bytes"],
            "failed": stats["failed"], "launches": ffs.kernel_launches() - launches0,
            "d2h": sum(8 * i["n_ops"] + 20 for i in infos),
            "h2d": sum(np.asarray(a, np.int32).nbytes for p in work.problems for a in (p.o, p.p, p.q, p.R, p.D))
            + sum(r.arrivals.p.nbytes + r.arrivals.R.nbytes + r.arrivals.D.nbytes
                  for r in work.requests if r.arrivals is not None)}


def bench_service(args):
    import torch

    from paper_1903_10741_gb300 import ffs

    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    G, Ps = args.generations, 2048
    ga_kw = dict(P=Ps, island=64, tour_k=TOUR_K, pc=PC, pm=PM, migrate_every=MIGRATE, seed=SEED)
    # warm-up: load the kernels and set their shared-memory limits on a small stream
    warm = wl.service_small(seed=99, n_instances=3, n_requests=max(3, args.warmup))
    wi = [ffs.Instance(p) for p in warm.problems]
    svc = ffs.Service(max_active=args.max_active, memory_bytes=1 << 30, **ga_kw)
    for t in [svc.submit(wi[r.instance], r.arrivals, r.t_now, 5) for r in warm.requests]:
        svc.wait(t, schedule=False)
    svc.close()

    clocks = ClockSampler(local)
    clocks.start()
    # (1) the stated arrival rate (50/s): far above what one GPU completes at these sizes,
    # so it measures the capacity (requests completed per second under a full queue)
    burst = run_service(ffs, wl.service(seed=1, n_requests=args.service_requests, rate=args.rate), G, ga_kw,
                        args.max_active, args.service_memory_gb, local)
    capacity = burst["requests_per_s"]
    # (2) at offered rates the GPU sustains, over `service_seconds` of Poisson arrivals
    sustained = []
    for frac in ([0.5, 1.0] if args.service_seconds > 0 else []):
        rate = frac * capacity
        # every arrival of the first `service_seconds` of the process (the same instance
        # and request draws as the burst, only the gaps scaled)
        work = wl.service(seed=1, n_requests=int(np.ceil(2 * args.service_seconds * rate)) + 16, rate=rate)
        work.requests[:] = [r for r in work.requests if r.at <= args.service_seconds]
        rec = run_service(ffs, work, G, ga_kw, args.max_active, args.service_memory_gb, local)
        rec["fraction_of_capacity"] = frac
        rec["process_rate_per_s"] = rate
        sustained.append(rec)
    clk = clocks.stop()
    line = {
        "metric": METRIC, "value": burst["decodes"] / burst["wall_s"], "unit": UNIT, "n_gpus": 1, "steps": 1,
        "warmup": args.warmup, "ms_per_step": burst["wall_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": SVC_WORKLOAD, "requests": burst["requests"], "offered_rate_per_s": args.rate,
                   "arrival_window_s": burst["arrival_window_s"], "generations_per_request": G,
                   "max_active": args.max_active, "service_memory_gb": args.service_memory_gb,
                   "genes": burst["genes"], "sustained_arrivals_s": args.service_seconds},
        "service": {k: burst[k] for k in ("p50_latency_ms", "p99_latency_ms", "p50_queue_ms", "p99_queue_ms",
                                           "p50_run_ms", "p99_run_ms", "requests_per_s", "warm_starts",
                                           "peak_memory_bytes", "failed")},
        "capacity_rps": capacity,
        "sustained_rates": [{k: r[k] for k in ("fraction_of_capacity", "process_rate_per_s", "offered_rate_per_s",
                                               "requests", "arrival_window_s", "requests_per_s", "p50_latency_ms",
                                               "p99_latency_ms", "p50_queue_ms", "p99_queue_ms", "p50_run_ms",
                                               "p99_run_ms", "warm_starts", "failed")} for r in sustained],
        "e2e": {"value": burst["decodes"] / burst["wall_s"], "unit": UNIT, "h2d_bytes_per_step": burst["h2d"],
                "d2h_bytes_per_step": burst["d2h"],
                "note": "the whole run is end to end: host arrays in, host schedules out, through ffs_service_*"},
        "gpu_launches": burst["launches"],
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- oracle
def _oracle_ga(dyn):
    import oracle
    inst = oracle.Instance(dyn.problem)
    return oracle.GA(inst, P=P, island=ISLAND, tour_k=TOUR_K, pc=PC, pm=PM, migrate_every=MIGRATE,
                     seed=SEED, instance_id=0).init()


def cpu_baseline(seconds: float) -> dict:
    """The oracle GA, single-threaded, on the initial solve of the same job for about
    `seconds` of CPU time."""
    dyn = wl.dynamic_medium(1)
    t0 = time.perf_counter()
    ga = _oracle_ga(dyn)
    gens = 0
    while time.perf_counter() - t0 < seconds:
        ga.step()
        gens += 1
    dt = time.perf_counter() - t0
    dec = P * (gens + 1)
    return {"value": dec / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle GA on the initial solve (population {P}): init + {gens} generations, "
                      f"{dec} exact decodes in {dt:.1f} s"}


def _oracle_decode_slice(args):
    """Worker of the all-cores oracle baseline: decode rows [lo, hi) of the generation-0
    population of the job's initial solve, repeatedly, for `seconds`."""
    lo, hi, seconds = args
    import oracle
    dyn = wl.dynamic_medium(1)
    inst = oracle.Instance(dyn.problem)
    ga = oracle.GA(inst, P=P, island=ISLAND, tour_k=TOUR_K, pc=PC, pm=PM, migrate_every=MIGRATE, seed=SEED,
                   instance_id=0).init()
    rows = ga.Y[lo:hi, :ga.K].copy()
    t0, n = time.perf_counter(), 0
    while time.perf_counter() - t0 < seconds:
        for y in rows:
            inst.decode(y)
            n += 1
    return n, time.perf_counter() - t0


def cpu_baseline_all_cores(seconds: float) -> dict:
    """The same oracle decoder as os.cpu_count() independent processes, each on its own
    slice of the initial solve's population (the paper's 1-core vs multi-core comparison).
    Processes are spawned, never forked from a process that has used the GPU."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    bounds = [(P * i // cores, P * (i + 1) // cores, seconds) for i in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_decode_slice, bounds)
    dec = sum(n for n, _ in res)
    wall = max(t for _, t in res)
    return {"value": dec / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} spawned processes decoding disjoint slices of the initial solve's population "
                      f"(population {P}) for about {seconds:.0f} s: {dec} exact decodes"}


def bench_reference(args):
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    dyn = wl.dynamic_medium(1)
    ga = _oracle_ga(dyn)
    for _ in range(args.warmup):
        ga.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ga.step(args.ref_generations)
    dt = time.perf_counter() - t0
    dec = P * args.ref_generations * args.steps
    v = dec / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{args.ref_generations} oracle GA generations per step "
                                                   "on the initial solve"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} x {args.ref_generations} generations x {P} decodes"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--generations", type=int, default=500, help="GA generations per solve")
    ap.add_argument("--ref-generations", type=int, default=2, help="oracle generations per reference step")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-all-cores", action="store_true",
                    help="also time the oracle as one process per host core on disjoint slices")
    ap.add_argument("--workload", choices=["dynamic", "batched", "surrogate", "service", "static-vs-reactive",
                                           "unrelated", "insert", "static"],
                    default="dynamic",
                    help="dynamic: the headline rescheduling job; batched: 256 uneven instances; "
                         "surrogate: time-to-objective of the surrogate-assisted GA; service: Poisson "
                         "rescheduling requests through the continuous-batching service")
    ap.add_argument("--service-requests", type=int, default=48)
    ap.add_argument("--service-seconds", type=float, default=60.0,
                    help="service: seconds of Poisson arrivals at 0.5x and 1x the measured capacity (0: skip)")
    ap.add_argument("--svr-seeds", type=int, default=20, help="instances per ratio (static-vs-reactive)")
    ap.add_argument("--rate", type=float, default=50.0, help="service request arrival rate (1/s)")
    ap.add_argument("--max-active", type=int, default=8, help="service requests on the device at once")
    ap.add_argument("--service-memory-gb", type=float, default=32.0)
    ap.add_argument("--chunk", type=int, default=20, help="generations between progress checks (surrogate)")
    ap.add_argument("--lr", type=float, default=1e-3, help="surrogate learning rate")
    ap.add_argument("--surrogate-cap", type=int, default=0, help="generation cap of the surrogate run")
    ap.add_argument("--train-steps", type=int, default=2, help="surrogate Adam steps per generation")
    ap.add_argument("--oversample", type=int, default=2, help="surrogate candidates per population slot")
    ap.add_argument("--screen", type=float, default=0.5, help="fraction of offspring slots that take the surrogate's pick")
    ap.add_argument("--pretrain-steps", type=int, default=50, help="surrogate Adam steps on generation 0")
    ap.add_argument("--keep", type=int, default=0, help="surrogate keep rule: 0 per-slot screening, 1 island top")
    ap.add_argument("--sur-arm", action="store_true",
                    help="surrogate workload: run only the arm given by --oversample/--keep/--screen/...")
    ap.add_argument("--no-tto", action="store_true",
                    help="default workload: skip the time-to-objective record of the surrogate workload")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--tune-generations", type=int, default=3)
    ap.add_argument("--batch-mapping", default="",
                    help="warps,smem_bytes,cluster of the batched kernel instead of autotuning")
    ap.add_argument("--eager", action="store_true",
                    help="launch every generation directly instead of replaying its CUDA graph "
                         "(for profilers that cannot follow graph launches)")
    args = ap.parse_args()
    if args.impl == "reference":
        bench_reference(args)
    elif args.workload == "batched":
        if args.generations == 500:
            args.generations = 300
        bench_batched(args)
    elif args.workload == "surrogate":
        if args.generations == 500:
            args.generations = 1000
        bench_surrogate(args)
    elif args.workload == "static":
        if args.generations == 500:
            args.generations = 100
        bench_static(args)
    elif args.workload == "insert":
        bench_insert(args)
    elif args.workload == "unrelated":
        bench_unrelated(args)
    elif args.workload == "static-vs-reactive":
        if args.generations == 500:
            args.generations = 100
        bench_static_vs_reactive(args)
    elif args.workload == "service":
        if args.generations == 500:
            args.generations = 200
        bench_service(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
