"""Algorithmic work per exact decode on the dynamic rescheduling workload, from the oracle.

TEST INFRASTRUCTURE: runs only the CPU oracle.  It replays the benchmark's job (50 jobs,
5 stages, population 1024, 500 generations at each of the initial solve and the three
rescheduling events) in the oracle GA and, every `--every` generations, decodes the whole
population to average the oracle's `slots` count: for every op, over every machine tried,
(earliest feasible start - earliest availability + p), plus p for the profile update.
That is the number of per-instant power checks (Eq. 7) and updates (Eq. 8) an exact
evaluation performs.  The stage-by-stage order adds a sort of each stage's free ops by
priority: sum over stages of n_s * ceil(log2 n_s) comparisons (n_s free ops at stage s),
a property of the instance at each rescheduling point.  Prints one JSON line.

    python -m oracle.work_per_decode --generations 500 --every 50
    python -m oracle.work_per_decode --workload batched --samples 8

The batched workload's figure averages, over its 256 rescheduling snapshots (each built
with the oracle's own decoder: a seeded plan, frozen at 30% of its makespan, 10% new jobs),
the slots of `--samples` uniformly random chromosomes per instance; every instance counts
equally because each decodes the same population size per generation.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_1903_10741_gb300 import workloads as wl  # noqa: E402


def batched(samples: int):
    per_inst = []
    for it in wl.batched(256, seed=1):
        inst = oracle.Instance(it.problem)
        y = np.random.default_rng(it.plan_seed).permutation(inst.K).astype(np.int16) + 1
        r = inst.decode(y)
        inst.commit(r["S"], r["M"])
        t_now = it.rs_permille * r["cmax"] // 1000
        inst.reschedule(wl.random_arrivals(np.random.default_rng(it.arrival_seed), it.arrivals_n,
                                           it.problem.g, t_now, 99), t_now)
        rng = np.random.default_rng(0)
        s = [inst.decode(rng.permutation(inst.K) + 1)["slots"] for _ in range(samples)]
        per_inst.append(float(np.mean(s)))
    print(json.dumps(dict(workload="batched(256, seed=1)", samples=samples,
                          slots_per_decode=float(np.mean(per_inst)),
                          min=min(per_inst), max=max(per_inst))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["dynamic", "batched"], default="dynamic")
    ap.add_argument("--samples", type=int, default=8)
    ap.add_argument("--generations", type=int, default=500)
    ap.add_argument("--every", type=int, default=50)
    ap.add_argument("--pop", type=int, default=1024)
    a = ap.parse_args()
    if a.workload == "batched":
        batched(a.samples)
        return
    dyn = wl.dynamic_medium(1)
    inst = oracle.Instance(dyn.problem)
    per_solve = []
    for solve in range(len(dyn.events) + 1):
        ga = oracle.GA(inst, P=a.pop, island=64, tour_k=2, pc=(4, 5), pm=(1, 10), seed=1,
                       instance_id=solve).init()
        samples = []
        for g in range(a.generations + 1):
            if g % a.every == 0:
                s = [inst.decode(ga.Y[i, :ga.K], None)["slots"] for i in range(a.pop)]
                samples.append(float(np.mean(s)))
            if g < a.generations:
                ga.step()
        y, x, _ = ga.best()
        r = inst.decode(y, x)
        _, gs = inst.gene_map()
        n_s = np.bincount(gs, minlength=inst.g)
        sort = int(sum(int(n) * int(np.ceil(np.log2(n))) for n in n_s if n > 1))
        per_solve.append(dict(K=ga.K, N=inst.N, rs=inst.RS, slots_mean=float(np.mean(samples)),
                              slots_first=samples[0], slots_last=samples[-1], sort_compares=sort,
                              best_obj=r["obj"]))
        inst.commit(r["S"], r["M"])
        if solve < len(dyn.events):
            t_now, arr = dyn.events[solve]
            inst.reschedule(arr, t_now)
    mean = float(np.mean([p["slots_mean"] for p in per_solve]))
    sort = float(np.mean([p["sort_compares"] for p in per_solve]))
    print(json.dumps(dict(workload="dynamic_medium(seed=1)", pop=a.pop, generations=a.generations,
                          every=a.every, slots_per_decode=mean, sort_compares_per_decode=sort,
                          work_per_decode=mean + sort, per_solve=per_solve)))


if __name__ == "__main__":
    main()
