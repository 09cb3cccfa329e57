"""Seeded synthetic EDFFS inputs.

This module only draws numbers: it builds problem instances (processing times, machine
powers, release and due dates, peak-power limit) and arrival events with the shapes and
value distributions of the workloads the library is measured on.  It holds none of the
method's arithmetic (no freezing, decoding, objective or GA step), so both the CUDA path
and the CPU oracle can consume its output.

Problem data follow Table 2 of the paper (Sec. 3.2): ``N`` jobs, ``g`` stages, ``o[s]``
identical parallel machines at stage ``s`` (processing time ``p[j, s]`` does not depend on
the machine, Table 5 reading), power ``q[m]`` per stage-machine (machines numbered
stage-major), release ``R[j]``, due ``D[j]``, peak limit ``Qmax``, tardiness weight ``WT``.
All values are int32.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

WT_DEFAULT = 100  # Table 5: WT = 100


@dataclass
class Problem:
    """An EDFFS instance (Table 2).  Arrays are int32 and C-contiguous."""

    o: np.ndarray            # [g] machines per stage
    p: np.ndarray            # [N, g] processing times
    q: np.ndarray            # [sum(o)] power per machine, stage-major
    R: np.ndarray            # [N] release times
    D: np.ndarray            # [N] due times
    Qmax: int                # peak power limit (Eq. 7)
    WT: int = WT_DEFAULT     # weight of total tardiness (Eq. 1)
    pm: np.ndarray = None    # [N, sum(o)] P_jsm per machine (unrelated machines), or None
    qm: np.ndarray = None    # [N, sum(o)] Q_jsm per machine, or None (then q per machine)

    def __post_init__(self):
        self.o = np.ascontiguousarray(self.o, dtype=np.int32)
        self.p = np.ascontiguousarray(self.p, dtype=np.int32)
        self.q = np.ascontiguousarray(self.q, dtype=np.int32)
        self.R = np.ascontiguousarray(self.R, dtype=np.int32)
        self.D = np.ascontiguousarray(self.D, dtype=np.int32)
        self.Qmax = int(self.Qmax)
        self.WT = int(self.WT)
        if self.pm is not None:
            self.pm = np.ascontiguousarray(self.pm, dtype=np.int32)
            self.qm = np.ascontiguousarray(self.qm, dtype=np.int32)

    @property
    def N(self) -> int:
        return int(self.p.shape[0])

    @property
    def g(self) -> int:
        return int(self.o.shape[0])

    @property
    def M(self) -> int:
        return int(self.o.sum())


@dataclass
class Arrivals:
    """New jobs J' arriving at a rescheduling point (Sec. 4.1)."""

    p: np.ndarray  # [n', g]
    R: np.ndarray  # [n']
    D: np.ndarray  # [n']
    pm: np.ndarray = None  # [n', sum(o)] P_jsm per machine (unrelated machines), or None
    qm: np.ndarray = None  # [n', sum(o)] Q_jsm per machine, or None

    def __post_init__(self):
        self.p = np.ascontiguousarray(self.p, dtype=np.int32)
        self.R = np.ascontiguousarray(self.R, dtype=np.int32)
        self.D = np.ascontiguousarray(self.D, dtype=np.int32)
        if self.pm is not None:
            self.pm = np.ascontiguousarray(self.pm, dtype=np.int32)
            self.qm = np.ascontiguousarray(self.qm, dtype=np.int32)

    @property
    def n(self) -> int:
        return int(self.p.shape[0])


@dataclass
class DynamicWorkload:
    """An initial problem plus a list of (t_now, arrivals) rescheduling events."""

    problem: Problem
    events: List[Tuple[int, Arrivals]] = field(default_factory=list)


def _u(rng: np.random.Generator, lo: int, hi: int, size=None) -> np.ndarray:
    """Inclusive integer uniform U{lo..hi}."""
    return rng.integers(lo, hi + 1, size=size, dtype=np.int64)


def _due(rng, release: np.ndarray, work: np.ndarray, f_lo: int, f_hi: int) -> np.ndarray:
    """D = R + floor(work * f / 1000) with f ~ U{f_lo..f_hi} per mille."""
    f = _u(rng, f_lo, f_hi, size=work.shape[0])
    return (release.astype(np.int64) + (work.astype(np.int64) * f) // 1000).astype(np.int32)


def _powers(rng, o: np.ndarray, q_lo: int, q_hi: int, pct_num: int, pct_den: int = 100):
    """Draw machine powers and Qmax = floor(pct * sum(q)); redraw until every single
    machine fits under the peak (otherwise no schedule exists)."""
    M = int(o.sum())
    for _ in range(1000):
        q = _u(rng, q_lo, q_hi, size=M)
        qmax = int(q.sum()) * pct_num // pct_den
        if q.max() <= qmax:
            return q.astype(np.int32), qmax
    raise RuntimeError("could not draw a feasible power table")


def static_small(seed: int = 1) -> Problem:
    """Static single instance: 10 jobs, 3 stages with [2, 3, 2] identical machines,
    p ~ U{1..20}, q ~ U{1..10}, Qmax = floor(60% of all-on power), all releases 0,
    D = floor(work * U{1000..1500} / 1000)."""
    rng = np.random.default_rng(seed)
    o = np.array([2, 3, 2], dtype=np.int32)
    N = 10
    p = _u(rng, 1, 20, size=(N, 3))
    q, qmax = _powers(rng, o, 1, 10, 60)
    R = np.zeros(N, dtype=np.int32)
    D = _due(rng, R, p.sum(axis=1), 1000, 1500)
    return Problem(o=o, p=p, q=q, R=R, D=D, Qmax=qmax)


def _arrivals(rng, n: int, g: int, t_now: int, p_lo: int, p_hi: int, f_lo: int, f_hi: int) -> Arrivals:
    p = _u(rng, p_lo, p_hi, size=(n, g))
    R = np.full(n, t_now, dtype=np.int32)
    D = _due(rng, R, p.sum(axis=1), f_lo, f_hi)
    return Arrivals(p=p, R=R, D=D)


def dynamic_medium(seed: int = 1) -> DynamicWorkload:
    """Dynamic rescheduling: 50 initial jobs, 5 stages with U{2..4} machines each,
    p ~ U{1..99}, q ~ U{5..30}, Qmax = floor(55% of all-on power), releases 0; events at
    t = 100, 250, 400 each adding 10 jobs released at the event with
    D = t + floor(work * U{1200..2000} / 1000).  Initial jobs use the same due factor."""
    rng = np.random.default_rng(seed)
    g, N = 5, 50
    o = _u(rng, 2, 4, size=g).astype(np.int32)
    p = _u(rng, 1, 99, size=(N, g))
    q, qmax = _powers(rng, o, 5, 30, 55)
    R = np.zeros(N, dtype=np.int32)
    D = _due(rng, R, p.sum(axis=1), 1200, 2000)
    prob = Problem(o=o, p=p, q=q, R=R, D=D, Qmax=qmax)
    events = [(t, _arrivals(rng, 10, g, t, 1, 99, 1200, 2000)) for t in (100, 250, 400)]
    return DynamicWorkload(problem=prob, events=events)


def random_instance(rng: np.random.Generator, N: int, g: int, o_lo: int, o_hi: int,
                    p_hi: int, q_lo: int, q_hi: int, pct: int, f_lo: int = 1200,
                    f_hi: int = 2000, p_lo: int = 1, release_hi: int = 0) -> Problem:
    """A generic instance with the given size and value ranges (all inclusive)."""
    o = _u(rng, o_lo, o_hi, size=g).astype(np.int32)
    p = _u(rng, p_lo, p_hi, size=(N, g))
    q, qmax = _powers(rng, o, q_lo, q_hi, pct)
    R = _u(rng, 0, release_hi, size=N).astype(np.int32) if release_hi > 0 else np.zeros(N, np.int32)
    D = _due(rng, R, p.sum(axis=1), f_lo, f_hi)
    return Problem(o=o, p=p, q=q, R=R, D=D, Qmax=qmax)


def random_arrivals(rng: np.random.Generator, n: int, g: int, t_now: int, p_hi: int,
                    f_lo: int = 1200, f_hi: int = 2000) -> Arrivals:
    return _arrivals(rng, n, g, t_now, 1, p_hi, f_lo, f_hi)


@dataclass
class BatchItem:
    """One instance of the batched workload: an initial problem, a seeded priority
    vector for the plan that was being executed, the rescheduling point as a fraction of
    that plan's makespan, and the jobs that arrive there."""

    problem: Problem
    plan_seed: int
    rs_permille: int
    arrivals_n: int
    arrival_seed: int


def batched(count: int = 256, seed: int = 1, n_lo: int = 20, n_hi: int = 200,
            g_lo: int = 3, g_hi: int = 8) -> List[BatchItem]:
    """Batched rescheduling: instances of uneven size, N ~ U{20..200}, g ~ U{3..8},
    machines U{1..6} per stage, p ~ U{1..99}, q ~ U{5..30}, peak U{40..70}% of the all-on
    power; each is rescheduled at 30% of an initial plan's makespan with 10% new jobs."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed * 1_000_003 + i)
        N = int(_u(rng, n_lo, n_hi))
        g = int(_u(rng, g_lo, g_hi))
        pct = int(_u(rng, 40, 70))
        prob = random_instance(rng, N, g, 1, 6, 99, 5, 30, pct)
        out.append(BatchItem(problem=prob, plan_seed=int(rng.integers(1, 2**31)),
                             rs_permille=300, arrivals_n=max(1, N // 10),
                             arrival_seed=int(rng.integers(1, 2**31))))
    return out


@dataclass
class ServiceRequest:
    """One rescheduling request of the service workload."""

    at: float                 # arrival time in seconds after the start (Poisson process)
    instance: int             # index into the workload's instance pool
    t_now: int                # rescheduling point; 0 for an instance's first request
    arrivals: Arrivals = None  # new jobs (None for an instance's first request)


@dataclass
class ServiceWorkload:
    problems: List[Problem]
    requests: List[ServiceRequest]


def service(seed: int = 1, n_instances: int = 16, n_requests: int = 48, rate: float = 50.0,
            n_range=(50, 500), g_range=(5, 10), o_range=(2, 8), p_hi: int = 199, q_range=(5, 30),
            pct_range=(40, 70), new_jobs=(5, 50), advance_pct=(5, 15)) -> ServiceWorkload:
    """Rescheduling service: a pool of instances (N ~ U{50..500}, g ~ U{5..10}, machines
    U{2..8} per stage, p ~ U{1..199}, q ~ U{5..30}, peak U{40..70}% of the all-on power) and
    requests arriving as a Poisson process of the given rate, each for a uniformly drawn
    instance.  An instance's first request solves it from scratch at t_now = 0; every
    later one moves its clock on by U{5..15}% of W = max_s (sum_j p_js) / o_s and brings
    U{5..50} jobs released at t_now (due factor U{1.2..2.0} of their work)."""
    rng = np.random.default_rng(seed)
    problems, clock, width = [], [], []
    for _ in range(n_instances):
        N = int(_u(rng, *n_range))
        g = int(_u(rng, *g_range))
        pct = int(_u(rng, *pct_range))
        prob = random_instance(rng, N, g, o_range[0], o_range[1], p_hi, q_range[0], q_range[1], pct)
        problems.append(prob)
        clock.append(None)
        width.append(int(max(prob.p[:, s].sum() // prob.o[s] for s in range(g))))
    reqs, t = [], 0.0
    for _ in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        i = int(rng.integers(0, n_instances))
        if clock[i] is None:
            clock[i] = 0
            reqs.append(ServiceRequest(at=t, instance=i, t_now=0, arrivals=None))
            continue
        clock[i] += max(1, width[i] * int(_u(rng, *advance_pct)) // 100)
        n = int(_u(rng, *new_jobs))
        reqs.append(ServiceRequest(at=t, instance=i, t_now=clock[i],
                                   arrivals=random_arrivals(rng, n, problems[i].g, clock[i], p_hi)))
    return ServiceWorkload(problems=problems, requests=reqs)


def service_small(seed: int = 1, n_instances: int = 5, n_requests: int = 15) -> ServiceWorkload:
    """A small service workload for parity tests: N ~ U{8..20}, g ~ U{2..4}, machines
    U{1..3}, p ~ U{1..30}, new jobs U{1..4}."""
    return service(seed, n_instances, n_requests, rate=1000.0, n_range=(8, 20), g_range=(2, 4),
                   o_range=(1, 3), p_hi=30, new_jobs=(1, 4), advance_pct=(10, 30))


def surrogate_large(seed: int = 1) -> Problem:
    """Surrogate-assisted workload: 200 jobs, 8 stages, machines U{2..6}, p ~ U{1..99},
    q ~ U{5..50}, Qmax = floor(50% of all-on power)."""
    rng = np.random.default_rng(seed)
    return random_instance(rng, 200, 8, 2, 6, 99, 5, 50, 50)


def table5_instance(n: int, g: int, o: int, qmax: int, seed: int = 1, scale: int = 100) -> Problem:
    """Table 5 generator, scaled to integers by ``scale``: p ~ U[1, 5] identical on every
    machine, q = 1, R ~ U[0, Pbar] with Pbar = sum_s p_js, D = R + Pbar (1 + sigma),
    sigma ~ U[0, 2].  Continuous draws are rounded to 1/scale."""
    rng = np.random.default_rng(seed)
    p = np.rint(rng.uniform(1, 5, size=(n, g)) * scale).astype(np.int64)
    pbar = p.sum(axis=1)
    R = np.rint(rng.uniform(0, 1, size=n) * pbar).astype(np.int64)
    sigma = rng.uniform(0, 2, size=n)
    D = R + np.rint(pbar * (1 + sigma)).astype(np.int64)
    o_arr = np.full(g, o, dtype=np.int32)
    q = np.ones(g * o, dtype=np.int32)
    return Problem(o=o_arr, p=p, q=q, R=R, D=D, Qmax=qmax, WT=WT_DEFAULT)


def _unrelated_tables(rng, n: int, o: np.ndarray, p_lo: int, p_hi: int, q_lo: int, q_hi: int):
    """P_jsm ~ U{p_lo..p_hi}, Q_jsm ~ U{q_lo..q_hi} per job and machine; p [n, g] is the
    fastest machine's time of each op (a per-op summary; schedules read pm)."""
    M = int(o.sum())
    pm = _u(rng, p_lo, p_hi, size=(n, M)).astype(np.int32)
    qm = _u(rng, q_lo, q_hi, size=(n, M)).astype(np.int32)
    off = np.concatenate([[0], np.cumsum(o)])
    p = np.stack([pm[:, off[s]:off[s + 1]].min(axis=1) for s in range(len(o))], axis=1)
    return p, pm, qm


def unrelated_instance(rng: np.random.Generator, N: int, g: int, o_lo: int, o_hi: int, p_hi: int,
                       q_lo: int, q_hi: int, pct: int, f_lo: int = 1200, f_hi: int = 2000) -> Problem:
    """Unrelated parallel machines (Table 2: P_jsm and Q_jsm differ per job and machine):
    P_jsm ~ U{1..p_hi}, Q_jsm ~ U{q_lo..q_hi}, Qmax = floor(pct% of the sum over machines of
    their largest Q_jsm), raised to the largest single Q_jsm; releases 0, D = floor(work *
    U{f_lo..f_hi} / 1000) with work the sum of the fastest machines' times."""
    o = _u(rng, o_lo, o_hi, size=g).astype(np.int32)
    p, pm, qm = _unrelated_tables(rng, N, o, 1, p_hi, q_lo, q_hi)
    qmax = max(int(qm.max(axis=0).sum()) * pct // 100, int(qm.max()))
    R = np.zeros(N, dtype=np.int32)
    D = _due(rng, R, p.sum(axis=1), f_lo, f_hi)
    return Problem(o=o, p=p, q=qm.max(axis=0), R=R, D=D, Qmax=qmax, pm=pm, qm=qm)


def unrelated_arrivals(rng: np.random.Generator, n: int, o: np.ndarray, t_now: int, p_hi: int, q_lo: int,
                       q_hi: int, qmax: int, f_lo: int = 1200, f_hi: int = 2000) -> Arrivals:
    """New jobs for an unrelated-machine instance, released at t_now; powers capped at Qmax."""
    p, pm, qm = _unrelated_tables(rng, n, np.asarray(o), 1, p_hi, q_lo, q_hi)
    qm = np.minimum(qm, qmax).astype(np.int32)
    R = np.full(n, t_now, dtype=np.int64)
    return Arrivals(p=p, R=R, D=_due(rng, R, p.sum(axis=1), f_lo, f_hi), pm=pm, qm=qm)


def table5_arrivals(rng: np.random.Generator, n: int, g: int, t_now: int, scale: int = 100) -> Arrivals:
    """New jobs for a Table 5 instance at rescheduling point t_now: p ~ U[1, 5] per stage,
    R = t_now + U[0, Pbar], D = R + Pbar (1 + sigma), sigma ~ U[0, 2], on the same 1/scale
    grid as table5_instance."""
    p = np.rint(rng.uniform(1, 5, size=(n, g)) * scale).astype(np.int64)
    pbar = p.sum(axis=1)
    R = t_now + np.rint(rng.uniform(0, 1, size=n) * pbar).astype(np.int64)
    D = R + np.rint(pbar * (1 + rng.uniform(0, 2, size=n))).astype(np.int64)
    return Arrivals(p=p, R=R, D=D)


def random_chromosomes(rng: np.random.Generator, count: int, K: int, gene_machines: np.ndarray):
    """``count`` random chromosomes over K genes: Y rows are permutations of 1..K
    (int16), X rows are uniform machine indices below ``gene_machines[k]`` (int8)."""
    Y = np.empty((count, K), dtype=np.int16)
    for i in range(count):
        Y[i] = rng.permutation(K) + 1
    X = (rng.random((count, K)) * gene_machines[None, :]).astype(np.int8)
    return Y, X
