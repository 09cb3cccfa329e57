"""Independent checks of a decoded schedule against the model of Sec. 3.2.

Nothing here decodes: these functions only verify a finished schedule against
Eq. (4)-(10) on a literal per-instant power array, and verify by brute force that every
placement was the earliest feasible one given the ops assigned before it.
"""
from __future__ import annotations

import numpy as np

ST_FREE, ST_EXEC, ST_DONE = 0, 1, 2


def machine_offsets(o):
    off = np.zeros(len(o) + 1, dtype=np.int64)
    off[1:] = np.cumsum(o)
    return off


def op_p(inst, j, s, m):
    """P_jsm (Table 2): per machine when the instance has per-machine tables."""
    pm = getattr(inst, "pm", None)
    if pm is None:
        return int(inst.p[j, s])
    return int(pm[j, machine_offsets(inst.o)[s] + m])


def op_q(inst, j, s, m):
    """Q_jsm (Table 2)."""
    qm = getattr(inst, "qm", None)
    mg = machine_offsets(inst.o)[s] + m
    return int(inst.q[mg]) if qm is None else int(qm[j, mg])


def durations(inst, M):
    N, g = inst.p.shape
    return np.array([[op_p(inst, j, s, int(M[j, s])) for s in range(g)] for j in range(N)], dtype=np.int64)


def check_invariants(inst, S, M, obj=None, tard=None, cmax=None):
    """Eq. (2)-(10) on a schedule of `inst` (an oracle.Instance-like object with arrays
    p, q, o, R, D, status, S0, M0 and scalars Qmax, WT, RS).  Raises AssertionError."""
    N, g = inst.p.shape
    RS = inst.RS
    off = machine_offsets(inst.o)
    end = S + durations(inst, M)
    for j in range(N):
        for s in range(g):
            assert 0 <= M[j, s] < inst.o[s], "machine out of range"
            if inst.status[j, s] != ST_FREE:
                assert S[j, s] == inst.S0[j, s] and M[j, s] == inst.M0[j, s], "frozen op moved"
            else:
                assert S[j, s] >= RS, "Eq. (10): start before the rescheduling point"
        assert S[j, 0] >= inst.R[j] or inst.status[j, 0] != ST_FREE, "Eq. (4): start before release"
        for s in range(1, g):
            assert S[j, s] >= end[j, s - 1], "Eq. (5): stage precedence"
    # Eq. (6): no two ops overlap on one machine (ops still relevant after RS)
    for s in range(g):
        for m in range(inst.o[s]):
            iv = sorted((S[j, s], end[j, s]) for j in range(N) if M[j, s] == m and end[j, s] > RS)
            for a, b in zip(iv, iv[1:]):
                assert a[1] <= b[0], f"Eq. (6): overlap on stage {s} machine {m}: {a} {b}"
    # Eq. (7)-(9): literal Q_t for every instant t >= RS
    horizon = int(end.max())
    if horizon > RS:
        Qt = np.zeros(horizon - RS, dtype=np.int64)
        for j in range(N):
            for s in range(g):
                a, b = max(int(S[j, s]), RS), int(end[j, s])
                if b > a:
                    Qt[a - RS:b - RS] += op_q(inst, j, s, int(M[j, s]))
        assert Qt.max() <= inst.Qmax, "Eq. (7): peak power exceeded"
    # Eq. (1)-(3)
    Cj = end[:, g - 1]
    T = np.maximum(Cj.astype(np.int64) - inst.D, 0)
    if tard is not None:
        assert tard == int(T.sum())
    if cmax is not None:
        assert cmax == int(Cj.max())
    if obj is not None:
        assert obj == inst.WT * int(T.sum()) + int(Cj.max())
    # makespan lower bound: every job needs its own work after its release
    lb = max(int(inst.R[j]) + sum(min(op_p(inst, j, s, m) for m in range(inst.o[s])) for s in range(g))
             for j in range(N))
    assert int(Cj.max()) >= min(lb, int(Cj.max())), "impossible"
    if RS == 0:
        assert int(Cj.max()) >= lb, "C_max below the longest job's work"


def stage_order(inst, y):
    """The stage-by-stage order: stages ascending, within a stage y descending."""
    gj, gs = gene_map(inst)
    return sorted(range(len(y)), key=lambda k: (gs[k], -int(y[k])))


def gene_map(inst):
    N, g = inst.p.shape
    gj, gs = [], []
    for j in range(N):
        for s in range(g):
            if inst.status[j, s] == ST_FREE:
                gj.append(j)
                gs.append(s)
    return np.array(gj, dtype=np.int64), np.array(gs, dtype=np.int64)


def check_greedy_earliest(inst, order, S, M, any_machine: bool, insert: bool = False):
    """Replay `order` and verify each op starts at the earliest integer instant at which it
    is available, its machine has finished every op assigned to it before, and the power
    of the ops assigned before it plus its own stays within Qmax at every instant; with
    `any_machine`, on the machine where that start gives the earliest completion (lowest
    index among equals; with identical machines, the earliest start).  With `insert`, an
    op may start in any idle gap of its machine after the machine's frozen ops, instead of
    after the op assigned to it last."""
    N, g = inst.p.shape
    RS = inst.RS
    off = machine_offsets(inst.o)
    gj, gs = gene_map(inst)
    end_all = S + durations(inst, M)
    H = int(end_all.max()) + 2
    Qt = np.zeros(max(H - RS, 1), dtype=np.int64)
    mfree = np.full(int(off[-1]), RS, dtype=np.int64)
    Cj = np.zeros(N, dtype=np.int64)
    placed = [[] for _ in range(int(off[-1]))]  # intervals of ops placed on each machine
    for j in range(N):
        for s in range(g):
            if inst.status[j, s] != ST_FREE:
                Cj[j] = end_all[j, s]
                if inst.status[j, s] == ST_EXEC:
                    mg = off[s] + M[j, s]
                    mfree[mg] = max(mfree[mg], end_all[j, s])
                    Qt[0:end_all[j, s] - RS] += op_q(inst, j, s, int(M[j, s]))
    for k in order:
        j, s = int(gj[k]), int(gs[k])
        est = max(RS, int(inst.R[j]), int(Cj[j]))
        machines = range(inst.o[s]) if any_machine else [int(M[j, s])]
        best = None
        for m in machines:
            mg = off[s] + m
            qm, p = op_q(inst, j, s, m), op_p(inst, j, s, m)
            t = max(est, int(mfree[mg]))
            while True:
                if t + p - RS > len(Qt):
                    Qt = np.concatenate([Qt, np.zeros(t + p - RS - len(Qt) + 1, np.int64)])
                idle = all(t + p <= a or b <= t for a, b in placed[mg]) if insert else True
                if idle and (p == 0 or int(Qt[t - RS:t - RS + p].max()) + qm <= inst.Qmax):
                    break
                t += 1
            if best is None or t + p < best[0] + best[2]:
                best = (t, m, p)
        assert (int(S[j, s]), int(M[j, s])) == best[:2], f"op ({j},{s}) not at its earliest slot: {S[j, s], M[j, s]} vs {best}"
        mg = off[s] + best[1]
        p = best[2]
        Qt[best[0] - RS:best[0] - RS + p] += op_q(inst, j, s, best[1])
        if insert:
            placed[mg].append((best[0], best[0] + p))
        else:
            mfree[mg] = best[0] + p
        Cj[j] = best[0] + p
