"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU)."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from oracle import MACH_EARLIEST, MACH_GENE, ORDER_GIVEN, ORDER_STAGE, ORDER_TOPO
from paper_1903_10741_gb300 import workloads as wl
from schedule_checks import check_greedy_earliest, check_invariants, stage_order

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ Philox

def test_philox_known_answers():
    """Philox4x32-10 reproduces the published known-answer vectors (Salmon et al. 2011)."""
    n = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            out = oracle.philox4x32_10(v[0:4], v[4:6])
            assert list(out) == v[6:10]
            n += 1
    assert n == 3


def test_draw_counter_map():
    """A draw is word d%4 of the block at counter (d/4, slot, gen, purpose<<24|instance)."""
    seed = 0x1234_5678_9ABC_DEF0
    for d in range(9):
        blk = oracle.philox4x32_10([d >> 2, 7, 3, (4 << 24) | 5], [seed & 0xFFFFFFFF, seed >> 32])
        assert oracle.draw(seed, 4, 5, 3, 7, d) == int(blk[d & 3])


# ------------------------------------------------------------------ worked example

def _worked_example():
    ex = json.load(open(os.path.join(GOLDEN, "worked_example.json")))
    n0, g = ex["n_original"], ex["g"]
    pst = np.array(ex["p_per_stage"])
    prob = wl.Problem(o=ex["o"], p=np.tile(pst, (n0, 1)), q=np.full(sum(ex["o"]), ex["q"]),
                      R=ex["R"][:n0], D=np.full(n0, 10**6), Qmax=ex["Qmax"], WT=ex["WT"])
    inst = oracle.Instance(prob)
    inst.commit(np.array(ex["S_original"]), np.array(ex["M_original"]))
    n1 = len(ex["R"]) - n0
    inst.reschedule(wl.Arrivals(p=np.tile(pst, (n1, 1)), R=ex["R"][n0:], D=[10**6] * n1), ex["RS"])
    return ex, inst


def test_worked_example_classification():
    """Alg. 1 first branch on Table 4 at RS = 7: r = 11 frozen ops, K = 13 genes, the
    executing ops are exactly the Z = 0 cells and the completed ones the Z = C cells."""
    ex, inst = _worked_example()
    Z = ex["Z_printed"]
    assert inst.K == ex["K"] == 8 * 3 - ex["r"]
    for j in range(8):
        for s in range(3):
            want = {"C": oracle.ST_DONE, 0: oracle.ST_EXEC}.get(Z[j][s], oracle.ST_FREE)
            assert inst.status[j, s] == want, (j, s)
    # the -1 cells of X and Y are exactly the frozen ops
    X, Y = np.array(ex["X"]), np.array(ex["Y"])
    assert np.array_equal(X < 0, inst.status != oracle.ST_FREE)
    assert np.array_equal(Y < 0, inst.status != oracle.ST_FREE)
    # the free Y values are a permutation of 1..K (Eq. 11)
    assert sorted(Y[Y > 0].tolist()) == list(range(1, ex["K"] + 1))


def _example_genes(ex, inst):
    gj, gs = inst.gene_map()
    Y, X, Z = np.array(ex["Y"]), np.array(ex["X"]), ex["Z_printed"]
    given = sorted(range(len(gj)), key=lambda k: Z[gj[k]][gs[k]])
    return Y[gj, gs], X[gj, gs], given, gj, gs


def test_worked_example_decode_printed_order():
    """Alg. 2 on the printed Z: job 7 at stage 0 is delayed to 13.91, the completion of
    job 5 at stage 2 on machine 4 (Sec. 4.3 narrative), and C_max = 20.42 (Fig. 8)."""
    ex, inst = _worked_example()
    y, x, given, gj, gs = _example_genes(ex, inst)
    r = inst.decode(y, x, ORDER_GIVEN, MACH_GENE, given=given)
    S, M = r["S"], r["M"]
    assert S[7, 0] == ex["expect_job7_stage0_start"]
    d = ex["expect_delay_until_end_of"]
    assert d["global_machine"] == 2 * d["stage"] + M[d["job"], d["stage"]]
    assert S[d["job"], d["stage"]] + inst.p[d["job"], d["stage"]] == S[7, 0]
    assert r["cmax"] == ex["expect_cmax"]
    check_invariants(inst, S, M, obj=r["obj"], tard=r["tard"], cmax=r["cmax"])
    check_greedy_earliest(inst, given, S, M, any_machine=False)
    # Without the power limit job 7 would have started when machine 0 freed (7.80).
    assert S[7, 0] > 780


def test_worked_example_topological_reading():
    """The topological reading of Alg. 1 (largest y among ready job heads) gives the same
    C_max as the printed Z on this example."""
    ex, inst = _worked_example()
    y, x, given, gj, gs = _example_genes(ex, inst)
    r = inst.decode(y, x, ORDER_TOPO, MACH_GENE)
    assert r["cmax"] == ex["expect_cmax"]
    # Kahn order respects both pairwise rules of Alg. 1 wherever they do not conflict:
    # within a job stages ascend; a ready head with larger y always goes first.
    check_invariants(inst, r["S"], r["M"], obj=r["obj"], tard=r["tard"], cmax=r["cmax"])


def _ops(order, gj, gs):
    return [(int(gj[k]), int(gs[k])) for k in order]


def test_worked_example_topological_order_itself():
    """The Z order of the topological reading on the Sec. 4.3 example, worked by hand.

    Free ops and their y (printed Y): (2,1)4 (2,2)2 | (3,1)10 (3,2)6 | (4,2)12 | (5,1)9
    (5,2)3 | (6,0)8 (6,1)13 (6,2)11 | (7,0)1 (7,1)5 (7,2)7.  Taking, each time, the ready job
    head with the largest y:
      heads 4,10,12,9,8,1  -> (4,2);   heads 4,10,9,8,1 -> (3,1);   heads 4,6,9,8,1 -> (5,1);
      heads 4,6,3,8,1      -> (6,0);   heads 4,6,3,13,1 -> (6,1);   heads 4,6,3,11,1 -> (6,2);
      heads 4,6,3,1        -> (3,2);   heads 4,3,1      -> (2,1);   heads 2,3,1      -> (5,2);
      heads 2,1            -> (2,2);   then (7,0), (7,1), (7,2).
    The printed Z agrees at positions 1-3 and 8-13 (nine of 13).  It lists (3,2) fourth, before
    the ready head (6,0) with the larger y, which no y rule gives; with (3,2) set aside the
    two orders are the same sequence.
    """
    ex, inst = _worked_example()
    y, x, given, gj, gs = _example_genes(ex, inst)
    got = _ops(inst.order(y, ORDER_TOPO), gj, gs)
    want = [(4, 2), (3, 1), (5, 1), (6, 0), (6, 1), (6, 2), (3, 2), (2, 1), (5, 2), (2, 2), (7, 0), (7, 1), (7, 2)]
    assert got == want
    printed = _ops(inst.order(y, ORDER_GIVEN, given=given), gj, gs)
    Z = ex["Z_printed"]
    assert [Z[j][s] for j, s in printed] == list(range(1, 14))  # ORDER_GIVEN is the printed Z
    agree = [n + 1 for n in range(13) if got[n] == printed[n]]
    assert agree == [1, 2, 3, 8, 9, 10, 11, 12, 13]
    assert [op for op in got if op != (3, 2)] == [op for op in printed if op != (3, 2)]


def test_worked_example_stage_order_itself():
    """The stage-by-stage order on the Sec. 4.3 example, by hand: stage 0 by y descending is
    (6,0)8, (7,0)1; stage 1 is (6,1)13, (3,1)10, (5,1)9, (7,1)5, (2,1)4; stage 2 is (4,2)12,
    (6,2)11, (7,2)7, (3,2)6, (5,2)3, (2,2)2."""
    ex, inst = _worked_example()
    y, x, given, gj, gs = _example_genes(ex, inst)
    assert _ops(inst.order(y, ORDER_STAGE), gj, gs) == [
        (6, 0), (7, 0), (6, 1), (3, 1), (5, 1), (7, 1), (2, 1), (4, 2), (6, 2), (7, 2), (3, 2), (5, 2), (2, 2)]


# ------------------------------------------------------------------ objective

@pytest.mark.parametrize("wt,tard,cmax,obj", [
    (0.01, 35.23, 40.54, 40.89), (0.1, 23.43, 40.78, 43.12), (0.4, 19.04, 41.14, 48.76),
    (0.7, 18.61, 41.23, 54.26), (1, 18.29, 41.44, 59.73), (4, 17.83, 42.15, 113.46),
    (7, 17.69, 42.18, 166.00), (10, 17.57, 42.12, 217.86), (100, 17.58, 42.39, 1800.43)])
def test_objective_table11(wt, tard, cmax, obj):
    """Eq. (1): objective = WT * total tardiness + C_max on rows of Table 11: the weight
    multiplies the tardiness and the makespan is added unweighted.  Times are on a 1/100
    grid and WT on a 1/100 grid, so obj_int = (100 WT) * (100 T) + 100 C_max * 100."""
    scale = 100
    # job 0 carries the whole tardiness; job 1 sets the makespan and is never late
    C_j = np.array([int(round(tard * scale)), int(round(cmax * scale))], np.int32)
    D = np.array([0, 10**8], np.int32)
    wt_i = int(round(wt * 100))
    o, t, cm = oracle.objective(C_j, D, wt_i)
    assert t == C_j[0] and cm == C_j[1]
    got = (o - cm) / (100 * scale) + cm / scale
    # the table prints 100-run averages rounded to 0.01: T carries +-0.005 * WT
    assert abs(got - obj) <= 0.005 * wt + 0.0051


# ------------------------------------------------------------------ invariants

def _random_problem(seed, N=8, g=3, o=(1, 3), p_hi=20, q=(1, 10), pct=55, release_hi=0):
    rng = np.random.default_rng(seed)
    return wl.random_instance(rng, N, g, o[0], o[1], p_hi, q[0], q[1], pct, release_hi=release_hi)


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("mode", [(ORDER_STAGE, MACH_EARLIEST), (ORDER_TOPO, MACH_GENE),
                                  (ORDER_STAGE, MACH_GENE), (ORDER_TOPO, MACH_EARLIEST)])
def test_decode_invariants_and_greedy(seed, mode):
    """Every decoded schedule satisfies Eq. (2)-(10) and each op sits at its earliest
    feasible slot given the ops before it (brute force over integer starts)."""
    prob = _random_problem(seed, release_hi=30 if seed % 2 else 0)
    inst = oracle.Instance(prob)
    rng = np.random.default_rng(100 + seed)
    Y, X = wl.random_chromosomes(rng, 4, inst.K, inst.gene_machines())
    for y, x in zip(Y, X):
        r = inst.decode(y, x, *mode)
        check_invariants(inst, r["S"], r["M"], obj=r["obj"], tard=r["tard"], cmax=r["cmax"])
        if mode[0] == ORDER_STAGE:
            order = stage_order(inst, y)
            check_greedy_earliest(inst, order, r["S"], r["M"], any_machine=mode[1] == MACH_EARLIEST)


@pytest.mark.parametrize("seed", range(6))
def test_reschedule_chain_invariants(seed):
    """Freeze at RS, append arrivals, decode again: frozen ops keep their plan, executing
    ops keep their machine busy and draw power until they end, and no new op starts
    before RS (Eq. 10)."""
    rng = np.random.default_rng(seed)
    prob = wl.random_instance(rng, 10, 4, 1, 3, 30, 5, 30, 50)
    inst = oracle.Instance(prob)
    r = inst.decode(np.arange(inst.K, 0, -1), None, ORDER_STAGE, MACH_EARLIEST)
    for ev in range(3):
        inst.commit(r["S"], r["M"])
        t_now = int(r["cmax"] * (2 + ev) // 6)
        inst.reschedule(wl.random_arrivals(rng, 3, inst.g, t_now, 30), t_now)
        assert (inst.status[inst.N - 3:] == oracle.ST_FREE).all()
        Y, X = wl.random_chromosomes(rng, 3, inst.K, inst.gene_machines())
        for y in Y:
            r = inst.decode(y, None, ORDER_STAGE, MACH_EARLIEST)
            check_invariants(inst, r["S"], r["M"], obj=r["obj"], tard=r["tard"], cmax=r["cmax"])
            check_greedy_earliest(inst, stage_order(inst, y), r["S"], r["M"], any_machine=True)


def test_classify_boundaries():
    """Alg. 1: S+P <= RS completed, S < RS < S+P executing, S >= RS free (half-open
    operation intervals, Eq. 9)."""
    p = np.array([[5, 5, 5]], np.int32)
    inst = oracle.Instance(wl.Problem(o=[1, 1, 1], p=p, q=[1, 1, 1], R=[0], D=[0], Qmax=3))
    inst.commit(np.array([[0, 5, 10]]), np.zeros((1, 3)))
    inst.reschedule(wl.Arrivals(p=np.zeros((0, 3)), R=[], D=[]), 5)
    assert inst.status.tolist() == [[oracle.ST_DONE, oracle.ST_FREE, oracle.ST_FREE]]
    inst.commit(np.array([[0, 5, 10]]), np.zeros((1, 3)))
    inst.reschedule(wl.Arrivals(p=np.zeros((0, 3)), R=[], D=[]), 6)
    assert inst.status.tolist() == [[oracle.ST_DONE, oracle.ST_EXEC, oracle.ST_FREE]]


# ------------------------------------------------------------------ closed forms

def test_single_machine_closed_form():
    """g = 1, o = 1, power not binding: ops run back to back in y-descending order, so
    C_j is the prefix sum of p in that order and C_max = sum p."""
    rng = np.random.default_rng(3)
    N = 9
    p = rng.integers(1, 30, size=(N, 1))
    D = rng.integers(10, 150, size=N)
    inst = oracle.Instance(wl.Problem(o=[1], p=p, q=[4], R=np.zeros(N), D=D, Qmax=10))
    y = rng.permutation(N) + 1
    r = inst.decode(y, None, ORDER_STAGE, MACH_EARLIEST)
    seq = np.argsort(-y)
    Cj = np.empty(N, np.int64)
    Cj[seq] = np.cumsum(p[seq, 0])
    assert r["cmax"] == p.sum()
    assert r["tard"] == int(np.maximum(Cj - D, 0).sum())
    assert r["obj"] == 100 * r["tard"] + r["cmax"]


def test_power_serialises_everything():
    """If Qmax equals every machine's power, only one op can run at any instant; with all
    releases 0 the stage-by-stage decode leaves no idle time: C_max = sum of all p."""
    rng = np.random.default_rng(5)
    N, g = 7, 3
    p = rng.integers(1, 15, size=(N, g))
    inst = oracle.Instance(wl.Problem(o=[2, 3, 2], p=p, q=np.full(7, 6), R=np.zeros(N),
                                      D=np.zeros(N), Qmax=6))
    for seed in range(5):
        y = np.random.default_rng(seed).permutation(inst.K) + 1
        r = inst.decode(y, None, ORDER_STAGE, MACH_EARLIEST)
        assert r["cmax"] == p.sum()


def test_permutation_flow_shop_recursion():
    """One machine per stage and power never binding: with y giving every stage the same
    job sequence, C_max follows the textbook permutation flow shop recursion
    C[k][s] = max(C[k-1][s], C[k][s-1]) + p."""
    rng = np.random.default_rng(11)
    N, g = 8, 4
    p = rng.integers(1, 25, size=(N, g))
    inst = oracle.Instance(wl.Problem(o=[1] * g, p=p, q=np.ones(g), R=np.zeros(N),
                                      D=np.zeros(N), Qmax=g))
    seq = rng.permutation(N)
    rank = np.empty(N, np.int64)
    rank[seq] = np.arange(N)
    # y: larger for earlier jobs, identical job order at every stage
    gj, gs = inst.gene_map()
    y = (N - rank[gj]) * g - gs  # unique, same job order in each stage
    y = np.argsort(np.argsort(y)) + 1
    r = inst.decode(y, None, ORDER_STAGE, MACH_EARLIEST)
    Cm = np.zeros((N + 1, g + 1), np.int64)
    for k, j in enumerate(seq, start=1):
        for s in range(1, g + 1):
            Cm[k, s] = max(Cm[k - 1, s], Cm[k, s - 1]) + p[j, s - 1]
    assert r["cmax"] == Cm[N, g]


def test_parallel_list_scheduling_closed_form():
    """One stage, o identical machines, power never binding: each op goes to the machine
    that frees first (lowest index on ties), i.e. classic list scheduling."""
    rng = np.random.default_rng(2)
    N, o = 12, 3
    p = rng.integers(1, 40, size=(N, 1))
    inst = oracle.Instance(wl.Problem(o=[o], p=p, q=[1, 2, 3], R=np.zeros(N), D=np.zeros(N), Qmax=6))
    y = rng.permutation(N) + 1
    r = inst.decode(y, None, ORDER_STAGE, MACH_EARLIEST)
    free = [0] * o
    for j in np.argsort(-y):
        m = min(range(o), key=lambda i: (free[i], i))
        assert r["S"][j, 0] == free[m] and r["M"][j, 0] == m
        free[m] += int(p[j, 0])


# ------------------------------------------------------------------ brute force

def _all_stage_orders(inst):
    """Every chromosome that yields a distinct per-stage order (y up to stage-wise rank)."""
    gj, gs = inst.gene_map()
    K = len(gj)
    stages = sorted(set(gs.tolist()))
    per = [[k for k in range(K) if gs[k] == s] for s in stages]
    for combo in itertools.product(*[itertools.permutations(v) for v in per]):
        y = np.zeros(K, np.int64)
        val = K
        for seq in combo:
            for k in seq:
                y[k] = val
                val -= 1
        yield y


def test_bruteforce_small_space_and_ga_reaches_it():
    """N = 4, g = 2: enumerate all (4!)^2 per-stage orders; the GA's best is never below
    the brute-force minimum and reaches it on this tiny space."""
    rng = np.random.default_rng(21)
    prob = wl.random_instance(rng, 4, 2, 2, 2, 20, 3, 9, 50)
    inst = oracle.Instance(prob)
    best = None
    for y in _all_stage_orders(inst):
        r = inst.decode(y, None, ORDER_STAGE, MACH_EARLIEST)
        check_invariants(inst, r["S"], r["M"], obj=r["obj"])
        best = r["obj"] if best is None else min(best, r["obj"])
    ga = oracle.GA(inst, P=32, island=16, seed=3).init()
    ga.step(60)
    assert ga.bobj.min() >= best
    assert ga.bobj.min() == best


# ------------------------------------------------------------------ GA operators

FIG11_A_X = [[-1, 1, 0], [-1, -1, 1], [1, 0, 1]]
FIG11_A_Y = [[-1, 6, 1], [-1, -1, 5], [4, 3, 2]]
FIG11_B_X = [[-1, 0, 0], [-1, -1, 0], [1, 1, 1]]
FIG11_B_Y = [[-1, 3, 6], [-1, -1, 1], [4, 2, 5]]


def _free(mat):
    a = np.array(mat)
    return a[a >= 0]


def _unfree(vals, like):
    a = np.array(like).copy()
    a[a >= 0] = vals
    return a.tolist()


def test_crossover_fig11():
    """Fig. 11: X cut after 2 free genes, Y cut after 1; child0 = head(A)+tail(B),
    child1 = head(B)+tail(A); the later duplicate takes the missing value."""
    y0, x0, y1, x1 = oracle.crossover(_free(FIG11_A_Y), _free(FIG11_A_X), _free(FIG11_B_Y),
                                      _free(FIG11_B_X), cx=2, cy=1)
    assert _unfree(x0, FIG11_A_X) == [[-1, 1, 0], [-1, -1, 0], [1, 1, 1]]
    assert _unfree(y0, FIG11_A_Y) == [[-1, 6, 3], [-1, -1, 1], [4, 2, 5]]
    assert _unfree(x1, FIG11_A_X) == [[-1, 0, 0], [-1, -1, 1], [1, 0, 1]]
    assert _unfree(y1, FIG11_A_Y) == [[-1, 3, 1], [-1, -1, 5], [4, 6, 2]]


def test_correction_several_duplicates():
    """Duplicates, in scan order, take the missing values in ascending order."""
    y = np.array([5, 2, 5, 1, 2, 5], np.int16)  # missing 3, 4, 6; dups at 2, 4, 5
    assert oracle.correct(y).tolist() == [5, 2, 3, 1, 4, 6]


def test_mutation_fig12():
    """Fig. 12 with two machines per stage: every free x flips; y swaps the first and last
    free genes (6 <-> 2)."""
    x = _free(FIG11_A_X)
    y = _free(FIG11_A_Y)
    go = np.full(len(y), 2)
    ym, xm = oracle.mutate(y, x, go, np.zeros(len(y), np.uint32), 0, len(y) - 1)
    assert _unfree(xm, FIG11_A_X) == [[-1, 0, 1], [-1, -1, 0], [0, 1, 0]]
    assert _unfree(ym, FIG11_A_Y) == [[-1, 2, 1], [-1, -1, 5], [4, 3, 6]]


def test_mutation_never_keeps_machine():
    """Each redraw lands on one of the other o-1 machines, all reachable."""
    go = np.full(4, 5)
    x = np.array([0, 2, 4, 3], np.int8)
    seen = set()
    for r in range(4):
        _, xm = oracle.mutate(np.arange(1, 5), x, go, np.full(4, r, np.uint32), 0, 1)
        assert (xm != x).all()
        seen.add(tuple(xm.tolist()))
    assert len(seen) == 4


# ------------------------------------------------------------------ selection, replacement, migration

def test_tournament_ties_to_lower_index():
    """Sec. 4.4 selection: the entrant with the larger fitness wins; equal fitness goes to
    the lower population index, whatever the entrants' order.  With fit = [5, 7, 7, 3, 7]:
    k=2 {2,1} -> 1 (7 = 7, 1 < 2); {0,3} -> 0 (5 > 3); {4,4} -> 4; k=3 {4,2,0} -> 2;
    {3,3,0} -> 0; {1,3,4} -> 1; all-equal fitness {3,1,2} -> 1."""
    fit = [5, 7, 7, 3, 7]
    assert oracle.tournament(fit, [2, 1]) == 1
    assert oracle.tournament(fit, [1, 2]) == 1
    assert oracle.tournament(fit, [0, 3]) == 0
    assert oracle.tournament(fit, [4, 4]) == 4
    assert oracle.tournament(fit, [4, 2, 0]) == 2
    assert oracle.tournament(fit, [3, 3, 0]) == 0
    assert oracle.tournament(fit, [1, 3, 4]) == 1
    assert oracle.tournament([9, 9, 9, 9], [3, 1, 2]) == 1


def test_l5_torus_cells():
    """The 5-cell neighbourhood (Sec. 4.4, Fig. 9) on the 4 x 4 torus, cells row-major
    (r = i // 4, c = i % 4), listed as the cell, N, S, W, E:
      cell 0  (0,0): N (3,0)=12, S (1,0)=4,  W (0,3)=3,  E (0,1)=1
      cell 6  (1,2): N (0,2)=2,  S (2,2)=10, W (1,1)=5,  E (1,3)=7
      cell 7  (1,3): N (0,3)=3,  S (2,3)=11, W (1,2)=6,  E (1,0)=4
      cell 15 (3,3): N (2,3)=11, S (0,3)=3,  W (3,2)=14, E (3,0)=12
    and on the 3 x 3 torus the centre cell 4: 1, 7, 3, 5."""
    assert oracle.l5_cells(16, 0) == [0, 12, 4, 3, 1]
    assert oracle.l5_cells(16, 6) == [6, 2, 10, 5, 7]
    assert oracle.l5_cells(16, 7) == [7, 3, 11, 6, 4]
    assert oracle.l5_cells(16, 15) == [15, 11, 3, 14, 12]
    assert oracle.l5_cells(9, 4) == [4, 1, 7, 3, 5]


def test_select_l5_picks_the_fittest_neighbour():
    """With tournament size 0 the parent of a slot is the fittest of its five cells: on the
    4 x 4 torus, slot 6 with fitness 50 at cell 7 (its E neighbour) and 40 elsewhere in the
    neighbourhood takes 7; slot 0 with equal fitness at 12 (N) and 1 (E) takes 1; cell 9,
    outside slot 6's neighbourhood, never wins it."""
    fit = np.full(16, 40, np.int64)
    fit[7], fit[9] = 50, 99
    assert oracle.select(fit, 16, 16, 0, 1, 0, 1, 6) == 7
    fit = np.zeros(16, np.int64)
    fit[12] = fit[1] = 8
    assert oracle.select(fit, 16, 16, 0, 1, 0, 1, 0) == 1


@pytest.mark.parametrize("k", [2, 3])
def test_select_tournament_draws(k):
    """Entrant t of slot i is island start + floor(u_t * I / 2^32), u_t = draw t of slot i's
    selection stream (purpose 3; the stream itself is pinned above).  Islands of 8 in a
    population of 32: with equal fitness the winner is the smallest entrant; with distinct
    fitness (larger for larger index) the largest; entrants never leave the slot's island."""
    P, I, seed, gen = 32, 8, 77, 5
    flat = np.zeros(P, np.int64)
    rising = np.arange(P, dtype=np.int64)
    for i in range(P):
        lo = (i // I) * I
        ent = [lo + (oracle.draw(seed, 3, 2, gen, i, t) * I >> 32) for t in range(k)]
        assert all(lo <= e < lo + I for e in ent)
        assert oracle.select(flat, P, I, k, seed, 2, gen, i) == min(ent)
        assert oracle.select(rising, P, I, k, seed, 2, gen, i) == max(ent)


def _marked_rows(n, K):
    """Row r holds y = [10 r + 1, 10 r + 2, ...] and x = [r, r, ...], so every copy is traceable."""
    Y = np.array([[10 * r + 1 + c for c in range(K)] for r in range(n)], np.int16)
    X = np.array([[r] * K for r in range(n)], np.int8)
    return Y, X


def test_island_replace_strict_improvement():
    """Elitist replacement (Sec. 4.4) of the second island (slots 4..7) of two, K = 3.
    Children's fitness 10, 30, 30, 5 (slots 4-7), objectives 90, 70, 70, 95; record fitness 20.
    The best child is slot 5 (30; slot 6 ties and loses on index), strictly fitter than 20,
    so the record becomes slot 5's row (y 51 52 53, obj 70, fit 30); then the record
    overwrites the worst child, slot 7 (fitness 5).  Island 0 is untouched."""
    Y, X = _marked_rows(8, 3)
    obj = np.array([1, 2, 3, 4, 90, 70, 70, 95], np.int64)
    fit = np.array([9, 9, 9, 9, 10, 30, 30, 5], np.int64)
    bY, bX = np.array([7, 7, 7], np.int16), np.array([1, 1, 1], np.int8)
    cY, cX, cobj, cfit, nbY, nbX, bo, bf = oracle.island_replace(Y, X, obj, fit, 4, 4, bY, bX, 80, 20)
    assert (bo, bf) == (70, 30) and nbY.tolist() == [51, 52, 53] and nbX.tolist() == [5, 5, 5]
    assert cY[7].tolist() == [51, 52, 53] and cX[7].tolist() == [5, 5, 5]
    assert cobj[7] == 70 and cfit[7] == 30
    assert np.array_equal(cY[:7], Y[:7]) and np.array_equal(cobj[:7], obj[:7]) and np.array_equal(cfit[:7], fit[:7])


def test_island_replace_tie_keeps_record_and_worst_tie_lowest():
    """Same island; the record has fitness 30 and the best child only equals it, so the
    record stays (y 7 7 7, obj 80).  Children's fitness 10, 5, 30, 5: the worst is slot 5
    (5; slot 7 ties and loses on index), and it takes the record."""
    Y, X = _marked_rows(8, 3)
    obj = np.array([1, 2, 3, 4, 90, 95, 70, 95], np.int64)
    fit = np.array([9, 9, 9, 9, 10, 5, 30, 5], np.int64)
    bY, bX = np.array([7, 7, 7], np.int16), np.array([1, 1, 1], np.int8)
    cY, cX, cobj, cfit, nbY, nbX, bo, bf = oracle.island_replace(Y, X, obj, fit, 4, 4, bY, bX, 80, 30)
    assert (bo, bf) == (80, 30) and nbY.tolist() == [7, 7, 7]
    assert cY[5].tolist() == [7, 7, 7] and cX[5].tolist() == [1, 1, 1] and cobj[5] == 80 and cfit[5] == 30
    assert cY[7].tolist() == Y[7].tolist() and cfit[7] == 5


def test_migrate_ring_from_snapshot():
    """Single-ring migration (Sec. 4.4) over three islands of two, K = 2, rows marked by slot.
    Fitness 3 3 | 8 2 | 5 9: bests are slots 0, 2, 5 and worsts 0, 3, 4 (island 0 ties: slot
    0 is both).  Island i's worst takes island i-1's best as it was before any copy:
      slot 0 <- slot 5 (y 51 52, obj 105, fit 9);  slot 3 <- slot 0 (y 1 2, obj 100, fit 3);
      slot 4 <- slot 2 (y 21 22, obj 102, fit 8).
    Copying in place, island 1 would have received slot 5's row through slot 0, and a ring
    turning the other way would put slot 2's row into slot 0."""
    Y, X = _marked_rows(6, 2)
    obj = np.arange(100, 106, dtype=np.int64)
    fit = np.array([3, 3, 8, 2, 5, 9], np.int64)
    cY, cX, cobj, cfit = oracle.migrate(Y, X, obj, fit, 2)
    assert cY.tolist() == [[51, 52], [11, 12], [21, 22], [1, 2], [21, 22], [51, 52]]
    assert cX[:, 0].tolist() == [5, 1, 2, 0, 2, 5]
    assert cobj.tolist() == [105, 101, 102, 100, 102, 105]
    assert cfit.tolist() == [9, 3, 8, 3, 8, 9]


def test_ga_migrants_are_post_replacement_bests():
    """Operator order of a generation: replacement, then migration.  After replacement each
    island's fittest member is its best-ever record (fitness bfit); migration then copies it
    into the next island.  So after every migration generation island i holds a member with
    fitness bfit[i-1]; migrating before replacement would move only the best child, whose
    fitness falls short of the record in most generations."""
    prob = wl.static_small(4)
    ga = oracle.GA(oracle.Instance(prob), P=64, island=8, tour_k=2, migrate_every=1, seed=9).init()
    nisl = 8
    for _ in range(25):
        ga.step()
        for i in range(nisl):
            members = ga.fit[8 * i:8 * i + 8]
            assert ga.bfit[(i - 1) % nisl] in members, (ga.gen, i)
            assert members.max() >= ga.bfit[i]


def test_candidates_with_one_per_slot_are_the_generation_children():
    """With one candidate per slot the offspring rows are exactly the children a generation
    builds before decoding; with F per slot, candidate 0 of every slot is that child, and
    every row is a permutation of 1..K."""
    prob = wl.static_small(5)
    ga = oracle.GA(oracle.Instance(prob), P=64, island=16, tour_k=2, migrate_every=0, seed=4, mach_mode=MACH_GENE)
    ga.init().step(3)
    cY, cX, _ = ga.candidates(1)
    cY8, cX8, new8 = ga.candidates(8)
    assert np.array_equal(cY8[:64], cY) and np.array_equal(cX8[:64], cX)
    assert all(sorted(r.tolist()) == list(range(1, ga.K + 1)) for r in cY8)
    ga.step()
    # the children after replacement: all but one slot per island (the record's) are cY
    same = (ga.Y[:, :ga.K] == cY).all(axis=1)
    assert same.reshape(4, 16).sum(axis=1).min() >= 15
    assert 0.5 < new8.mean() < 1.0  # crossover 0.8, mutation 0.1


# ------------------------------------------------------------------ GA properties

def test_ga_population_stays_valid_and_elitist():
    """Every generation keeps each Y a permutation of 1..K, the best-ever objective never
    rises, and each island holds its best-ever individual."""
    prob = wl.static_small(1)
    inst = oracle.Instance(prob)
    ga = oracle.GA(inst, P=64, island=16, seed=7, migrate_every=5).init()
    K = inst.K
    prev = ga.bobj.copy()
    for _ in range(30):
        ga.step()
        for row in ga.Y[:, :K]:
            assert sorted(row.tolist()) == list(range(1, K + 1))
        assert (ga.bobj <= prev).all()
        prev = ga.bobj.copy()
        for isl in range(4):
            assert ga.obj[isl * 16:(isl + 1) * 16].min() <= ga.bobj[isl]
        assert ((ga.fit == np.maximum(ga.emax - ga.obj, 0))).all()


def test_ga_emax_rule():
    """E_max = 10^a with the smallest a >= 1 such that every initial objective is below it
    (Sec. 5)."""
    inst = oracle.Instance(wl.static_small(1))
    ga = oracle.GA(inst, P=64, seed=1).init()
    mx = int(ga.obj.max())
    assert ga.emax > mx and (ga.emax // 10 <= mx or ga.emax == 10)
    assert str(ga.emax).strip("0") == "1"


def test_ga_resume_is_bit_exact():
    """The stream is counter based: 20 generations equal 10 + 10 from a copied state."""
    inst = oracle.Instance(wl.static_small(2))
    a = oracle.GA(inst, P=64, island=32, seed=9).init()
    a.step(20)
    b = oracle.GA(inst, P=64, island=32, seed=9).init()
    b.step(10)
    c = oracle.GA(inst, P=64, island=32, seed=9)
    for name in ("Y", "X", "obj", "fit", "bY", "bX", "bobj", "bfit"):
        getattr(c, name)[...] = getattr(b, name)
    c.st.emax, c.st.gen = b.st.emax, b.st.gen
    c.step(10)
    for name in ("Y", "obj", "bY", "bobj"):
        assert np.array_equal(getattr(a, name), getattr(c, name))


def test_ga_paper_mode_runs():
    """Paper mode (Kahn order, machine genes, local 5-neighbourhood selection) keeps X in
    range and improves on the initial population."""
    inst = oracle.Instance(wl.static_small(1))
    ga = oracle.GA(inst, P=64, island=16, tour_k=0, order_mode=ORDER_TOPO, mach_mode=MACH_GENE,
                   pc=(9, 10), seed=4).init()
    first = int(ga.bobj.min())
    ga.step(40)
    gm = inst.gene_machines()
    assert (ga.X[:, :inst.K] < gm[None, :]).all() and (ga.X >= 0).all()
    assert int(ga.bobj.min()) <= first


# ---------------------------------------------------------------- warm start (not in the paper)

def test_warm_remap_worked_example():
    # genes (keys) 0..3 before; keys 0 and 2 froze, keys 4 and 5 belong to a new job.
    # Survivors by old priority: key 1 (y=1) then key 3 (y=2) -> priorities 3 and 4;
    # new genes in index order take 2 and 1.
    Y, X = oracle.warm_remap(np.array([[3, 1, 4, 2]]), np.array([[1, 0, 1, 2]]), [0, 1, 2, 3],
                             [1, 3, 4, 5], 1)
    assert Y.tolist() == [[3, 4, 2, 1]]
    assert X.tolist() == [[0, 2, 0, 0]]


def test_warm_remap_identity_and_row_cycling():
    rng = np.random.default_rng(3)
    Y0 = np.stack([rng.permutation(9) + 1 for _ in range(4)]).astype(np.int16)
    X0 = rng.integers(0, 3, size=(4, 9)).astype(np.int8)
    keys = list(range(0, 18, 2))
    Y, X = oracle.warm_remap(Y0, X0, keys, keys, 10)
    for r in range(10):  # nothing froze, nothing arrived: row r is old row r mod 4
        assert np.array_equal(Y[r], Y0[r % 4]) and np.array_equal(X[r], X0[r % 4])


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_warm_remap_properties_after_reschedule(seed):
    rng = np.random.default_rng(seed)
    pr = wl.random_instance(rng, 12, 3, 1, 3, 30, 5, 20, 60)
    inst = oracle.Instance(pr)
    keys0 = oracle.gene_keys(inst)
    ga = oracle.GA(inst, P=16, island=8, seed=seed, mach_mode=MACH_GENE).init().step(3)
    y, x, _ = ga.best()
    r = inst.decode(y, x, mach_mode=MACH_GENE)
    inst.commit(r["S"], r["M"])
    t_now = r["cmax"] // 3
    inst.reschedule(wl.random_arrivals(rng, 4, 3, t_now, 30), t_now)
    keys1 = oracle.gene_keys(inst)
    Y, X = oracle.warm_remap(ga.Y[:, :ga.K], ga.X[:, :ga.K], keys0, keys1, 24)
    K1 = len(keys1)
    old = {k: i for i, k in enumerate(keys0.tolist())}
    surv = [i for i, k in enumerate(keys1.tolist()) if k in old]
    fresh = [i for i, k in enumerate(keys1.tolist()) if k not in old]
    assert fresh and len(surv) < len(keys0)  # some genes froze, a job arrived
    for r_ in range(24):
        yo, xo = ga.Y[r_ % 16, :ga.K], ga.X[r_ % 16, :ga.K]
        assert sorted(Y[r_].tolist()) == list(range(1, K1 + 1))
        assert min(Y[r_, surv]) > max(Y[r_, fresh])  # new genes below every survivor
        # survivors in the same relative order, with their machine genes
        for a in surv:
            assert X[r_, a] == xo[old[keys1[a]]]
            for b in surv:
                assert (Y[r_, a] < Y[r_, b]) == (yo[old[keys1[a]]] < yo[old[keys1[b]]])
        assert [Y[r_, i] for i in fresh] == list(range(len(fresh), 0, -1))
        inst.decode(Y[r_], X[r_], mach_mode=MACH_GENE)  # a valid chromosome of the new instance


def test_ga_init_from_random_rows_equals_init():
    inst = oracle.Instance(wl.static_small(2))
    a = oracle.GA(inst, P=32, island=8, seed=5, mach_mode=MACH_GENE).init()
    b = oracle.GA(inst, P=32, island=8, seed=5, mach_mode=MACH_GENE).init_from(a.Y, a.X)
    for f in ("Y", "X", "obj", "fit", "bY", "bX", "bobj", "bfit"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    assert a.emax == b.emax and b.gen == 0
    a.step(4)
    b.step(4)
    assert np.array_equal(a.Y, b.Y) and np.array_equal(a.bobj, b.bobj)


# ---------------------------------------------------------------- static approach (Sec. 5.3)

def _worked_example_static():
    ex = json.load(open(os.path.join(GOLDEN, "worked_example.json")))
    n0 = ex["n_original"]
    pst = np.array(ex["p_per_stage"])
    prob = wl.Problem(o=ex["o"], p=np.tile(pst, (n0, 1)), q=np.full(sum(ex["o"]), ex["q"]),
                      R=ex["R"][:n0], D=np.full(n0, 10**6), Qmax=ex["Qmax"], WT=ex["WT"])
    inst = oracle.Instance(prob)
    inst.commit(np.array(ex["S_original"]), np.array(ex["M_original"]))
    n1 = len(ex["R"]) - n0
    inst.reschedule(wl.Arrivals(p=np.tile(pst, (n1, 1)), R=ex["R"][n0:], D=[10**6] * n1), ex["RS"], static=True)
    return ex, inst


def _check_static(inst, S, M):
    """The plan is kept; every new op follows the last planned op of its machine."""
    N, g = inst.p.shape
    frozen = inst.status != oracle.ST_FREE
    assert np.array_equal(S[frozen], inst.S0[frozen]) and np.array_equal(M[frozen], inst.M0[frozen])
    for s in range(g):
        for m in range(inst.o[s]):
            last = max([int(inst.S0[j, s] + inst.p[j, s]) for j in range(N)
                        if frozen[j, s] and inst.M0[j, s] == m] + [inst.RS])
            for j in range(N):
                if not frozen[j, s] and M[j, s] == m:
                    assert S[j, s] >= last, (j, s, m)


def test_static_worked_example_fig7():
    """Fig. 7 (static environment) on Table 4 at RS = 7: the original plan is kept, jobs 6
    and 7 are the only genes, and the best makespan over every order and machine choice
    of their six ops is 19.91, the figure's C_max (Fig. 8's reactive schedule has 20.42)."""
    ex, inst = _worked_example_static()
    assert inst.K == 6
    assert (inst.status[:6] != oracle.ST_FREE).all() and (inst.status[6:] == oracle.ST_FREE).all()
    # ops not yet completed at RS are being executed (Z = 0 cells) or fixed in the plan
    Z = ex["Z_printed"]
    for j in range(6):
        for s in range(3):
            want = oracle.ST_DONE if Z[j][s] == "C" else oracle.ST_EXEC if Z[j][s] == 0 else oracle.ST_FIXED
            assert inst.status[j, s] == want, (j, s)
    best = None
    for perm in itertools.permutations(range(1, 7)):
        y = np.array(perm, np.int16)
        for xm in range(64):
            x = np.array([(xm >> k) & 1 for k in range(6)], np.int8)
            r = inst.decode(y, x, ORDER_STAGE, MACH_GENE)
            best = r["cmax"] if best is None else min(best, r["cmax"])
        r = inst.decode(y, None, ORDER_STAGE, MACH_EARLIEST)
        assert r["cmax"] == 1991
    assert best == 1991
    check_invariants(inst, r["S"], r["M"], obj=r["obj"], tard=r["tard"], cmax=r["cmax"])
    _check_static(inst, r["S"], r["M"])


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_static_chain_invariants(seed):
    """Static rescheduling chains on random instances: schedules satisfy Eq. (4)-(10), the
    kept plan never moves, and new ops follow each machine's last planned op."""
    rng = np.random.default_rng(seed)
    pr = wl.random_instance(rng, 10, 3, 1, 3, 20, 5, 20, 55)
    inst = oracle.Instance(pr)
    ga = oracle.GA(inst, P=32, island=16, seed=seed, mach_mode=MACH_GENE).init().step(3)
    y, x, _ = ga.best()
    r = inst.decode(y, x, mach_mode=MACH_GENE)
    inst.commit(r["S"], r["M"])
    t_now = 0
    for ev in range(3):
        t_now = t_now + max(1, r["cmax"] // 5)
        inst.reschedule(wl.random_arrivals(rng, 3, 3, t_now, 20), t_now, static=True)
        assert inst.K == 9  # only the new jobs are genes
        yy = rng.permutation(inst.K).astype(np.int16) + 1
        for mode in (MACH_EARLIEST, MACH_GENE):
            xx = (rng.random(inst.K) * inst.gene_machines()).astype(np.int8)
            r = inst.decode(yy, xx, ORDER_STAGE, mode)
            check_invariants(inst, r["S"], r["M"], obj=r["obj"], tard=r["tard"], cmax=r["cmax"])
            _check_static(inst, r["S"], r["M"])
        inst.commit(r["S"], r["M"])


def test_static_equals_reactive_without_plan_left():
    """When every op of the plan has completed by RS, nothing is kept and the two
    approaches give the same instance: the same genes and the same decoded schedules."""
    rng = np.random.default_rng(4)
    pr = wl.random_instance(rng, 8, 3, 1, 2, 20, 5, 20, 60)
    a, b = oracle.Instance(pr), oracle.Instance(pr)
    y = (rng.permutation(a.K) + 1).astype(np.int16)
    r = a.decode(y)
    for inst in (a, b):
        inst.commit(r["S"], r["M"])
    arr = wl.random_arrivals(rng, 4, 3, r["cmax"], 20)
    a.reschedule(arr, r["cmax"])
    b.reschedule(arr, r["cmax"], static=True)
    assert np.array_equal(a.status, b.status) and a.K == b.K == 12
    y2 = (rng.permutation(a.K) + 1).astype(np.int16)
    assert a.decode(y2)["obj"] == b.decode(y2)["obj"]


# ---------------------------------------------------------------- unrelated machines (Table 2)

def test_unrelated_hand_example_earliest_completion():
    """One stage, two machines, no binding peak.  Job 0 takes 5 on machine 0 and 2 on
    machine 1: both start at 0, so earliest start would pick machine 0 but earliest
    completion picks machine 1 (0..2).  Job 1 takes 3 / 4: machine 0 completes at 3,
    machine 1 at 2 + 4 = 6, so machine 0 (0..3).  C_max = 3."""
    pr = wl.Problem(o=[2], p=[[2], [3]], q=[1, 1], R=[0, 0], D=[100, 100], Qmax=10,
                    pm=[[5, 2], [3, 4]], qm=[[1, 1], [1, 1]])
    inst = oracle.Instance(pr)
    r = inst.decode(np.array([2, 1], np.int16), None, ORDER_STAGE, MACH_EARLIEST)
    assert r["S"].ravel().tolist() == [0, 0] and r["M"].ravel().tolist() == [1, 0]
    assert r["cmax"] == 3
    # machine genes: job 0 on machine 0 takes 5
    r = inst.decode(np.array([2, 1], np.int16), np.array([0, 1], np.int8), ORDER_STAGE, MACH_GENE)
    assert r["S"].ravel().tolist() == [0, 0] and r["cmax"] == 5


def test_unrelated_hand_example_power():
    """Q_jsm per job: job 0 draws 3 on machine 0 and 1 on machine 1, job 1 draws 2 on
    either; peak 3.  Job 0 (p 2 / 2) goes to machine 0 at 0 (ties to the lower index).
    Job 1 (p 1 / 1): machine 1 is free but 3 + 2 > 3 until job 0 ends at 2, on either
    machine; machine 0 is free at 2 as well, so job 1 runs on machine 0 at 2..3."""
    pr = wl.Problem(o=[2], p=[[2], [1]], q=[3, 2], R=[0, 0], D=[100, 100], Qmax=3,
                    pm=[[2, 2], [1, 1]], qm=[[3, 1], [2, 2]])
    inst = oracle.Instance(pr)
    r = inst.decode(np.array([2, 1], np.int16), None, ORDER_STAGE, MACH_EARLIEST)
    assert r["S"].ravel().tolist() == [0, 2] and r["M"].ravel().tolist() == [0, 0]
    check_invariants(inst, r["S"], r["M"], obj=r["obj"], tard=r["tard"], cmax=r["cmax"])


@pytest.mark.parametrize("seed", [1, 2])
def test_unrelated_replicated_tables_equal_identical_machines(seed):
    """Per-machine tables that repeat each op's time and each machine's power reduce to the
    identical-machine model: the same schedules in every mode, along a rescheduling chain."""
    rng = np.random.default_rng(seed)
    pr = wl.random_instance(rng, 12, 3, 1, 3, 30, 5, 20, 55)
    off = np.concatenate([[0], np.cumsum(pr.o)])
    rep = lambda p: np.concatenate([np.repeat(p[:, s:s + 1], pr.o[s], axis=1) for s in range(pr.g)], axis=1)
    pr_u = wl.Problem(o=pr.o, p=pr.p, q=pr.q, R=pr.R, D=pr.D, Qmax=pr.Qmax, pm=rep(pr.p),
                      qm=np.tile(pr.q, (pr.N, 1)))
    a, b = oracle.Instance(pr), oracle.Instance(pr_u)
    for ev in range(3):
        Y, X = wl.random_chromosomes(rng, 20, a.K, a.gene_machines())
        for i in range(20):
            for order, mach in ((ORDER_STAGE, MACH_EARLIEST), (ORDER_TOPO, MACH_GENE), (ORDER_STAGE, MACH_GENE)):
                ra, rb = a.decode(Y[i], X[i], order, mach), b.decode(Y[i], X[i], order, mach)
                assert ra["obj"] == rb["obj"] and np.array_equal(ra["S"], rb["S"]) and np.array_equal(ra["M"], rb["M"])
        r = a.decode(Y[0], X[0])
        t_now = a.RS + (r["cmax"] - a.RS) // 3
        arr = wl.random_arrivals(rng, 2, pr.g, t_now, 30)
        arr_u = wl.Arrivals(p=arr.p, R=arr.R, D=arr.D, pm=rep(arr.p), qm=np.tile(pr.q, (arr.n, 1)))
        for inst, ar in ((a, arr), (b, arr_u)):
            inst.commit(r["S"], r["M"])
            inst.reschedule(ar, t_now)
        assert np.array_equal(a.status, b.status)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_unrelated_invariants_and_greedy(seed):
    """Eq. (4)-(10) with per-machine times and powers, and every placement the earliest
    completion (earliest feasible start on each machine, then the earliest end), checked
    on an independent per-instant replay, along a rescheduling chain."""
    rng = np.random.default_rng(seed)
    pr = wl.unrelated_instance(rng, 14, 3, 1, 3, 30, 2, 15, 50)
    inst = oracle.Instance(pr)
    for ev in range(3):
        Y, X = wl.random_chromosomes(rng, 6, inst.K, inst.gene_machines())
        for i in range(6):
            for mach in (MACH_EARLIEST, MACH_GENE):
                r = inst.decode(Y[i], X[i], ORDER_STAGE, mach)
                check_invariants(inst, r["S"], r["M"], obj=r["obj"], tard=r["tard"], cmax=r["cmax"])
                check_greedy_earliest(inst, stage_order(inst, Y[i]), r["S"], r["M"],
                                      any_machine=mach == MACH_EARLIEST)
        inst.commit(r["S"], r["M"])
        t_now = inst.RS + (r["cmax"] - inst.RS) // 3
        inst.reschedule(wl.unrelated_arrivals(rng, 3, pr.o, t_now, 30, 2, 15, pr.Qmax), t_now)


# ---------------------------------------------------------------- idle-gap insertion (option)

def test_insert_hand_example():
    """One machine.  Job A (released at 10, p 5) is assigned first and runs 10..15.  Job B
    (released at 0, p 3) comes second: appended it waits for A (15..18); inserted it fills
    the idle gap before A (0..3)."""
    pr = wl.Problem(o=[1], p=[[5], [3]], q=[1], R=[10, 0], D=[100, 100], Qmax=5)
    inst = oracle.Instance(pr)
    y = np.array([2, 1], np.int16)
    a = inst.decode(y, None, ORDER_STAGE, MACH_EARLIEST)
    b = inst.decode(y, None, ORDER_STAGE, MACH_EARLIEST | oracle.PLACE_INSERT)
    assert a["S"].ravel().tolist() == [10, 15] and a["cmax"] == 18
    assert b["S"].ravel().tolist() == [10, 0] and b["cmax"] == 15


def test_insert_gap_too_short_or_power_bound():
    """The gap before A (0..10) holds B only if B fits in it and the power allows: with
    p_B = 11 it does not fit, so B follows A; with a second job C drawing power over 0..4
    that leaves no room for B, B starts once C ends."""
    pr = wl.Problem(o=[1, 1], p=[[5, 1], [11, 1], [4, 1]], q=[2, 2], R=[10, 0, 0], D=[99] * 3, Qmax=3)
    inst = oracle.Instance(pr)
    # genes job-major: A0 A1 B0 B1 C0 C1; stage 0 order A, B, C (B too long for the gap)
    y = np.array([6, 3, 5, 2, 4, 1], np.int16)
    r = inst.decode(y, None, ORDER_STAGE, MACH_EARLIEST | oracle.PLACE_INSERT)
    assert r["S"][1, 0] == 15  # after A
    # C (p 4) fits the gap 0..10 on machine 0 of stage 0
    assert r["S"][2, 0] == 0
    check_invariants(inst, r["S"], r["M"], obj=r["obj"], tard=r["tard"], cmax=r["cmax"])
    # stage 1 (one machine, power 2 each, peak 3): ops cannot overlap each other in power
    # either; A1 after A0 ends (15), C1 fills the gap before it
    assert r["S"][2, 1] == 4


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_insert_invariants_and_greedy(seed):
    """Eq. (4)-(10) on insertion schedules and every placement the earliest idle, power-
    feasible start (earliest completion across machines), checked by the independent
    replay; identical and unrelated machines, along a rescheduling chain."""
    rng = np.random.default_rng(seed)
    for pr in (wl.random_instance(rng, 12, 3, 1, 3, 30, 5, 20, 55, release_hi=40),
               wl.unrelated_instance(rng, 12, 3, 1, 3, 30, 2, 15, 50)):
        inst = oracle.Instance(pr)
        for ev in range(3):
            Y, X = wl.random_chromosomes(rng, 5, inst.K, inst.gene_machines())
            for i in range(5):
                for mach in (MACH_EARLIEST, MACH_GENE):
                    r = inst.decode(Y[i], X[i], ORDER_STAGE, mach | oracle.PLACE_INSERT)
                    check_invariants(inst, r["S"], r["M"], obj=r["obj"], tard=r["tard"], cmax=r["cmax"])
                    check_greedy_earliest(inst, stage_order(inst, Y[i]), r["S"], r["M"],
                                          any_machine=mach == MACH_EARLIEST, insert=True)
            inst.commit(r["S"], r["M"])
            t_now = inst.RS + (r["cmax"] - inst.RS) // 3
            arr = (wl.random_arrivals(rng, 3, pr.g, t_now, 30) if pr.pm is None else
                   wl.unrelated_arrivals(rng, 3, pr.o, t_now, 30, 2, 15, pr.Qmax))
            inst.reschedule(arr, t_now)


def test_insert_equals_append_without_gaps():
    """One stage, every release at 0 and a peak no schedule reaches: each machine runs its
    ops back to back from 0, no gap ever opens, and insertion gives the appended schedule."""
    rng = np.random.default_rng(9)
    pr = wl.random_instance(rng, 10, 1, 3, 3, 30, 5, 20, 100)
    pr.Qmax = int(pr.q.sum())
    inst = oracle.Instance(pr)
    for _ in range(10):
        y = (rng.permutation(inst.K) + 1).astype(np.int16)
        a = inst.decode(y, None, ORDER_STAGE, MACH_EARLIEST)
        b = inst.decode(y, None, ORDER_STAGE, MACH_EARLIEST | oracle.PLACE_INSERT)
        assert np.array_equal(a["S"], b["S"]) and np.array_equal(a["M"], b["M"])


def test_insert_ga_runs():
    """The GA with insertion keeps valid populations and is elitist."""
    inst = oracle.Instance(wl.static_small(3))
    ga = oracle.GA(inst, P=32, island=16, seed=2, mach_mode=MACH_GENE | oracle.PLACE_INSERT).init()
    best = ga.bobj.min()
    for _ in range(5):
        ga.step()
        assert ga.bobj.min() <= best
        best = ga.bobj.min()
    for i in range(32):
        assert sorted(ga.Y[i, :ga.K].tolist()) == list(range(1, ga.K + 1))
