"""Whole GA runs on the GPU vs the CPU oracle: every generation's population, objectives,
fitness and island best-ever individuals are bit-identical (all integer, one Philox map)."""
import numpy as np
import pytest

import oracle
from paper_1903_10741_gb300 import ffs
from paper_1903_10741_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def assert_same_state(pop, ga, K, gene_mode):
    d = pop.read()
    assert d["gen"] == ga.gen
    assert d["emax"] == ga.emax
    assert np.array_equal(d["obj"], ga.obj), np.nonzero(d["obj"] != ga.obj)
    assert np.array_equal(d["fit"], ga.fit)
    assert np.array_equal(d["Y"], ga.Y[:, :K])
    if gene_mode:
        assert np.array_equal(d["X"], ga.X[:, :K])
    assert np.array_equal(d["bobj"], ga.bobj)
    assert np.array_equal(d["bY"], ga.bY[:, :K])


def _pair(problem, **kw):
    lib_i, orc_i = ffs.Instance(problem), oracle.Instance(problem)
    pop = ffs.Population(lib_i, **kw)
    okw = dict(kw)
    ga = oracle.GA(orc_i, **okw).init()
    return lib_i, orc_i, pop, ga


def test_static_small_full_run_every_generation():
    """10 jobs, 3 stages [2,3,2], population 64, 100 generations, k = 2, pc 0.8, pm 0.1."""
    lib_i, orc_i, pop, ga = _pair(wl.static_small(1), P=64, island=64, tour_k=2, pc=(4, 5), pm=(1, 10), seed=1)
    K = orc_i.K
    assert_same_state(pop, ga, K, False)
    for g in range(100):
        pop.run(1, want_schedule=False)
        ga.step()
        assert_same_state(pop, ga, K, False)
    res = pop.run(0)
    y, x, obj = ga.best()
    ref = orc_i.decode(y, x, oracle.ORDER_STAGE, oracle.MACH_EARLIEST)
    assert res["obj"] == obj == ref["obj"]
    assert np.array_equal(res["S"], ref["S"]) and np.array_equal(res["M"], ref["M"])


def test_paper_mode_islands_and_migration():
    """Alg. 1 topological order, machine genes, 5-neighbourhood selection on the 8x8 torus,
    islands of 16, pc 0.9, ring migration every 5 generations."""
    kw = dict(P=64, island=16, tour_k=0, pc=(9, 10), pm=(1, 10), order_mode=ffs.ORDER_TOPO,
              mach_mode=ffs.MACH_GENE, migrate_every=5, seed=5)
    lib_i, orc_i, pop, ga = _pair(wl.static_small(2), **kw)
    for _ in range(6):
        pop.run(5, want_schedule=False)
        ga.step(5)
        assert_same_state(pop, ga, orc_i.K, True)


def test_tournament3_machine_genes():
    kw = dict(P=128, island=32, tour_k=3, pc=(3, 4), pm=(1, 5), order_mode=ffs.ORDER_STAGE,
              mach_mode=ffs.MACH_GENE, migrate_every=4, seed=77, instance_id=9)
    rng = np.random.default_rng(4)
    prob = wl.random_instance(rng, 23, 4, 1, 4, 40, 2, 12, 45, release_hi=60)
    lib_i, orc_i, pop, ga = _pair(prob, **kw)
    pop.run(13, want_schedule=False)
    ga.step(13)
    assert_same_state(pop, ga, orc_i.K, True)


def test_dynamic_chain_reduced_generations():
    """50 jobs, 5 stages, population 1024 (16 islands), 3 rescheduling events; each solve
    runs 12 generations; the best schedule is committed and frozen at the next event."""
    dyn = wl.dynamic_medium(1)
    lib_i, orc_i = ffs.Instance(dyn.problem), oracle.Instance(dyn.problem)
    for solve in range(len(dyn.events) + 1):
        kw = dict(P=1024, island=64, tour_k=2, pc=(4, 5), pm=(1, 10), seed=1, instance_id=solve)
        pop = ffs.Population(lib_i, **kw)
        ga = oracle.GA(orc_i, **kw).init()
        res = pop.run(12)
        ga.step(12)
        assert_same_state(pop, ga, orc_i.K, False)
        y, x, obj = ga.best()
        ref = orc_i.decode(y, x, oracle.ORDER_STAGE, oracle.MACH_EARLIEST)
        assert res["obj"] == ref["obj"]
        assert np.array_equal(res["S"], ref["S"])
        orc_i.commit(ref["S"], ref["M"])
        pop.close()
        if solve < len(dyn.events):
            t_now, arr = dyn.events[solve]
            orc_i.reschedule(arr, t_now)
            lib_i.reschedule(arr, t_now)


def test_split_runs_and_checkpoint_restore():
    prob = wl.static_small(3)
    kw = dict(P=64, island=32, seed=11)
    lib_i = ffs.Instance(prob)
    a = ffs.Population(lib_i, **kw)
    a.run(7, want_schedule=False)
    ck = a.checkpoint()
    a.run(8, want_schedule=False)
    sa = a.read()
    b = ffs.Population(lib_i, **kw)
    b.restore(ck)
    assert b.read()["gen"] == 7
    b.run(8, want_schedule=False)
    sb = b.read()
    for k in ("Y", "obj", "fit", "bY", "bobj"):
        assert np.array_equal(sa[k], sb[k])
    ga = oracle.GA(oracle.Instance(prob), **kw).init()
    ga.step(15)
    assert_same_state(b, ga, ga.K, False)


def test_stale_population_rejected():
    lib_i = ffs.Instance(wl.static_small(1))
    pop = ffs.Population(lib_i, P=64, seed=1)
    pop.run(2)
    lib_i.reschedule(wl.Arrivals(p=np.ones((1, 3)), R=[5], D=[99]), 5)
    with pytest.raises(ffs.FFSError) as e:
        pop.run(1)
    assert e.value.code == -7


def test_service_sized_instance_sampled():
    """The service workload's largest shape: 500 jobs, 10 stages of U{2..8} machines, p up
    to 199 (K = 5000 genes), population 2048 after one generation; sampled rows of the
    device population decode in the oracle to the objectives the GPU recorded."""
    rng = np.random.default_rng(41)
    prob = wl.random_instance(rng, 500, 10, 2, 8, 199, 5, 30, 55)
    lib_i, orc_i = ffs.Instance(prob), oracle.Instance(prob)
    pop = ffs.Population(lib_i, P=2048, island=64, seed=3)
    pop.run(1, want_schedule=False)
    d = pop.read()
    assert d["gen"] == 1 and d["Y"].shape[1] == orc_i.K == 5000
    for i in range(0, 2048, 409):
        assert d["obj"][i] == orc_i.decode(d["Y"][i], d["X"][i])["obj"], i
    for isl in range(0, 32, 11):
        assert d["bobj"][isl] == orc_i.decode(d["bY"][isl], d["bX"][isl])["obj"], isl
