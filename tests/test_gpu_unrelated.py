"""Unrelated parallel machines (Table 2: P_jsm, Q_jsm per job and machine) on the GPU vs the
oracle, bit for bit: decoding in every mode along a rescheduling chain, the reduction to
identical machines, whole GA runs, and the global-profile fallback."""
import numpy as np
import pytest

import oracle
from paper_1903_10741_gb300 import ffs
from paper_1903_10741_gb300 import workloads as wl
from test_gpu_decode import MODES, compare

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", MODES)
def test_unrelated_chain_decode(mode):
    rng = np.random.default_rng(21)
    pr = wl.unrelated_instance(rng, 40, 4, 1, 4, 60, 2, 20, 50)
    lib_i, orc_i = ffs.Instance(pr), oracle.Instance(pr)
    for ev in range(3):
        Y, X = wl.random_chromosomes(rng, 197, orc_i.K, orc_i.gene_machines())
        compare(lib_i, orc_i, Y, X, *mode, schedule=True, sample=range(0, 197, 4))
        compare(lib_i, orc_i, Y, X, *mode, schedule=False, sample=range(1, 197, 9))
        r = orc_i.decode(Y[0], X[0], *mode)
        orc_i.commit(r["S"], r["M"])
        lib_i.commit(r["S"], r["M"])
        t_now = orc_i.RS + (r["cmax"] - orc_i.RS) // 3
        arr = wl.unrelated_arrivals(rng, 6, pr.o, t_now, 60, 2, 20, pr.Qmax)
        orc_i.reschedule(arr, t_now)
        lib_i.reschedule(arr, t_now)
        assert np.array_equal(lib_i.status(), orc_i.status)


def test_unrelated_replicated_tables_equal_identical_on_gpu():
    """The unrelated-machine kernels on tables that repeat the identical-machine values
    give the identical-machine kernels' schedules."""
    import torch
    rng = np.random.default_rng(22)
    pr = wl.random_instance(rng, 30, 4, 1, 4, 50, 5, 20, 55)
    rep = lambda p: np.concatenate([np.repeat(p[:, s:s + 1], pr.o[s], axis=1) for s in range(pr.g)], axis=1)
    pu = wl.Problem(o=pr.o, p=pr.p, q=pr.q, R=pr.R, D=pr.D, Qmax=pr.Qmax, pm=rep(pr.p), qm=np.tile(pr.q, (pr.N, 1)))
    a, b = ffs.Instance(pr), ffs.Instance(pu)
    Y, X = wl.random_chromosomes(rng, 256, a.K, oracle.Instance(pr).gene_machines())
    yd, xd = torch.from_numpy(Y).cuda(), torch.from_numpy(X).cuda()
    for order, mach in MODES:
        ra = a.decode(yd, xd, order, mach, schedule=True)
        rb = b.decode(yd, xd, order, mach, schedule=True)
        for k in ("obj", "S", "M"):
            assert torch.equal(ra[k], rb[k]), (order, mach, k)


@pytest.mark.parametrize("mach", [ffs.MACH_EARLIEST, ffs.MACH_GENE])
def test_unrelated_ga_run_matches_oracle(mach):
    rng = np.random.default_rng(23)
    pr = wl.unrelated_instance(rng, 20, 3, 2, 4, 40, 2, 15, 50)
    lib_i, orc_i = ffs.Instance(pr), oracle.Instance(pr)
    kw = dict(P=128, island=32, tour_k=2, pc=(4, 5), pm=(1, 10), migrate_every=3, seed=8)
    pop = ffs.Population(lib_i, **kw, mach_mode=mach)
    ga = oracle.GA(orc_i, **kw, mach_mode=mach).init()
    for _ in range(4):
        pop.run(3, want_schedule=False)
        ga.step(3)
        d = pop.read()
        assert np.array_equal(d["Y"], ga.Y[:, :ga.K]) and np.array_equal(d["obj"], ga.obj)
        if mach == ffs.MACH_GENE:
            assert np.array_equal(d["X"], ga.X[:, :ga.K])
    res = pop.run(0)
    y, x, obj = ga.best()
    ref = orc_i.decode(y, x, oracle.ORDER_STAGE, mach)
    assert res["obj"] == obj == ref["obj"] and np.array_equal(res["S"], ref["S"]) and np.array_equal(res["M"], ref["M"])


def test_unrelated_global_profile_fallback():
    """A 220-job, 8-stage unrelated instance whose schedules outgrow the shared-memory
    profile: the global-memory path gives the oracle's results."""
    rng = np.random.default_rng(24)
    pr = wl.unrelated_instance(rng, 220, 8, 2, 5, 99, 2, 20, 40)
    lib_i, orc_i = ffs.Instance(pr), oracle.Instance(pr)
    Y, X = wl.random_chromosomes(rng, 40, orc_i.K, orc_i.gene_machines())
    compare(lib_i, orc_i, Y, X, ffs.ORDER_STAGE, ffs.MACH_EARLIEST, schedule=False, sample=range(0, 40, 5))
    compare(lib_i, orc_i, Y, X, ffs.ORDER_STAGE, ffs.MACH_GENE, schedule=False, sample=range(2, 40, 5))


def test_batch_refuses_unrelated_instances():
    rng = np.random.default_rng(25)
    inst = ffs.Instance(wl.unrelated_instance(rng, 10, 2, 1, 2, 20, 2, 10, 60))
    with pytest.raises(ffs.FFSError):
        ffs.Batch([inst], P=128, island=64)
