"""The traditional static approach (Sec. 4.1 Fig. 7, Sec. 5.3) on the GPU vs the oracle:
decoding with the kept plan's fixed ops, and whole GA runs, bit for bit."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1903_10741_gb300 import ffs
from paper_1903_10741_gb300 import workloads as wl
from test_gpu_decode import MODES, compare

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", MODES)
def test_static_chain_decode(mode):
    """Three static events on the dynamic workload: fixed ops draw power over their
    planned interval and block their machines; only new jobs are decoded."""
    dyn = wl.dynamic_medium(2)
    lib_i, orc_i = ffs.Instance(dyn.problem), oracle.Instance(dyn.problem)
    rng = np.random.default_rng(5)
    Y, X = wl.random_chromosomes(rng, 1, orc_i.K, orc_i.gene_machines())
    r = orc_i.decode(Y[0], X[0], *mode)
    for ev, (t_now, arr) in enumerate(dyn.events):
        orc_i.commit(r["S"], r["M"])
        lib_i.commit(r["S"], r["M"])
        orc_i.reschedule(arr, t_now, static=True)
        lib_i.reschedule(arr, t_now, static=True)
        assert np.array_equal(lib_i.status(), orc_i.status)
        Y, X = wl.random_chromosomes(rng, 130, orc_i.K, orc_i.gene_machines())
        compare(lib_i, orc_i, Y, X, *mode, schedule=True, sample=range(0, 130, 3))
        r = orc_i.decode(Y[0], X[0], *mode)


def test_static_worked_example_fig7_on_gpu():
    """Table 4 kept at RS = 7, jobs 6 and 7 appended: the earliest-machine decode gives
    Fig. 7's C_max = 19.91 for every order of the six new ops tried here."""
    import torch
    ex = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")))
    n0 = ex["n_original"]
    pst = np.array(ex["p_per_stage"])
    prob = wl.Problem(o=ex["o"], p=np.tile(pst, (n0, 1)), q=np.ones(6), R=ex["R"][:n0],
                      D=np.full(n0, 10**6), Qmax=ex["Qmax"], WT=ex["WT"])
    arr = wl.Arrivals(p=np.tile(pst, (2, 1)), R=ex["R"][n0:], D=[10**6] * 2)
    lib_i, orc_i = ffs.Instance(prob), oracle.Instance(prob)
    for inst in (lib_i, orc_i):
        inst.commit(np.array(ex["S_original"]), np.array(ex["M_original"]))
        inst.reschedule(arr, ex["RS"], static=True)
    rng = np.random.default_rng(0)
    Y = np.stack([rng.permutation(6) + 1 for _ in range(64)]).astype(np.int16)
    X = np.zeros_like(Y, dtype=np.int8)
    compare(lib_i, orc_i, Y, X, ffs.ORDER_STAGE, ffs.MACH_EARLIEST)
    out = lib_i.decode(torch.from_numpy(Y).cuda(), None, ffs.ORDER_STAGE, ffs.MACH_EARLIEST)
    assert (out["cmax"].cpu().numpy() == 1991).all()


def test_static_ga_run_matches_oracle():
    """The GA over the new jobs only, after a static event, equals the oracle's run."""
    dyn = wl.dynamic_medium(1)
    lib_i, orc_i = ffs.Instance(dyn.problem), oracle.Instance(dyn.problem)
    kw = dict(P=256, island=64, tour_k=2, pc=(4, 5), pm=(1, 10), seed=4)
    pop = ffs.Population(lib_i, **kw, instance_id=0)
    res = pop.run(6)
    ga = oracle.GA(orc_i, **kw, instance_id=0).init().step(6)
    y, x, _ = ga.best()
    ref = orc_i.decode(y, x)
    assert res["obj"] == ref["obj"]
    orc_i.commit(ref["S"], ref["M"])
    t_now, arr = dyn.events[0]
    lib_i.reschedule(arr, t_now, static=True)
    orc_i.reschedule(arr, t_now, static=True)
    pop2 = ffs.Population(lib_i, **kw, instance_id=1)
    ga2 = oracle.GA(orc_i, **kw, instance_id=1).init()
    for _ in range(3):
        pop2.run(4, want_schedule=False)
        ga2.step(4)
        d = pop2.read()
        assert np.array_equal(d["Y"], ga2.Y[:, :ga2.K]) and np.array_equal(d["obj"], ga2.obj)
    res2 = pop2.run(0)
    y2, x2, o2 = ga2.best()
    assert res2["obj"] == o2 == orc_i.decode(y2, x2)["obj"]
