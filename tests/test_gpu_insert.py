"""Idle-gap insertion placement (an option beside Alg. 2's append placement) on the GPU vs
the oracle, bit for bit: decoding with identical and unrelated machines along
rescheduling chains, the global-profile fallback, GA runs, and the refused combinations."""
import numpy as np
import pytest

import oracle
from paper_1903_10741_gb300 import ffs
from paper_1903_10741_gb300 import workloads as wl
from test_gpu_decode import compare

pytestmark = pytest.mark.gpu

INS_MODES = [(ffs.ORDER_STAGE, ffs.MACH_EARLIEST | ffs.PLACE_INSERT),
             (ffs.ORDER_STAGE, ffs.MACH_GENE | ffs.PLACE_INSERT)]


@pytest.mark.parametrize("mode", INS_MODES)
@pytest.mark.parametrize("unrelated", [False, True])
def test_insert_chain_decode(mode, unrelated):
    rng = np.random.default_rng(31 + unrelated)
    pr = (wl.unrelated_instance(rng, 36, 4, 1, 4, 60, 2, 20, 50) if unrelated else
          wl.random_instance(rng, 36, 4, 1, 4, 60, 5, 20, 55, release_hi=150))
    lib_i, orc_i = ffs.Instance(pr), oracle.Instance(pr)
    for ev in range(3):
        Y, X = wl.random_chromosomes(rng, 133, orc_i.K, orc_i.gene_machines())
        compare(lib_i, orc_i, Y, X, *mode, schedule=True, sample=range(0, 133, 4))
        compare(lib_i, orc_i, Y, X, *mode, schedule=False, sample=range(1, 133, 7))
        r = orc_i.decode(Y[0], X[0], *mode)
        orc_i.commit(r["S"], r["M"])
        lib_i.commit(r["S"], r["M"])
        t_now = orc_i.RS + (r["cmax"] - orc_i.RS) // 3
        arr = (wl.unrelated_arrivals(rng, 5, pr.o, t_now, 60, 2, 20, pr.Qmax) if unrelated else
               wl.random_arrivals(rng, 5, pr.g, t_now, 60))
        orc_i.reschedule(arr, t_now)
        lib_i.reschedule(arr, t_now)


def test_insert_differs_from_append_and_fallback():
    """On a 220-job, 8-stage instance (global profiles) insertion schedules equal the
    oracle's, and differ from appended ones somewhere."""
    import torch
    rng = np.random.default_rng(33)
    pr = wl.random_instance(rng, 220, 8, 2, 5, 99, 5, 30, 40, release_hi=2000)
    lib_i, orc_i = ffs.Instance(pr), oracle.Instance(pr)
    Y, X = wl.random_chromosomes(rng, 24, orc_i.K, orc_i.gene_machines())
    ins = compare(lib_i, orc_i, Y, X, *INS_MODES[0], schedule=False, sample=range(0, 24, 6))
    app = lib_i.decode(torch.from_numpy(Y).cuda(), None, ffs.ORDER_STAGE, ffs.MACH_EARLIEST)["obj"].cpu().numpy()
    assert (ins != app).any()


@pytest.mark.parametrize("mach", [ffs.MACH_EARLIEST, ffs.MACH_GENE])
def test_insert_ga_run_matches_oracle(mach):
    rng = np.random.default_rng(34)
    pr = wl.random_instance(rng, 24, 3, 2, 4, 40, 5, 20, 50, release_hi=80)
    lib_i, orc_i = ffs.Instance(pr), oracle.Instance(pr)
    kw = dict(P=128, island=32, tour_k=2, pc=(4, 5), pm=(1, 10), migrate_every=3, seed=6)
    pop = ffs.Population(lib_i, **kw, mach_mode=mach | ffs.PLACE_INSERT)
    ga = oracle.GA(orc_i, **kw, mach_mode=mach | oracle.PLACE_INSERT).init()
    for _ in range(3):
        pop.run(4, want_schedule=False)
        ga.step(4)
        d = pop.read()
        assert np.array_equal(d["Y"], ga.Y[:, :ga.K]) and np.array_equal(d["obj"], ga.obj)
    res = pop.run(0)
    y, x, obj = ga.best()
    ref = orc_i.decode(y, x, oracle.ORDER_STAGE, mach | oracle.PLACE_INSERT)
    assert res["obj"] == obj == ref["obj"] and np.array_equal(res["S"], ref["S"])


def test_insert_refused_combinations():
    import torch
    inst = ffs.Instance(wl.static_small(1))
    y = torch.from_numpy((np.random.default_rng(0).permutation(inst.K) + 1).astype(np.int16)[None, :]).cuda()
    with pytest.raises(ffs.FFSError):
        inst.decode(y, None, ffs.ORDER_TOPO, ffs.MACH_EARLIEST | ffs.PLACE_INSERT)
    with pytest.raises(ffs.FFSError):
        ffs.Batch([inst], P=128, island=64, mach_mode=ffs.MACH_EARLIEST | ffs.PLACE_INSERT)
