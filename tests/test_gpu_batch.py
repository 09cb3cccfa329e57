"""The batched persistent GA: every instance of a batch equals its own single-population
run (and the oracle), whatever the launch mapping; the tuner leaves the state intact."""
import numpy as np
import pytest

import oracle
from paper_1903_10741_gb300 import ffs
from paper_1903_10741_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _problems(count, seed, n_hi=40):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = int(rng.integers(5, n_hi + 1))
        g = int(rng.integers(2, 6))
        out.append(wl.random_instance(rng, N, g, 1, 5, 60, 3, 25, int(rng.integers(40, 71)),
                                      release_hi=int(rng.integers(0, 50))))
    return out


def _same(a, b, gene):
    for k in ("Y", "obj", "fit", "bY", "bobj", "bfit", "gen", "emax"):
        assert np.array_equal(a[k], b[k]), k
    if gene:
        assert np.array_equal(a["X"], b["X"])


@pytest.mark.parametrize("mode", [(ffs.ORDER_STAGE, ffs.MACH_EARLIEST), (ffs.ORDER_TOPO, ffs.MACH_GENE)])
def test_batch_equals_single_runs(mode):
    probs = _problems(11, 5)
    kw = dict(P=64, island=16, tour_k=2, pc=(4, 5), pm=(1, 5), order_mode=mode[0], mach_mode=mode[1],
              migrate_every=3, seed=42)
    insts = [ffs.Instance(p) for p in probs]
    batch = ffs.Batch(insts, instance_id=100, **kw)
    batch.run(4)
    batch.run(3)
    for i, p in enumerate(probs):
        single = ffs.Population(ffs.Instance(p), instance_id=100 + i, **kw)
        single.run(7, want_schedule=False)
        _same(batch.read(i), single.read(), mode[1] == ffs.MACH_GENE)
    # two instances against the oracle itself
    for i in (0, 7):
        ga = oracle.GA(oracle.Instance(probs[i]), instance_id=100 + i, **kw).init()
        ga.step(7)
        d = batch.read(i)
        K = ga.K
        assert np.array_equal(d["obj"], ga.obj) and np.array_equal(d["Y"], ga.Y[:, :K])
        assert np.array_equal(d["bobj"], ga.bobj)


def test_mapping_does_not_change_results_and_tuner_restores():
    probs = _problems(9, 8, n_hi=60)
    kw = dict(P=128, island=32, seed=3, migrate_every=4)
    a = ffs.Batch([ffs.Instance(p) for p in probs], **kw)
    b = ffs.Batch([ffs.Instance(p) for p in probs], **kw)
    b.set_config(4, 56 * 1024, 2)
    assert b.config()["cluster"] == 2
    c = ffs.Batch([ffs.Instance(p) for p in probs], **kw)
    chosen = c.tune(2)
    assert chosen["warps_per_cta"] in (4, 8, 16, 32) and chosen["ms_per_generation"] > 0
    for x in (a, b, c):
        x.run(9)
    for i in range(len(probs)):
        ra, rb, rc = a.read(i), b.read(i), c.read(i)
        assert ra["gen"] == 9
        _same(ra, rb, False)
        _same(ra, rc, False)


def test_batch_results_are_committed_best_schedules():
    probs = _problems(5, 13)
    kw = dict(P=64, island=32, seed=9)
    insts = [ffs.Instance(p) for p in probs]
    batch = ffs.Batch(insts, **kw)
    res = batch.run(6, results=True)
    for i, p in enumerate(probs):
        single = ffs.Population(ffs.Instance(p), instance_id=i, **kw)
        r = single.run(6)
        assert res[i]["obj"] == r["obj"] and np.array_equal(res[i]["S"], r["S"])
    # committed: the instance can now be rescheduled at a later point
    insts[0].reschedule(wl.Arrivals(p=np.ones((1, probs[0].g)), R=[5], D=[99]), 5)


def test_batched_workload_shape_sampled():
    """32 instances of the batched workload's shape (sizes U{20..200} x U{3..8}), each a
    rescheduling snapshot; population 512, 3 generations; three instances checked
    against their single-population runs."""
    import torch
    items = wl.batched(32, seed=1)
    insts, probs = [], []
    for it in items:
        inst = ffs.Instance(it.problem)
        K = inst.K
        y = np.random.default_rng(it.plan_seed).permutation(K).astype(np.int16) + 1
        yd = torch.from_numpy(y[None, :]).cuda()
        cm = int(inst.decode(yd)["cmax"][0])
        sch = inst.decode(yd, schedule=True)
        inst.commit(sch["S"][0].cpu().numpy(), sch["M"][0].cpu().numpy())
        t_now = it.rs_permille * cm // 1000
        arr = wl.random_arrivals(np.random.default_rng(it.arrival_seed), it.arrivals_n, it.problem.g, t_now, 99)
        inst.reschedule(arr, t_now)
        insts.append(inst)
        probs.append((it, sch["S"][0].cpu().numpy(), sch["M"][0].cpu().numpy(), t_now, arr))
    kw = dict(P=512, island=64, seed=1)
    batch = ffs.Batch(insts, **kw)
    batch.run(3)
    for i in (0, 13, 31):
        it, S, M, t_now, arr = probs[i]
        inst = ffs.Instance(it.problem)
        inst.commit(S, M)
        inst.reschedule(arr, t_now)
        single = ffs.Population(inst, instance_id=i, **kw)
        single.run(3, want_schedule=False)
        _same(batch.read(i), single.read(), False)


def test_stop_request_ends_a_run_at_generation_boundaries():
    """ga_batch_stop from another thread ends a long persistent run early; every instance is
    left after a whole number of generations, equal to its own single run of that many, and
    the batch runs on normally afterwards.  A request made while no run is in progress is
    cleared by the next run."""
    import threading
    import time

    probs = _problems(12, 21)
    kw = dict(P=64, island=16, tour_k=2, pc=(4, 5), pm=(1, 5), migrate_every=3, seed=9)
    batch = ffs.Batch([ffs.Instance(p) for p in probs], instance_id=300, **kw)
    batch.stop()  # no run in progress: the next run clears it
    batch.run(2)
    assert all(batch.read(i)["gen"] == 2 for i in range(len(probs)))

    G = 200000  # far longer than the test waits
    box = {}

    def worker():
        try:
            batch.run(G)
            box["rc"] = ffs.FFS_OK
        except ffs.FFSError as e:
            box["rc"] = e.code

    th = threading.Thread(target=worker)
    t0 = time.perf_counter()
    th.start()
    time.sleep(0.3)
    batch.stop()
    th.join(timeout=120)
    assert not th.is_alive()
    assert box["rc"] == ffs.E_STOPPED
    assert time.perf_counter() - t0 < 60
    gens = [batch.read(i)["gen"] for i in range(len(probs))]
    assert all(2 < g < 2 + G for g in gens), gens
    for i, p in enumerate(probs):
        single = ffs.Population(ffs.Instance(p), instance_id=300 + i, **kw)
        single.run(gens[i], want_schedule=False)
        _same(batch.read(i), single.read(), False)
    # the next run starts from each instance's own generation
    batch.run(3)
    for i, p in enumerate(probs):
        single = ffs.Population(ffs.Instance(p), instance_id=300 + i, **kw)
        single.run(gens[i] + 3, want_schedule=False)
        _same(batch.read(i), single.read(), False)
