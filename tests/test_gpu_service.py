"""Warm start and the rescheduling service on the GPU.

- The warm-started generation 0, and the GA run that follows it, equal the oracle's
  (oracle GA -> commit -> reschedule -> oracle.warm_remap -> GA.init_from) bit for bit.
- Every request's result through the service is the same alone (one request on the device
  at a time) and in a mix (many requests overlapping), and the same as the direct calls
  (ffs_reschedule + ga_population_create(_warm) + ga_run).
- Admission by memory: a budget that holds two populations still completes everything
  with unchanged results; a population larger than the budget is refused; the memory the
  service reports equals ga_population_footprint.
"""
import time

import numpy as np
import pytest

import oracle
from paper_1903_10741_gb300 import ffs
from paper_1903_10741_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GA = dict(P=64, island=16, tour_k=2, pc=(4, 5), pm=(1, 10), seed=3)


def _oracle_chain(problem, events, gens, kw, mach_mode):
    """Oracle: solve, then for each (t_now, arrivals) freeze, warm-start and solve again."""
    inst = oracle.Instance(problem)
    out = []
    ga = oracle.GA(inst, **kw, mach_mode=mach_mode, instance_id=0).init().step(gens)
    for solve, (t_now, arr) in enumerate(events, start=1):
        y, x, _ = ga.best()
        r = inst.decode(y, x, mach_mode=mach_mode)
        inst.commit(r["S"], r["M"])
        keys0 = oracle.gene_keys(inst)
        Y0, X0 = ga.Y[:, :ga.K].copy(), ga.X[:, :ga.K].copy()
        inst.reschedule(arr, t_now)
        Y, X = oracle.warm_remap(Y0, X0, keys0, oracle.gene_keys(inst), kw["P"])
        ga = oracle.GA(inst, **kw, mach_mode=mach_mode, instance_id=solve).init_from(Y, X)
        out.append((Y, X, ga.obj.copy(), ga.emax, ga.bobj.copy()))
        ga.step(gens)
        out.append((ga.Y[:, :ga.K].copy(), ga.X[:, :ga.K].copy(), ga.obj.copy(), ga.emax, ga.bobj.copy()))
    y, x, obj = ga.best()
    return out, obj, inst.decode(y, x, mach_mode=mach_mode)


@pytest.mark.parametrize("mach_mode", [ffs.MACH_EARLIEST, ffs.MACH_GENE])
def test_warm_start_chain_matches_oracle(mach_mode):
    rng = np.random.default_rng(11)
    prob = wl.random_instance(rng, 18, 3, 1, 3, 30, 5, 20, 55)
    events, t = [], 0
    for _ in range(3):
        t += 40
        events.append((t, wl.random_arrivals(rng, 3, 3, t, 30)))
    gens = 7
    ref, ref_obj, ref_dec = _oracle_chain(prob, events, gens, GA, mach_mode)
    inst = ffs.Instance(prob)
    pop = ffs.Population(inst, **GA, mach_mode=mach_mode, instance_id=0)
    pop.run(gens)
    got = []
    for solve, (t_now, arr) in enumerate(events, start=1):
        inst.reschedule(arr, t_now)
        nxt = ffs.Population(inst, **GA, mach_mode=mach_mode, instance_id=solve, prev=pop)
        pop.close()
        pop = nxt
        d = pop.read()
        got.append((d["Y"], d["X"], d["obj"], d["emax"], d["bobj"]))
        res = pop.run(gens)
        d = pop.read()
        got.append((d["Y"], d["X"], d["obj"], d["emax"], d["bobj"]))
    for i, (g_, r_) in enumerate(zip(got, ref)):
        assert np.array_equal(g_[0], r_[0]), f"Y differs at step {i}"
        if mach_mode == ffs.MACH_GENE:
            assert np.array_equal(g_[1], r_[1]), f"X differs at step {i}"
        assert np.array_equal(g_[2], r_[2]) and g_[3] == r_[3] and np.array_equal(g_[4], r_[4]), i
    assert res["obj"] == ref_obj == ref_dec["obj"]
    assert np.array_equal(res["S"], ref_dec["S"]) and np.array_equal(res["M"], ref_dec["M"])


def test_warm_start_identity_when_nothing_changes():
    """Rescheduling at the same point with no new jobs keeps every gene: the warm
    population is the old one row for row."""
    inst = ffs.Instance(wl.static_small(3))
    pop = ffs.Population(inst, **GA)
    pop.run(5, want_schedule=False)  # commits a plan that starts at 0: nothing freezes at 0
    before = pop.read()
    inst.reschedule(wl.Arrivals(np.zeros((0, 3), np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32)), 0)
    warm = ffs.Population(inst, **GA, prev=pop)
    after = warm.read()
    assert np.array_equal(after["Y"], before["Y"]) and np.array_equal(after["obj"], before["obj"])


def _direct(work, gens, kw):
    """Reference: the direct calls, one request after the other."""
    insts = [ffs.Instance(p) for p in work.problems]
    pops, solves, out = {}, {}, []
    for rq in work.requests:
        inst = insts[rq.instance]
        if rq.arrivals is not None or rq.t_now:
            inst.reschedule(rq.arrivals, rq.t_now)
        n = solves.get(rq.instance, 0)
        prev = pops.get(rq.instance)
        pop = ffs.Population(inst, **kw, instance_id=n, prev=prev)
        if prev is not None:
            prev.close()
        pops[rq.instance] = pop
        solves[rq.instance] = n + 1
        r = pop.run(gens)
        out.append((r["obj"], r["S"].ravel().copy(), r["M"].ravel().copy()))
    return out


def _through_service(work, gens, kw, max_active, memory=1 << 30, sequential=False):
    insts = [ffs.Instance(p) for p in work.problems]
    svc = ffs.Service(max_active=max_active, memory_bytes=memory, **kw)
    tickets, infos = [], []
    for rq in work.requests:
        tk = svc.submit(insts[rq.instance], rq.arrivals, rq.t_now, gens)
        tickets.append(tk)
        if sequential:
            infos.append(svc.wait(tk))
    if not sequential:
        infos = [svc.wait(tk) for tk in tickets]
    stats = svc.stats()
    svc.close()
    return infos, stats


def test_service_alone_equals_mix_equals_direct():
    work = wl.service_small(seed=4, n_instances=5, n_requests=16)
    gens = 9
    ref = _direct(work, gens, GA)
    alone, _ = _through_service(work, gens, GA, max_active=1, sequential=True)
    mix, stats = _through_service(work, gens, GA, max_active=6)
    assert stats["completed"] == len(work.requests) and stats["failed"] == 0
    seen = set()
    for i, (r, a, m) in enumerate(zip(ref, alone, mix)):
        first = work.requests[i].instance not in seen
        seen.add(work.requests[i].instance)
        assert a["warm"] == m["warm"] == (0 if first else 1), i
        assert a["obj"] == m["obj"] == r[0], i
        assert np.array_equal(a["S"], r[1]) and np.array_equal(m["S"], r[1]), i
        assert np.array_equal(a["M"], r[2]) and np.array_equal(m["M"], r[2]), i


def test_service_requests_overlap_on_the_device():
    rng = np.random.default_rng(6)
    insts = [ffs.Instance(wl.random_instance(rng, 40, 4, 1, 3, 40, 5, 20, 55)) for _ in range(6)]
    svc = ffs.Service(max_active=6, memory_bytes=1 << 30, **GA)
    tickets = [svc.submit(inst, None, 0, 2000) for inst in insts]
    infos = [svc.wait(tk, schedule=False) for tk in tickets]
    svc.close()
    # distinct instances, all admitted at once: every request was admitted before the
    # first one finished
    first_done = min(i["done_ns"] for i in infos)
    assert all(i["admit_ns"] < first_done for i in infos)


def test_service_memory_admission_and_footprint():
    work = wl.service_small(seed=8, n_instances=4, n_requests=12)
    gens = 6
    ref = _direct(work, gens, GA)
    insts = [ffs.Instance(p) for p in work.problems]
    fp = max(ffs.footprint(i, **GA) for i in insts)
    # room for about two populations (plus the transient gene map) at a time
    budget = 2 * fp + 3 * fp // 4
    svc = ffs.Service(max_active=8, memory_bytes=budget, **GA)
    tickets = [svc.submit(insts[rq.instance], rq.arrivals, rq.t_now, gens) for rq in work.requests]
    infos = [svc.wait(tk) for tk in tickets]
    st = svc.stats()
    assert st["peak_bytes"] <= budget and st["completed"] == len(work.requests)
    # an instance's requests match the direct chain as long as none of them (after its
    # first) had to start cold because its kept population was dropped for memory
    intact, seen, checked = {}, set(), 0
    for i, (r, got) in enumerate(zip(ref, infos)):
        k = work.requests[i].instance
        if k in seen and not got["warm"]:
            intact[k] = False
        seen.add(k)
        if intact.get(k, True):
            assert got["obj"] == r[0] and np.array_equal(got["S"], r[1]), i
            checked += 1
    assert checked >= len(work.problems)
    # what the service holds now is exactly the kept populations' footprints
    held = st["used_bytes"]
    kept = st["warm"]
    assert kept >= 1 and held > 0
    for inst in insts:
        svc.forget(inst)
    for _ in range(200):
        if svc.stats()["used_bytes"] == 0:
            break
        time.sleep(0.01)
    assert svc.stats()["used_bytes"] == 0 and svc.stats()["warm"] == 0
    svc.close()


def test_service_footprint_is_what_a_population_holds():
    """While a request runs its population holds ga_population_footprint; once it is kept
    as the instance's warm state, only the chromosomes (two buffers of int16 Y and int8 X)
    and the generation counter stay, each block rounded to 256 bytes."""
    work = wl.service_small(seed=9, n_instances=1, n_requests=1)
    inst = ffs.Instance(work.problems[0])
    fp = ffs.footprint(inst, **GA)
    K = inst.K
    svc = ffs.Service(max_active=2, memory_bytes=64 << 20, **GA)
    svc.wait(svc.submit(inst, None, 0, 3))
    st = svc.stats()
    r = lambda n: (n + 255) // 256 * 256
    kept = 2 * r(GA["P"] * K * 2) + 2 * r(GA["P"] * K) + r(24) + r(4)
    assert st["used_bytes"] == kept < fp and st["warm"] == 1
    assert st["peak_bytes"] >= fp
    svc.close()


def test_service_refuses_a_population_larger_than_its_memory():
    work = wl.service_small(seed=10, n_instances=1, n_requests=1)
    inst = ffs.Instance(work.problems[0])
    fp = ffs.footprint(inst, **GA)
    svc = ffs.Service(max_active=2, memory_bytes=fp // 2, **GA)
    tk = svc.submit(inst, None, 0, 3)
    with pytest.raises(ffs.FFSError) as e:
        svc.wait(tk)
    assert e.value.code == -6
    # a later request of another instance still runs
    inst2 = ffs.Instance(wl.static_small(1))
    svc2 = ffs.Service(max_active=1, memory_bytes=64 << 20, **GA)
    assert svc2.wait(svc2.submit(inst2, None, 0, 2))["state"] == 2
    svc.close()
    svc2.close()


def test_service_bad_request_fails_alone():
    """A request whose rescheduling point precedes the instance's fails; the others of the
    mix still finish."""
    insts = [ffs.Instance(wl.static_small(s)) for s in (1, 2)]
    svc = ffs.Service(max_active=4, memory_bytes=256 << 20, **GA)
    a = svc.submit(insts[0], None, 0, 3)
    b = svc.submit(insts[1], None, 5, 3)  # no plan yet: t_now must equal RS = 0
    c = svc.submit(insts[0], None, 10, 3)
    assert svc.wait(a)["state"] == 2
    with pytest.raises(ffs.FFSError):
        svc.wait(b)
    assert svc.wait(c)["warm"] == 1
    svc.close()


def test_service_stop_request_ends_requests_early():
    """A long admitted request stopped mid-run finishes with the best schedule of the
    generations it ran, equal to a request of exactly that many; a queued request of the
    same instance stopped before its rescheduling was applied ends with FFS_E_STOPPED and
    leaves the instance alone, so the next request equals the direct calls without it.
    A multi-chunk request that is not stopped equals its direct run too."""
    rng = np.random.default_rng(12)
    prob = wl.random_instance(rng, 30, 4, 1, 3, 40, 5, 20, 55)
    arr = wl.random_arrivals(rng, 4, 4, 60, 40)
    inst = ffs.Instance(prob)
    svc = ffs.Service(max_active=2, memory_bytes=1 << 30, **GA)
    big = 10 ** 6
    t1 = svc.submit(inst, None, 0, big)
    t2 = svc.submit(inst, arr, 60, 50)  # waits behind t1 (same instance)
    time.sleep(0.3)
    svc.stop(t2)
    with pytest.raises(ffs.FFSError) as e:
        svc.wait(t2, timeout_ms=60000)
    assert e.value.code == ffs.E_STOPPED
    svc.stop(t1)
    r1 = svc.wait(t1, timeout_ms=60000)
    assert r1["state"] == 2 and r1["status"] == 0 and 0 < r1["generations"] < big
    t3 = svc.submit(inst, arr, 60, 150)  # three chunks, not stopped
    r3 = svc.wait(t3, timeout_ms=60000)
    assert r3["generations"] == 150 and r3["warm"] == 1
    svc.close()
    # the direct calls: a solve of r1's generation count, then the warm request
    ref = ffs.Instance(prob)
    pop = ffs.Population(ref, **GA, instance_id=0)
    d1 = pop.run(r1["generations"])
    assert r1["obj"] == d1["obj"] and np.array_equal(r1["S"], d1["S"].ravel())
    ref.reschedule(arr, 60)
    warm = ffs.Population(ref, **GA, instance_id=1, prev=pop)
    d3 = warm.run(150)
    assert r3["obj"] == d3["obj"] and np.array_equal(r3["S"], d3["S"].ravel())
