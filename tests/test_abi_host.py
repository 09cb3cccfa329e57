"""The C ABI on the host (no GPU): the library loads, exports what include/ffs.h
declares, validates its inputs, and its rescheduling freeze and gene numbering agree with
the oracle's."""
import numpy as np
import pytest

import oracle
from paper_1903_10741_gb300 import ffs
from paper_1903_10741_gb300 import workloads as wl


def test_library_exports_every_declared_function():
    L = ffs.lib()
    names = ffs.header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_strerror_names_every_code():
    for code in range(0, -10, -1):
        assert ffs.lib().ffs_strerror(code).decode() != "unknown status"


def test_stop_requests_and_bounds_reader_validate_arguments():
    """The early-stop calls reject a missing handle without touching a device, and an
    ordinary build says that it does not check device indices."""
    import ctypes as C
    L = ffs.lib()
    assert L.ga_batch_stop(None) == -1
    assert L.ffs_service_stop_request(None, 1) == -1
    assert L.ffs_debug_bounds_faults(None) == -1
    n = C.c_uint32(7)
    assert L.ffs_debug_bounds_faults(C.byref(n)) == -7 and n.value == 0


def test_create_rejects_infeasible_and_bad_input():
    prob = wl.static_small(1)
    bad = wl.Problem(o=prob.o, p=prob.p, q=prob.q, R=prob.R, D=prob.D, Qmax=int(prob.q.max()) - 1)
    with pytest.raises(ffs.FFSError) as e:
        ffs.Instance(bad)
    assert e.value.code == -2
    empty_stage = wl.Problem(o=[2, 0, 2], p=prob.p, q=prob.q[:4], R=prob.R, D=prob.D, Qmax=prob.Qmax)
    with pytest.raises(ffs.FFSError) as e:
        ffs.Instance(empty_stage)
    assert e.value.code == -2
    neg = wl.Problem(o=prob.o, p=-prob.p, q=prob.q, R=prob.R, D=prob.D, Qmax=prob.Qmax)
    with pytest.raises(ffs.FFSError) as e:
        ffs.Instance(neg)
    assert e.value.code == -1


def _pair(problem):
    return ffs.Instance(problem), oracle.Instance(problem)


def test_fresh_instance_all_free():
    lib_i, orc_i = _pair(wl.static_small(1))
    inf = lib_i.info()
    assert inf["n_genes"] == orc_i.K == 30 and inf["rs"] == 0
    gj, gs = lib_i.genes()
    ogj, ogs = orc_i.gene_map()
    assert np.array_equal(gj, ogj) and np.array_equal(gs, ogs)
    assert (lib_i.status() == 0).all()
    # the profile bound covers running every op back to back
    assert inf["horizon"] >= int(orc_i.p.sum()) + 1


@pytest.mark.parametrize("seed", range(4))
def test_reschedule_chain_matches_oracle(seed):
    """Alg. 1 freeze + arrival append on the library's host side equals the oracle's."""
    dyn = wl.dynamic_medium(seed + 1)
    lib_i, orc_i = _pair(dyn.problem)
    rng = np.random.default_rng(seed)
    for t_now, arr in dyn.events:
        y = rng.permutation(orc_i.K) + 1
        r = orc_i.decode(y, None, oracle.ORDER_STAGE, oracle.MACH_EARLIEST)
        orc_i.commit(r["S"], r["M"])
        lib_i.commit(r["S"], r["M"])
        orc_i.reschedule(arr, t_now)
        lib_i.reschedule(arr, t_now)
        assert np.array_equal(lib_i.status(), orc_i.status)
        gj, gs = lib_i.genes()
        ogj, ogs = orc_i.gene_map()
        assert np.array_equal(gj, ogj) and np.array_equal(gs, ogs)
        inf = lib_i.info()
        assert inf["rs"] == t_now and inf["n_jobs"] == orc_i.N and inf["n_genes"] == orc_i.K


@pytest.mark.parametrize("seed", range(3))
def test_static_reschedule_chain_matches_oracle(seed):
    """The static approach's classification (completed / executing / fixed) and gene
    numbering (new jobs only) on the library's host side equal the oracle's."""
    dyn = wl.dynamic_medium(seed + 1)
    lib_i, orc_i = _pair(dyn.problem)
    rng = np.random.default_rng(seed)
    for t_now, arr in dyn.events:
        y = rng.permutation(orc_i.K) + 1
        r = orc_i.decode(y, None, oracle.ORDER_STAGE, oracle.MACH_EARLIEST)
        orc_i.commit(r["S"], r["M"])
        lib_i.commit(r["S"], r["M"])
        orc_i.reschedule(arr, t_now, static=True)
        lib_i.reschedule(arr, t_now, static=True)
        assert np.array_equal(lib_i.status(), orc_i.status)
        assert (orc_i.status == oracle.ST_FIXED).any()
        gj, gs = lib_i.genes()
        ogj, ogs = orc_i.gene_map()
        assert np.array_equal(gj, ogj) and np.array_equal(gs, ogs) and orc_i.K == arr.n * dyn.problem.g
        inf = lib_i.info()
        # the bound covers the kept plan's end plus every new op back to back
        assert inf["horizon"] >= int((orc_i.S0 + orc_i.p)[orc_i.status == oracle.ST_FIXED].max()) - t_now


def test_unrelated_instance_validation():
    """Per-machine tables: both or neither; a job's power on a machine above the peak is
    infeasible; arrivals of such an instance need their own tables."""
    rng = np.random.default_rng(1)
    pr = wl.unrelated_instance(rng, 6, 2, 1, 3, 20, 2, 10, 60)
    inst = ffs.Instance(pr)
    assert inst.info()["n_genes"] == 12
    bad = wl.Problem(o=pr.o, p=pr.p, q=pr.q, R=pr.R, D=pr.D, Qmax=pr.Qmax, pm=pr.pm, qm=pr.qm.copy())
    bad.qm[0, 0] = pr.Qmax + 1
    with pytest.raises(ffs.FFSError) as e:
        ffs.Instance(bad)
    assert e.value.code == -2
    # arrivals without per-machine tables are refused by an unrelated instance
    with pytest.raises(ffs.FFSError):
        inst.reschedule(wl.Arrivals(p=np.ones((1, 2)), R=[0], D=[9]), 0)
    inst.reschedule(wl.unrelated_arrivals(rng, 2, pr.o, 0, 20, 2, 10, pr.Qmax), 0)
    assert inst.info()["n_genes"] == 16


def test_reschedule_rules():
    lib_i = ffs.Instance(wl.static_small(1))
    arr = wl.Arrivals(p=np.ones((1, 3)), R=[5], D=[50])
    with pytest.raises(ffs.FFSError) as e:  # no plan committed and time moved on
        lib_i.reschedule(arr, 5)
    assert e.value.code == -7
    lib_i.reschedule(arr, 0)                # nothing has run yet: append only
    assert lib_i.info()["n_jobs"] == 11
    orc_i = oracle.Instance(wl.static_small(1))
    orc_i.reschedule(arr, 0)
    r = orc_i.decode(np.arange(orc_i.K, 0, -1), None, oracle.ORDER_STAGE, oracle.MACH_EARLIEST)
    lib_i.commit(r["S"], r["M"])
    lib_i.reschedule(wl.Arrivals(p=np.ones((0, 3)), R=[], D=[]), 10)
    with pytest.raises(ffs.FFSError) as e:  # time cannot go backwards
        lib_i.reschedule(arr, 9)
    assert e.value.code in (-1, -7)


def test_commit_validation():
    lib_i = ffs.Instance(wl.static_small(1))
    S = np.zeros((10, 3), np.int32)
    M = np.zeros((10, 3), np.int32)
    M[0, 1] = 3  # stage 1 has 3 machines: 0..2
    with pytest.raises(ffs.FFSError):
        lib_i.commit(S, M)
    M[0, 1] = 2
    lib_i.commit(S, M)
