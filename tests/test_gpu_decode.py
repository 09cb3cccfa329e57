"""CUDA decoder vs the CPU oracle, element by element (all integer: bit-exact)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1903_10741_gb300 import ffs
from paper_1903_10741_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

MODES = [(ffs.ORDER_STAGE, ffs.MACH_EARLIEST), (ffs.ORDER_TOPO, ffs.MACH_GENE),
         (ffs.ORDER_STAGE, ffs.MACH_GENE), (ffs.ORDER_TOPO, ffs.MACH_EARLIEST)]


def _torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def compare(lib_i, orc_i, Y, X, order, mach, schedule=True, sample=None):
    """Decode Y/X on the GPU and in the oracle; assert equal objectives and schedules."""
    torch = _torch()
    yd = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
    xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    out = lib_i.decode(yd, xd if (mach & 1) == ffs.MACH_GENE else None, order, mach, schedule=schedule)
    obj = out["obj"].cpu().numpy()
    idx = range(len(Y)) if sample is None else sample
    S = out["S"].cpu().numpy() if schedule else None
    M = out["M"].cpu().numpy() if schedule else None
    if not schedule:
        tard = out["tard"].cpu().numpy()
        cmax = out["cmax"].cpu().numpy()
    for i in idx:
        r = orc_i.decode(Y[i], X[i], order, mach)
        assert obj[i] == r["obj"], (i, obj[i], r["obj"])
        if schedule:
            assert np.array_equal(S[i], r["S"]), i
            assert np.array_equal(M[i], r["M"]), i
        else:
            assert tard[i] == r["tard"] and cmax[i] == r["cmax"], i
    return obj


@pytest.mark.parametrize("mode", MODES)
def test_static_small_random(mode):
    prob = wl.static_small(1)
    lib_i, orc_i = ffs.Instance(prob), oracle.Instance(prob)
    rng = np.random.default_rng(7)
    Y, X = wl.random_chromosomes(rng, 333, orc_i.K, orc_i.gene_machines())  # ragged tail of warps
    compare(lib_i, orc_i, Y, X, *mode, schedule=True)
    compare(lib_i, orc_i, Y[:70], X[:70], *mode, schedule=False)


@pytest.mark.parametrize("mode", MODES[:2])
def test_dynamic_chain(mode):
    """Initial solve plus three rescheduling events (executing ops, frozen prefixes,
    released new jobs), K not a multiple of 32."""
    dyn = wl.dynamic_medium(1)
    lib_i, orc_i = ffs.Instance(dyn.problem), oracle.Instance(dyn.problem)
    rng = np.random.default_rng(3)
    for ev in range(len(dyn.events) + 1):
        Y, X = wl.random_chromosomes(rng, 300, orc_i.K, orc_i.gene_machines())
        compare(lib_i, orc_i, Y, X, *mode, schedule=True, sample=range(0, 300, 7))
        compare(lib_i, orc_i, Y, X, *mode, schedule=False, sample=range(3, 300, 11))
        if ev == len(dyn.events):
            break
        r = orc_i.decode(Y[0], X[0], *mode)
        orc_i.commit(r["S"], r["M"])
        lib_i.commit(r["S"], r["M"])
        t_now, arr = dyn.events[ev]
        orc_i.reschedule(arr, t_now)
        lib_i.reschedule(arr, t_now)
        assert np.array_equal(lib_i.status(), orc_i.status)


def test_worked_example_on_gpu():
    """Sec. 4.3 worked example, Alg. 1 read as a topological order, machine genes."""
    ex = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")))
    n0 = ex["n_original"]
    pst = np.array(ex["p_per_stage"])
    prob = wl.Problem(o=ex["o"], p=np.tile(pst, (n0, 1)), q=np.ones(6), R=ex["R"][:n0],
                      D=np.full(n0, 10**6), Qmax=ex["Qmax"], WT=ex["WT"])
    arr = wl.Arrivals(p=np.tile(pst, (2, 1)), R=ex["R"][n0:], D=[10**6] * 2)
    lib_i, orc_i = ffs.Instance(prob), oracle.Instance(prob)
    for inst in (lib_i, orc_i):
        inst.commit(np.array(ex["S_original"]), np.array(ex["M_original"]))
        inst.reschedule(arr, ex["RS"])
    gj, gs = orc_i.gene_map()
    Y = np.array(ex["Y"])[gj, gs][None, :].astype(np.int16)
    X = np.array(ex["X"])[gj, gs][None, :].astype(np.int8)
    compare(lib_i, orc_i, Y, X, ffs.ORDER_TOPO, ffs.MACH_GENE)
    torch = _torch()
    out = lib_i.decode(torch.from_numpy(Y).cuda(), torch.from_numpy(X).cuda(), ffs.ORDER_TOPO,
                       ffs.MACH_GENE)
    # Fig. 8: C_max = 20.42 (the topological reading reaches the printed Z's makespan)
    assert int(out["cmax"][0]) == ex["expect_cmax"]


@pytest.mark.parametrize("case", ["one_gene", "single_machine", "serialised", "tiny_peak_tall_p"])
def test_edge_cases(case):
    rng = np.random.default_rng(5)
    if case == "one_gene":
        prob = wl.Problem(o=[1], p=[[7]], q=[3], R=[4], D=[2], Qmax=3)
    elif case == "single_machine":
        prob = wl.Problem(o=[1], p=rng.integers(1, 50, (40, 1)), q=[2], R=np.zeros(40),
                          D=rng.integers(0, 500, 40), Qmax=2)
    elif case == "serialised":
        prob = wl.Problem(o=[3, 2, 3], p=rng.integers(1, 30, (37, 3)), q=np.full(8, 5), R=np.zeros(37),
                          D=rng.integers(0, 900, 37), Qmax=5)
    else:
        prob = wl.Problem(o=[4, 4], p=rng.integers(200, 900, (9, 2)), q=[3, 4, 5, 6, 1, 2, 3, 4],
                          R=rng.integers(0, 100, 9), D=rng.integers(0, 3000, 9), Qmax=7)
    lib_i, orc_i = ffs.Instance(prob), oracle.Instance(prob)
    Y, X = wl.random_chromosomes(rng, 65, orc_i.K, orc_i.gene_machines())
    for mode in MODES:
        compare(lib_i, orc_i, Y, X, *mode)


def test_all_frozen_but_one():
    """Only one free op remains after the freeze: K = 1."""
    prob = wl.Problem(o=[1, 1], p=[[5, 5], [5, 5]], q=[1, 1], R=[0, 0], D=[0, 0], Qmax=2)
    lib_i, orc_i = ffs.Instance(prob), oracle.Instance(prob)
    S = np.array([[0, 5], [5, 12]])  # job 1 stage 1 starts after RS = 11: the only free op
    M = np.zeros((2, 2), int)
    for inst in (lib_i, orc_i):
        inst.commit(S, M)
        inst.reschedule(wl.Arrivals(p=np.zeros((0, 2)), R=[], D=[]), 11)
    assert orc_i.K == 1 and lib_i.K == 1
    Y = np.ones((3, 1), np.int16)
    X = np.zeros((3, 1), np.int8)
    for mode in MODES:
        compare(lib_i, orc_i, Y, X, *mode)


def test_profile_overflow_fallback():
    """An instance whose profile bound exceeds the shared-memory slice: schedules that
    outgrow it are redone with a global-memory profile, with identical results."""
    rng = np.random.default_rng(11)
    prob = wl.random_instance(rng, 260, 10, 2, 5, 99, 5, 40, 50)
    lib_i, orc_i = ffs.Instance(prob), oracle.Instance(prob)
    Y, X = wl.random_chromosomes(rng, 24, orc_i.K, orc_i.gene_machines())
    compare(lib_i, orc_i, Y, X, ffs.ORDER_STAGE, ffs.MACH_EARLIEST, schedule=False)
    compare(lib_i, orc_i, Y[:6], X[:6], ffs.ORDER_TOPO, ffs.MACH_GENE, schedule=True)


def test_surrogate_size_instance_sampled():
    """The 200-job, 8-stage instance: 600 chromosomes decoded, a sample checked."""
    prob = wl.surrogate_large(1)
    lib_i, orc_i = ffs.Instance(prob), oracle.Instance(prob)
    rng = np.random.default_rng(2)
    Y, X = wl.random_chromosomes(rng, 600, orc_i.K, orc_i.gene_machines())
    compare(lib_i, orc_i, Y, X, ffs.ORDER_STAGE, ffs.MACH_EARLIEST, schedule=False,
            sample=range(0, 600, 37))


def test_malformed_chromosome_reported():
    """A row that is not a permutation is reported as FFS_E_DEVICE, the others decode."""
    prob = wl.static_small(1)
    lib_i, orc_i = ffs.Instance(prob), oracle.Instance(prob)
    rng = np.random.default_rng(1)
    Y, X = wl.random_chromosomes(rng, 8, orc_i.K, orc_i.gene_machines())
    Y[3, 5] = Y[3, 6]
    torch = _torch()
    with pytest.raises(ffs.FFSError) as e:
        lib_i.decode(torch.from_numpy(Y).cuda())
    assert e.value.code == -8
    out = lib_i.decode(torch.from_numpy(Y[:3]).cuda())  # the flag was cleared
    assert out["obj"].shape[0] == 3
