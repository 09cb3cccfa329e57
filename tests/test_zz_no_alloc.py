"""The allocation-free decode entry point, ffs_decode_noalloc.

It exists for callers that may not allocate device memory (a fixed device-memory budget
set at start-up, a framework allocator that owns the memory, loops that must not wait on
the allocator); it keeps all of its scratch in one fixed device array inside the library.
Its results must equal the oracle's and ffs_decode's exactly (integer arithmetic), call
after call, since every call reuses the same array; and after its first call on a device
it must not change the device's free memory.  This file is collected last so that a
failure here cannot stop the other GPU tests from running first.
"""
import numpy as np
import pytest

import oracle
from paper_1903_10741_gb300 import ffs
from paper_1903_10741_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def _same(a, b):
    for key in ("obj", "tard", "cmax"):
        assert np.array_equal(a[key].cpu().numpy(), b[key].cpu().numpy()), key


@pytest.mark.parametrize("mode", [(ffs.ORDER_STAGE, ffs.MACH_EARLIEST), (ffs.ORDER_TOPO, ffs.MACH_GENE)])
def test_noalloc_matches_decode_twice(mode):
    torch = _torch()
    dyn = wl.dynamic_medium(2)
    inst = ffs.Instance(dyn.problem)
    orc = oracle.Instance(dyn.problem)
    rng = np.random.default_rng(17)
    gj, gs = inst.genes()
    machines = dyn.problem.o[gs]
    # first call: all ops free; second call: after a rescheduling point with executing ops
    for call in range(2):
        Y, X = wl.random_chromosomes(rng, 257, inst.K, machines)
        y = torch.from_numpy(Y).cuda()
        x = torch.from_numpy(X).cuda() if mode[1] == ffs.MACH_GENE else None
        want = inst.decode(y, x, *mode)
        got = inst.decode_noalloc(y, x, *mode)
        _same(want, got)
        got_again = inst.decode_noalloc(y, x, *mode)  # the array keeps the last call's data
        _same(want, got_again)
        for i in range(0, 257, 16):  # a sample of rows against the oracle itself
            r = orc.decode(Y[i], X[i], *mode)
            assert (int(got["obj"][i]), int(got["tard"][i]), int(got["cmax"][i])) == (r["obj"], r["tard"], r["cmax"])
        if call == 0:
            out = inst.decode(y[:1], x[:1] if x is not None else None, *mode, schedule=True)
            S, M = out["S"][0].cpu().numpy(), out["M"][0].cpu().numpy()
            inst.commit(S, M)
            orc.commit(S, M)
            t_now, arr = dyn.events[0]
            inst.reschedule(arr, t_now)
            orc.reschedule(arr, t_now)
            gj, gs = inst.genes()
            machines = dyn.problem.o[gs]
    assert (inst.status() == ffs.ST_EXEC).any()


def test_noalloc_rejects_oversized_instance():
    torch = _torch()
    rng = np.random.default_rng(3)
    N, g = 1000, 10
    p = rng.integers(200, 260, size=(N, g))  # free work above the 16 MiB scratch's reach
    prob = wl.Problem(o=np.full(g, 3), p=p, q=np.full(3 * g, 2), R=np.zeros(N), D=np.zeros(N), Qmax=60)
    inst = ffs.Instance(prob)
    y = torch.arange(1, inst.K + 1, dtype=torch.int16, device="cuda")[None, :]
    with pytest.raises(ffs.FFSError) as e:
        inst.decode_noalloc(y)
    assert e.value.code == -1
    assert "limit" in ffs.lib().ffs_last_error().decode()


def test_noalloc_leaves_device_memory_unchanged():
    """After the first call on the device (which looks up the array's address), further
    calls into preallocated outputs leave the device's free memory exactly as it was."""
    torch = _torch()
    import ctypes as C
    dyn = wl.dynamic_medium(3)
    inst = ffs.Instance(dyn.problem)
    rng = np.random.default_rng(5)
    Y, _ = wl.random_chromosomes(rng, 300, inst.K, dyn.problem.o[inst.genes()[1]])
    y = torch.from_numpy(Y).cuda()
    want = inst.decode(y)
    obj = torch.empty(300, dtype=torch.int64, device="cuda")
    tard = torch.empty(300, dtype=torch.int64, device="cuda")
    cmax = torch.empty(300, dtype=torch.int32, device="cuda")
    L = ffs.lib()

    def call():
        rc = L.ffs_decode_noalloc(inst.handle, ffs.ORDER_STAGE, ffs.MACH_EARLIEST, C.c_void_p(y.data_ptr()), None,
                                  300, C.c_void_p(obj.data_ptr()), C.c_void_p(tard.data_ptr()),
                                  C.c_void_p(cmax.data_ptr()), None)
        assert rc == 0, rc

    call()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        call()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    _same(want, {"obj": obj, "tard": tard, "cmax": cmax})
