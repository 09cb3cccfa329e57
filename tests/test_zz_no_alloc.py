"""The allocation-free decode entry point, ffs_decode_noalloc.

It exists for callers that may not allocate device memory (inside a CUDA graph capture,
under a fixed up-front memory budget, in loops that must not wait on the allocator); it
keeps all of its scratch in one fixed device array inside the library.  Its results must
equal ffs_decode's exactly (integer arithmetic), call after call, since every call reuses
the same array.  This file is collected last so that a failure here cannot stop the other
GPU tests from running first.
"""
import numpy as np
import pytest

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
        if call == 0:
            out = inst.decode(y[:1], x[:1] if x is not None else None, *mode, schedule=True)
            inst.commit(out["S"][0].cpu().numpy(), out["M"][0].cpu().numpy())
            t_now, arr = dyn.events[0]
            inst.reschedule(arr, t_now)
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
