"""Bounded device waits that run out come back as FFS_E_TIMEOUT, and the context stays
usable.  The failure is injected without any copy in flight (ffs_debug_inject): the table
copy of the decode kernel, or the operand loads of the tensor-core GEMM, are not issued,
so the kernel's own bounded wait expires, the CTA records the timeout and returns (the
GEMM CTA first frees its tensor memory).  Nothing faults, traps or hangs."""
import numpy as np
import pytest

import oracle
from paper_1903_10741_gb300 import ffs
from paper_1903_10741_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture
def injected():
    yield ffs.debug_inject
    ffs.debug_inject(ffs.INJECT_NONE)


def test_decode_table_wait_times_out(injected):
    prob = wl.static_small(3)
    inst, orc = ffs.Instance(prob), oracle.Instance(prob)
    Y, _ = wl.random_chromosomes(np.random.default_rng(1), 40, orc.K, orc.gene_machines())
    y = torch.from_numpy(Y).cuda()
    injected(ffs.INJECT_TABLE_COPY)
    with pytest.raises(ffs.FFSError) as e:
        inst.decode(y)
    assert e.value.code == ffs.E_TIMEOUT
    injected(ffs.INJECT_NONE)
    got = inst.decode(y)["obj"].cpu().numpy()  # the same instance and context work again
    assert np.array_equal(got, [orc.decode(r)["obj"] for r in Y])


def test_gemm_operand_wait_times_out(injected):
    a = np.random.default_rng(2).integers(-3, 4, size=(256, 128)).astype(np.float32)
    b = np.random.default_rng(3).integers(-3, 4, size=(256, 128)).astype(np.float32)
    A = torch.from_numpy(a).to(torch.bfloat16).cuda()
    B = torch.from_numpy(b).to(torch.bfloat16).cuda()
    injected(ffs.INJECT_GEMM_LOADS)
    with pytest.raises(ffs.FFSError) as e:
        ffs.tensor_gemm(A, B)
    assert e.value.code == ffs.E_TIMEOUT
    injected(ffs.INJECT_NONE)
    C = ffs.tensor_gemm(A, B).cpu().numpy()  # tensor memory was freed: the next GEMM runs
    assert np.array_equal(C, a @ b.T)


def test_inject_rejects_unknown_modes():
    with pytest.raises(ffs.FFSError):
        ffs.debug_inject(8)
