"""The bounds-checked build (FFS_CHECKED): decodes and GA generations run in a separate
process on the checked library, equal the oracle, and find no device index out of range."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import sys
sys.path.insert(0, ROOT)
import numpy as np, torch
import oracle
from paper_1903_10741_gb300 import ffs, workloads as wl
assert ffs.lib()._name.endswith("_build_checked/libffs.so"), ffs.lib()._name
torch.cuda.set_device(0)
rng = np.random.default_rng(5)
checked = 0
for N, g, P in ((12, 3, 64), (40, 5, 128), (90, 6, 64)):
    prob = wl.random_instance(rng, N, g, 1, 4, 60, 3, 25, 55)
    li, oi = ffs.Instance(prob), oracle.Instance(prob)
    Y, X = wl.random_chromosomes(rng, 33, oi.K, oi.gene_machines())
    for order, mach in ((ffs.ORDER_STAGE, ffs.MACH_EARLIEST), (ffs.ORDER_TOPO, ffs.MACH_GENE)):
        out = li.decode(torch.from_numpy(Y).cuda(), torch.from_numpy(X).cuda(), order_mode=order, mach_mode=mach)
        ref = [oi.decode(y, x, order_mode=order, mach_mode=mach)["obj"] for y, x in zip(Y, X)]
        assert np.array_equal(out["obj"].cpu().numpy(), np.array(ref)), (N, order, mach)
        checked += len(Y)
    pop = ffs.Population(li, P=P, island=32, seed=2, migrate_every=3)
    pop.run(7, want_schedule=False)
    ga = oracle.GA(oracle.Instance(prob), P=P, island=32, seed=2, migrate_every=3).init()
    ga.step(7)
    st = pop.read()
    assert np.array_equal(st["Y"], ga.Y[:, :ga.K]) and np.array_equal(st["obj"], ga.obj), N
# unrelated machines (earliest completion) and idle-gap insertion, the other grouped and
# one-step paths
up = wl.unrelated_instance(rng, 30, 4, 2, 4, 60, 5, 25, 55)
li, oi = ffs.Instance(up), oracle.Instance(up)
Y, X = wl.random_chromosomes(rng, 33, oi.K, oi.gene_machines())
out = li.decode(torch.from_numpy(Y).cuda(), torch.from_numpy(X).cuda(), order_mode=ffs.ORDER_STAGE,
                mach_mode=ffs.MACH_EARLIEST)
ref = [oi.decode(y, x, order_mode=oracle.ORDER_STAGE, mach_mode=oracle.MACH_EARLIEST)["obj"] for y, x in zip(Y, X)]
assert np.array_equal(out["obj"].cpu().numpy(), np.array(ref)), "unrelated"
prob = wl.random_instance(rng, 40, 4, 2, 4, 60, 3, 25, 50)
li, oi = ffs.Instance(prob), oracle.Instance(prob)
Y, X = wl.random_chromosomes(rng, 33, oi.K, oi.gene_machines())
out = li.decode(torch.from_numpy(Y).cuda(), torch.from_numpy(X).cuda(), order_mode=ffs.ORDER_STAGE,
                mach_mode=ffs.MACH_EARLIEST | ffs.PLACE_INSERT)
ref = [oi.decode(y, x, order_mode=oracle.ORDER_STAGE, mach_mode=oracle.MACH_EARLIEST | oracle.PLACE_INSERT)["obj"]
       for y, x in zip(Y, X)]
assert np.array_equal(out["obj"].cpu().numpy(), np.array(ref)), "insertion"
checked += 66
faults = ffs.bounds_faults()
assert faults == 0, faults
print("checked build ok:", checked, "decodes and 3 GA runs, no index out of range")
"""


def test_checked_build_finds_no_index_out_of_range():
    env = dict(os.environ, FFS_CHECKED="1")
    code = "ROOT = " + repr(ROOT) + "\n" + _CHILD
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked build ok" in r.stdout
