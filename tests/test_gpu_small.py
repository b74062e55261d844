"""The one-CTA check of small instances (strategy 4, and strategy 0 when an
instance fits): every interval, its classification and barrier agreement in
one launch.  Its reports are compared with the oracle across the parity
suite (tests/test_gpu_parity.py runs strategy 4 on every case); here: that a
small check is one kernel launch, that instances it cannot take fall back
with the same report, and its per-check time."""
import time

import numpy as np
import pytest

from paper_1308_3203_gb300 import workloads as W
from tests.test_gpu_parity import same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1308_3203_gb300 import build as gpu_build
    gpu_build.build()
    from paper_1308_3203_gb300 import racecheck
    racecheck.load()
    racecheck.set_engine("auto")
    yield racecheck
    racecheck.set_strategy(0)


def test_one_launch_per_small_check(rc, oracle):
    rc.set_strategy(4)
    for seed in range(20):
        inst = W.small_kernel(seed)
        bc = rc.compile(inst.src)
        n0 = rc.kernel_launches()
        got = rc.check(bc, inst.groups, inst.group_size, inst.globals)
        assert rc.kernel_launches() - n0 == 1, inst.name
        same(got, oracle.check(inst.src, inst.groups, inst.group_size, inst.globals), inst.name)
    rc.set_strategy(0)


def test_instances_it_cannot_take_fall_back(rc, oracle):
    """More work-items than one CTA holds, and more logged accesses per
    interval than it sorts: the same report through the other paths."""
    rc.set_strategy(4)
    cases = [W.small_kernel(3, group_size=256, groups=5),                   # 1280 work-items
             W.large_kernel(1, groups=4, group_size=256, global_len=8192, local_len=512),
             W.Instance("loop", "kernel e(global int A[]) { for i in 0 .. 80 { A[(gtid + i) % size(A)] = i; } }",
                        1, 64, [np.zeros(128, np.int32)])]                  # 80 x 64 > 4096 records
    for inst in cases:
        same(rc.check(rc.compile(inst.src), inst.groups, inst.group_size, inst.globals),
             oracle.check(inst.src, inst.groups, inst.group_size, inst.globals), inst.name)
    rc.set_strategy(0)


def test_small_check_latency(rc):
    """Per-check time of 1 x 64 work-item kernels (32 statements, one
    barrier) from host inputs, printed; the automatic strategy takes the
    one-CTA path."""
    rc.set_strategy(0)
    insts = [W.small_kernel(s) for s in range(100)]
    bcs = [rc.compile(i.src) for i in insts]
    for b, i in zip(bcs[:5], insts[:5]):
        rc.check(b, i.groups, i.group_size, i.globals, want_final=False)
    t0 = time.perf_counter()
    for b, i in zip(bcs, insts):
        rc.check(b, i.groups, i.group_size, i.globals, want_final=False)
    dt = (time.perf_counter() - t0) / len(insts)
    rc.profile_reset()
    rc.profile_enable(True)
    for b, i in zip(bcs, insts):
        rc.check(b, i.groups, i.group_size, i.globals, want_final=False)
    rc.profile_enable(False)
    p = rc.profile_get(0)
    print(f"small check: {dt * 1e6:.1f} us per check, kernel {1e3 * p['ms'] / max(p['launches'], 1):.1f} us")
    assert dt < 1e-3
