"""Work-group-scoped barriers on the GPU (RC_GROUP_BARRIERS): the per-group
barrier-release rule and the cross-group records of the whole run, against
the oracle's group-scope mode record for record (status, interval and
access counters, every record, final global memory), under both
classification strategies.
"""
import numpy as np
import pytest

from paper_1308_3203_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STRATEGIES = (1, 2)


@pytest.fixture(scope="module")
def rc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1308_3203_gb300 import build as gpu_build
    gpu_build.build()
    from paper_1308_3203_gb300 import racecheck
    racecheck.load()
    yield racecheck
    racecheck.set_strategy(0)


def same(got, want, what=""):
    for k in ("status", "n_intervals", "n_access", "n_global", "n_local"):
        assert got[k] == want[k], (what, k, got[k], want[k])
    np.testing.assert_array_equal(got["records"], want["records"], err_msg=what)
    np.testing.assert_array_equal(got["final"], want["final"], err_msg=what)


def run_both(rc, oracle, src, G, S, globals_, name=""):
    want = oracle.check(src, G, S, globals_, group_barriers=True)
    bc = rc.compile(src)
    for s in STRATEGIES:
        rc.set_strategy(s)
        got = rc.check(bc, G, S, globals_, group_barriers=True)
        same(got, want, f"{name} strategy {s}")
    rc.set_strategy(0)
    return want


HAND = [
    ("kernel t(global int A[]) { A[tid % 3] = wg + 7; }", 3, 8, 3),
    ("kernel t(global int A[]) { A[tid % 5] = 7; }", 4, 32, 5),
    ("kernel t(global int A[]) {\n A[gtid] = 1;\n barrier;\n x = A[(gtid + 5) % 12];\n}", 3, 4, 12),
    ("kernel t(global int A[]) {\n if (wg == 0) { A[0] = 5; }\n barrier;\n x = A[0];\n}", 2, 4, 1),
    ("kernel t(global int A[]) {\n A[0] = wg;\n barrier;\n if (wg == 0) { x = A[0]; }\n}", 2, 4, 1),
    ("kernel t(global int A[]) {\n if (wg == 0) { A[0] = 1; }\n barrier;\n if (wg == 1) { A[0] = 2; }\n}", 2, 4, 1),
    ("kernel t(global int A[]) { if (wg == 0) { barrier; A[0] = 3; } }", 2, 4, 1),
    ("kernel t(global int A[]) {\n if (wg == 0) { barrier; } else { barrier; }\n A[gtid] = 1;\n}", 2, 4, 8),
    ("kernel t(global int A[]) { if (tid == 0) { barrier; } }", 2, 4, 1),
    ("kernel t(global int A[]) { if (wg == 1) { if (tid < 2) { barrier; } } }", 2, 4, 1),
    ("kernel t(global int A[], local int L[1]) {\n L[0] = wg;\n barrier;\n A[gtid] = L[0];\n}", 3, 4, 12),
]


@pytest.mark.parametrize("case", range(len(HAND)))
def test_hand_cases(rc, oracle, case):
    src, G, S, n = HAND[case]
    for init in (0, 5):
        run_both(rc, oracle, src, G, S, [np.full(n, init, np.int32)], f"hand {case} init {init}")


def test_group_kernels(rc, oracle):
    for seed in range(40):
        inst = W.group_kernel(seed)
        run_both(rc, oracle, inst.src, inst.groups, inst.group_size, inst.globals, inst.name)


@pytest.mark.parametrize("shape", [(7, 33), (16, 64), (2, 1024), (64, 32)])
def test_group_kernels_shapes(rc, oracle, shape):
    """Ragged and full group sizes, many groups."""
    G, S = shape
    for seed in range(3):
        inst = W.group_kernel(100 + seed, groups=G, group_size=S)
        run_both(rc, oracle, inst.src, G, S, inst.globals, inst.name)


def test_other_generators_in_group_scope(rc, oracle):
    """The kernel-wide families checked with group-scoped barriers."""
    insts = [W.tiny_kernel(s) for s in range(60)]
    insts += [W.small_kernel(s, group_size=32, groups=4, n_stmts=24, n_barriers=2) for s in range(20)]
    insts += [W.large_kernel(s, groups=8, group_size=64, global_len=4096, local_len=64, n_stmts=60,
                             n_barriers=4) for s in range(4)]
    for inst in insts:
        run_both(rc, oracle, inst.src, inst.groups, inst.group_size, inst.globals, inst.name)


def test_large_instance_group_scope(rc, oracle):
    """A config-2 kernel at 64 x 256 (the oracle runs it in seconds)."""
    inst = W.large_kernel(1, groups=64, group_size=256)
    run_both(rc, oracle, inst.src, inst.groups, inst.group_size, inst.globals, inst.name)


def test_group_scope_is_rejected_where_unsupported(rc):
    bc = rc.compile("kernel t(global int A[]) { A[gtid] = 1; }")
    A = np.zeros(8, np.int32)
    inp, keep = rc._marshal([A], None, False)
    inp.flags |= rc.RC_GROUP_BARRIERS
    import ctypes
    out = (rc._ExploreInterval * 4)()
    n = ctypes.c_uint32()
    code = rc.load().rc_explore(bc.handle, 2, 4, ctypes.byref(inp), 0, out, 4, ctypes.byref(n))
    assert code == 2  # RC_E_INVALID
    del keep
