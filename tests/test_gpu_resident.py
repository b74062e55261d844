"""Resident runs (strategy 3, and the automatic choice when every work-group
fits on the GPU at once): one cooperative launch runs all barrier intervals
with in-kernel commits, grid barriers and compaction, the exact sort after
the run.  Reports must equal the oracle's record for record; runs that fill
the record buffer or the interval table fall back to the interval-by-
interval path with the same result.
"""
import numpy as np
import pytest

from paper_1308_3203_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


def check(rc, oracle, src, G, S, globals_, name="", launches=None):
    want = oracle.check(src, G, S, globals_)
    bc = rc.compile(src)
    for strategy in (3, 0):
        rc.set_strategy(strategy)
        before = rc.kernel_launches()
        got = rc.check(bc, G, S, globals_)
        n = rc.kernel_launches() - before
        same(got, want, f"{name} strategy {strategy}")
        if launches is not None:
            assert n == launches, (name, strategy, n)
    rc.set_strategy(0)
    return want


def test_race_free_run_is_one_launch(rc, oracle):
    """Eight barriers, private cells: the whole check is one kernel launch."""
    body = "\n".join(f"A[gtid] = A[gtid] + {k};\nbarrier;" for k in range(8))
    src = f"kernel t(global int A[]) {{\n{body}\n}}\n"
    want = check(rc, oracle, src, 16, 128, [np.arange(2048, dtype=np.int32)], "private", launches=1)
    assert want["status"] == 0 and want["n_intervals"] == 9


def test_small_kernels(rc, oracle):
    for seed in range(60):
        inst = W.small_kernel(seed)
        check(rc, oracle, inst.src, inst.groups, inst.group_size, inst.globals, inst.name)


@pytest.mark.parametrize("shape", [(8, 256), (1, 1024), (33, 32), (64, 64)])
def test_large_kernels_reduced(rc, oracle, shape):
    G, S = shape
    for seed in range(3):
        inst = W.large_kernel(seed, groups=G, group_size=S, global_len=1 << 16, local_len=256, n_stmts=80,
                              n_barriers=6)
        check(rc, oracle, inst.src, G, S, inst.globals, inst.name)


def test_large_instance_full_size(rc, oracle):
    """The bench workload (1024 x 256): the resident report equals the
    interval-by-interval shadow path's, which test_gpu_parity compares with
    the oracle at this size."""
    inst = W.large_kernel(0)
    bc = rc.compile(inst.src)
    rc.set_strategy(2)
    want = rc.check(bc, inst.groups, inst.group_size, inst.globals)
    rc.set_strategy(3)
    before = rc.kernel_launches()
    got = rc.check(bc, inst.groups, inst.group_size, inst.globals)
    assert rc.kernel_launches() - before < 60  # resident: one launch plus the exact sort of shared cells
    rc.set_strategy(0)
    same(got, want, inst.name)


def test_owner_tag_wraps(rc, oracle):
    """70 intervals: the 6-bit owner-table tag wraps and the table is cleared in-kernel."""
    src = ("kernel t(global int A[]) {\n for i in 0 .. 70 {\n  A[(gtid + i) % 64] = i;\n"
           "  x = A[(gtid + i + 1) % 64];\n  barrier;\n }\n}\n")
    want = check(rc, oracle, src, 2, 32, [np.zeros(64, np.int32)], "wrap")
    assert want["n_intervals"] == 71


def test_races_errors_and_divergence_across_intervals(rc, oracle):
    src = ("kernel t(global int A[], local int L[64]) {\n"
           " A[gtid % 7] = tid;\n barrier;\n L[tid % 3] = wg;\n x = L[(tid + 1) % 3];\n barrier;\n"
           " if (gtid == 37) { x = A[1000]; }\n assert(gtid != 90);\n barrier;\n"
           " A[gtid] = x;\n if (wg == 1) { barrier; }\n}\n")
    for G, S in [(4, 32), (2, 64)]:
        want = check(rc, oracle, src, G, S, [np.zeros(G * S, np.int32)], f"mixed {G}x{S}")
        assert want["status"] == 1


def test_record_buffer_overflow_falls_back(rc, oracle):
    """Every interval's accesses need the exact sort and together they exceed
    the resident run's record buffer: the check restarts interval by interval."""
    src = ("kernel t(global int A[]) {\n for i in 0 .. 12 {\n"
           + "".join(f"  A[{k}] = tid + i;\n" for k in range(8)) + "  barrier;\n }\n}\n")
    check(rc, oracle, src, 4, 256, [np.zeros(8, np.int32)], "overflow")


def test_interval_cap_falls_back(rc, oracle):
    src = "kernel t(global int A[]) {\n for i in 0 .. 4100 {\n  A[gtid] = i;\n  barrier;\n }\n}\n"
    want = check(rc, oracle, src, 1, 32, [np.zeros(32, np.int32)], "cap")
    assert want["n_intervals"] == 4101


def test_owner_table_reuse_across_instances(rc, oracle):
    """A small instance whose in-kernel tag wrap must also clear the owner-table
    words of a larger instance checked before and after it."""
    big = W.large_kernel(2, groups=8, group_size=64, global_len=8192, local_len=256)
    wrap = ("kernel t(global int A[]) {\n for i in 0 .. 70 {\n  A[(gtid + i) % 64] = i;\n"
            "  x = A[(gtid + i + 1) % 64];\n  barrier;\n }\n}\n")
    wb = oracle.check(big.src, big.groups, big.group_size, big.globals)
    ww = oracle.check(wrap, 2, 32, [np.zeros(64, np.int32)])
    bb, bw = rc.compile(big.src), rc.compile(wrap)
    rc.set_strategy(3)
    for _ in range(4):
        same(rc.check(bb, big.groups, big.group_size, big.globals), wb, "big")
        same(rc.check(bw, 2, 32, [np.zeros(64, np.int32)]), ww, "wrap")
    rc.set_strategy(0)


def test_grid_barrier_gives_up_and_reports(rc, oracle):
    """A grid barrier that cannot complete (one arrival more than the launch
    has) gives up after its limit and reports it; the device stays usable."""
    timed_out, seconds = rc.diag_grid_barrier(2000)
    assert timed_out and seconds < 5.0
    inst = W.small_kernel(7)
    check(rc, oracle, inst.src, inst.groups, inst.group_size, inst.globals, "after the probe")
