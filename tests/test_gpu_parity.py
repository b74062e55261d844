"""GPU parity: reports of the CUDA path through the C ABI against the oracle.

Race reports are integer results, so the bar is bit-exact equality of every
record (interval, cell, class, witness pair, counts), the status, the access
counters and the final global memory.  Each case runs under both
classification strategies (full sort, shadow owner table), the resident
run (one cooperative launch for every interval) and the one-CTA check of
small instances, each where the shape allows it.
"""
import numpy as np
import pytest

from paper_1308_3203_gb300 import workloads as W
from tests.golden import golden

pytestmark = pytest.mark.gpu

STRATEGIES = (1, 2, 3, 4)


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
    if got["final"] is not None:
        np.testing.assert_array_equal(got["final"], want["final"], err_msg=what)


def run_both(rc, oracle, inst, strategies=STRATEGIES):
    want = oracle.check(inst.src, inst.groups, inst.group_size, inst.globals)
    bc = rc.compile(inst.src)
    for s in strategies:
        rc.set_strategy(s)
        got = rc.check(bc, inst.groups, inst.group_size, inst.globals)
        same(got, want, f"{inst.name} strategy {s}")
    rc.set_strategy(0)
    return want


@pytest.mark.parametrize("name", golden.names())
def test_golden(rc, name):
    g = golden.load(name)
    bc = rc.compile(g["src"])
    for s in STRATEGIES:
        rc.set_strategy(s)
        r = rc.check(bc, g["groups"], g["group_size"], g["globals"])
        for k, v in g["expect"].items():
            assert r[k] == v, (name, s, k)
        np.testing.assert_array_equal(r["records"], g["records"])
        np.testing.assert_array_equal(r["final"], g["final"])
    rc.set_strategy(0)


@pytest.mark.parametrize("chunk", range(5))
def test_small_kernels(rc, oracle, chunk):
    """1 group x 64, 1 barrier, 32 statements over A[256] (seeds 0..199)."""
    for seed in range(chunk * 40, chunk * 40 + 40):
        run_both(rc, oracle, W.small_kernel(seed))


def test_tiny_kernels(rc, oracle):
    for seed in range(150):
        run_both(rc, oracle, W.tiny_kernel(seed))


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("shape", [(8, 256), (3, 100), (5, 1), (1, 1024), (33, 32)])
def test_large_kernels_reduced(rc, oracle, seed, shape):
    """Config-2 statement mix (loops, local memory, planted collisions) at
    shapes the oracle finishes quickly, incl. ragged group sizes."""
    G, S = shape
    inst = W.large_kernel(seed, groups=G, group_size=S, global_len=max(16 * G * S, 4096),
                          local_len=16 * S)
    run_both(rc, oracle, inst)


@pytest.mark.parametrize("seed", range(3))
def test_stress_kernels_reduced(rc, oracle, seed):
    """Config-5 statement mix (nested loops, branches on loaded values)."""
    run_both(rc, oracle, W.stress_kernel(seed, groups=16, group_size=1024))


@pytest.mark.parametrize("seed", range(3))
def test_batch_shapes(rc, oracle, seed):
    """Config-3 kernels (uneven shapes) through rc_check_batch."""
    insts = W.batch_kernels(seed, 12)
    insts = [i for i in insts if i.n_threads * 300 < 2_000_000][:6]
    want = [oracle.check(i.src, i.groups, i.group_size, i.globals) for i in insts]
    bcs = [rc.compile(i.src) for i in insts]
    for s in STRATEGIES:
        rc.set_strategy(s)
        got = rc.check_batch([(b, i.groups, i.group_size, i.globals) for b, i in zip(bcs, insts)])
        for g, w, i in zip(got, want, insts):
            same(g, w, i.name)
    rc.set_strategy(0)


def test_batch_pinned_inputs(rc, oracle):
    """Inputs in page-locked host memory reach a batch through the copy kernel
    (the SMs read them over the CPU-GPU link), pageable ones through
    cudaMemcpyAsync: the same reports and final memories under each
    strategy, in lock-step rounds (shadow rounds classify beside the next
    round) and resident."""
    import torch
    insts = W.batch_kernels(7, 12)
    insts = [i for i in insts if i.n_threads * 300 < 2_000_000][:6]
    want = [oracle.check(i.src, i.groups, i.group_size, i.globals) for i in insts]
    bcs = [rc.compile(i.src) for i in insts]
    pinned = [[torch.from_numpy(g).pin_memory().numpy() for g in i.globals] for i in insts]
    for s in (0, 1, 2, 3):
        rc.set_strategy(s)
        got = rc.check_batch([(b, i.groups, i.group_size, p) for b, i, p in zip(bcs, insts, pinned)])
        for g, w, i in zip(got, want, insts):
            same(g, w, f"{i.name} strategy {s}")
    rc.set_strategy(0)


@pytest.mark.parametrize("shape", [(1, 65, 8), (1, 66, 32), (3, 97, 16), (2, 200, 8), (1, 300, 64), (5, 129, 4)])
def test_large_cells(rc, oracle, shape):
    """Cells touched by more than 64 work-items are classified by a whole
    CTA (three sweeps with block reductions); small arrays make every cell
    crowded, with affine and constant values, so witnesses of every kind
    come from those sweeps."""
    G, S, L = shape
    for seed in range(8):
        run_both(rc, oracle, W.small_kernel(1000 + seed, group_size=S, groups=G, n_stmts=24, n_barriers=2, L=L))


EDGE = [
    ("kernel e() { }", 2, 3, []),
    ("kernel e(global int A[]) { A[tid] = tid; }", 1, 1, [np.zeros(1, np.int32)]),
    ("kernel e(global int A[]) { A[tid] = 1; }", 2, 3, [np.zeros(0, np.int32)]),
    ("kernel e(global int A[]) { A[0] = tid; }", 4, 1024, [np.zeros(1, np.int32)]),
    ("kernel e(global int A[]) { x = A[0]; A[0] = 3; }", 7, 999, [np.array([3], np.int32)]),
    ("kernel e(global int A[]) { if (tid < 2) { barrier; } else { barrier; } A[tid] = 1; }",
     1, 4, [np.zeros(4, np.int32)]),
    ("kernel e(global int A[]) { if (tid == 0) { barrier; } }", 1, 3, [np.zeros(1, np.int32)]),
    ("kernel e(global int A[]) { assert(tid != 1); assume(tid != 2); A[tid] = 1; }",
     2, 4, [np.zeros(8, np.int32)]),
    ("kernel e(global int A[], local int L[2]) { L[tid] = 1; barrier; A[gtid] = L[tid % 2]; }",
     3, 3, [np.zeros(9, np.int32)]),
    ("kernel e(global int A[], local int L[4]) { L[0] = tid; barrier; A[gtid] = L[0]; "
     "if (tid == 0) { L[1] = wg; } }", 5, 2, [np.zeros(10, np.int32)]),
    ("kernel e(global int A[]) { for i in 0 .. 40 { barrier; A[(gtid + i) % size(A)] = i; } }",
     2, 64, [np.zeros(128, np.int32)]),
    ("kernel e(global int A[]) { x = 2147483647; A[tid] = x + tid; A[tid + 4] = -2147483648 / -1; "
     "A[tid + 8] = -7 % 3; A[tid + 12] = 7 / 0; }", 1, 4, [np.zeros(16, np.int32)]),
    # a work-item reads back its own store while its neighbour reads the
    # same cell: the read-back is logged (the cell's read/write record counts it)
    ("kernel e(global int A[]) { A[gtid] = 1; x = A[gtid]; y = A[(gtid + 1) % size(A)]; }",
     2, 64, [np.zeros(128, np.int32)]),
    ("kernel e(global int A[], local int L[64]) { L[tid] = tid; x = L[tid]; y = L[(tid + 1) % 64]; "
     "A[gtid] = x + y; }", 2, 64, [np.zeros(128, np.int32)]),
]


def test_every_opcode_on_its_boundaries(rc, oracle):
    """Every expression and branch form the compiler emits, on values at
    each comparison's boundary (the kernel of the translator's CPU test)."""
    from tests.test_translate_cpu import opcode_kernel
    for S in (8, 64):
        run_both(rc, oracle, opcode_kernel(S))


@pytest.mark.parametrize("case", range(len(EDGE)))
def test_edge_cases(rc, oracle, case):
    src, G, S, glob = EDGE[case]
    run_both(rc, oracle, W.Instance(f"edge{case}", src, G, S, glob))


def test_device_inputs_and_stream(rc, oracle):
    import torch
    inst = W.large_kernel(1, groups=4, group_size=128, global_len=8192, local_len=512)
    want = oracle.check(inst.src, inst.groups, inst.group_size, inst.globals)
    bc = rc.compile(inst.src)
    s = torch.cuda.Stream()
    dev = [torch.from_numpy(a).cuda() for a in inst.globals]
    with torch.cuda.stream(s):
        got = rc.check(bc, inst.groups, inst.group_size, dev)
    same(got, want)
    # the caller's device input is not modified
    np.testing.assert_array_equal(dev[0].cpu().numpy(), inst.globals[0])


def test_repeat_calls_reuse_workspace(rc, oracle):
    a = W.large_kernel(2, groups=8, group_size=64, global_len=8192, local_len=256)
    b = W.small_kernel(3)
    wa = oracle.check(a.src, a.groups, a.group_size, a.globals)
    wb = oracle.check(b.src, b.groups, b.group_size, b.globals)
    ba, bb = rc.compile(a.src), rc.compile(b.src)
    for _ in range(3):
        same(rc.check(ba, a.groups, a.group_size, a.globals), wa)
        same(rc.check(bb, b.groups, b.group_size, b.globals), wb)


def test_large_kernel_full_size(rc, oracle):
    """1024 groups x 256, 8 barriers, 200 statements, global int[4M], local
    int[4096] per group: the full report against the oracle (both strategies)."""
    inst = W.large_kernel(0)
    want = run_both(rc, oracle, inst)
    assert want["n_access"] > 10_000_000


def test_long_program_runs_from_global_memory(rc, oracle):
    """Programs longer than the constant-memory bytecode window run from
    global memory; the report must not change."""
    inst = W.large_kernel(7, groups=4, group_size=64, global_len=4096, local_len=256, n_stmts=3000)
    assert rc.compile(inst.src).info()["n_insn"] > 4000
    run_both(rc, oracle, inst)


def test_batch_mixed_instances(rc, oracle):
    """One rc_check_batch over instances of every kind (different programs,
    shapes, barrier counts, errors, divergence): each report equals the
    oracle's for that instance alone."""
    insts = [W.small_kernel(s) for s in range(12)] + [W.tiny_kernel(s) for s in range(12)]
    insts += [W.large_kernel(s, groups=3, group_size=100, global_len=4800, local_len=1600) for s in range(3)]
    insts += [W.Instance(f"edge{i}", *EDGE[i]) for i in range(len(EDGE))]
    want = [oracle.check(i.src, i.groups, i.group_size, i.globals) for i in insts]
    bcs = [rc.compile(i.src) for i in insts]
    for s in STRATEGIES:
        rc.set_strategy(s)
        got = rc.check_batch([(b, i.groups, i.group_size, i.globals) for b, i in zip(bcs, insts)])
        for g, w, i in zip(got, want, insts):
            same(g, w, f"{i.name} strategy {s}")
    rc.set_strategy(0)


def test_resident_batch_is_one_launch(rc, oracle):
    """Strategy 3 runs every round of a batch in one cooperative launch
    (barriers up to 8, divergence, errors, crowded cells): one interpreter
    launch for the call, reports equal to the oracle's, final memories
    included."""
    insts = [W.small_kernel(s, n_barriers=b) for s, b in zip(range(40), [0, 1, 2, 3, 5, 8] * 7)]
    insts += [W.Instance(f"edge{i}", *EDGE[i]) for i in range(len(EDGE))]
    insts += W.batch_kernels(11, 8)[:4]
    insts = [i for i in insts if i.n_threads * 300 < 4_000_000]
    want = [oracle.check(i.src, i.groups, i.group_size, i.globals) for i in insts]
    bcs = [rc.compile(i.src) for i in insts]
    rc.set_strategy(3)
    rc.profile_enable(True)
    rc.profile_reset()
    try:
        got = rc.check_batch([(b, i.groups, i.group_size, i.globals) for b, i in zip(bcs, insts)])
        assert rc.profile_get(0)["launches"] == 1
    finally:
        rc.profile_enable(False)
        rc.set_strategy(0)
    for g, w, i in zip(got, want, insts):
        same(g, w, i.name)


def test_autotuner_decides_and_persists(rc, oracle, tmp_path):
    """Strategy 0 alternates both exact strategies per interval until it has
    two samples of each, then keeps the cheaper one and writes it to the
    cache; reports stay identical throughout.  (A group size that is not a
    multiple of 32 keeps the run interval by interval: resident runs take
    no strategy.)"""
    cache = str(tmp_path / "tune.json")
    rc.autotune_config(cache)
    rc.set_strategy(0)
    inst = W.large_kernel(3, groups=16, group_size=250, global_len=65536, local_len=4096)
    want = oracle.check(inst.src, inst.groups, inst.group_size, inst.globals)
    bc = rc.compile(inst.src)
    bound = bc.info()["max_access_per_interval"]
    assert rc.autotune_lookup(0, inst.n_threads, bound) == 0
    same(rc.check(bc, inst.groups, inst.group_size, inst.globals), want)  # 9 intervals: decides
    best = rc.autotune_lookup(0, inst.n_threads, bound)
    assert best in (1, 2)
    same(rc.check(bc, inst.groups, inst.group_size, inst.globals), want)
    assert '"best": %d' % best in open(cache).read()
    rc.autotune_reset()
    assert rc.autotune_lookup(0, inst.n_threads, bound) == 0
    rc.autotune_config(cache)  # reload from the file
    assert rc.autotune_lookup(0, inst.n_threads, bound) == best
    # batches decide per round the same way, then time each block shape
    # (128, 256, 512 threads per CTA) on two rounds and keep the fastest
    insts = [W.small_kernel(s, n_barriers=3) for s in range(20)]
    wants = [oracle.check(i.src, i.groups, i.group_size, i.globals) for i in insts]
    bcs = [rc.compile(i.src) for i in insts]
    tasks = sum((i.n_threads + 31) // 32 for i in insts)
    bound = sum((i.n_threads + 31) // 32 * max(b.info()["max_access_per_interval"], 1)
                for i, b in zip(insts, bcs)) // tasks
    for _ in range(4):  # 4 rounds per call: strategy samples, then shape samples
        got = rc.check_batch([(b, i.groups, i.group_size, i.globals) for b, i in zip(bcs, insts)])
        for g, w, i in zip(got, wants, insts):
            same(g, w, i.name)
    assert rc.autotune_lookup(1, tasks, bound) in (1, 2)
    threads = rc.autotune_lookup(2, tasks, bound)
    assert threads in (128, 256, 512)
    assert '"threads": %d' % threads in open(cache).read()
    # the log capacity: twice the fullest slice seen, in permille of the bound
    log_pm = rc.autotune_lookup(3, tasks, bound)
    assert 16 <= log_pm <= 1000
    assert '"log_permille": %d' % log_pm in open(cache).read()
    rc.autotune_config("")


def test_batch_log_capacity_overflow_recovers(rc, oracle, tmp_path):
    """A batch class whose tuned log capacity is too small (one record per
    work-item and interval, planted in the cache file) overflows its slices:
    the call is checked again at the static bound, the reports equal the
    oracle's, and the class keeps the bound (1000 permille) from then on.
    Both schedules: lock-step rounds and resident."""
    insts = [W.small_kernel(s, n_barriers=2) for s in range(300, 312)]
    wants = [oracle.check(i.src, i.groups, i.group_size, i.globals) for i in insts]
    bcs = [rc.compile(i.src) for i in insts]
    tasks = sum((i.n_threads + 31) // 32 for i in insts)
    bound = sum((i.n_threads + 31) // 32 * max(b.info()["max_access_per_interval"], 1)
                for i, b in zip(insts, bcs)) // tasks
    key = "batch:T%d:B%d" % (tasks.bit_length(), bound.bit_length())
    for strategy in (0, 3):
        cache = tmp_path / f"tune{strategy}.json"
        cache.write_text('{"racecheck_autotune": 1, "entries": {"%s": {"best": 2, "threads": 256, '
                         '"log_permille": 1}}}' % key)
        rc.autotune_reset()
        rc.autotune_config(str(cache))
        assert rc.autotune_lookup(3, tasks, bound) == 1
        rc.set_strategy(strategy)
        try:
            got = rc.check_batch([(b, i.groups, i.group_size, i.globals) for b, i in zip(bcs, insts)])
        finally:
            rc.set_strategy(0)
        for g, w, i in zip(got, wants, insts):
            same(g, w, i.name)
        assert rc.autotune_lookup(3, tasks, bound) == 1000
    rc.autotune_reset()
    rc.autotune_config("")


def test_pinned_host_inputs(rc, oracle):
    """Page-locked host inputs are read by a copy kernel over the CPU-GPU
    link; ragged lengths and offsets that are not 16-byte aligned."""
    import torch
    src = ("kernel t(global int A[], global int B[], global int C[]) {\n"
           " x = A[gtid % 37];\n y = B[(gtid * 3) % 1001];\n C[gtid] = x + y;\n}\n")
    arrs = [np.arange(37, dtype=np.int32) * 7, np.arange(1001, dtype=np.int32) - 500,
            np.zeros(4 * 96, np.int32)]
    want = oracle.check(src, 4, 96, arrs)
    pinned = [torch.from_numpy(a.copy()).pin_memory() for a in arrs]
    bc = rc.compile(src)
    for s in STRATEGIES:
        rc.set_strategy(s)
        same(rc.check(bc, 4, 96, pinned), want, f"pinned strategy {s}")
    rc.set_strategy(0)
    inst = W.large_kernel(1, groups=8, group_size=256, global_len=65536, local_len=256)
    want = oracle.check(inst.src, inst.groups, inst.group_size, inst.globals)
    pinned = [torch.from_numpy(a.copy()).pin_memory() for a in inst.globals]
    same(rc.check(rc.compile(inst.src), inst.groups, inst.group_size, pinned), want, "pinned large")
