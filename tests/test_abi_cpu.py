"""Host-side checks of the C ABI library (no GPU compute calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1308_3203_gb300 import build as gpu_build
from paper_1308_3203_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rc():
    gpu_build.build()
    from paper_1308_3203_gb300 import racecheck
    racecheck.load()
    return racecheck


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(rc_\w+)\s*\(", text, re.M))
    return names


def test_library_exports_every_declared_symbol(rc):
    lib = ctypes.CDLL(rc.LIB_PATH)
    syms = declared_symbols()
    assert {"rc_compile", "rc_check", "rc_check_batch", "rc_report_free"} <= syms
    for s in sorted(syms):
        assert hasattr(lib, s), s


def test_compile_reports_static_facts(rc):
    b = rc.compile("kernel k(global int A[], local int L[8], global int g) {\n"
                   "  x = A[tid];\n  barrier;\n  for i in 0 .. 4 { L[i] = x + A[i]; }\n"
                   "  assert(x >= 0);\n  g = x;\n}\n")
    i = b.info()
    assert i["n_mems"] == 3 and i["n_global"] == 2 and i["n_barriers"] == 1
    assert i["n_asserts"] == 1 and i["local_cells"] == 8
    # interval 0: one read; interval 1: 4 x (read + write) + write of g
    assert i["max_access_per_interval"] == 9
    assert i["max_write_per_interval"] == 5


@pytest.mark.parametrize("bad", [
    "kernel k(global int A[]) { A[0] = ; }",
    "kernel k(global int A[4]) { }",
    "kernel k(local int L[]) { }",
    "kernel k() { B[0] = 1; }",
    "kernel k() { for i in 0 .. 3 { i = 2; } }",
    "kernel k() { for i in 0 .. 3 { for i in 0 .. 2 { } } }",
    "kernel k() { tid = 1; }",
    "kernel k() { x = 99999999999; }",
    "kernel k(global int A[], global int A[]) { }",
    "kernel k() { x = 1 }",
    "kernel k() { x = 1; } trailing",
    "kernel k() { x = @; }",
])
def test_compile_rejects_bad_programs(rc, bad):
    with pytest.raises(rc.RaceCheckError) as e:
        rc.compile(bad)
    assert e.value.code == 1


def test_static_bounds_cover_every_run(rc, oracle):
    """The per-interval access/write bounds the runtime sizes its logs with
    are never exceeded by a real run (checked against the oracle)."""
    for s in range(25):
        for f in (W.small_kernel(s),
                  W.large_kernel(s, groups=2, group_size=64, global_len=4096, local_len=256),
                  W.stress_kernel(s, groups=2, group_size=64),
                  W.tiny_kernel(s)):
            o = oracle.check(f.src, f.groups, f.group_size, f.globals)
            i = rc.compile(f.src).info()
            assert o["max_acc"] <= i["max_access_per_interval"], f.name
            assert o["max_wr"] <= i["max_write_per_interval"], f.name


def test_bad_arguments_rejected_without_gpu_work(rc):
    b = rc.compile("kernel k(global int A[]) { A[tid] = 1; }")
    with pytest.raises(rc.RaceCheckError) as e:
        rc.check(b, 0, 32, [np.zeros(4, np.int32)])
    assert e.value.code == 2
    with pytest.raises(rc.RaceCheckError):
        rc.check(b, 1, 2048, [np.zeros(4, np.int32)])
    with pytest.raises(rc.RaceCheckError):
        rc.check(b, 1, 32, [])
    with pytest.raises(rc.RaceCheckError):
        rc.set_strategy(7)


def test_strategy_values(rc):
    """0 auto, 1 sort, 2 shadow, 3 resident, 4 one CTA are accepted; nothing else."""
    for s in (0, 1, 2, 3, 4):
        rc.set_strategy(s)
    for bad in (5, -1):
        with pytest.raises(rc.RaceCheckError):
            rc.set_strategy(bad)
    rc.set_strategy(0)


def test_diag_grid_barrier_rejects_bad_limits(rc):
    """The diagnostic checks its argument before touching a device."""
    with pytest.raises(rc.RaceCheckError):
        rc.diag_grid_barrier(0)
    with pytest.raises(rc.RaceCheckError):
        rc.diag_grid_barrier(20_000_000)


def test_group_scope_rejected_where_unsupported_without_gpu_work(rc):
    """Batches and the explorers take kernel-wide barriers only: the request
    is refused before any device work."""
    import ctypes
    bc = rc.compile("kernel k(global int A[]) { A[gtid] = 1; }")
    A = np.zeros(8, np.int32)
    inp, keep = rc._marshal([A], None, False)
    inp.flags |= rc.RC_GROUP_BARRIERS
    lib = rc.load()
    out = (rc._ExploreInterval * 4)()
    n = ctypes.c_uint32()
    assert lib.rc_explore(bc.handle, 2, 4, ctypes.byref(inp), 0, out, 4, ctypes.byref(n)) == 2
    pairs = (rc._PairInterval * 4)()
    assert lib.rc_explore_pairs(bc.handle, 2, 4, ctypes.byref(inp), 0, pairs, 4, ctypes.byref(n), None) == 2
    hs = (ctypes.c_void_p * 1)(bc.handle.value)
    gs = (ctypes.c_uint32 * 1)(2)
    ss = (ctypes.c_uint32 * 1)(4)
    ins = (rc._Input * 1)(inp)
    outs = (ctypes.POINTER(rc._Report) * 1)()
    assert lib.rc_check_batch(hs, gs, ss, ins, 1, outs) == 2
    del keep


def test_prove_private_checks_its_flag_array(rc):
    import ctypes
    bc = rc.compile("kernel k(global int A[]) { A[gtid] = 1; }")
    inp, keep = rc._marshal([np.zeros(8, np.int32)], None, False)
    flags = (ctypes.c_uint8 * 1)()
    n = ctypes.c_uint32()
    assert rc.load().rc_prove_private(bc.handle, 1, 8, ctypes.byref(inp), flags, 1, ctypes.byref(n)) == 2
    del keep


def test_search_ranked_checks_its_arguments_without_gpu_work(rc):
    """Unknown flags and missing arrays are refused, and an empty candidate
    list is an empty search, before any device or feature work."""
    import ctypes
    lib = rc.load()
    res = rc._RankedResult()
    assert lib.rc_search_ranked(None, None, None, None, None, 0, 0, 0, ctypes.byref(res), None) == 0
    assert res.first == -1 and res.checks == 0
    assert lib.rc_search_ranked(None, None, None, None, None, 0, 0, 2, ctypes.byref(res), None) == 2
    assert lib.rc_search_ranked(None, None, None, None, None, 3, 0, 0, ctypes.byref(res), None) == 2
    assert lib.rc_search_ranked(None, None, None, None, None, 0, 0, 0, None, None) == 2


@pytest.mark.filterwarnings("ignore:This process .* is multi-threaded")
def test_features_worker_pool_survives_a_fork(rc):
    """The feature threads are per process: a child forked after they
    started computes the same features with a pool of its own."""
    import multiprocessing as mp
    from paper_1308_3203_gb300 import proposal
    _, items = proposal.kernel_candidates(7)
    want = rc.features(items, n_threads=4)
    ctx = mp.get_context("fork")
    q = ctx.Queue()
    p = ctx.Process(target=_features_in_child, args=(q, 7))
    p.start()
    got = q.get(timeout=120)
    p.join(timeout=60)
    assert p.exitcode == 0
    np.testing.assert_array_equal(got, want)


def _features_in_child(q, seed):
    from paper_1308_3203_gb300 import proposal, racecheck
    _, items = proposal.kernel_candidates(seed)
    q.put(racecheck.features(items, n_threads=4))


def test_report_arrays_view_the_library_report(monkeypatch):
    """A Python report's record and final-memory arrays are views of the
    library's arrays: the rc_report is freed once, when the last view is
    gone, and not before."""
    import gc
    from paper_1308_3203_gb300 import racecheck
    freed = []

    class FakeLib:
        def rc_report_free(self, p):
            freed.append(p)

    monkeypatch.setattr(racecheck, "load", lambda: FakeLib())
    recs = (ctypes.c_uint32 * 30)(*range(30))
    fin = (ctypes.c_int32 * 5)(-1, 2, 3, 4, 5)
    r = racecheck._Report(1, 5, 1000, 900, 100, 3, ctypes.cast(recs, ctypes.c_void_p), 5,
                          ctypes.cast(fin, ctypes.c_void_p), 800)
    d = racecheck._report(ctypes.pointer(r))
    assert d["records"].shape == (3, 10) and d["records"][2, 9] == 29
    assert list(d["final"]) == [-1, 2, 3, 4, 5]
    assert (d["status"], d["n_intervals"], d["n_access"], d["n_logged"]) == (1, 5, 1000, 800)
    kept = d["records"]
    del d
    gc.collect()
    assert not freed  # the records still view the report
    assert kept[1, 0] == 10
    del kept
    gc.collect()
    assert len(freed) == 1
    empty = racecheck._Report(0, 1, 0, 0, 0, 0, None, 0, None, 0)
    d = racecheck._report(ctypes.pointer(empty))
    assert d["records"].shape == (0, 10) and d["final"] is None
    del d
    gc.collect()
    assert len(freed) == 2
