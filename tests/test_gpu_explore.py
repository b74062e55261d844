"""Exhaustive interleavings on the GPU (rc_explore) against the oracle's
brute-force explorer.

The oracle explores every schedule of the whole run (all states reachable
at each barrier); the GPU explores each interval from the checker's own
state at its start.  Those starts coincide while every earlier interval has
one reachable shared state and no schedule-dependent read (then every
schedule leaves every work-item in the same state), so intervals are
compared up to the first one where the oracle sees several."""
import numpy as np
import pytest

from paper_1308_3203_gb300 import workloads as W
from tests.golden import golden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1308_3203_gb300 import build as gpu_build
    gpu_build.build()
    from paper_1308_3203_gb300 import racecheck
    racecheck.load()
    return racecheck


def compare(rc, oracle, src, G, S, globals_, what):
    want = oracle.explore(src, G, S, globals_)
    assert not want["overflow"], what
    got = rc.explore(rc.compile(src), G, S, globals_)
    assert all(g["complete"] for g in got), what
    n = 0
    for k, (ends, dev) in enumerate(zip(want["end_states"], want["deviated"])):
        assert k < len(got), (what, k)
        assert got[k]["n_end_states"] == ends, (what, k, got[k], ends)
        assert got[k]["deviated"] == dev, (what, k, got[k], dev)
        n += 1
        if ends != 1 or dev:
            break
    return got, want, n


@pytest.mark.parametrize("chunk", range(4))
def test_tiny_kernels_match_the_oracle_explorer(rc, oracle, chunk):
    compared = 0
    for seed in range(chunk * 50, chunk * 50 + 50):
        inst = W.tiny_kernel(seed)
        _, _, n = compare(rc, oracle, inst.src, inst.groups, inst.group_size, inst.globals, inst.name)
        compared += n
    assert compared >= 50


def test_fig2_race_is_confirmed(rc, oracle):
    """Fig. 2 (4 work-items): the checker flags RW races in interval 1 and
    the schedules leave g = 0 or 1 (two shared states); with A[n] = 0 the
    reads still depend on the schedule but memory does not (one state)."""
    for name, n_states in (("fig2_n4.txt", 2), ("fig2_n4_lastzero.txt", 1)):
        g = golden.load(name)
        got, want, _ = compare(rc, oracle, g["src"], g["groups"], g["group_size"], g["globals"], name)
        assert got[0]["n_end_states"] == 1 and not got[0]["deviated"], (name, got)
        assert got[1]["deviated"] and got[1]["n_end_states"] == n_states, (name, got)


def test_race_free_intervals_have_one_state(rc, oracle):
    """Invariant I1 on the GPU side: where the checker reports no race record
    for an interval (from a start every schedule shares), every schedule
    reaches the same shared state and no read depends on the schedule."""
    checked = 0
    for seed in range(300, 360):
        inst = W.tiny_kernel(seed)
        rep = oracle.check(inst.src, inst.groups, inst.group_size, inst.globals)
        got = rc.explore(rc.compile(inst.src), inst.groups, inst.group_size, inst.globals)
        flagged = {int(r[0]) for r in rep["records"] if r[4] in (1, 2, 3)}
        for g in got:
            if g["interval"] in flagged:
                break
            assert g["n_end_states"] == 1 and not g["deviated"], (inst.name, got)
            checked += 1
    assert checked > 40


def test_rejects_large_instances(rc):
    bc = rc.compile("kernel k(global int A[]) { A[tid] = 1; }")
    with pytest.raises(rc.RaceCheckError):
        rc.explore(bc, 2, 16, [np.zeros(64, np.int32)])


# ---- interleaving product of two work-items (rc_explore_pairs)

def compare_pairs(rc, oracle, src, G, S, globals_, what):
    want = oracle.explore_pairs(src, G, S, globals_)
    got = rc.explore_pairs(rc.compile(src), G, S, globals_, detail=True)
    full = oracle.explore(src, G, S, globals_)
    n = 0
    for k, w in enumerate(want):
        if w is None:
            break
        assert got[k]["complete"], (what, k)
        assert got[k]["pairs"] == w, (what, k, got[k]["pairs"], w)
        n += 1
        if full["end_states"][k] != 1 or full["deviated"][k]:
            break  # later intervals may start from several states on the oracle side
    return got, n


def test_pairs_match_the_oracle(rc, oracle):
    compared = 0
    for seed in range(0, 120):
        inst = W.tiny_kernel(seed)
        _, n = compare_pairs(rc, oracle, inst.src, inst.groups, inst.group_size, inst.globals, inst.name)
        compared += n
    assert compared >= 120


def test_pairs_find_the_fig2_race(rc, oracle):
    """Fig. 2: the neighbouring pair (2, 3) reaches g = 0 and g = 1."""
    g = golden.load("fig2_n4.txt")
    got, _ = compare_pairs(rc, oracle, g["src"], g["groups"], g["group_size"], g["globals"], "fig2")
    assert got[1]["n_racy"] == 1 and got[1]["first"] == (2, 3)


def test_two_work_items_pairs_equal_the_full_search(rc, oracle):
    """With two work-items the only pair is the whole instance."""
    for seed in range(40):
        inst = W.tiny_kernel(1000 + seed)
        if inst.n_threads != 2:
            continue
        bc = rc.compile(inst.src)
        full = rc.explore(bc, inst.groups, inst.group_size, inst.globals)
        pairs = rc.explore_pairs(bc, inst.groups, inst.group_size, inst.globals, detail=True)
        for f, p in zip(full, pairs):
            assert p["pairs"] == [(f["n_end_states"], f["deviated"])], (inst.name, f, p)


def test_pairs_scale_past_the_full_search(rc):
    """64 work-items (2016 pairs): each copies its right neighbour's cell,
    which the neighbour overwrites in the same interval, so exactly the pairs
    (t, t + 1) reach two memories; any other pair reads a cell of a
    work-item that does not run."""
    src = "kernel k(global int A[]) { A[tid] = 0; barrier; A[tid] = 1; x = A[tid + 1]; A[tid + 64] = x; }"
    S = 64
    got = rc.explore_pairs(rc.compile(src), 1, S, [np.zeros(2 * S, np.int32)], detail=True)
    assert got[1]["n_pairs"] == S * (S - 1) // 2 and got[1]["complete"]
    racy = [(i, j) for p, (i, j) in zip(got[1]["pairs"], [(i, j) for i in range(S) for j in range(i + 1, S)])
            if p[0] >= 2]
    assert racy == [(t, t + 1) for t in range(S - 1)], racy[:5]
