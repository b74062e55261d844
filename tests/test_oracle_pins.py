"""Pins for the CPU oracle: values fixed by the paper and by mathematics.

Nothing here trusts the oracle's own code: expected values are hand-derived
from the paper's figures (fixtures in tests/golden), closed forms for
affine access patterns, the definition of int32 arithmetic, and the
brute-force interleaving explorer, which runs the paper's Sec. 4 global
semantics literally over every schedule.
"""
import numpy as np
import pytest

from paper_1308_3203_gb300 import workloads as W
from tests.golden import golden

pytestmark = pytest.mark.filterwarnings("ignore")


def rec(interval, addr, cls, t_a, t_b, nr, nw, na, space=0, wg=0):
    return [interval, space, wg, addr, cls, t_a, t_b, nr, nw, na]


# ---------------------------------------------------------------- goldens

@pytest.mark.parametrize("name", golden.names())
def test_golden_fixture(oracle, name):
    g = golden.load(name)
    r = oracle.check(g["src"], g["groups"], g["group_size"], g["globals"])
    for k, v in g["expect"].items():
        assert r[k] == v, (k, r[k], v)
    np.testing.assert_array_equal(r["records"], g["records"])
    np.testing.assert_array_equal(r["final"], g["final"])


FIG1 = golden.load("fig1_n6.txt")["src"]
FIG2 = golden.load("fig2_n4.txt")["src"]


@pytest.mark.parametrize("n", [3, 4, 7, 12])
@pytest.mark.parametrize("seed", [0, 1])
def test_fig1_closed_form(oracle, n, seed):
    """Fig. 1: OOB for work-items 0 and n-1; in interval 1 a read/write race
    at R[k+1] (reader k, writer k+1) exactly when 2*R0[k+2] != R0[k+1], where
    R0 is R after interval 0, for k = 1..n-3."""
    rng = np.random.default_rng(seed)
    A = rng.integers(-5, 5, n).astype(np.int32)
    B = rng.integers(-5, 5, n).astype(np.int32)
    R = rng.integers(-5, 5, n).astype(np.int32)
    if seed == 1:  # make some cells agree so that both outcomes occur
        A[:] = 0
        B[:] = 0
        R[:] = 0
    r = oracle.check(FIG1, 1, n, [A, B, R])
    R0 = R.astype(np.int64).copy()
    for k in range(1, n - 1):
        R0[k] = A[k - 1] + B[k + 1]
    baseR = 2 * n
    exp = []
    for k in range(1, n - 2):
        if 2 * R0[k + 2] != R0[k + 1]:
            exp.append(rec(1, baseR + k + 1, 3, k, k + 1, 1, 1, 2))
    exp.append(rec(0, 2**32 - 1, 16, 0, 0, 0, 0, 0))
    exp.append(rec(0, n, 16, n - 1, 1, 0, 0, 0))
    np.testing.assert_array_equal(r["records"], np.array(exp, dtype=np.uint32).reshape(-1, 10))
    Rf = R0.copy()
    for k in range(1, n - 1):
        Rf[k] = 2 * R0[k + 1]
    np.testing.assert_array_equal(r["final"], np.concatenate([A, B, Rf.astype(np.int32)]))
    assert r["status"] == (1 if any(e[4] == 3 for e in exp) else 2)
    assert r["n_intervals"] == 2
    assert r["n_access"] == 3 * (n - 2) + 1 + 2 * (n - 2)


def test_fig2_schedules_reach_both_values_of_g(oracle):
    """Sec. 6.1 (Fig. 2): depending on the schedule, g ends as 0 or as 1."""
    n = 3
    e = oracle.explore(FIG2, 1, n, [np.ones(n + 1, np.int32), np.array([5], np.int32)])
    assert not e["overflow"]
    gs = sorted(int(f[-1]) for f in e["finals"])
    assert gs == [0, 1]
    assert e["end_states"][0] == 1 and e["end_states"][1] == 2
    assert e["deviated"] == [False, True, False]
    # variant where the last cell is 0: one final memory, reads still racy
    A = np.ones(n + 1, np.int32)
    A[n] = 0
    e = oracle.explore(FIG2, 1, n, [A, np.array([5], np.int32)])
    assert len(e["finals"]) == 1 and int(e["finals"][0][-1]) == 1
    assert e["deviated"][1]


# ---------------------------------------------------------------- arithmetic

ARITH = [
    ("2147483647 + 1", -2147483648),
    ("-2147483648 - 1", 2147483647),
    ("65536 * 65536", 0),
    ("65537 * 65537", 131073),
    ("-7 / 2", -3), ("7 / -2", -3), ("-7 / -2", 3), ("7 / 0", 0),
    ("-7 % 3", 2), ("7 % -3", 1), ("-7 % -3", 2), ("7 % 0", 0), ("6 % 3", 0),
    ("-2147483648 / -1", -2147483648), ("-2147483648 % -1", 0),
    ("-2147483648 % 3", 1),
    ("3 < 5", 1), ("5 <= 5", 1), ("5 > 5", 0), ("5 >= 6", 0), ("4 == 4", 1), ("4 != 4", 0),
    ("-1 < 0", 1),
    ("3 && 0", 0), ("3 && -1", 1), ("0 || 0", 0), ("0 || 7", 1), ("!0", 1), ("!9", 0),
    ("-(-5)", 5), ("4294967295", -1), ("2147483648", -2147483648),
    ("2 + 3 * 4", 14), ("(2 + 3) * 4", 20), ("10 - 3 - 2", 5), ("100 / 10 / 5", 2),
    ("1 < 2 == 1", 1), ("1 + 2 < 4 && 5 > 3", 1), ("!1 + 1", 1), ("-3 % 5 * 2", 4),
]


def test_int32_arithmetic(oracle):
    body = "\n".join(f"  A[{i}] = {e};" for i, (e, _) in enumerate(ARITH))
    src = f"kernel arith(global int A[]) {{\n{body}\n}}\n"
    r = oracle.check(src, 1, 1, [np.zeros(len(ARITH), np.int32)])
    assert r["status"] == 0 and len(r["records"]) == 0
    np.testing.assert_array_equal(r["final"], np.array([v for _, v in ARITH], dtype=np.int32))


def test_builtins_and_private_state(oracle):
    src = """kernel ids(global int A[], global int B[]) {
  if (gtid == 6) {
    A[0] = tid; A[1] = wg; A[2] = gtid; A[3] = gsize; A[4] = ngroups;
    A[5] = size(A); A[6] = size(B); A[7] = x;
    x = 3; x = x * x; A[8] = x;
    for i in 2 .. 5 { y = y + i; }
    A[9] = y; A[10] = i;
    for j in 5 .. 2 { y = 100; }
    A[11] = j; A[12] = y;
  }
}
"""
    r = oracle.check(src, 3, 4, [np.zeros(13, np.int32), np.zeros(5, np.int32)])
    np.testing.assert_array_equal(r["final"][:13], [2, 1, 6, 4, 3, 13, 5, 0, 9, 9, 5, 5, 9])


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("a", [0, 1, 2])
@pytest.mark.parametrize("n", [1, 2, 5, 64, 129, 200, 256])
@pytest.mark.parametrize("c,d", [(0, 3), (1, 0), (-3, 7), (2**25, 1)])
def test_affine_store_closed_form(oracle, a, n, c, d):
    """A[(a*tid + b) % 256] = c*tid + d by n work-items in one interval.
    a = 0: one cell, benign iff c = 0 (or one writer), witness (0, 1);
    a = 1: no collision; a = 2: tid and tid+128 collide, values differ iff
    128*c != 0 mod 2^32."""
    b = 17
    src = f"kernel aff(global int A[]) {{\n  A[({a} * tid + {b}) % 256] = {c} * tid + {d};\n}}\n"
    r = oracle.check(src, 1, n, [np.zeros(256, np.int32)])
    exp = []
    if a == 0 and n >= 2:
        exp.append(rec(0, b, 2 if c == 0 else 1, 0, 1, 0, n, n))
    if a == 2:
        for cell in range(256):
            ts = [t for t in range(n) if (2 * t + b) % 256 == cell]
            if len(ts) == 2:
                benign = (128 * c) % 2**32 == 0
                exp.append(rec(0, cell, 2 if benign else 1, ts[0], ts[1], 0, 2, 2))
        assert len(exp) == max(0, n - 128)
    np.testing.assert_array_equal(r["records"], np.array(exp, dtype=np.uint32).reshape(-1, 10))


# ---------------------------------------------------------------- rule details

def _run(oracle, body, n, A, groups=1, decl="global int A[]"):
    src = f"kernel t({decl}) {{\n{body}\n}}\n"
    return oracle.check(src, groups, n, [np.array(A, np.int32)])


def test_ww_uses_last_write_of_each_thread(oracle):
    # thread 0 writes 6 then 5, thread 1 writes 5: the cell ends 5 either way
    r = _run(oracle, "if (tid == 0) { A[0] = 6; A[0] = 5; }\nif (tid == 1) { A[0] = 5; }", 2, [0])
    np.testing.assert_array_equal(r["records"], [rec(0, 0, 2, 0, 1, 0, 2, 3)])
    # last values 5,5,6,5: race, witness (smallest writer, first differing)
    r = _run(oracle, "A[0] = 5;\nif (tid == 2) { A[0] = 6; }", 4, [0])
    np.testing.assert_array_equal(r["records"], [rec(0, 0, 1, 0, 2, 0, 4, 5)])


def test_rw_witness_is_smallest_conflicting_pair(oracle):
    body = "x = A[0];\nif (tid == 2) { A[0] = 7; }\nif (tid == 3) { A[0] = 9; }"
    # every work-item reads 7; writer 2 writes 7 (no conflict), writer 3 writes 9
    r = _run(oracle, body, 4, [7])
    np.testing.assert_array_equal(r["records"], [rec(0, 0, 1, 2, 3, 4, 2, 6),
                                                 rec(0, 0, 3, 0, 3, 4, 2, 6)])
    r = _run(oracle, "if (tid != 0) { x = A[0]; }\n" + body.split("\n", 1)[1], 4, [7])
    np.testing.assert_array_equal(r["records"][1], rec(0, 0, 3, 1, 3, 3, 2, 5))
    # a reader that wrote the cell itself sees its own value; only others count
    body2 = "if (tid == 3) { A[0] = 9; x = A[0]; }\nif (tid == 1) { A[0] = 9; }"
    r = _run(oracle, body2, 4, [7])
    np.testing.assert_array_equal(r["records"], [rec(0, 0, 2, 1, 3, 1, 2, 3)])
    body3 = "if (tid == 3) { A[0] = 8; x = A[0]; }\nif (tid == 1) { A[0] = 9; }"
    r = _run(oracle, body3, 4, [7])
    np.testing.assert_array_equal(r["records"], [rec(0, 0, 1, 1, 3, 1, 2, 3),
                                                 rec(0, 0, 3, 3, 1, 1, 2, 3)])
    # reads of a cell nobody else writes: never a race
    r = _run(oracle, "x = A[tid];\nA[tid] = x + 1;", 4, [1, 2, 3, 4])
    assert len(r["records"]) == 0
    np.testing.assert_array_equal(r["final"], [2, 3, 4, 5])


def test_reads_see_snapshot_and_own_writes(oracle):
    # thread 1 writes A[0] = 5 while thread 0 reads A[0] twice around its own write
    body = ("if (tid == 0) { x = A[0]; A[1] = x; A[0] = 3; y = A[0]; A[2] = y; }\n"
            "if (tid == 1) { A[0] = 5; }\nbarrier;\nif (tid == 0) { z = A[0]; A[3] = z; }")
    r = _run(oracle, body, 2, [9, 0, 0, 0])
    # commit: the highest writer (1) wins -> A[0] = 5 after the barrier
    np.testing.assert_array_equal(r["final"], [5, 9, 3, 5])
    recs = r["records"]
    assert [tuple(x[[0, 3, 4, 5, 6]]) for x in recs] == [(0, 0, 1, 0, 1), (0, 0, 3, 0, 1)]


def test_commit_takes_highest_writer_last_write(oracle):
    r = _run(oracle, "if (tid == 0) { A[0] = 1; }\nif (tid == 2) { A[0] = 3; A[0] = 4; }\n"
                     "if (tid == 1) { A[0] = 2; }", 3, [0])
    assert r["final"][0] == 4


def test_errors_assert_assume_divergence(oracle):
    r = _run(oracle, "assert(tid != 1);\nassert(tid != 2);\nA[tid] = 1;", 4, [0, 0, 0, 0])
    np.testing.assert_array_equal(r["records"], [rec(0, 0, 17, 1, 0, 0, 0, 0),
                                                 rec(0, 0, 17, 2, 1, 0, 0, 0)])
    assert r["status"] == 3
    np.testing.assert_array_equal(r["final"], [1, 0, 0, 1])
    r = _run(oracle, "assume(tid != 1);\nA[tid] = 1;", 3, [0, 0, 0])
    assert len(r["records"]) == 0 and r["status"] == 0
    np.testing.assert_array_equal(r["final"], [1, 0, 1])
    # barrier inside a branch: work-items 0,1 wait at barrier 0, 2,3 at barrier 1
    r = _run(oracle, "if (tid < 2) { barrier; } else { barrier; }\nA[tid] = 1;", 4, [0] * 4)
    np.testing.assert_array_equal(r["records"], [rec(0, 0, 18, 0, 0, 0, 0, 2),
                                                 rec(0, 0, 18, 2, 1, 0, 0, 2)])
    assert r["status"] == 4 and r["n_intervals"] == 1
    # some work-items exit while others wait
    r = _run(oracle, "if (tid == 0) { barrier; }", 3, [0])
    np.testing.assert_array_equal(r["records"], [rec(0, 0, 18, 0, 0, 0, 0, 1),
                                                 rec(0, 0, 18, 1, 2**32 - 1, 0, 0, 2)])
    # errors of one interval are ordered by kind, then work-item: work-item 2
    # stores out of bounds (A[4] of 4 cells), work-item 0 fails the assert;
    # the failed assert decides the status, the out-of-bounds store is not
    # performed and not counted
    r = _run(oracle, "assert(tid != 0);\nA[tid + 2] = 1;", 3, [0] * 4)
    np.testing.assert_array_equal(r["records"], [rec(0, 4, 16, 2, 0, 0, 0, 0),
                                                 rec(0, 0, 17, 0, 0, 0, 0, 0)])
    assert r["status"] == 3 and r["n_access"] == 1
    np.testing.assert_array_equal(r["final"], [0, 0, 0, 1])


def test_local_memory_is_per_group(oracle):
    src = ("kernel t(global int A[], local int L[2]) {\n  L[0] = tid;\n  barrier;\n"
           "  A[gtid] = L[0];\n  if (tid == 0) { L[1] = wg; }\n}\n")
    r = oracle.check(src, 3, 2, [np.zeros(6, np.int32)])
    # two writers per group with values 0, 1: a race in each group's own cell
    # witnesses are global ids (gtid = wg * gsize + tid)
    np.testing.assert_array_equal(r["records"], [rec(0, 0, 1, 2 * w, 2 * w + 1, 0, 2, 2,
                                                     space=1, wg=w) for w in range(3)])
    np.testing.assert_array_equal(r["final"], [1] * 6)
    assert r["n_local"] == 6 + 6 + 3 and r["n_global"] == 6


def test_local_oob_and_empty(oracle):
    src = "kernel t(global int A[], local int L[2]) {\n  L[tid] = 1;\n}\n"
    r = oracle.check(src, 2, 3, [np.zeros(1, np.int32)])
    np.testing.assert_array_equal(r["records"], [rec(0, 2, 16, 2, 1, 0, 0, 0, space=1, wg=0),
                                                 rec(0, 2, 16, 5, 1, 0, 0, 0, space=1, wg=1)])
    r = oracle.check("kernel e() { }", 4, 32, [])
    assert r["status"] == 0 and r["n_access"] == 0 and r["n_intervals"] == 1
    r = oracle.check("kernel e(global int A[]) { A[tid] = 1; }", 1, 3, [np.zeros(0, np.int32)])
    assert r["status"] == 2 and len(r["records"]) == 3


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
])
def test_parse_errors(oracle, bad):
    with pytest.raises(oracle.OracleError):
        oracle.check(bad, 1, 1, [np.zeros(1, np.int32)] * bad.count("global"))


# ---------------------------------------------------------------- metamorphic

@pytest.mark.parametrize("seed", range(20))
def test_thread_order_does_not_matter(oracle, seed):
    i = W.small_kernel(seed)
    a = oracle.check(i.src, i.groups, i.group_size, i.globals)
    b = oracle.check(i.src, i.groups, i.group_size, i.globals, reverse=True)
    np.testing.assert_array_equal(a["records"], b["records"])
    np.testing.assert_array_equal(a["final"], b["final"])


def test_thread_order_does_not_matter_large(oracle):
    i = W.large_kernel(0, groups=4, group_size=64, global_len=4096, local_len=256, n_stmts=80)
    a = oracle.check(i.src, i.groups, i.group_size, i.globals)
    b = oracle.check(i.src, i.groups, i.group_size, i.globals, reverse=True)
    assert a["n_access"] > 1000
    np.testing.assert_array_equal(a["records"], b["records"])
    np.testing.assert_array_equal(a["final"], b["final"])


# ---------------------------------------------------------------- brute force

def _first_flagged(records):
    races = [r for r in records if r[4] in (1, 3)]
    return min((int(r[0]) for r in races), default=None)


@pytest.mark.parametrize("chunk", range(8))
def test_bruteforce_schedules(oracle, chunk):
    """I1: no race record -> every schedule reaches one shared state at every
    barrier, reads never depend on the schedule, and the final memory is the
    oracle's.  I2: the first flagged interval holds a write/write race and
    no read/write race -> two schedules reach different shared states at its
    barrier.  I3: it holds a read/write race -> some schedule changes a read."""
    seen = {"free": 0, "ww": 0, "rw": 0}
    for seed in range(chunk * 60, chunk * 60 + 60):
        i = W.tiny_kernel(seed)
        r = oracle.check(i.src, i.groups, i.group_size, i.globals)
        e = oracle.explore(i.src, i.groups, i.group_size, i.globals)
        assert not e["overflow"], seed
        k = _first_flagged(r["records"])
        diverges = any(x[4] == 18 for x in r["records"])
        upto = r["n_intervals"] if k is None else k
        for j in range(upto):
            assert e["end_states"][j] == 1, (seed, j, i.src)
            assert not e["deviated"][j], (seed, j, i.src)
        if k is None:
            seen["free"] += 1
            assert e["diverged"] == diverges, (seed, i.src)
            if not diverges:
                assert len(e["finals"]) == 1, (seed, i.src)
                np.testing.assert_array_equal(e["finals"][0], r["final"])
            continue
        classes = {int(x[4]) for x in r["records"] if x[0] == k}
        if 3 in classes:
            seen["rw"] += 1
            assert e["deviated"][k], (seed, i.src)
        else:
            seen["ww"] += 1
            assert e["end_states"][k] >= 2, (seed, i.src)
    assert seen["free"] and seen["rw"], seen


# ---------------------------------------------------------------- interleaving product of two work-items
# The explorer's pair mode runs two work-items over every schedule while the
# others stay where the interval started (it is compared with the GPU's).

def test_pair_product_fig2(oracle):
    """Fig. 2, n = 4, pairs in order (0,1) (0,2) (0,3) (1,2) (1,3) (2,3).
    Interval 0: writes only, one end state per pair.  Interval 1: in a pair
    (k, k+1), k reads A[k+1] before or after k+1 writes it (a read that
    depends on the schedule); only for (2, 3) does that change memory, since
    work-item 3 reads A[4] = 1 and leaves g alone, while in (0, 1) and
    (1, 2) the second work-item reads its frozen neighbour's 0 and sets g = 1
    anyway.  Interval 2 starts from g = 0 or g = 1: no pair result."""
    g = golden.load("fig2_n4.txt")
    r = oracle.explore_pairs(g["src"], g["groups"], g["group_size"], g["globals"])
    assert r[0] == [(1, False)] * 6
    assert r[1] == [(1, True), (1, False), (1, False), (1, True), (1, False), (2, True)]
    assert r[2] is None


@pytest.mark.parametrize("S", [3, 4, 5])
def test_pair_product_neighbour_copy(oracle, S):
    """Each work-item copies its right neighbour's cell, which the neighbour
    overwrites in the same interval: exactly the pairs (t, t + 1) reach two
    memories and a schedule-dependent read; any other pair reads a cell of a
    work-item that does not run.  (Work-item S - 1 reads A[S], where work-item
    0 stores its copy; in the pair (0, S - 1) that copy is of a frozen cell,
    0, the value A[S] already holds.  With S = 2 the pair (0, 1) is both.)"""
    src = f"kernel k(global int A[]) {{ A[tid] = 0; barrier; A[tid] = 1; x = A[tid + 1]; A[tid + {S}] = x; }}"
    r = oracle.explore_pairs(src, 1, S, [np.zeros(2 * S, np.int32)])
    pairs = [(i, j) for i in range(S) for j in range(i + 1, S)]
    assert r[0] == [(1, False)] * len(pairs)
    assert r[1] == [(2, True) if j == i + 1 else (1, False) for i, j in pairs]


def test_bruteforce_pair_product_of_two_work_items(oracle):
    """With two work-items the only pair is the whole instance, so the pair
    mode must agree with the full interleaving search interval by interval
    (as long as the interval starts from one state)."""
    n = 0
    for seed in range(300):
        i = W.tiny_kernel(seed)
        if i.n_threads != 2:
            continue
        full = oracle.explore(i.src, i.groups, i.group_size, i.globals)
        pairs = oracle.explore_pairs(i.src, i.groups, i.group_size, i.globals)
        for k, p in enumerate(pairs):
            if p is None:
                break
            assert p == [(full["end_states"][k], full["deviated"][k])], (seed, k, i.src)
            n += 1
    assert n >= 50


# ---------------------------------------------------------------- work-group-scoped barriers
# Closed forms for the cross-group classification of the whole run and the
# per-group barrier-release rule (OpenCL barriers wait for their own group
# only), and two reductions to the kernel-wide checker.

XG = 2**32 - 1  # interval field of the cross-group records


def _grp(oracle, body, G, S, A, gb=True, decl="global int A[]"):
    src = f"kernel t({decl}) {{\n{body}\n}}\n"
    return oracle.check(src, G, S, [np.array(A, np.int32)], group_barriers=gb)


def _xg(r):
    return [list(map(int, x)) for x in r["records"] if x[0] == XG]


@pytest.mark.parametrize("G,S,m", [(2, 4, 4), (3, 8, 3), (4, 32, 5)])
@pytest.mark.parametrize("same", [False, True])
def test_group_scope_cross_group_writes(oracle, G, S, m, same):
    # every group writes cells 0..m-1 (work-items tid = c mod m): writers in
    # all G groups; values wg + 7 differ between groups, 7 does not
    r = _grp(oracle, f"A[tid % {m}] = {'7' if same else 'wg + 7'};", G, S, [0] * m)
    want = []
    for c in range(m):
        tids = [t for t in range(S) if t % m == c]
        nw = G * len(tids)
        want.append(rec(XG, c, 5 if same else 4, tids[0], (G - 1) * S + tids[-1], 0, nw, nw))
    assert _xg(r) == want
    assert r["status"] == (0 if same else 1)


@pytest.mark.parametrize("G,S,k", [(2, 4, 1), (3, 4, 5), (4, 8, 3), (2, 16, 16)])
def test_group_scope_neighbour_read_after_barrier(oracle, G, S, k):
    # A[gtid] = 1 | barrier | read A[(gtid + k) % N]: the barrier orders the
    # pair only inside a group; cell c (written by c, read by (c - k) mod N)
    # races across groups: value 0 before, 1 after the write
    N = G * S
    body = f"A[gtid] = 1;\nbarrier;\nx = A[(gtid + {k}) % {N}];"
    want = [rec(XG, c, 6, (c - k) % N, c, 1, 1, 2) for c in range(N) if ((c - k) % N) // S != c // S]
    r = _grp(oracle, body, G, S, [0] * N)
    assert _xg(r) == want and r["status"] == (1 if want else 0)
    r = _grp(oracle, body, G, S, [0] * N, gb=False)
    assert len(r["records"]) == 0 and r["status"] == 0


def test_group_scope_read_of_a_value_held_all_along(oracle):
    # group 0 writes 5, everyone reads after the barrier: a race unless the
    # cell held 5 before the run; witness: all readers r0 = 0, r1 = 7 and all
    # writers (0..3) -> (r1, w0) = (7, 0)
    body = "if (wg == 0) { A[0] = 5; }\nbarrier;\nx = A[0];"
    r = _grp(oracle, body, 2, 4, [0])
    assert _xg(r) == [rec(XG, 0, 6, 7, 0, 8, 4, 12)] and r["status"] == 1
    r = _grp(oracle, body, 2, 4, [5])
    assert _xg(r) == [] and r["status"] == 0
    # the same with the writer in group 1: (r0, w0) = (0, 4)
    r = _grp(oracle, body.replace("wg == 0", "wg == 1"), 2, 4, [0])
    assert _xg(r) == [rec(XG, 0, 6, 0, 4, 8, 4, 12)]
    # writers 0..3 and 4..7 both: (r0, w1) = (0, 7), and a cross-group WW
    r = _grp(oracle, "A[0] = wg;\nbarrier;\nif (wg == 0) { x = A[0]; }", 2, 4, [0])
    assert _xg(r) == [rec(XG, 0, 4, 0, 7, 4, 8, 12), rec(XG, 0, 6, 0, 7, 4, 8, 12)]
    # reader 0 alone, writers 1..7 (value 1, read back as 1, 0 before the
    # run): r0 = 0 and w0 = 1 are different work-items of one group, so the
    # witness is (r0, w1) = (0, 7); the writes agree: XG_WW_BENIGN (1, 7)
    r = _grp(oracle, "if (gtid != 0) { A[0] = 1; }\nbarrier;\nif (gtid == 0) { x = A[0]; }", 2, 4, [0])
    assert _xg(r) == [rec(XG, 0, 5, 1, 7, 1, 7, 8), rec(XG, 0, 6, 0, 7, 1, 7, 8)]


def test_group_scope_cross_round_writes(oracle):
    # group 0 writes in round 0, group 1 in round 1: no race with a kernel-wide
    # barrier, a cross-group race with a group-scoped one
    body = "if (wg == 0) { A[0] = 1; }\nbarrier;\nif (wg == 1) { A[0] = 2; }"
    r = _grp(oracle, body, 2, 4, [0], gb=False)
    assert r["status"] == 0 and all(x[4] == 2 for x in r["records"])
    r = _grp(oracle, body, 2, 4, [0])
    assert _xg(r) == [rec(XG, 0, 4, 0, 7, 0, 8, 8)] and r["status"] == 1
    np.testing.assert_array_equal(r["final"], [2])


def test_group_scope_barrier_agreement_per_group(oracle):
    # a barrier only group 0 takes: divergence kernel-wide, fine per group
    r = _grp(oracle, "if (wg == 0) { barrier; A[0] = 3; }", 2, 4, [0], gb=False)
    assert r["status"] == 4
    r = _grp(oracle, "if (wg == 0) { barrier; A[0] = 3; }", 2, 4, [0])
    assert r["status"] == 0 and r["n_intervals"] == 2
    np.testing.assert_array_equal(r["final"], [3])
    # groups at different barriers in one round
    r = _grp(oracle, "if (wg == 0) { barrier; } else { barrier; }\nA[gtid] = 1;", 2, 4, [0] * 8)
    assert r["status"] == 0 and r["n_intervals"] == 2 and len(r["records"]) == 0
    # divergence inside each group: one record per stop point, wg = the group
    r = _grp(oracle, "if (tid == 0) { barrier; }", 2, 4, [0])
    np.testing.assert_array_equal(r["records"], [rec(0, 0, 18, 0, 0, 0, 0, 1, wg=0),
                                                 rec(0, 0, 18, 1, XG, 0, 0, 3, wg=0),
                                                 rec(0, 0, 18, 4, 0, 0, 0, 1, wg=1),
                                                 rec(0, 0, 18, 5, XG, 0, 0, 3, wg=1)])
    assert r["status"] == 4 and r["n_intervals"] == 1
    # only group 1 diverges
    r = _grp(oracle, "if (wg == 1) { if (tid < 2) { barrier; } }", 2, 4, [0])
    np.testing.assert_array_equal(r["records"], [rec(0, 0, 18, 4, 0, 0, 0, 2, wg=1),
                                                 rec(0, 0, 18, 6, XG, 0, 0, 2, wg=1)])


@pytest.mark.parametrize("seed", range(12))
def test_group_scope_with_one_group_is_kernel_scope(oracle, seed):
    inst = W.tiny_kernel(seed) if seed % 2 else W.small_kernel(seed, group_size=16, n_stmts=12, n_barriers=2)
    a = oracle.check(inst.src, 1, inst.group_size, inst.globals)
    b = oracle.check(inst.src, 1, inst.group_size, inst.globals, group_barriers=True)
    for k in ("status", "n_intervals", "n_access"):
        assert a[k] == b[k]
    np.testing.assert_array_equal(a["records"], b["records"])
    np.testing.assert_array_equal(a["final"], b["final"])


@pytest.mark.parametrize("seed", range(6))
def test_group_scope_private_slabs_are_kernel_scope(oracle, seed):
    # each group touches only its own slab of A and takes the same barriers:
    # no cross-group pair, so the report is the kernel-wide one
    G, S = 3, 8
    rng = np.random.default_rng([12, seed])
    lines = []
    for _ in range(10):
        c = int(rng.integers(S))
        if rng.random() < 0.2:
            lines.append("barrier;")
        elif rng.random() < 0.5:
            lines.append(f"A[wg * {S} + (tid + {c}) % {S}] = tid + {int(rng.integers(3))};")
        else:
            lines.append(f"x = A[wg * {S} + (tid * 2 + {c}) % {S}];")
    src = "kernel t(global int A[]) {\n" + "\n".join(lines) + "\n}\n"
    A = rng.integers(0, 4, size=G * S).astype(np.int32)
    a = oracle.check(src, G, S, [A])
    b = oracle.check(src, G, S, [A], group_barriers=True)
    np.testing.assert_array_equal(a["records"], b["records"])
    np.testing.assert_array_equal(a["final"], b["final"])


@pytest.mark.parametrize("seed", range(8))
def test_group_scope_thread_order_does_not_matter(oracle, seed):
    inst = W.group_kernel(seed)
    a = oracle.check(inst.src, inst.groups, inst.group_size, inst.globals, group_barriers=True)
    b = oracle.check(inst.src, inst.groups, inst.group_size, inst.globals, reverse=True, group_barriers=True)
    np.testing.assert_array_equal(a["records"], b["records"])
    np.testing.assert_array_equal(a["final"], b["final"])


def test_group_scope_local_cells_stay_in_their_group(oracle):
    # every group writes its own L[0] with its own value: no cross-group record
    src = "kernel t(global int A[], local int L[1]) {\n L[0] = wg;\n barrier;\n A[gtid] = L[0];\n}\n"
    r = oracle.check(src, 3, 4, [np.zeros(12, np.int32)], group_barriers=True)
    assert _xg(r) == [] and r["status"] == 0
    np.testing.assert_array_equal(r["final"], np.repeat(np.arange(3), 4))


def test_group_scope_barriers_in_a_loop_of_one_group(oracle):
    # only group 0 loops over four barriers: five rounds, group 1 finished
    # after the first; each round's four writers store one value
    r = _grp(oracle, "if (wg == 0) { for i in 0 .. 4 { A[i] = wg; barrier; } }", 2, 4, [9] * 4)
    assert r["status"] == 0 and r["n_intervals"] == 5
    np.testing.assert_array_equal(r["records"], [rec(k, k, 2, 0, 1, 0, 4, 4) for k in range(4)])
    np.testing.assert_array_equal(r["final"], [0, 0, 0, 0])


def test_group_scope_read_rounds_before_the_write(oracle):
    # group 1 reads in round 0, group 0 writes in round 2: ordered by the
    # kernel-wide barriers, unordered by group-scoped ones; witness (r0, w0) = (4, 0)
    body = "if (wg == 1) { x = A[0]; }\nbarrier;\nbarrier;\nif (wg == 0) { A[0] = 3; }"
    r = _grp(oracle, body, 2, 4, [0], gb=False)
    assert r["status"] == 0
    r = _grp(oracle, body, 2, 4, [0])
    assert r["status"] == 1 and _xg(r) == [rec(XG, 0, 6, 4, 0, 4, 4, 8)]


@pytest.mark.parametrize("gb", [False, True])
def test_address_sharded_runs_merge_to_the_full_report(oracle, gb):
    """P address shards (each logging and classifying its cells, committing
    all) merge to the unsharded report, record for record."""
    insts = [W.tiny_kernel(s) for s in range(12)] + [W.small_kernel(s, group_size=32, groups=2) for s in range(4)]
    insts += [W.large_kernel(1, groups=4, group_size=32, global_len=4096, local_len=64, n_stmts=40,
                             n_barriers=3), W.group_kernel(2)]
    for inst in insts:
        want = oracle.check(inst.src, inst.groups, inst.group_size, inst.globals, group_barriers=gb)
        for P in (2, 3):
            got = oracle.check_sharded(inst.src, inst.groups, inst.group_size, inst.globals, P, group_barriers=gb)
            assert got["status"] == want["status"], inst.name
            np.testing.assert_array_equal(got["records"], want["records"], err_msg=inst.name)
            np.testing.assert_array_equal(got["final"], want["final"], err_msg=inst.name)


def test_address_sharded_runs_in_processes(oracle):
    inst = W.large_kernel(2, groups=4, group_size=32, global_len=4096, local_len=64, n_stmts=40, n_barriers=3)
    want = oracle.check(inst.src, inst.groups, inst.group_size, inst.globals)
    got = oracle.check_sharded(inst.src, inst.groups, inst.group_size, inst.globals, 4, processes=2)
    np.testing.assert_array_equal(got["records"], want["records"])
    np.testing.assert_array_equal(got["final"], want["final"])
