"""The seeded input generators: same seed, same instance; the shapes and
value ranges the documented workloads promise; every kernel compiles."""
import numpy as np
import pytest

from paper_1308_3203_gb300 import workloads as W


@pytest.fixture(scope="module")
def rc():
    from paper_1308_3203_gb300 import build as gpu_build
    gpu_build.build()
    from paper_1308_3203_gb300 import racecheck
    racecheck.load()
    return racecheck


GENS = {
    "tiny": lambda s: W.tiny_kernel(s),
    "small": lambda s: W.small_kernel(s),
    "large": lambda s: W.large_kernel(s, groups=4, group_size=64, global_len=4096, local_len=256),
    "stress": lambda s: W.stress_kernel(s, groups=4, group_size=64),
    "group": lambda s: W.group_kernel(s),
    "proposal": lambda s: W.proposal_kernel(s).instance(*W.proposal_candidates(s)[0]),
    "batch_proposal": lambda s: W.batch_proposal_kernel(s, max_stmts=64).instance(*W.proposal_candidates(s)[0]),
}


@pytest.mark.parametrize("name", sorted(GENS))
def test_same_seed_same_instance(name):
    a, b, c = GENS[name](3), GENS[name](3), GENS[name](4)
    assert a.src == b.src and (a.groups, a.group_size) == (b.groups, b.group_size)
    for x, y in zip(a.globals, b.globals):
        np.testing.assert_array_equal(x, y)
    assert a.src != c.src


@pytest.mark.parametrize("name", sorted(GENS))
def test_every_kernel_compiles(rc, name):
    for s in range(10):
        inst = GENS[name](s)
        info = rc.compile(inst.src).info()
        assert info["n_global"] == len(inst.globals)
        assert all(g.dtype == np.int32 for g in inst.globals)


def test_documented_shapes_and_ranges():
    s = W.small_kernel(0)
    assert (s.groups, s.group_size) == (1, 64) and s.globals[0].size == 256
    assert s.globals[0].min() >= 0 and s.globals[0].max() < 16
    big = W.large_kernel(0)
    assert (big.groups, big.group_size) == (1024, 256) and big.globals[0].size == 4 << 20
    assert big.globals[0].min() >= 0 and big.globals[0].max() < 1024
    assert big.src.count("barrier;") == 8
    t = W.tiny_kernel(0)
    assert 2 <= t.n_threads <= 4 and t.globals[0].max() < 4
    params = W._batch_params(0, 200)
    for (_, _, S, G, n_stmts, n_bar, L) in params:
        assert 32 <= S <= 1024 and 1 <= G <= 64 and 16 <= n_stmts <= 512 and 0 <= n_bar <= 8
        assert 1024 <= L <= 1 << 20
    for (G, S, _) in W.proposal_candidates(0):
        assert 1 <= G <= 64 and S % 32 == 0 and 32 <= S <= 1024
    # config-3 programs as proposal kernels: the program does not depend on
    # the candidate, the input does (A of the kernel's length, values [0, 16))
    bp = W.batch_proposal_kernel(5)
    a, b = bp.instance(2, 64, 1), bp.instance(8, 1024, 2)
    assert a.src == b.src and a.globals[0].size == b.globals[0].size == bp.L
    assert 1024 <= bp.L <= 1 << 20 and 0 <= a.globals[0].min() and a.globals[0].max() < 16
    assert not np.array_equal(a.globals[0], b.globals[0])
