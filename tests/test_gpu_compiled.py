"""Compiled intervals on the GPU: every instance checked with the interval
kernel compiled from its own program (rc_set_engine(2)) against the oracle,
bit for bit, under each classification strategy (sort, shadow owner table,
resident run).  The instances cover what the compiled engine does
differently from the interpreter: lanes of a warp diverging and appending
to the log at different times (branches on tid and on loaded values,
loops), out-of-bounds accesses and failed asserts inside compiled code,
barriers reached from different code paths, programs whose accesses the
pre-filter proves private (no log append compiled in)."""
import numpy as np
import pytest

from paper_1308_3203_gb300 import workloads as W
from tests.golden import golden
from tests.test_gpu_parity import EDGE, run_both, same

STRATEGIES = (1, 2, 3)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1308_3203_gb300 import build as gpu_build
    gpu_build.build()
    from paper_1308_3203_gb300 import racecheck
    racecheck.load()
    racecheck.set_engine("compiled")
    yield racecheck
    racecheck.set_engine("auto")
    racecheck.set_strategy(0)


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


def test_small_and_tiny_kernels(rc, oracle):
    for seed in range(8):
        run_both(rc, oracle, W.small_kernel(seed), STRATEGIES)
    for seed in range(8):
        run_both(rc, oracle, W.tiny_kernel(seed), STRATEGIES)


@pytest.mark.parametrize("shape", [(8, 256), (3, 100), (5, 1), (33, 32)])
def test_large_kernels_reduced(rc, oracle, shape):
    G, S = shape
    inst = W.large_kernel(shape[0], groups=G, group_size=S, global_len=max(16 * G * S, 4096), local_len=16 * S)
    run_both(rc, oracle, inst, STRATEGIES)


@pytest.mark.parametrize("seed", range(2))
def test_stress_kernels_reduced(rc, oracle, seed):
    """Nested loops and branches on loaded values: lanes diverge inside the
    compiled code."""
    run_both(rc, oracle, W.stress_kernel(seed, groups=16, group_size=1024), STRATEGIES)


def test_every_opcode_on_its_boundaries(rc, oracle):
    from tests.test_translate_cpu import opcode_kernel
    for S in (8, 64):
        run_both(rc, oracle, opcode_kernel(S), STRATEGIES)


@pytest.mark.parametrize("case", range(len(EDGE)))
def test_edge_cases(rc, oracle, case):
    src, G, S, glob = EDGE[case]
    run_both(rc, oracle, W.Instance(f"edge{case}", src, G, S, glob), STRATEGIES)


def test_large_kernel_full_size(rc, oracle):
    """The 1024 x 256 large instance, resident and interval by interval."""
    inst = W.large_kernel(0)
    want = run_both(rc, oracle, inst, STRATEGIES)
    assert want["n_access"] > 10_000_000


def test_engines_agree_and_compiles_are_cached(rc, oracle):
    """The same instance under the interpreter and compiled intervals gives
    the same report; a second check of the same program and shape compiles
    nothing."""
    inst = W.stress_kernel(2, groups=8, group_size=512)
    bc = rc.compile(inst.src)
    want = oracle.check(inst.src, inst.groups, inst.group_size, inst.globals)
    rc.set_strategy(2)
    same(rc.check(bc, inst.groups, inst.group_size, inst.globals), want)
    n0 = rc.jit_stats()["compiles"]
    same(rc.check(bc, inst.groups, inst.group_size, inst.globals), want)
    assert rc.jit_stats()["compiles"] == n0
    rc.set_engine("interpreter")
    same(rc.check(bc, inst.groups, inst.group_size, inst.globals), want)
    rc.set_engine("compiled")
    rc.set_strategy(0)
