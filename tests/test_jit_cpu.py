"""Compiled intervals without a GPU: the interval kernel generated for an
instance (translated program, engine headers, private-site table) compiles
for sm_103a with NVRTC, for both launch modes, on programs of every
workload family and on the kernel that holds every expression and branch
form."""
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


def instances():
    from tests.test_translate_cpu import opcode_kernel
    return [W.small_kernel(0), W.tiny_kernel(3), opcode_kernel(8),
            W.large_kernel(1, groups=4, group_size=64, global_len=4096, local_len=256),
            W.stress_kernel(1, groups=4, group_size=64),
            W.Instance("empty", "kernel e() { }", 2, 3, []),
            W.Instance("oob", "kernel e(global int A[]) { A[tid + 1] = tid; assert(tid != 2); }", 1, 8,
                       [np.zeros(4, np.int32)])]


@pytest.mark.parametrize("k", range(7))
def test_interval_kernel_compiles(rc, k):
    inst = instances()[k]
    bc = rc.compile(inst.src)
    for resident in (False, True):
        r = rc.jit_compile(bc, inst.groups, inst.group_size, inst.globals, resident=resident)
        assert r["cubin_bytes"] > 0
    # cached: the same source is not compiled twice
    n = rc.jit_stats()["compiles"]
    rc.jit_compile(bc, inst.groups, inst.group_size, inst.globals)
    assert rc.jit_stats()["compiles"] == n


def test_engine_values(rc):
    for e in ("auto", "interpreter", "compiled", 0, 1, 2):
        rc.set_engine(e)
    with pytest.raises(Exception):
        rc.set_engine(3)
    rc.set_engine("auto")
