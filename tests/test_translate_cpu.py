"""The kernel text rc_translate writes, run on the CPU against the oracle.

rc_translate turns a compiled kernel into a C++ function that runs one
work-item through one barrier interval (Sec. 4's thread-local rules).  Here
the functions of many generated kernels are compiled together with a host
harness (tests/jit/harness.cpp) and each work-item of each interval runs on
its own, its loads answered with the values the oracle's run read.  What
the work-item then does must be what the oracle's work-item did: the same
loads and stores in the same order (command, array, index, stored value),
the same out-of-bounds access or failed assert, and the same stop (the
barrier all live work-items wait at, or the exit).
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_1308_3203_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1308_3203_gb300", "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
TS_BARRIER, TS_EXIT, TS_DEAD = 1, 2, 3


@pytest.fixture(scope="module")
def rc():
    from paper_1308_3203_gb300 import build as gpu_build
    gpu_build.build()
    from paper_1308_3203_gb300 import racecheck
    racecheck.load()
    return racecheck


# every expression and branch form the compiler emits (register and
# immediate comparisons, the six branch senses, not, and, or, negation,
# division and remainder by negative numbers and zero, multiply-add, masks),
# on values that sit on each comparison's boundary for some work-item
OPCODE_EXPRS = ["x + 7", "x - tid", "x * -5", "x / 2", "x % 3", "10 / (x + 1)", "10 % (x - 1)", "7 - x", "-x",
                "!x", "x < 1", "x <= 1", "x > 1", "x >= 1", "x == 1", "x != 1", "x < tid", "x <= tid - 3",
                "x > tid - 4", "x >= tid", "x == tid - 3", "x != tid - 3", "(x > 0) && (tid < 5)",
                "(x > 0) || (tid == 0)", "x * 3 + tid", "(x + 8) % 8", "(x + 8) % 4 + 1", "x / -2", "x % -3",
                "-2147483647 - 1 - x", "size(A) - x", "!(x < 2)"]
OPCODE_BRANCHES = ["x >= 1", "x > 1", "x <= 1", "x < 1", "x == 1", "x != 1", "!x", "x", "(x > 0) && (tid < 5)",
                   "(x > 0) || (tid == 0)", "x >= tid", "x < tid - 2"]


def opcode_kernel(group_size=8):
    """x = tid - 3 runs over -3 .. group_size - 4; each work-item stores every
    expression and the sense of every branch into its own 64 cells."""
    body = ["  x = tid - 3;"]
    body += [f"  A[gtid * 64 + {i}] = {e};" for i, e in enumerate(OPCODE_EXPRS)]
    k0 = len(OPCODE_EXPRS)
    body += [f"  if ({b}) {{ A[gtid * 64 + {k0 + j}] = {j + 1}; }} else {{ A[gtid * 64 + {k0 + j}] = -{j + 1}; }}"
             for j, b in enumerate(OPCODE_BRANCHES)]
    src = "kernel ops(global int A[]) {\n" + "\n".join(body) + "\n}\n"
    return W.Instance("opcodes", src, 1, group_size, [np.zeros(64 * group_size, np.int32)])


def instances():
    out = [opcode_kernel()]
    out += [W.tiny_kernel(s) for s in range(120)]
    out += [W.small_kernel(s, group_size=8, n_stmts=16) for s in range(60)]
    out += [W.small_kernel(s, group_size=4, groups=2, n_stmts=24, n_barriers=2, L=8) for s in range(30)]
    # the batch workload's long programs (hundreds of statements, up to 8 barriers) at a small shape
    out += [W.small_kernel(500 + s, group_size=8, groups=2, n_stmts=300 + 10 * s, n_barriers=s % 9, L=64)
            for s in range(20)]
    out += [W.large_kernel(s, groups=2, group_size=8, global_len=256, local_len=32, n_stmts=40, n_barriers=3)
            for s in range(10)]
    out += [W.stress_kernel(s, groups=2, group_size=8) for s in range(6)]
    for s in range(6):
        pk = W.proposal_kernel(s)
        out.append(pk.instance(2, 8, 0))
    out.append(W.Instance("edges", "kernel e(global int A[], local int L[4]) {\n"
                          " x = 2147483647; A[tid] = x + tid; A[tid + 4] = -2147483648 / -1;\n"
                          " A[tid + 8] = -7 % 3; A[tid + 12] = 7 / 0; A[tid + 16] = size(A);\n"
                          " assume(tid != 1);\n L[tid] = tid; barrier; A[tid + 20] = L[(tid + 1) % 4];\n"
                          " assert(tid != 2);\n}", 1, 4, [np.zeros(24, np.int32)]))
    return out


@pytest.fixture(scope="module")
def harness(rc, tmp_path_factory):
    insts = instances()
    d = tmp_path_factory.mktemp("jit")
    text, regs = [], []
    for k, inst in enumerate(insts):
        bc = rc.compile(inst.src)
        n_regs = bc.info()["n_regs"]
        text.append(rc.translate(bc, f"k{k}"))
        text.append(f"RC_HARNESS_WRAPPER(k{k}, {n_regs})\n")
        regs.append(n_regs)
    gen = d / "kernels.inc"
    gen.write_text("\n".join(text))
    lib = d / "libjit.so"
    subprocess.run(["g++", "-O0", "-std=c++17", "-shared", "-fPIC", f"-I{CSRC}", f"-I{INCLUDE}",
                    f"-DRC_JIT_TEXT=\"{gen}\"", "-o", str(lib), os.path.join(HERE, "jit", "harness.cpp")],
                   check=True, capture_output=True)
    return insts, regs, ctypes.CDLL(str(lib))


def _run_instance(rc, oracle, lib, k, inst, n_regs):
    r = oracle.check(inst.src, inst.groups, inst.group_size, inst.globals, trace=True)
    bc = rc.compile(inst.src)
    sites = rc.access_sites(bc)
    np.testing.assert_array_equal(sites[:, 1:], r["sites"], err_msg=inst.name)
    # memory objects in declared order: lengths, and flat bases inside their space
    lens, spaces = _mem_layout(inst)
    bases, tot = [], [0, 0]
    for ln, sp in zip(lens, spaces):
        bases.append(tot[sp])
        tot[sp] += ln
    mem_len = np.array(lens, dtype=np.int64)
    t = r["trace"]
    recs = r["records"]
    G, S = inst.groups, inst.group_size
    N = G * S
    fn = getattr(lib, f"k{k}_run")
    regs = np.zeros((N, n_regs), np.int32)
    for g in range(N):
        regs[g, :5] = (g % S, g // S, g, S, G)
    pc = np.zeros(N, np.uint32)
    st = np.zeros(N, np.uint32)
    ev = np.zeros(5 * 65536, np.uint32)
    errs = []
    order = np.lexsort((np.arange(len(t)), t[:, 1], t[:, 0])) if len(t) else np.zeros(0, np.int64)
    t = t[order]
    keys = t[:, 0].astype(np.int64) * N + t[:, 1] if len(t) else np.zeros(0, np.int64)
    for iv in range(r["n_intervals"]):
        stops = {}
        for g in range(N):
            if st[g] in (TS_EXIT, TS_DEAD):
                continue
            lo, hi = np.searchsorted(keys, iv * N + g), np.searchsorted(keys, iv * N + g + 1)
            rows = t[lo:hi]
            loads = np.ascontiguousarray(rows[rows[:, 5] == 0][:, 7].astype(np.uint32).view(np.int32))
            row_regs = np.ascontiguousarray(regs[g])
            c_pc, c_st = ctypes.c_uint32(int(pc[g])), ctypes.c_uint32(int(st[g]))
            n_ev, bar = ctypes.c_uint32(), ctypes.c_int32()
            rc_ = fn(row_regs.ctypes.data_as(ctypes.c_void_p), ctypes.byref(c_pc), ctypes.byref(c_st),
                     loads.ctypes.data_as(ctypes.c_void_p), len(loads), mem_len.ctypes.data_as(ctypes.c_void_p),
                     ev.ctypes.data_as(ctypes.c_void_p), 65536, ctypes.byref(n_ev), ctypes.byref(bar))
            assert rc_ == 0, (inst.name, iv, g, "loads left over")
            regs[g] = row_regs
            pc[g], st[g] = c_pc.value, c_st.value
            e = ev[:5 * n_ev.value].reshape(-1, 5)
            acc = e[e[:, 0] <= 1]
            # the same accesses in the same order: load/store, command, index, value
            base = np.array([bases[int(m)] for m in sites[rows[:, 6], 2]], np.uint32)
            want = np.stack([rows[:, 5], rows[:, 6], rows[:, 4] - base.reshape(-1), rows[:, 7]], axis=1)
            got = acc[:, [0, 1, 3, 4]]
            np.testing.assert_array_equal(got, want, err_msg=f"{inst.name} interval {iv} work-item {g}")
            for x in e[e[:, 0] >= 2]:
                if x[0] == 2:  # out of bounds: (interval, kind, work-item) -> index, array
                    errs.append((iv, 16, g, int(x[3]), int(x[2])))
                else:
                    errs.append((iv, 17, g, 0, int(x[3])))
            if st[g] == TS_BARRIER:
                stops.setdefault(bar.value, []).append(g)
            elif st[g] == TS_EXIT:
                stops.setdefault(0xFFFFFFFF, []).append(g)
        div = [x for x in recs if x[4] == 18 and x[0] == iv]
        if div:  # the oracle stopped here: the stop points and who stopped there
            assert sorted((int(x[6]), int(x[5]), int(x[9])) for x in div) == \
                sorted((b, min(v), len(v)) for b, v in stops.items()), inst.name
        elif iv + 1 < r["n_intervals"]:
            assert len(stops) == 1 and 0xFFFFFFFF not in stops, (inst.name, iv, stops.keys())
        else:
            assert set(stops) <= {0xFFFFFFFF}, (inst.name, iv, stops.keys())
    want_errs = sorted((int(x[0]), int(x[4]), int(x[5]), int(x[3]) if x[4] == 16 else 0, int(x[6]))
                       for x in recs if x[4] in (16, 17))
    assert sorted(errs) == want_errs, inst.name


def _mem_layout(inst):
    """lengths and spaces of the memory objects in declared order, from the
    kernel's declaration list"""
    head = inst.src[inst.src.index("(") + 1:inst.src.index(")")]
    lens, spaces, gi = [], [], 0
    for decl in [x.strip() for x in head.split(",") if x.strip()]:
        if decl.startswith("local"):
            lens.append(int(decl[decl.index("[") + 1:decl.index("]")]))
            spaces.append(1)
        else:
            lens.append(int(np.asarray(inst.globals[gi]).size))
            spaces.append(0)
            gi += 1
    return lens, spaces


def test_translated_kernels_follow_the_oracle(rc, oracle, harness):
    insts, regs, lib = harness
    for k, inst in enumerate(insts):
        _run_instance(rc, oracle, lib, k, inst, regs[k])


def test_translate_rejects_bad_names(rc):
    bc = rc.compile("kernel e() { }")
    for bad in ("", "1x", "a-b", "a b", "x" * 129):
        with pytest.raises(Exception):
            rc.translate(bc, bad)
    assert "RC_JIT_FN void ok_name(" in rc.translate(bc, "ok_name")


DEVICE_SHIM = r'''
#include <cstdint>
#include "semantics.cuh"
struct Ctx { const int32_t *snap; const uint32_t *len; int32_t *log; uint32_t *n; };
__device__ __forceinline__ bool hk_ld(Ctx &cx, uint32_t, uint32_t mem, int32_t idx, int32_t &out) {
  if ((uint32_t)idx >= cx.len[mem]) return false;
  out = cx.snap[idx];
  return true;
}
__device__ __forceinline__ bool hk_st(Ctx &cx, uint32_t, uint32_t mem, int32_t idx, int32_t v) {
  if ((uint32_t)idx >= cx.len[mem]) return false;
  cx.log[atomicAdd(cx.n, 1u)] = v;
  return true;
}
#define RC_JIT_FN __device__ __forceinline__
#define RC_JIT_CTX Ctx
#define RC_LD(cx, s, m, i, o) hk_ld(cx, s, m, i, o)
#define RC_ST(cx, s, m, i, v) hk_st(cx, s, m, i, v)
#define RC_SIZE(cx, m) ((int32_t)(cx).len[m])
#define RC_ASSERT_FAIL(cx, id) ((void)0)
#define RC_AT_BARRIER(cx, id) ((void)0)
#include "gen.inc"
__global__ void probe(Ctx cx, uint32_t *out) {
  int32_t r[NREGS] = {};
  r[0] = threadIdx.x; r[1] = blockIdx.x; r[2] = blockIdx.x * blockDim.x + threadIdx.x;
  r[3] = blockDim.x; r[4] = gridDim.x;
  uint32_t pc = 0, st = 0;
  for (int iv = 0; iv < 64 && st != 2 && st != 3; iv++) {
    run_item(cx, r, pc, st);
    __syncthreads();
  }
  out[r[2]] = st;
}
'''


def test_translated_bench_kernel_compiles_for_sm103a_without_a_stack_frame(rc, tmp_path):
    """The bench kernel's function compiled as CUDA C++ for sm_103a (no GPU
    needed): its register array is indexed by constants only, so ptxas keeps
    it in machine registers -- no stack frame, no spills."""
    from paper_1308_3203_gb300 import build as B
    inst = W.large_kernel(0)
    bc = rc.compile(inst.src)
    (tmp_path / "gen.inc").write_text(rc.translate(bc, "run_item"))
    (tmp_path / "probe.cu").write_text(DEVICE_SHIM)
    p = subprocess.run([B._nvcc()] + B.ARCH + ["-O3", "-std=c++17", f"-I{CSRC}", f"-I{INCLUDE}",
                                                f"-DNREGS={bc.info()['n_regs']}", "-Xptxas", "-v", "-c",
                                                str(tmp_path / "probe.cu"), "-o", str(tmp_path / "probe.o")],
                       capture_output=True, text=True, cwd=str(tmp_path))
    assert p.returncode == 0, p.stderr[-2000:]
    assert "0 bytes stack frame, 0 bytes spill stores, 0 bytes spill loads" in p.stderr, p.stderr[-2000:]
