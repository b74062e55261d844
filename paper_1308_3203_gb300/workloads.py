"""Seeded synthetic kernel instances.

This module only produces program text and input arrays; it evaluates no
program and holds none of the race checker's arithmetic, so the GPU path and
the CPU oracle can both be fed from it.

Kernel shapes follow the workloads the checker is built for:

* ``small_kernel``  one work-group of 64, one barrier, 32 random statements
  over ``global int A[256]`` at ``(a*tid+b) % 256`` with a in {0,1,2}, values
  affine in tid or constant, ``if (tid < k)`` branches, input in [0,16).
* ``large_kernel``  1024 groups x 256, 8 barriers, 200 statements with
  constant-trip loops (1..16), a global array of 4M ints and a local array of
  4096 ints per group, indices affine in gtid/tid modulo the slab they stay
  in; about 5% of stores are planted to collide with differing values and 5%
  with equal values.
* ``batch_kernels`` many config-1-style kernels of uneven shape (group size
  log-uniform 32..1024, 1..64 groups, 16..512 statements, 0..8 barriers,
  arrays 1K..1M).
* ``stress_kernel`` 65,536 groups x 1024 (2^26 work-items), 16 barriers, 512
  statements, nested loops up to 32 trips, branches on loaded values, a 64M
  global array; every interval that writes ends with a benign cell, a racy
  cell and reads of the racy cell in each group.
* ``tiny_kernel``   2-4 work-items with a handful of accesses and values in
  [0,4), small enough to enumerate every schedule.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Instance:
    name: str
    src: str
    groups: int
    group_size: int
    globals: list  # one int32 numpy array per `global` declaration

    @property
    def n_threads(self) -> int:
        return self.groups * self.group_size


# ----------------------------------------------------------------------------
# small / batch kernels: index (a*tid + b) % L


class _AffineGen:
    """Random statements over one global array, config-1 style."""

    def __init__(self, rng, L, n_vars=6, S=64):
        self.rng = rng
        self.L = L
        self.n_vars = n_vars
        self.S = S
        self.assigned = {0}

    def var(self):
        return f"v{int(self.rng.integers(self.n_vars))}"

    def used_var(self):
        return f"v{int(self.rng.choice(sorted(self.assigned)))}"

    def index(self):
        a = int(self.rng.integers(3))
        b = int(self.rng.integers(self.L))
        if a == 0:
            return f"{b}"
        return f"({a} * tid + {b}) % {self.L}"

    def value(self):
        r = self.rng.random()
        if r < 0.4:
            c = int(self.rng.integers(-3, 4))
            d = int(self.rng.integers(0, 16))
            return f"{c} * tid + {d}"
        if r < 0.7:
            return f"{int(self.rng.integers(0, 16))}"
        return self.used_var()

    def stmt(self, depth):
        r = self.rng.random()
        if r < 0.22:
            v = self.var()
            self.assigned.add(int(v[1:]))
            k = self.rng.random()
            if k < 0.4:
                rhs = f"{int(self.rng.integers(-3, 4))} * tid + {int(self.rng.integers(16))}"
            elif k < 0.7:
                rhs = f"{self.used_var()} + {int(self.rng.integers(-4, 5))}"
            else:
                rhs = f"{self.used_var()} * {int(self.rng.integers(-2, 3))} - {self.used_var()}"
            return [f"{v} = {rhs};"], 1
        if r < 0.52:
            v = self.var()
            self.assigned.add(int(v[1:]))
            return [f"{v} = A[{self.index()}];"], 1
        if r < 0.85 or depth > 0:
            return [f"A[{self.index()}] = {self.value()};"], 1
        k = int(self.rng.integers(1, self.S + 1))
        body, n = [], 0
        for _ in range(int(self.rng.integers(1, 4))):
            lines, c = self.stmt(depth + 1)
            body += ["  " + x for x in lines]
            n += c
        out = [f"if (tid < {k}) {{"] + body + ["}"]
        return out, n + 1


def small_kernel(seed: int, group_size: int = 64, groups: int = 1, n_stmts: int = 32,
                 n_barriers: int = 1, L: int = 256) -> Instance:
    """One config-1 kernel: 1 x 64 work-items, 1 barrier, 32 statements."""
    rng = np.random.default_rng([1, seed])
    g = _AffineGen(rng, L, S=group_size)
    lines, count = [], 0
    while count < n_stmts:
        ls, c = g.stmt(0)
        lines += ls
        count += c
    # barriers at distinct top-level positions
    tops = [i for i, x in enumerate(lines) if not x.startswith(" ") and not x.startswith("}")]
    pos = sorted(rng.choice(len(tops), size=min(n_barriers, len(tops)), replace=False).tolist())
    for p in reversed(pos):
        lines.insert(tops[p], "barrier;")
    src = "kernel small(global int A[]) {\n" + "\n".join("  " + x for x in lines) + "\n}\n"
    A = rng.integers(0, 16, size=L, dtype=np.int32)
    return Instance(f"small-s{seed}", src, groups, group_size, [A])


def _batch_params(seed: int, n_kernels: int) -> list:
    rng = np.random.default_rng([3, seed])
    out = []
    for k in range(n_kernels):
        S = int(round(math.exp(rng.uniform(math.log(32), math.log(1024)))))
        S = max(32, min(1024, S))
        G = int(rng.integers(1, 65))
        n_stmts = int(rng.integers(16, 513))
        n_bar = int(rng.integers(0, 9))
        L = int(round(math.exp(rng.uniform(math.log(1024), math.log(1 << 20)))))
        out.append((f"batch-s{seed}-k{k}", int(rng.integers(1 << 31)), S, G, n_stmts, n_bar, L))
    return out


def _batch_one(p):
    name, kseed, S, G, n_stmts, n_bar, L = p
    inst = small_kernel(kseed, group_size=S, groups=G, n_stmts=n_stmts, n_barriers=n_bar, L=L)
    inst.name = name
    return inst


def batch_kernels(seed: int, n_kernels: int, processes: int = 0) -> list:
    """Config-3 batch: uneven shapes, config-1 statement/index distributions.

    processes > 1 builds the kernels in a spawn-started process pool (the
    parameters are drawn first, so the result does not depend on it)."""
    params = _batch_params(seed, n_kernels)
    if processes > 1 and n_kernels > 64:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            return pool.map(_batch_one, params, chunksize=64)
    return [_batch_one(p) for p in params]


# ----------------------------------------------------------------------------
# large / stress kernels: slab-structured indices


class _SlabGen:
    """Statements for large instances.

    The global array is viewed as ``n_slab`` slabs of N cells (N = work-items)
    and each local array as slabs of S cells.  In every barrier interval one
    slab takes planted stores only, a quarter are "write" slabs, where each
    work-item writes and re-reads only its own cell, and the rest are
    read-only, where work-items read neighbours.  Planted stores collide on
    purpose: a few work-items per group write one cell of the plant slab,
    with differing values (a race) or one value (benign).  With a single slab
    (N cells in all) intervals alternate between a write phase (own cells
    only, plants collide with own-cell writes) and a read phase (neighbour
    reads, no stores).
    """

    def __init__(self, rng, N, S, L, LL, n_vars, max_trip, plant_frac, loads_on_branch,
                 max_depth, mix="dense"):
        self.rng, self.N, self.S, self.L, self.LL = rng, N, S, L, LL
        self.mix = mix
        self.n_slab = max(1, L // N)
        self.n_lslab = max(1, LL // S) if LL else 0
        self.n_vars = n_vars
        self.max_trip = max_trip
        self.plant = plant_frac
        self.loads_on_branch = loads_on_branch
        self.max_depth = max_depth
        self.loopvars = []
        self.phase = 0
        self.new_interval()

    @staticmethod
    def _roles(rng, n):
        if n >= 3:
            perm = rng.permutation(n).tolist()
            k = max(1, n // 4)
            return [perm[0]], sorted(perm[1:1 + k]), sorted(perm[1 + k:])
        return None

    def new_interval(self):
        r = self.rng
        self.phase += 1
        roles = self._roles(r, self.n_slab)
        if roles:
            self.pslabs, self.wslabs, self.rslabs = roles
        elif self.phase % 2:  # single slab, write phase
            self.pslabs, self.wslabs, self.rslabs = [0], [0], []
        else:                 # single slab, read phase
            self.pslabs, self.wslabs, self.rslabs = [0], [], [0]
        if self.n_lslab:
            self.lp, self.lw, self.lr = self._roles(r, self.n_lslab) or ([0], [0], [])

    def var(self):
        return f"x{int(self.rng.integers(self.n_vars))}"

    def term(self):
        r = self.rng.random()
        if r < 0.3:
            return self.var()
        if r < 0.5 and self.loopvars:
            return self.loopvars[int(self.rng.integers(len(self.loopvars)))]
        if r < 0.7:
            return "tid"
        return str(int(self.rng.integers(0, 32)))

    def value(self):
        r = self.rng.random()
        if r < 0.5:
            return f"{self.var()} + {self.term()}"
        if r < 0.8:
            return f"{self.var()} * {int(self.rng.integers(1, 4))} + {self.term()}"
        return f"{self.term()} - {self.var()}"

    def shift(self):
        if self.loopvars and self.rng.random() < 0.5:
            return f"{self.loopvars[-1]} + {int(self.rng.integers(0, 8))}"
        return str(int(self.rng.integers(0, 64)))

    @staticmethod
    def _plus(base, e):
        return f"{base} + {e}" if base else e

    def gaddr_read(self):
        if not self.rslabs:
            return self.gaddr_own(any_slab=True)
        s = int(self.rng.choice(self.rslabs))
        return self._plus(s * self.N, f"(gtid + {self.shift()}) % {self.N}")

    def gaddr_own(self, any_slab=False):
        slabs = self.wslabs or (self.rslabs if any_slab else [])
        s = int(self.rng.choice(slabs))
        return self._plus(s * self.N, "gtid")

    def laddr_read(self):
        if not self.lr:
            return self.laddr_own()
        s = int(self.rng.choice(self.lr)) * self.S
        return self._plus(s, f"(tid + {self.shift()}) % {self.S}")

    def laddr_own(self):
        s = int(self.rng.choice(self.lw)) * self.S
        return self._plus(s, "tid")

    def planted(self):
        """Stores that collide on purpose (one cell per group)."""
        r = self.rng
        benign = r.random() < 0.5
        use_local = self.n_lslab and r.random() < 0.3
        step = min(int(r.choice([8, 16, 32, 64])), self.S)
        off = int(r.integers(self.S))
        if use_local:
            tgt = f"Lc[{self._plus(int(self.lp[0]) * self.S, str(off))}]"
        else:
            s = int(self.pslabs[0])
            tgt = f"A[{self._plus(s * self.N, f'wg * {self.S} + {off}')}]"
        val = f"wg * 3 + {int(r.integers(8))}" if benign else f"tid + {int(r.integers(8))}"
        return [f"if (tid % {step} == 0) {{", f"  {tgt} = {val};", "}"], 2

    def can_plant(self):
        return self.S >= 2 and bool(self.wslabs or self.n_slab >= 3)

    def closing_plants(self):
        """Three statements that end a write interval, so that every group
        carries each class of record whatever the random draws were: a
        benign cell (its owner is among the writers, all of whom store one
        value and write nothing after it), a racy cell (writers store
        ``tid + c``: pairwise different values) and reads of the racy cell
        by work-items that do not write it (every reader sees a value some
        writer differs from)."""
        r, S = self.rng, self.S
        base = int(self.pslabs[0]) * self.N
        off1 = int(r.integers(S))
        off2 = (off1 + 1 + int(r.integers(S - 1))) % S
        st1, st2, st3 = (min(int(r.choice([8, 16, 32, 64])), S) for _ in range(3))
        c1, c2 = int(r.integers(8)), int(r.integers(8))
        cell1 = self._plus(base, f"wg * {S} + {off1}")
        cell2 = self._plus(base, f"wg * {S} + {off2}")
        lines = [f"if (tid % {st1} == {off1 % st1}) {{", f"  A[{cell1}] = wg * 3 + {c1};", "}",
                 f"if (tid % {st2} == 0) {{", f"  A[{cell2}] = tid + {c2};", "}"]
        if st2 % 2 == 0 and st3 >= 2:  # readers are odd, writers even: disjoint
            lines += [f"if (tid % {st3} == 1) {{", f"  {self.var()} = A[{cell2}];", "}"]
        return lines, 3

    # cumulative thresholds: assign, neighbour load, own load, local load,
    # store, local store, loop; the rest are branches
    MIX = {"dense": (0.2, 0.42, 0.5, 0.56, 0.72, 0.78, 0.88),
           "sparse": (0.55, 0.64, 0.68, 0.68, 0.78, 0.78, 0.8)}

    def stmt(self, depth, in_loop):
        t = self.MIX[self.mix]
        r = self.rng.random()
        if r < t[0]:
            return [f"{self.var()} = {self.value()};"], 1
        if r < t[1]:
            return [f"{self.var()} = A[{self.gaddr_read()}];"], 1
        if r < t[2]:
            return [f"{self.var()} = {self.var()} + A[{self.gaddr_own(any_slab=True)}];"], 1
        if r < t[3] and self.n_lslab:
            return [f"{self.var()} = Lc[{self.laddr_read()}];"], 1
        if r < t[4]:
            if self.rng.random() < self.plant * 2 and (self.wslabs or self.n_slab >= 3):
                return self.planted()
            if not self.wslabs:
                return [f"{self.var()} = {self.value()};"], 1
            return [f"A[{self.gaddr_own()}] = {self.value()};"], 1
        if r < t[5] and self.n_lslab:
            return [f"Lc[{self.laddr_own()}] = {self.value()};"], 1
        if r < t[6] and depth < self.max_depth:
            v = f"i{len(self.loopvars)}"
            trip = int(self.rng.integers(1, self.max_trip + 1))
            self.loopvars.append(v)
            body, n = [], 0
            for _ in range(int(self.rng.integers(1, 4))):
                ls, c = self.stmt(depth + 1, True)
                body += ["  " + x for x in ls]
                n += c
            self.loopvars.pop()
            return [f"for {v} in 0 .. {trip} {{"] + body + ["}"], n + 1
        if depth < self.max_depth + 1:
            if self.loads_on_branch and self.rng.random() < 0.5:
                cond = f"{self.var()} % {int(self.rng.integers(2, 5))} == 0"
            else:
                cond = f"tid < {int(self.rng.integers(1, self.S + 1))}"
            body, n = [], 0
            for _ in range(int(self.rng.integers(1, 3))):
                ls, c = self.stmt(depth + 1, in_loop)
                body += ["  " + x for x in ls]
                n += c
            return [f"if ({cond}) {{"] + body + ["}"], n + 1
        return [f"{self.var()} = {self.value()};"], 1


def _slab_kernel(name, rng, G, S, L, LL, n_stmts, n_barriers, max_trip, plant, loads_on_branch,
                 max_depth, n_vars=8, mix="dense", closing_plants=False):
    N = G * S
    g = _SlabGen(rng, N, S, L, LL, n_vars, max_trip, plant, loads_on_branch, max_depth, mix)
    per = n_stmts / (n_barriers + 1)
    lines, count, next_bar, bars = [], 0, per, 0

    def close_interval():
        nonlocal count
        if closing_plants and g.can_plant():
            ls, c = g.closing_plants()
            lines.extend(ls)
            count += c

    while count < n_stmts:
        ls, c = g.stmt(0, False)
        lines += ls
        count += c
        if bars < n_barriers and count >= next_bar:
            close_interval()
            lines.append("barrier;")
            bars += 1
            next_bar += per
            g.new_interval()
    while bars < n_barriers:
        close_interval()
        lines.append("barrier;")
        bars += 1
        if closing_plants:
            g.new_interval()
    close_interval()
    decl = "global int A[]" + (f", local int Lc[{LL}]" if LL else "")
    src = f"kernel {name}({decl}) {{\n" + "\n".join("  " + x for x in lines) + "\n}\n"
    return src


def large_kernel(seed: int, groups: int = 1024, group_size: int = 256,
                 global_len: int = 4 << 20, local_len: int = 4096, n_stmts: int = 200,
                 n_barriers: int = 8) -> Instance:
    """Config-2 instance (defaults: 1024 x 256, 8 barriers, 200 statements)."""
    rng = np.random.default_rng([2, seed])
    N = groups * group_size
    L = max(global_len, N)
    src = _slab_kernel("large", rng, groups, group_size, L, local_len, n_stmts, n_barriers,
                       max_trip=16, plant=0.05, loads_on_branch=False, max_depth=1)
    A = rng.integers(0, 1 << 10, size=L, dtype=np.int32)
    return Instance(f"large-s{seed}-{groups}x{group_size}", src, groups, group_size, [A])


def stress_kernel(seed: int, groups: int = 65536, group_size: int = 1024, n_stmts: int = 512,
                  n_barriers: int = 16, global_len: int | None = None, closing_plants: bool = True) -> Instance:
    """Config-5 instance (defaults: 65,536 x 1024, 16 barriers, 512 statements).
    ``closing_plants=False``: the same statement mix without the planted
    cells that end each writing interval (often race-free)."""
    rng = np.random.default_rng([5, seed])
    N = groups * group_size
    L = global_len or N
    src = _slab_kernel("stress", rng, groups, group_size, L, 0, n_stmts, n_barriers,
                       max_trip=32, plant=0.02, loads_on_branch=True, max_depth=2,
                       mix="sparse", closing_plants=closing_plants)
    A = rng.integers(0, 1 << 10, size=L, dtype=np.int32)
    return Instance(f"stress-s{seed}-{groups}x{group_size}", src, groups, group_size, [A])


# ----------------------------------------------------------------------------
# tiny kernels for exhaustive schedule enumeration


def tiny_kernel(seed: int) -> Instance:
    """2-4 work-items, <= 3 intervals, few accesses, values in [0,4)."""
    rng = np.random.default_rng([9, seed])
    G = int(rng.integers(1, 3))
    S = int(rng.integers(1, 3)) if G == 2 else int(rng.integers(2, 5))
    L = int(rng.integers(3, 7))
    use_local = rng.random() < 0.5
    n_bar = int(rng.integers(0, 3))
    lines = []
    budget = int(rng.integers(3, 8))

    def idx():
        k = rng.random()
        if k < 0.5:
            return f"({int(rng.integers(3))} * tid + {int(rng.integers(L))}) % {L}"
        if k < 0.75:
            return f"(gtid + {int(rng.integers(L))}) % {L}"
        return f"(x{int(rng.integers(2))} + tid) % {L}"

    def val():
        k = rng.random()
        if k < 0.4:
            return str(int(rng.integers(4)))
        if k < 0.7:
            return f"(tid + {int(rng.integers(4))}) % 4"
        return f"(x{int(rng.integers(2))} + {int(rng.integers(3))}) % 4"

    def st(depth):
        k = rng.random()
        if k < 0.35:
            return [f"x{int(rng.integers(2))} = A[{idx()}];"]
        if k < 0.7:
            return [f"A[{idx()}] = {val()};"]
        if k < 0.8 and use_local:
            return [f"Lc[tid % 3] = {val()};"] if rng.random() < 0.5 else \
                   [f"x{int(rng.integers(2))} = Lc[(tid + 1) % 3];"]
        if depth == 0:
            cond = f"x{int(rng.integers(2))} == {int(rng.integers(4))}" if rng.random() < 0.6 \
                else f"tid < {int(rng.integers(1, S + 1))}"
            return [f"if ({cond}) {{", "  " + st(1)[0], "}"]
        return [f"x{int(rng.integers(2))} = x{int(rng.integers(2))} + {int(rng.integers(3))};"]

    for _ in range(budget):
        lines += st(0)
    tops = [i for i, x in enumerate(lines) if not x.startswith(" ") and not x.startswith("}")]
    pos = sorted(rng.choice(len(tops), size=min(n_bar, len(tops)), replace=False).tolist())
    for p in reversed(pos):
        lines.insert(tops[p], "barrier;")
    decl = "global int A[]" + (", local int Lc[3]" if use_local else "")
    src = f"kernel tiny({decl}) {{\n" + "\n".join("  " + x for x in lines) + "\n}\n"
    A = rng.integers(0, 4, size=L, dtype=np.int32)
    return Instance(f"tiny-s{seed}", src, G, S, [A])


# ----------------------------------------------------------------------------
# proposal kernels: races that appear only for some candidate instances


@dataclasses.dataclass
class ProposalKernel:
    name: str
    src: str
    L: int        # global A[] length
    LI: int       # global In[] length
    V: int        # In[] values are uniform in [0, V)
    seed: int

    def instance(self, groups: int, group_size: int, input_seed: int) -> Instance:
        rng = np.random.default_rng([11, self.seed, input_seed])
        A = rng.integers(0, 16, size=self.L, dtype=np.int32)
        In = rng.integers(0, self.V, size=self.LI, dtype=np.int32)
        return Instance(f"{self.name}-G{groups}-S{group_size}-i{input_seed}", self.src, groups, group_size, [A, In])


def proposal_kernel(seed: int) -> ProposalKernel:
    """A kernel whose races depend on the launch shape and the input, each
    racy statement on roughly one candidate in eight: stores gated on
    ``tid >= K`` (K in [700, 1024)) or ``wg >= K`` (K in [24, 64)),
    indices ``(a*gtid + B) % L`` that collide only past L/gcd(a, L)
    work-items (L log-uniform in [8K, 256K]), a local array indexed
    ``tid % m`` (m in [700, 1024): racy for larger groups), a store under a
    branch on an input value that few positions hold, and read-then-write
    neighbours under ``tid >= K``.  One to four such statements among
    private arithmetic and plain loads, up to two barriers."""
    rng = np.random.default_rng([10, seed])
    L = int(round(math.exp(rng.uniform(math.log(8192), math.log(262144)))))
    LI = int(round(math.exp(rng.uniform(math.log(256), math.log(4096)))))
    V = LI * int(rng.integers(2, 17))
    lines = []

    def filler():
        k = rng.random()
        v = f"v{int(rng.integers(4))}"
        if k < 0.5:
            return [f"{v} = {int(rng.integers(-3, 4))} * tid + {int(rng.integers(16))};"]
        if k < 0.8:
            return [f"{v} = A[(tid + {int(rng.integers(L))}) % {L}];"]
        return [f"{v} = {v} * {int(rng.integers(1, 4))} + wg;"]

    def gated():
        k = int(rng.integers(6))
        B = int(rng.integers(L))
        d = int(rng.integers(16))
        if k == 0:
            K = int(rng.integers(700, 1024))
            return [f"if (tid >= {K}) {{", f"  A[{B}] = {int(rng.choice([-2, -1, 1, 2, 3]))} * tid + {d};", "}"]
        if k == 1:
            K = int(rng.integers(24, 64))
            return [f"if (wg >= {K}) {{", f"  A[(wg + {B}) % {L}] = tid + {d};", "}"]
        if k == 2:
            a = int(rng.integers(1, 4))
            return [f"A[({a} * gtid + {B}) % {L}] = gtid + {d};"]
        if k == 3:
            m = int(rng.integers(700, 1024))
            return [f"Lc[tid % {m}] = tid + {d};"]
        if k == 4:
            t = int(rng.integers(V))
            return [f"x = In[gtid % {LI}];", f"if (x == {t}) {{", f"  A[{B}] = gtid;", "}"]
        K = int(rng.integers(700, 1024))
        return [f"y = A[(tid + {B}) % {L}];", f"if (tid >= {K}) {{", f"  A[(tid + {B + 1}) % {L}] = y + 1;", "}"]

    n_gated = int(rng.integers(1, 5))
    n_fill = int(rng.integers(2, 9))
    kinds = ["g"] * n_gated + ["f"] * n_fill
    rng.shuffle(kinds)
    for kd in kinds:
        lines += gated() if kd == "g" else filler()
    tops = [i for i, x in enumerate(lines) if not x.startswith(" ") and not x.startswith("}")]
    n_bar = int(rng.integers(0, 3))
    pos = sorted(rng.choice(len(tops), size=min(n_bar, len(tops)), replace=False).tolist())
    for p in reversed(pos):
        lines.insert(tops[p], "barrier;")
    src = ("kernel proposal(global int A[], global int In[], local int Lc[1024]) {\n"
           + "\n".join("  " + x for x in lines) + "\n}\n")
    return ProposalKernel(f"prop-s{seed}", src, L, LI, V, seed)


@dataclasses.dataclass
class BatchProposalKernel:
    """A config-3 kernel as a proposal kernel: its program is fixed (drawn
    for group size 1024, so `if (tid < k)` guards take k in [1, 1024]) and
    each candidate brings its own launch shape and input."""
    name: str
    src: str
    L: int
    seed: int

    def instance(self, groups: int, group_size: int, input_seed: int) -> Instance:
        rng = np.random.default_rng([15, self.seed, input_seed])
        A = rng.integers(0, 16, size=self.L, dtype=np.int32)
        return Instance(f"{self.name}-G{groups}-S{group_size}-i{input_seed}", self.src, groups, group_size, [A])


def batch_proposal_kernel(seed: int, max_stmts: int = 512) -> BatchProposalKernel:
    """Proposal kernels from the config-3 generator: the config-1 statement
    and index mix, 16..max_stmts statements, 0-8 barriers, A of length
    log-uniform in [1K, 1M]."""
    rng = np.random.default_rng([14, seed])
    n_stmts = int(rng.integers(16, max_stmts + 1))
    n_bar = int(rng.integers(0, 9))
    L = int(round(math.exp(rng.uniform(math.log(1024), math.log(1 << 20)))))
    inst = small_kernel(int(rng.integers(1 << 31)), group_size=1024, groups=1, n_stmts=n_stmts,
                        n_barriers=n_bar, L=L)
    return BatchProposalKernel(f"bprop-s{seed}", inst.src, L, seed)


def proposal_candidates(seed: int, n: int = 64) -> list:
    """The candidate instances of a proposal kernel, in enumeration order:
    (groups, group_size, input_seed) with group size a multiple of 32 in
    [32, 1024], group count log-uniform in [1, 64]."""
    rng = np.random.default_rng([12, seed])
    out = []
    for _ in range(n):
        S = 32 * int(rng.integers(1, 33))
        G = int(round(math.exp(rng.uniform(0.0, math.log(64)))))
        out.append((max(1, min(64, G)), S, int(rng.integers(1 << 31))))
    return out


# ----------------------------------------------------------------------------
# work-group-scoped barrier kernels


def group_kernel(seed: int, groups: int = 4, group_size: int = 32, n_stmts: int = 24) -> Instance:
    """Kernels for work-group-scoped barriers: each group has a slab of its
    own in A (accesses there can race only inside the group), a shared tail
    of 16 cells that every group reads and writes, a local array, barriers
    every work-item takes, and barriers only some groups take (under a
    condition on wg, so a whole group agrees)."""
    rng = np.random.default_rng([13, seed])
    G, S = groups, group_size
    L = G * S + 16
    lines = []

    def own():
        return f"A[wg * {S} + ({int(rng.integers(1, 3))} * tid + {int(rng.integers(S))}) % {S}]"

    def shared():
        return f"A[{G * S} + (tid + {int(rng.integers(16))}) % {int(rng.choice([1, 4, 16]))}]"

    def val():
        k = rng.random()
        if k < 0.3:
            return str(int(rng.integers(4)))
        if k < 0.6:
            return f"(wg + {int(rng.integers(3))}) % 3"
        return f"x + {int(rng.integers(3))}"

    def stmt(depth):
        k = rng.random()
        if k < 0.25:
            return [f"x = {own()};"]
        if k < 0.45:
            return [f"{own()} = {val()};"]
        if k < 0.55:
            return [f"x = {shared()};"]
        if k < 0.63:
            return [f"{shared()} = {val()};"]
        if k < 0.72:
            return [f"Lc[(tid + {int(rng.integers(8))}) % 8] = {val()};"] if rng.random() < 0.5 else \
                   [f"x = Lc[tid % 8];"]
        if k < 0.8 or depth > 0:
            return ["barrier;"] if depth == 0 else [f"x = x + {int(rng.integers(3))};"]
        m = int(rng.integers(2, 4))
        body = [f"if (wg % {m} == {int(rng.integers(m))}) {{", "  barrier;"]
        body += ["  " + x for x in stmt(1)]
        return body + ["}"]

    for _ in range(n_stmts):
        lines += stmt(0)
    src = "kernel grp(global int A[], local int Lc[8]) {\n" + "\n".join("  " + x for x in lines) + "\n}\n"
    A = rng.integers(0, 4, size=L, dtype=np.int32)
    return Instance(f"group-s{seed}-{G}x{S}", src, G, S, [A])
