// Two-work-item NoRace pre-filter for one launch shape (a restricted,
// sound take on the symbolic method of Sec. 5-6: two renamed work-items
// i != j, their accesses in one barrier interval, race freedom when no cell
// can be shared with a conflicting value; Table 1's bounds premise for the
// array indices).
//
// Every register is described at every instruction by an affine form
//   v = ((c0 + ct * tid + cw * wg + sum_L cv[L] * i_L) mod M) + off    (M = 0: no reduction)
// over the work-item's (tid, wg) and the counters i_L of the constant-trip
// loops around it, i_L in [lo_L, max(lo_L, hi_L - 1)]; or "unknown".  The
// forms come from a fixpoint over the bytecode's control-flow graph: a join
// of two different forms is unknown, except that a loop's counter is the
// variable i_L at the loop head (other registers a loop updates become
// unknown there); a loaded value is unknown.  The forms are exact modulo
// 2^32, so a form whose range fits in int32 is the register's value; a
// Euclidean remainder or an index needs that.  Barriers are kernel-wide:
// two accesses may meet in one interval when some barrier region (code
// reachable from the start, or from just after a barrier, without crossing
// a barrier) contains both.  A compare-and-branch on an affine function of
// tid (or of wg) narrows the work-items that can execute the accesses of its
// single-entry fall-through region.  A pair of accesses to one array, one of
// them a store, by two different work-items (each with its own loop
// counters) is harmless when the index ranges are disjoint, or when both use
// the same index form and equal values of it force equal work-items (for
// local arrays: within one group), or -- on launches small enough to
// enumerate every work-item and loop counter -- when no cell is reached by
// two different work-items, or when every work-item stores one and the
// same value.  The verdict "race-free" holds for every schedule
// (Sec. 4's Definition); otherwise the pre-filter says nothing and the
// checker decides.
#include <algorithm>
#include <array>
#include <cstdint>
#include <cstdlib>
#include <unordered_map>
#include <vector>

#include "racecheck.h"
#include "bytecode.h"

namespace rc {
namespace {

constexpr int kLoops = 8;  // loop counters tracked as variables; the counters of further loops are unknown

struct AF {
  enum Kind : uint8_t { BOT, AFF, TOP } kind = BOT;
  int64_t c0 = 0, ct = 0, cw = 0, M = 0, off = 0;
  std::array<int64_t, kLoops> cv{};
  bool operator==(const AF &o) const {
    return kind == o.kind && (kind != AFF || (c0 == o.c0 && ct == o.ct && cw == o.cw && M == o.M &&
                                              off == o.off && cv == o.cv));
  }
  bool no_vars() const {
    for (int64_t k : cv)
      if (k) return false;
    return true;
  }
  bool is_const() const { return kind == AFF && ct == 0 && cw == 0 && M == 0 && no_vars(); }
  bool plain() const { return kind == AFF && M == 0; }
};

AF top() {
  AF f;
  f.kind = AF::TOP;
  return f;
}
AF konst(int64_t v) {
  AF f;
  f.kind = AF::AFF;
  f.c0 = v;
  return f;
}
AF var(int L) {
  AF f;
  f.kind = AF::AFF;
  f.cv[L] = 1;
  return f;
}
AF join(const AF &a, const AF &b) {
  if (a.kind == AF::BOT) return b;
  if (b.kind == AF::BOT) return a;
  return a == b ? a : top();
}

constexpr int64_t kBig = (int64_t)1 << 40;  // coefficients beyond this: unknown (keeps int64 exact)
AF clamp(AF f) {
  if (f.kind != AF::AFF) return f;
  bool big = std::llabs(f.c0) > kBig || std::llabs(f.ct) > kBig || std::llabs(f.cw) > kBig || std::llabs(f.off) > kBig;
  for (int64_t k : f.cv) big = big || std::llabs(k) > kBig;
  return big ? top() : f;
}
AF add(const AF &a, const AF &b) {
  if (a.kind != AF::AFF || b.kind != AF::AFF) return a.kind == AF::BOT || b.kind == AF::BOT ? AF() : top();
  if (a.plain() && b.plain()) {
    AF f = a;
    f.c0 += b.c0;
    f.ct += b.ct;
    f.cw += b.cw;
    for (int L = 0; L < kLoops; L++) f.cv[L] += b.cv[L];
    return clamp(f);
  }
  if (b.is_const()) {
    AF f = a;
    f.off += b.c0;
    return clamp(f);
  }
  if (a.is_const()) return add(b, a);
  return top();
}
AF scale(const AF &a, int64_t k) {
  if (a.kind != AF::AFF) return a;
  if (!a.plain()) return k == 1 ? a : top();
  AF f = a;
  f.c0 *= k;
  f.ct *= k;
  f.cw *= k;
  for (int64_t &c : f.cv) c *= k;
  return clamp(f);
}

// The work-items (tid, wg) in [t0, t1] x [w0, w1] of a launch [0, S) x [0, G),
// with the ranges of the loop counters.
struct Shape {
  int64_t S, G;
  int64_t t0, t1, w0, w1;
  std::array<int64_t, kLoops> vlo{}, vhi{};
  Shape(int64_t s, int64_t g) : S(s), G(g), t0(0), t1(s - 1), w0(0), w1(g - 1) {}
  bool empty() const { return t1 < t0 || w1 < w0; }
  int64_t nt() const { return t1 - t0 + 1; }
  int64_t nw() const { return w1 - w0 + 1; }
};
Shape hull(const Shape &a, const Shape &b) {
  if (a.empty()) return b;
  if (b.empty()) return a;
  Shape h = a;
  h.t0 = std::min(a.t0, b.t0);
  h.t1 = std::max(a.t1, b.t1);
  h.w0 = std::min(a.w0, b.w0);
  h.w1 = std::max(a.w1, b.w1);
  return h;
}

// floor division for a positive divisor
int64_t fdiv(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
int64_t cdiv(int64_t a, int64_t b) { return -fdiv(-a, b); }

constexpr int64_t kSat = (int64_t)1 << 62;
int64_t sat(__int128 v) { return v > kSat ? kSat : v < -kSat ? -kSat : (int64_t)v; }

struct Range {
  int64_t lo, hi;
};
// Value range of a known form over the work-items of sh (saturated at
// +-2^62, which keeps order).  A reduced form takes its inner values' own
// range when they lie in one period of M, where the remainder is a plain
// shift, else all of [0, M).
Range range_of(const AF &f, const Shape &sh) {
  __int128 lo = f.c0, hi = f.c0;
  auto span = [&](int64_t k, int64_t a, int64_t b) {
    const __int128 x = (__int128)k * a, y = (__int128)k * b;
    lo += std::min(x, y);
    hi += std::max(x, y);
  };
  span(f.ct, sh.t0, sh.t1);
  span(f.cw, sh.w0, sh.w1);
  for (int L = 0; L < kLoops; L++)
    if (f.cv[L]) span(f.cv[L], sh.vlo[L], sh.vhi[L]);
  if (f.M > 0) {
    const int64_t l = sat(lo), h = sat(hi), q = fdiv(l, f.M);
    if (fdiv(h, f.M) == q && l > -kSat && h < kSat) return Range{l - q * f.M + f.off, h - q * f.M + f.off};
    return Range{f.off, f.off + f.M - 1};
  }
  return Range{sat(lo + f.off), sat(hi + f.off)};
}
Range inner_range(const AF &f, const Shape &sh) {  // the part before the reduction
  AF g = f;
  g.M = 0;
  g.off = 0;
  return range_of(g, sh);
}
bool fits32(const Range &r) { return r.lo >= INT32_MIN && r.hi <= INT32_MAX; }
// the form equals the register's int32 value on every work-item of sh
bool exact(const AF &f, const Shape &sh) {
  if (f.kind != AF::AFF) return false;
  if (f.M > 0 && !fits32(inner_range(f, sh))) return false;
  return fits32(range_of(f, sh));
}

// Do equal values of the form force equal work-items (same_group: equal
// tid within one group), whatever loop counters either work-item has?  A
// term whose weight exceeds what every other term not yet shown equal can
// add up to must be equal on both sides; repeat until nothing changes.
bool injective(const AF &f, const Shape &sh, bool same_group) {
  if (f.kind != AF::AFF) return false;
  struct Dim {
    __int128 k, n1;  // |coefficient|, extent - 1
    bool item, fixed;
  };
  Dim d[2 + kLoops];
  int nd = 0;
  d[nd++] = Dim{std::llabs(f.ct), sh.nt() - 1, true, false};
  if (!same_group) d[nd++] = Dim{std::llabs(f.cw), sh.nw() - 1, true, false};
  for (int L = 0; L < kLoops; L++)
    if (f.cv[L]) d[nd++] = Dim{std::llabs(f.cv[L]), sh.vhi[L] - sh.vlo[L], false, false};
  __int128 span = 0;
  for (int i = 0; i < nd; i++) {
    d[i].fixed = d[i].n1 == 0;  // a single value never differs
    span += d[i].k * d[i].n1;
  }
  for (bool changed = true; changed;) {
    changed = false;
    for (int i = 0; i < nd; i++) {
      if (d[i].fixed || d[i].k == 0) continue;
      __int128 rest = 0;
      for (int j = 0; j < nd; j++)
        if (j != i && !d[j].fixed) rest += d[j].k * d[j].n1;
      if (d[i].k > rest) d[i].fixed = changed = true;
    }
  }
  for (int i = 0; i < nd; i++)
    if (d[i].item && !d[i].fixed) return false;
  // distinct inner values stay distinct after the reduction when they span less than M
  return f.M == 0 || span < f.M;
}

// Every (work-item, loop counters) point of the box, with the form's value
// there (the form is exact on the box).  Returns false, visiting nothing,
// when the box has more than `limit` points.
template <class F>
bool enumerate(const AF &f, const Shape &sh, uint64_t limit, F visit) {
  uint64_t n = (uint64_t)sh.nt() * (uint64_t)sh.nw();
  int vars[kLoops], nv = 0;
  for (int L = 0; L < kLoops; L++)
    if (f.cv[L]) {
      vars[nv++] = L;
      n *= (uint64_t)(sh.vhi[L] - sh.vlo[L] + 1);
      if (n > limit) return false;
    }
  if (n > limit || sh.empty()) return n <= limit;
  int64_t v[kLoops];
  for (int64_t w = sh.w0; w <= sh.w1; w++)
    for (int64_t t = sh.t0; t <= sh.t1; t++) {
      for (int k = 0; k < nv; k++) v[k] = sh.vlo[vars[k]];
      for (;;) {
        __int128 y = (__int128)f.c0 + (__int128)f.ct * t + (__int128)f.cw * w;
        for (int k = 0; k < nv; k++) y += (__int128)f.cv[vars[k]] * v[k];
        int64_t x = (int64_t)y;  // the form is exact on the box: the inner value fits int32
        if (f.M > 0) x = x - fdiv(x, f.M) * f.M;  // Euclidean remainder
        visit(t, w, x + f.off);
        int k = 0;
        while (k < nv && ++v[k] > sh.vhi[vars[k]]) v[k] = sh.vlo[vars[k]], k++;
        if (k == nv) break;
      }
    }
  return true;
}

// Exact check of a pair on small launches: can a work-item's access a and a
// different work-item's access b reach one cell (for local arrays: one cell
// of one group)?  a == b asks it of one instruction.  Returns 1 for "never",
// 0 for "they can", -1 when the points to enumerate exceed *budget (which
// the points visited are taken from).
int never_meet(const AF &fa, const Shape &ba, const AF &fb, const Shape &bb, bool same, bool local,
               uint64_t *budget) {
  const uint64_t kLimit = std::min<uint64_t>(*budget, 1u << 16);
  // cell (and group, for local arrays) -> the one work-item seen there, or kMany
  constexpr int64_t kMany = -1;
  std::unordered_map<uint64_t, int64_t> seen;
  const auto cell = [&](int64_t w, int64_t x) {
    return ((uint64_t)(local ? w : 0) << 32) ^ (uint64_t)(uint32_t)x;
  };
  const auto item = [&](int64_t t, int64_t w) { return w * (ba.S) + t; };
  bool clash = false;
  uint64_t visited = 0;
  const auto spend = [&]() { *budget -= std::min(*budget, visited); };
  if (!enumerate(fa, ba, kLimit, [&](int64_t t, int64_t w, int64_t x) {
        visited++;
        auto it = seen.emplace(cell(w, x), item(t, w));
        if (!it.second && it.first->second != item(t, w)) {
          if (same) clash = true;  // two work-items of the one instruction
          it.first->second = kMany;
        }
      }))
    return -1;
  if (clash || same) {
    spend();
    return clash ? 0 : 1;
  }
  if (!enumerate(fb, bb, kLimit, [&](int64_t t, int64_t w, int64_t x) {
        visited++;
        auto it = seen.find(cell(w, x));
        if (it != seen.end() && it->second != item(t, w)) clash = true;
      })) {
    spend();
    return -1;
  }
  spend();
  return clash ? 0 : 1;
}

// Restrict sh to the work-items where (x op imm) holds, op = 0 <, 1 <=, 2 >,
// 3 >=, 4 ==, 5 != (not representable: left out, a weaker constraint).
// Only x = c + k * tid or x = c + k * wg (exact on sh), or a constant, is used.
void restrict_box(Shape &sh, const AF &x, uint32_t op, int64_t imm) {
  if (!x.plain() || !x.no_vars() || !exact(x, sh) || op == 5) return;
  const bool on_t = x.ct != 0 && x.cw == 0, on_w = x.cw != 0 && x.ct == 0;
  if (!on_t && !on_w) {
    if (x.ct == 0 && x.cw == 0) {  // a constant condition
      const int64_t v = x.c0;
      const bool holds = op == 0 ? v < imm : op == 1 ? v <= imm : op == 2 ? v > imm : op == 3 ? v >= imm : v == imm;
      if (!holds) sh.t1 = sh.t0 - 1;
    }
    return;
  }
  int64_t k = on_t ? x.ct : x.cw, r = imm - x.c0;  // k * v op r
  if (k < 0) {  // flip to a positive multiplier
    k = -k;
    r = -r;
    op = op == 0 ? 2 : op == 1 ? 3 : op == 2 ? 0 : op == 3 ? 1 : op;
  }
  int64_t lo = INT64_MIN / 4, hi = INT64_MAX / 4;
  switch (op) {
    case 0: hi = cdiv(r, k) - 1; break;  // v < r / k
    case 1: hi = fdiv(r, k); break;
    case 2: lo = fdiv(r, k) + 1; break;
    case 3: lo = cdiv(r, k); break;
    default:  // ==
      if (r % k) lo = 1, hi = 0;
      else lo = hi = r / k;
  }
  if (on_t) {
    sh.t0 = std::max(sh.t0, lo);
    sh.t1 = std::min(sh.t1, hi);
  } else {
    sh.w0 = std::max(sh.w0, lo);
    sh.w1 = std::min(sh.w1, hi);
  }
}

struct Acc {
  uint32_t pc, mem;
  bool store, local;
  AF idx, val;
  Shape box{1, 1};  // the work-items that can execute the access
  Range ir{0, 0}, vr{0, 0};  // ranges of idx and val over box (known forms only)
};

// A counted loop: the back edge `reg = reg + 1; if reg < hi: goto head`
struct Loop {
  uint32_t pc, head, reg;
  int64_t hi;
  AF entry;  // the counter's value on the edges into the head from outside
  bool broken = false;  // the body changes the counter
};

uint32_t insn_class(const Insn &in) { return (in.ctl >> CTL_CLASS_SHIFT) & 0xFu; }

struct Prover {
  const Program &p;
  Shape sh;
  std::vector<std::vector<AF>> in;  // register forms on entry to each instruction
  std::vector<uint64_t> region;     // bit r: reachable from region entry r without crossing a barrier
  std::vector<uint32_t> mem_len;
  std::vector<Loop> loops;
  std::vector<int> head_loop;  // per pc: the loop whose head it is, or -1
  std::vector<uint32_t> guards;  // compare-and-branch instructions with a single-entry fall-through region

  Prover(const Program &prog, Shape s, std::vector<uint32_t> lens) : p(prog), sh(s), mem_len(std::move(lens)) {}

  std::vector<uint32_t> succ(uint32_t pc) const {
    const Insn &in = p.code[pc];
    const uint32_t cls = insn_class(in);
    if (cls == CC_EXIT) return {};
    if (cls == CC_ALU) {
      const uint32_t mode = (in.ctl >> AL_MODE_SHIFT) & 3u;
      if (mode == 2) return {(uint32_t)in.imm2};
      if (mode == 1) return {(uint32_t)in.imm2, pc + 1};
    }
    return {pc + 1};
  }

  AF step(const Insn &in, const std::vector<AF> &R, uint32_t &dest, bool &writes) const {
    const uint32_t cls = insn_class(in);
    const AF x = R[in.a], y = R[in.b];
    dest = in.d;
    writes = false;
    switch (cls) {
      case CC_ALU:
        writes = (in.ctl & AL_WRITE) != 0;
        switch (in.op) {
          case OP_MOVI: return konst(in.imm);
          case OP_MOV: return x;
          case OP_ADD: return add(x, y);
          case OP_SUB: return add(x, scale(y, -1));
          case OP_MUL:
            if (y.is_const()) return scale(x, y.c0);
            if (x.is_const()) return scale(y, x.c0);
            return x.kind == AF::BOT || y.kind == AF::BOT ? AF() : top();
          case OP_ADDI: return add(x, konst(in.imm));
          case OP_MULI: return scale(x, in.imm);
          case OP_RSUBI: return add(scale(x, -1), konst(in.imm));
          case OP_NEG: return scale(x, -1);
          case OP_MADI: return add(scale(x, in.imm), y);
          case OP_LOOP: return add(x, konst(1));
          case OP_ANDI: {  // x mod 2^k for a mask 2^k - 1 (k <= 31), exact on the wrapped value
            const uint64_t m = (uint64_t)(uint32_t)in.imm + 1;
            if (x.kind == AF::AFF && x.plain() && in.imm >= 0 && (m & (m - 1)) == 0) {
              AF f = x;
              f.M = (int64_t)m;
              return f;
            }
            return x.kind == AF::BOT ? AF() : top();
          }
          default: return x.kind == AF::BOT ? AF() : top();  // comparisons, branch results
        }
      case CC_DIVMOD:
        writes = true;
        if ((in.ctl & DM_MOD) && (in.ctl & DM_YIMM) && in.imm != 0 && x.kind == AF::AFF && x.plain() &&
            exact(x, sh)) {
          AF f = x;
          f.M = std::llabs((long long)in.imm);
          return f;
        }
        return x.kind == AF::BOT ? AF() : top();
      case CC_SIZE:
        writes = true;
        return konst(mem_len[in.ctl >> CTL_MEM_SHIFT]);
      case CC_LOGIC: writes = true; return top();
      case CC_LD: writes = true; return top();
      default: return AF();  // ST, ASSUME, ASSERT, BARRIER, EXIT write no register
    }
  }

  void find_loops() {
    const uint32_t n = (uint32_t)p.code.size();
    head_loop.assign(n, -1);
    for (uint32_t pc = 0; pc < n && loops.size() < (size_t)kLoops; pc++) {
      const Insn &in = p.code[pc];
      if (in.op != OP_LOOP || insn_class(in) != CC_ALU || ((in.ctl >> AL_MODE_SHIFT) & 3u) != 1u ||
          !(in.ctl & AL_LOOPCOND) || !(in.ctl & AL_WRITE) || in.d != in.a || in.d < kBuiltinRegs ||
          (uint32_t)in.imm2 > pc || head_loop[(uint32_t)in.imm2] >= 0)
        continue;
      head_loop[(uint32_t)in.imm2] = (int)loops.size();
      Loop lp;
      lp.pc = pc;
      lp.head = (uint32_t)in.imm2;
      lp.reg = in.a;
      lp.hi = in.imm;
      loops.push_back(lp);
    }
  }

  // the counter's form at the head of loop L, from what is known so far
  AF counter_at_head(int L) {
    Loop &lp = loops[L];
    if (lp.entry.kind == AF::BOT) return AF();
    if (lp.broken || !lp.entry.is_const()) return top();
    sh.vlo[L] = lp.entry.c0;
    sh.vhi[L] = std::max<int64_t>(lp.entry.c0, lp.hi - 1);
    return var(L);
  }

  void dataflow() {
    const uint32_t n = (uint32_t)p.code.size();
    const uint32_t nr = std::max<uint32_t>(p.n_regs, kBuiltinRegs);
    in.assign(n, std::vector<AF>(nr));
    std::vector<AF> init(nr, konst(0));  // registers start at 0
    init[REG_TID] = konst(0);
    init[REG_TID].ct = sh.S > 1;  // a coordinate with one value is the constant 0
    init[REG_WG] = konst(0);
    init[REG_WG].cw = sh.G > 1;
    init[REG_GTID] = konst(0);
    init[REG_GTID].ct = sh.S > 1;
    init[REG_GTID].cw = sh.G > 1 ? sh.S : 0;
    init[REG_GSIZE] = konst(sh.S);
    init[REG_NGROUPS] = konst(sh.G);
    find_loops();
    if (!n) return;
    in[0] = init;
    std::vector<uint32_t> work{0};
    std::vector<char> queued(n, 0);
    queued[0] = 1;
    uint64_t steps = 0;
    while (!work.empty() && steps++ < (uint64_t)n * nr * 8 + 1000) {
      const uint32_t pc = work.back();
      work.pop_back();
      queued[pc] = 0;
      std::vector<AF> out = in[pc];
      uint32_t d = 0;
      bool w = false;
      const AF r = step(p.code[pc], in[pc], d, w);
      if (w && d >= kBuiltinRegs && d < nr) out[d] = r;
      for (uint32_t s : succ(pc)) {
        if (s >= n) continue;
        bool changed = false;
        const int L = head_loop[s];
        for (uint32_t k = 0; k < nr; k++) {
          AF j;
          if (L >= 0 && k == loops[L].reg) {
            if (pc == loops[L].pc) {  // back edge: the counter must still be i_L at the loop instruction
              const AF &at = in[pc][k];
              if (!(at.kind == AF::BOT || at == var(L))) loops[L].broken = true;
            } else {
              loops[L].entry = join(loops[L].entry, out[k]);
            }
            j = counter_at_head(L);
          } else {
            j = join(in[s][k], out[k]);
          }
          if (!(j == in[s][k])) {
            in[s][k] = j;
            changed = true;
          }
        }
        if (changed && !queued[s]) {
          queued[s] = 1;
          work.push_back(s);
        }
      }
    }
    if (!work.empty())  // did not settle (cannot happen on this finite lattice): give up on everything
      for (auto &v : in)
        for (auto &f : v)
          if (f.kind == AF::AFF) f = top();
  }

  void regions() {
    const uint32_t n = (uint32_t)p.code.size();
    region.assign(n, 0);
    std::vector<uint32_t> entries{0};
    for (uint32_t pc = 0; pc < n; pc++)
      if (insn_class(p.code[pc]) == CC_BARRIER && pc + 1 < n) entries.push_back(pc + 1);
    if (entries.size() > 64) {  // more barrier regions than bits: every access may meet every other
      for (auto &r : region) r = ~0ull;
      return;
    }
    for (size_t e = 0; e < entries.size(); e++) {
      std::vector<uint32_t> st{entries[e]};
      while (!st.empty()) {
        const uint32_t pc = st.back();
        st.pop_back();
        if (pc >= n || (region[pc] >> e) & 1) continue;
        region[pc] |= 1ull << e;
        if (insn_class(p.code[pc]) == CC_BARRIER) continue;
        for (uint32_t s : succ(pc)) st.push_back(s);
      }
    }
  }

  // The forward "jump unless (a op imm)" instructions whose fall-through
  // region [b + 1, target) is entered only from b: no edge from outside the
  // region lands inside it (edges within it, loops included, are fine).
  void find_guards() {
    const uint32_t n = (uint32_t)p.code.size();
    std::vector<std::pair<uint32_t, uint32_t>> edges;
    for (uint32_t q = 0; q < n; q++)
      for (uint32_t s : succ(q)) edges.emplace_back(q, s);
    for (uint32_t b = 0; b < n; b++) {
      const Insn &in = p.code[b];
      if (in.op < OP_BFLTI || in.op > OP_BFNEI || insn_class(in) != CC_ALU ||
          ((in.ctl >> AL_MODE_SHIFT) & 3u) != 1u || (in.ctl & AL_LOOPCOND))
        continue;
      const uint32_t tgt = (uint32_t)in.imm2;
      if (tgt <= b + 1) continue;
      bool single_entry = true;
      for (const auto &e : edges)
        if ((e.first < b || e.first >= tgt) && e.second > b && e.second < tgt) {
          single_entry = false;
          break;
        }
      if (single_entry) guards.push_back(b);
    }
  }

  // Work-items that can reach pc: the launch, narrowed by the condition of
  // every guard whose region contains pc.  Guards are taken in program
  // order, so each one sits inside the regions of those before it and its
  // condition's form is exact on the box narrowed so far.
  Shape reach(uint32_t pc) const {
    Shape box = sh;
    for (uint32_t b : guards) {
      if (b >= pc) break;
      const Insn &in = p.code[b];
      if (pc < (uint32_t)in.imm2) restrict_box(box, this->in[b][in.a], (uint32_t)(in.op - OP_BFLTI), in.imm);
    }
    return box;
  }

  void index_form(const Insn &in, const std::vector<AF> &R, AF &f) const {
    const AF x = R[in.a];
    if (in.ctl & CTL_AM) {  // ((x + imm) mod 2^k) + imm2
      const uint32_t k = (in.ctl >> CTL_K_SHIFT) & 0x1Fu;
      f = add(x, konst(in.imm));
      if (f.kind != AF::AFF || !f.plain()) {
        f = top();
        return;
      }
      f.M = (int64_t)1 << k;
      f.off = in.imm2;
      return;
    }
    f = add(x, konst((int64_t)in.imm + in.imm2));
  }
};

}  // namespace
}  // namespace rc

namespace rc {

// The pre-filter over one launch shape.  out: the verdicts (see rc_prove);
// priv (if not null, one byte per instruction): 1 for a load or store that
// shares no cell with another work-item in its barrier interval, so that
// the cells it touches never carry a race or benign record:
//  * a store: every pair with an access of the same array that may meet it
//    in an interval (its own instruction included, run by another
//    work-item) is cleared by disjoint cells or a one-to-one index (or
//    cannot happen);
//  * a load: likewise every pair with a store; and no pair with another
//    load L' left open where L' itself has a store pair left open.
//    Otherwise a work-item t could read back its own store of a cell c
//    while another work-item reads c through L': the writers of c are then
//    {t} (the load's store pairs are cleared), but the cell carries a
//    read/write record that counts t's read.  If every load L' that may
//    meet the load has its store pairs cleared, no work-item reads a cell
//    another one writes through L', so no such record exists.
//  Equal values never clear a pair here.
// enum_budget: how many (work-item, loop counter) points the exact check of
// small launches may enumerate in all (0: none).
void prove_analyze(const Program &p, uint32_t groups, uint32_t group_size, const std::vector<uint32_t> &lens,
                   rc_prove_result *out, std::vector<uint8_t> *priv, uint64_t enum_budget) {
  uint64_t budget = enum_budget;
  Prover pr(p, Shape(group_size, groups), lens);
  pr.dataflow();
  pr.regions();
  pr.find_guards();
  std::vector<Acc> acc;
  for (uint32_t pc = 0; pc < p.code.size(); pc++) {
    const Insn &ins = p.code[pc];
    const uint32_t cls = insn_class(ins);
    if (cls != CC_LD && cls != CC_ST) continue;
    bool reached = false;
    for (const AF &f : pr.in[pc]) reached = reached || f.kind != AF::BOT;
    if (!reached) continue;
    Acc a;
    a.pc = pc;
    a.mem = ins.ctl >> CTL_MEM_SHIFT;
    a.store = cls == CC_ST;
    a.local = p.mems[a.mem].space != 0;
    a.box = pr.reach(pc);
    pr.index_form(ins, pr.in[pc], a.idx);
    if (!a.box.empty() && !exact(a.idx, a.box)) a.idx = top();
    a.val = a.store ? pr.in[pc][ins.b] : top();
    if (a.store && !a.box.empty() && !exact(a.val, a.box)) a.val = top();
    if (a.idx.kind == AF::AFF) a.ir = range_of(a.idx, a.box);
    if (a.val.kind == AF::AFF) a.vr = range_of(a.val, a.box);
    acc.push_back(a);
  }
  *out = rc_prove_result{};
  out->race_free = 1;
  out->in_bounds = 1;
  out->first_pc_a = out->first_pc_b = 0xFFFFFFFFu;
  if (priv) {
    priv->assign(p.code.size(), 0);
    for (const Acc &a : acc) (*priv)[a.pc] = 1;
  }
  for (const Acc &a : acc) {  // Table 1 bounds premise
    if (a.box.empty()) continue;  // no work-item gets there
    if (a.idx.kind != AF::AFF || a.ir.lo < 0 || a.ir.hi >= (int64_t)lens[a.mem]) out->in_bounds = 0;
  }
  std::vector<std::pair<uint32_t, uint32_t>> open_reads;  // load pairs that may share a cell
  for (size_t i = 0; i < acc.size(); i++)
    for (size_t j = i; j < acc.size(); j++) {
      const Acc &a = acc[i], &b = acc[j];
      if (a.mem != b.mem) continue;
      if (!(pr.region[a.pc] & pr.region[b.pc])) continue;
      const bool reads = !a.store && !b.store;
      if (reads && !priv) continue;
      if (!reads) out->n_pairs++;
      const Shape h = hull(a.box, b.box);
      // nobody executes one of them, or one work-item (per group, for local arrays) executes both
      bool ok = a.box.empty() || b.box.empty() || (h.nt() == 1 && (a.local || h.nw() == 1));
      if (!ok && a.idx.kind == AF::AFF && b.idx.kind == AF::AFF) {
        const Range &ra = a.ir, &rb = b.ir;
        ok = ra.hi < rb.lo || rb.hi < ra.lo;                            // disjoint cells
        ok = ok || (a.idx == b.idx && injective(a.idx, h, a.local));  // only with itself
        // small launches: every work-item's cells, enumerated
        ok = ok || (budget && never_meet(a.idx, a.box, b.idx, b.box, i == j, a.local, &budget) == 1);
      }
      if (reads) {
        if (!ok && i != j) open_reads.push_back({a.pc, b.pc});
        continue;
      }
      if (!ok && priv) (*priv)[a.pc] = (*priv)[b.pc] = 0;  // the two may share a cell
      if (!ok && a.store && b.store && a.val.kind == AF::AFF && b.val.kind == AF::AFF) {
        const Range &va = a.vr, &vb = b.vr;
        ok = va.lo == va.hi && vb.lo == vb.hi && va.lo == vb.lo;  // every writer stores one value: benign
      }
      if (!ok) {
        if (out->race_free) {
          out->first_pc_a = a.pc;
          out->first_pc_b = b.pc;
        }
        out->race_free = 0;
        out->n_unresolved++;
      }
    }
  if (priv) {
    const std::vector<uint8_t> store_pairs_clear = *priv;
    for (const auto &rr : open_reads) {
      if (!store_pairs_clear[rr.second]) (*priv)[rr.first] = 0;
      if (!store_pairs_clear[rr.first]) (*priv)[rr.second] = 0;
    }
  }
}

// per memory object: the input's length (global) or the declared one (local)
bool prove_lengths(const Program &p, const rc_input *in, std::vector<uint32_t> &lens) {
  if (in->n_global != p.n_global || (in->n_global && !in->global_len)) return false;
  lens.clear();
  uint32_t gi = 0;
  for (const MemDecl &m : p.mems)
    lens.push_back(m.space == 0 ? (uint32_t)std::min<uint64_t>(in->global_len[gi++], 0x7FFFFFFFu)
                                : (uint32_t)m.decl_len);
  return true;
}

}  // namespace rc

extern "C" int rc_prove(const rc_bytecode *bc, uint32_t groups, uint32_t group_size, const rc_input *in,
                        rc_prove_result *out) {
  using namespace rc;
  if (!bc || !in || !out || !groups || !group_size) {
    set_last_error("null argument or empty launch");
    return RC_E_INVALID;
  }
  std::vector<uint32_t> lens;
  if (!prove_lengths(bc->prog, in, lens)) {
    set_last_error("input count differs from the kernel's global declarations");
    return RC_E_INVALID;
  }
  prove_analyze(bc->prog, groups, group_size, lens, out, nullptr, 1u << 20);
  return RC_OK;
}

extern "C" int rc_prove_private(const rc_bytecode *bc, uint32_t groups, uint32_t group_size, const rc_input *in,
                                uint8_t *flags, uint32_t n_flags, uint32_t *n_private) {
  using namespace rc;
  if (!bc || !in || !flags || !n_private || !groups || !group_size || n_flags < bc->prog.code.size()) {
    set_last_error("null argument, empty launch or flag array shorter than the bytecode");
    return RC_E_INVALID;
  }
  std::vector<uint32_t> lens;
  if (!prove_lengths(bc->prog, in, lens)) {
    set_last_error("input count differs from the kernel's global declarations");
    return RC_E_INVALID;
  }
  rc_prove_result r;
  std::vector<uint8_t> priv;
  prove_analyze(bc->prog, groups, group_size, lens, &r, &priv, 0);  // as the checker does
  uint32_t n = 0;
  for (size_t k = 0; k < priv.size(); k++) {
    flags[k] = priv[k];
    n += priv[k];
  }
  *n_private = n;
  return RC_OK;
}

extern "C" int rc_access_sites(const rc_bytecode *bc, uint32_t *pc, uint8_t *is_store, uint32_t *mem, uint32_t cap,
                               uint32_t *n_sites) {
  using namespace rc;
  if (!bc || !n_sites || (cap && (!pc || !is_store || !mem))) {
    set_last_error("null argument");
    return RC_E_INVALID;
  }
  uint32_t n = 0;
  for (uint32_t k = 0; k < bc->prog.code.size(); k++) {
    const Insn &ins = bc->prog.code[k];
    const uint32_t cls = insn_class(ins);
    if (cls != CC_LD && cls != CC_ST) continue;
    if (n < cap) {
      pc[n] = k;
      is_store[n] = cls == CC_ST;
      mem[n] = ins.ctl >> CTL_MEM_SHIFT;
    }
    n++;
  }
  *n_sites = n;
  return RC_OK;
}
