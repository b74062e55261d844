// Features of candidate instances for the learned proposal.
//
// A candidate is (kernel, work-groups G, group size S, input).  Its feature
// vector has rc_features' fixed layout of RC_N_FEATURES floats:
//  * the kernel: opcode histogram, instruction / register / barrier counts;
//  * per access class (global load, global store, local load, local store):
//    how its index depends on tid and wg (uniform, tid only, through wg,
//    unknown), how many work-items reach it, whether a branch on a loaded
//    value guards it, whether the stored value varies between work-items,
//    and whether two work-items of this launch shape must meet on a cell;
//  * collisions seen when the accesses are evaluated for a sample of the
//    candidate's work-items on the candidate's input;
//  * the launch shape.
//
// The index and value of every access are found by one forward pass over the
// bytecode that keeps, per register, an affine form c0 + ct*tid + cw*wg
// (optionally reduced modulo M and offset), a loaded value (which access
// produced it), or "unknown".  Fused compare-and-branch instructions guard
// the code up to their target.  Loops are read once, their counters unknown
// afterwards.  The features only steer the order in which candidates are
// checked: every race the search reports comes from the exact checker.
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <functional>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "racecheck.h"
#include "bytecode.h"
#include "candidate_features.h"

namespace rc {
namespace {

struct Form {
  enum Kind : uint8_t { AFF, LOAD, TOP };
  Kind kind = TOP;
  int64_t c0 = 0, ct = 0, cw = 0;  // c0 + ct*tid + cw*wg
  int64_t M = 0;                   // > 0: the affine part is reduced modulo M (Euclidean)
  int64_t off = 0;                 // added after the reduction
  int32_t load = -1;               // LOAD: access that produced the value
  bool is_const() const { return kind == AFF && ct == 0 && cw == 0 && M == 0; }
  bool plain() const { return kind == AFF && M == 0; }
};

Form konst(int64_t v) {
  Form f;
  f.kind = Form::AFF;
  f.c0 = v;
  return f;
}
Form top() { return Form(); }

struct Guard {
  Form x;
  uint8_t op;   // 0 <, 1 <=, 2 >, 3 >=, 4 ==, 5 !=  (the condition that holds inside)
  bool neg;     // region of the else branch: the condition does not hold
  int64_t imm;
  uint32_t end; // first pc after the guarded region
};

struct Access {
  bool store;
  uint32_t mem, space;
  Form idx, val;
  std::vector<Guard> guards;
  uint32_t interval;
};

struct Analysis {
  std::vector<Access> acc;
};

Form add(const Form &a, const Form &b) {
  if (a.plain() && b.plain()) {
    Form f = a;
    f.c0 += b.c0;
    f.ct += b.ct;
    f.cw += b.cw;
    return f;
  }
  if (a.kind == Form::AFF && b.is_const()) {
    Form f = a;
    f.off += b.c0;
    return f;
  }
  if (b.kind == Form::AFF && a.is_const()) return add(b, a);
  return top();
}
Form scale(const Form &a, int64_t k) {
  if (!a.plain()) return top();
  Form f = a;
  f.c0 *= k;
  f.ct *= k;
  f.cw *= k;
  return f;
}
Form addc(const Form &a, int64_t c) { return add(a, konst(c)); }

// Forward pass over the bytecode for group size S (gtid = wg * S + tid).
Analysis analyse(const Program &p, uint32_t S, uint32_t G) {
  Analysis an;
  std::vector<Form> R(std::max<uint32_t>(p.n_regs, kBuiltinRegs));
  R[REG_TID].kind = Form::AFF;
  R[REG_TID].ct = 1;
  R[REG_WG].kind = Form::AFF;
  R[REG_WG].cw = 1;
  R[REG_GTID].kind = Form::AFF;
  R[REG_GTID].ct = 1;
  R[REG_GTID].cw = S;
  R[REG_GSIZE] = konst(S);
  R[REG_NGROUPS] = konst(G);
  std::vector<Guard> guards;
  uint32_t interval = 0;
  for (uint32_t pc = 0; pc < p.code.size(); pc++) {
    while (!guards.empty() && guards.back().end <= pc) guards.pop_back();
    const Insn &in = p.code[pc];
    const Form x = R[in.a], y = R[in.b];
    Form r = top();
    bool writes = true;
    switch (in.op) {
      case OP_MOVI: r = konst(in.imm); break;
      case OP_MOV: r = x; break;
      case OP_ADD: r = add(x, y); break;
      case OP_SUB: r = add(x, y.is_const() ? konst(-y.c0) : scale(y, -1)); break;
      case OP_MUL:
        r = y.is_const() ? scale(x, y.c0) : x.is_const() ? scale(y, x.c0) : top();
        break;
      case OP_ADDI: r = addc(x, in.imm); break;
      case OP_MULI: r = scale(x, in.imm); break;
      case OP_RSUBI: r = addc(scale(x, -1), in.imm); break;
      case OP_NEG: r = scale(x, -1); break;
      case OP_MADI: r = add(scale(x, in.imm), y); break;
      case OP_MODI:
        if (x.plain() && in.imm != 0) {
          r = x;
          r.M = std::llabs((long long)in.imm);
        }
        break;
      case OP_ANDI: {
        const uint64_t m = (uint64_t)(uint32_t)in.imm + 1;
        if (x.plain() && in.imm >= 0 && (m & (m - 1)) == 0) {
          r = x;
          r.M = (int64_t)m;
        }
        break;
      }
      case OP_LD:
      case OP_ST: {
        Access a;
        a.store = in.op == OP_ST;
        a.mem = in.ctl >> CTL_MEM_SHIFT;
        a.space = a.mem < p.mems.size() ? p.mems[a.mem].space : 0;
        if (in.ctl & CTL_AM) {
          const uint32_t k = (in.ctl >> CTL_K_SHIFT) & 0x1Fu;
          if (x.plain()) {
            a.idx = addc(x, in.imm);
            a.idx.M = (int64_t)1 << k;
            a.idx.off = in.imm2;
          }
        } else {
          a.idx = addc(x, (int64_t)in.imm + in.imm2);
        }
        a.val = a.store ? y : top();
        a.guards = guards;
        a.interval = interval;
        if (!a.store) {
          r.kind = Form::LOAD;
          r.load = (int32_t)an.acc.size();
        } else {
          writes = false;
        }
        an.acc.push_back(std::move(a));
        break;
      }
      case OP_BFLTI: case OP_BFLEI: case OP_BFGTI: case OP_BFGEI: case OP_BFEQI: case OP_BFNEI:
        writes = false;
        if ((uint32_t)in.imm2 > pc + 1)
          guards.push_back(Guard{x, (uint8_t)(in.op - OP_BFLTI), false, in.imm, (uint32_t)in.imm2});
        break;
      case OP_BZ:
        writes = false;
        if ((uint32_t)in.imm2 > pc + 1) guards.push_back(Guard{top(), 5, false, 0, (uint32_t)in.imm2});
        break;
      case OP_JMP:
        writes = false;
        // end of a then-branch that an else-branch follows: the else region
        // holds where the then-condition does not
        if ((uint32_t)in.imm2 > pc + 1 && !guards.empty() && guards.back().end == pc + 1) {
          Guard g = guards.back();
          g.neg = !g.neg;
          g.end = (uint32_t)in.imm2;
          guards.pop_back();
          guards.push_back(g);
        }
        break;
      case OP_BARRIER:
        writes = false;
        interval++;
        break;
      case OP_LOOP: r = top(); break;
      case OP_ASSUME: case OP_ASSERT: case OP_EXIT: case OP_NOP: writes = false; break;
      default: r = top(); break;
    }
    if (writes && in.d < R.size() && in.d >= kBuiltinRegs) R[in.d] = r;
  }
  return an;
}

struct Cand {
  const Program *p;
  uint32_t G, S;
  std::vector<const int32_t *> gdata;  // per memory object: input (global) or null (local)
  std::vector<uint64_t> len;           // per memory object
  std::vector<uint64_t> base;          // per memory object: first cell in its space
};

int64_t eval(const Form &f, int64_t tid, int64_t wg, const Analysis &an, const Cand &c, bool &known);

int64_t eval_aff(const Form &f, int64_t tid, int64_t wg) {
  int64_t v = f.c0 + f.ct * tid + f.cw * wg;
  if (f.M > 0) {  // Euclidean remainder
    v %= f.M;
    if (v < 0) v += f.M;
  }
  return v + f.off;
}

// value the access's load observes: the input (global) or 0 (local) at its index
int64_t eval(const Form &f, int64_t tid, int64_t wg, const Analysis &an, const Cand &c, bool &known) {
  if (f.kind == Form::AFF) return eval_aff(f, tid, wg);
  if (f.kind == Form::LOAD && f.load >= 0) {
    const Access &a = an.acc[f.load];
    bool k2 = true;
    const int64_t i = eval(a.idx, tid, wg, an, c, k2);
    if (!k2 || i < 0 || (uint64_t)i >= c.len[a.mem]) {
      known = false;
      return 0;
    }
    if (a.space == 0 && c.gdata[a.mem]) return c.gdata[a.mem][i];
    return 0;
  }
  known = false;
  return 0;
}

bool holds(const Guard &g, int64_t tid, int64_t wg, const Analysis &an, const Cand &c, bool &certain) {
  bool known = true;
  const int64_t x = eval(g.x, tid, wg, an, c, known);
  if (!known) {
    certain = false;
    return true;
  }
  bool r;
  switch (g.op) {
    case 0: r = x < g.imm; break;
    case 1: r = x <= g.imm; break;
    case 2: r = x > g.imm; break;
    case 3: r = x >= g.imm; break;
    case 4: r = x == g.imm; break;
    default: r = x != g.imm; break;
  }
  return r != g.neg;
}

bool enabled(const Access &a, int64_t tid, int64_t wg, const Analysis &an, const Cand &c, bool &certain) {
  for (const Guard &g : a.guards)
    if (!holds(g, tid, wg, an, c, certain)) return false;
  return true;
}

bool data_guarded(const Access &a) {
  for (const Guard &g : a.guards)
    if (g.x.kind != Form::AFF) return true;
  return false;
}

int64_t gcd64(int64_t a, int64_t b) {
  a = std::llabs((long long)a);
  b = std::llabs((long long)b);
  while (b) {
    const int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

struct Ev {  // one evaluated access of one sampled work-item
  uint64_t cell;  // space, (wg for local), flat index
  uint32_t gtid;
  int64_t val;
  bool store, vknown;
  uint32_t interval;
};

float lg(double x) { return (float)std::log2(1.0 + x); }

void features_one(const Cand &c, float *out) {
  const Program &p = *c.p;
  std::fill(out, out + RC_N_FEATURES, 0.0f);
  const uint32_t S = c.S, G = c.G;
  const uint64_t N = (uint64_t)S * G;
  const double n_insn = (double)std::max<size_t>(p.code.size(), 1);
  for (const Insn &in : p.code)
    if (in.op < 52) out[in.op] += (float)(1.0 / n_insn);
  out[52] = lg(n_insn) / 10.0f;
  out[53] = p.n_barriers / 8.0f;
  out[54] = lg(p.n_regs) / 6.0f;
  out[55] = p.mems.size() / 4.0f;

  const Analysis an = analyse(p, S, G);
  // work-item sample: all of them when few, else both ends and an even spread
  // -- 256 in all, fewer for long programs so that a candidate evaluates at
  // most about kEvalBudget accesses (at least 32 work-items): the ranking
  // must cost less than the checks it saves
  constexpr uint64_t kEvalBudget = 4096;
  const uint64_t n_acc = std::max<uint64_t>(an.acc.size(), 1);
  const uint32_t m = (uint32_t)std::max<uint64_t>(32, std::min<uint64_t>(256, (kEvalBudget / n_acc) & ~(uint64_t)3));
  std::vector<uint32_t> smp;
  if (N <= m) {
    smp.resize(N);
    std::iota(smp.begin(), smp.end(), 0u);
  } else {
    const uint32_t q = m / 4;
    for (uint32_t i = 0; i < q; i++) smp.push_back(i);
    for (uint32_t i = 0; i < q; i++) smp.push_back((uint32_t)(N - q + i));
    for (uint32_t i = 0; i < m / 2; i++) smp.push_back((uint32_t)((N * (2 * i + 1)) / m));
    std::sort(smp.begin(), smp.end());
    smp.erase(std::unique(smp.begin(), smp.end()), smp.end());
  }
  const double scale = (double)N / smp.size();
  // each sampled work-item's (tid, wg), once for every access
  thread_local std::vector<int64_t> smp_tid, smp_wg;
  smp_tid.resize(smp.size());
  smp_wg.resize(smp.size());
  for (size_t i = 0; i < smp.size(); i++) {
    smp_tid[i] = smp[i] % S;
    smp_wg[i] = smp[i] / S;
  }

  thread_local std::vector<Ev> evs;
  evs.clear();
  struct ClassAcc {
    double n = 0, uni = 0, tido = 0, wgi = 0, unk = 0, en = 0, dg = 0, maxen = 0, vv = 0, col = 0, race = 0, oob = 0;
  } cls[4];
  bool any_pred = false;
  for (const Access &a : an.acc) {
    const int k = (a.space ? 2 : 0) + (a.store ? 1 : 0);
    ClassAcc &C = cls[k];
    C.n += 1;
    const Form &f = a.idx;
    const bool known_idx = f.kind == Form::AFF;
    if (!known_idx) C.unk += 1;
    else if (f.ct == 0 && f.cw == 0) C.uni += 1;
    else if (f.cw == 0) C.tido += 1;
    else C.wgi += 1;
    const bool dg = data_guarded(a);
    if (dg) C.dg += 1;
    const bool vvar = a.store && !(a.val.kind == Form::AFF && a.val.ct == 0 && a.val.cw == 0 && a.val.M == 0);
    if (vvar) C.vv += 1;
    // enabled work-items in the sample; enabled tids of the first enabled group, groups of the first tid
    uint64_t en = 0, oob = 0;
    int64_t first_wg = -1, first_tid = -1;
    for (size_t si = 0; si < smp.size(); si++) {
      const uint32_t g = smp[si];
      const int64_t tid = smp_tid[si], wg = smp_wg[si];
      bool certain = true;
      if (!enabled(a, tid, wg, an, c, certain)) continue;
      en++;
      if (first_wg < 0) {
        first_wg = wg;
        first_tid = tid;
      }
      bool ki = true, kv = true;
      const int64_t idx = eval(f, tid, wg, an, c, ki);
      if (!ki) continue;
      if (idx < 0 || (uint64_t)idx >= c.len[a.mem]) {
        oob++;
        continue;
      }
      const int64_t v = a.store ? eval(a.val, tid, wg, an, c, kv) : 0;
      uint64_t cell = c.base[a.mem] + (uint64_t)idx;
      if (a.space) cell |= ((uint64_t)wg + 1) << 40;
      evs.push_back(Ev{cell, g, v, a.store, kv, a.interval});
    }
    const double frac = smp.empty() ? 0.0 : (double)en / smp.size();
    C.en += frac;
    const double n_en = en * scale;
    C.maxen = std::max(C.maxen, (double)lg(n_en) / 16.0);
    if (en) C.oob += (double)oob / en;
    // work-items of the first enabled group that reach the access (counted
    // over at most 64 of them spread evenly, then scaled to the group), and
    // groups of its first work-item that do, counted as far as 2
    auto group_items = [&]() {
      const uint32_t n_t = std::min<uint32_t>(S, 64);
      uint64_t k = 0;
      for (uint32_t i = 0; i < n_t; i++) {
        const int64_t t = S <= 64 ? i : ((int64_t)S * (2 * i + 1)) / 128;
        bool certain = true;
        if (enabled(a, t, first_wg, an, c, certain)) k++;
      }
      return (double)k * S / n_t;
    };
    auto item_groups = [&](uint64_t limit) {  // G <= 64
      uint64_t k = 0;
      for (int64_t w = 0; w < G && k <= limit; w++) {
        bool certain = true;
        if (enabled(a, first_tid, w, an, c, certain)) k++;
      }
      return k;
    };
    // must two work-items meet on a cell?
    bool col = false, race = false;
    if (known_idx && n_en >= 2) {
      const bool v_tid = !a.store || a.val.kind != Form::AFF || a.val.ct != 0 || a.val.M != 0;
      const bool v_wg = !a.store || a.val.kind != Form::AFF || a.val.cw != 0;
      if (f.ct == 0 && f.cw == 0) {  // one cell for everybody
        col = true;
        race = a.store && vvar;
      } else if (f.ct == 0) {  // depends on wg only: a whole group on one cell
        if (group_items() >= 2) {
          col = true;
          race = a.store && v_tid;
        }
      } else if (f.cw == 0) {  // depends on tid only
        if (a.space == 0 && item_groups(1) >= 2) {
          col = true;
          race = race || (a.store && v_wg);
        }
        if (f.M > 0 && f.M / gcd64(f.ct, f.M) < (int64_t)S && group_items() > (double)(f.M / gcd64(f.ct, f.M))) {
          col = true;
          race = race || (a.store && v_tid);
        }
      } else if (f.M > 0) {
        const int64_t g = gcd64(gcd64(f.ct, f.cw), f.M);
        if (f.cw == f.ct * (int64_t)S && (double)n_en > (double)f.M / gcd64(f.ct, f.M)) col = true;
        else if (n_en > (double)f.M / g) col = true;
        race = col && a.store && vvar;
      }
    }
    if (col) C.col += 1;
    if (race) C.race += 1;
    any_pred = any_pred || race;
  }
  for (int k = 0; k < 4; k++) {
    const ClassAcc &C = cls[k];
    float *o = out + 56 + 12 * k;
    const double n = std::max(C.n, 1.0);
    o[0] = lg(C.n) / 5.0f;
    o[1] = (float)(C.uni / n);
    o[2] = (float)(C.tido / n);
    o[3] = (float)(C.wgi / n);
    o[4] = (float)(C.unk / n);
    o[5] = (float)(C.en / n);
    o[6] = (float)(C.dg / n);
    o[7] = (float)C.maxen;
    o[8] = (float)(C.vv / n);
    o[9] = (float)(C.col / n);
    o[10] = (float)(C.race / n);
    o[11] = (float)(C.oob / n);
  }
  // collisions among the sampled work-items, per interval and cell: one
  // pass over the events in evaluation order (access by access, work-items
  // in sample order) into a table of cells (open addressing over indices
  // into the list of cells met)
  struct CellAcc {
    uint64_t cell;
    uint32_t interval;
    bool wrace, wben, two_readers;
    int64_t w0g, w0v, w1g, r0;
  };
  thread_local std::vector<CellAcc> cells;
  thread_local std::vector<uint32_t> tab;
  size_t cap = 16;
  while (cap < 2 * evs.size()) cap <<= 1;
  tab.assign(cap, 0xFFFFFFFFu);
  cells.clear();
  for (const Ev &e : evs) {
    size_t h = (size_t)(((e.cell ^ ((uint64_t)e.interval << 52)) * 0x9E3779B97F4A7C15ull) >> 20) & (cap - 1);
    while (tab[h] != 0xFFFFFFFFu && (cells[tab[h]].cell != e.cell || cells[tab[h]].interval != e.interval))
      h = (h + 1) & (cap - 1);
    if (tab[h] == 0xFFFFFFFFu) {
      tab[h] = (uint32_t)cells.size();
      cells.push_back(CellAcc{e.cell, e.interval, false, false, false, -1, 0, -1, -1});
    }
    CellAcc &t = cells[tab[h]];
    const int64_t g = (int64_t)e.gtid;
    if (e.store) {
      // writers: the first writer's value against the others' (other work-items)
      if (t.w0g < 0) {
        t.w0g = g;
        t.w0v = e.val;
      } else if (g != t.w0g) {
        if (t.w1g < 0) t.w1g = g;
        if (!e.vknown || e.val != t.w0v) t.wrace = true;
        else t.wben = true;
      }
    } else if (t.r0 < 0) {
      t.r0 = g;
    } else if (g != t.r0) {
      t.two_readers = true;
    }
  }
  double ww = 0, rw = 0, benign = 0;
  for (const CellAcc &t : cells) {
    if (t.w0g < 0) continue;
    // a read meets a write by another work-item (the value it observes is
    // unknown here: any other writer may differ): with two distinct writers
    // every read does; with one, a read by anyone else does
    const bool rrace = t.r0 >= 0 && (t.w1g >= 0 || t.two_readers || t.r0 != t.w0g);
    ww += t.wrace;
    benign += t.wben && !t.wrace;
    rw += rrace;
  }
  out[104] = lg(ww) / 10.0f;
  out[105] = lg(rw) / 10.0f;
  out[106] = lg(benign) / 10.0f;
  out[107] = (ww + rw) > 0 ? 1.0f : 0.0f;
  out[108] = any_pred ? 1.0f : 0.0f;
  out[109] = (float)std::log2((double)S) / 10.0f;
  out[110] = (float)std::log2((double)G) / 6.0f;
  out[111] = (float)std::log2((double)N) / 16.0f;
  out[112] = S / 1024.0f;
  out[113] = G / 64.0f;
  out[114] = (float)(N / 65536.0);
  out[115] = (float)smp.size() / (float)N;
  out[116] = (p.n_barriers + 1) / 9.0f;
}

Cand make_cand(const rc_bytecode *bc, uint32_t G, uint32_t S, const rc_input *in) {
  if (!bc || !in || G == 0 || S == 0 || S > 1024) throw std::string("bad arguments");
  if (in->on_device) throw std::string("features read host inputs only");
  const Program &p = bc->prog;
  if (in->n_global != p.n_global) throw std::string("input count differs from the kernel's global declarations");
  Cand c;
  c.p = &p;
  c.G = G;
  c.S = S;
  uint32_t gi = 0;
  uint64_t gb = 0, lb = 0;
  for (const MemDecl &m : p.mems) {
    if (m.space == 0) {
      c.gdata.push_back(in->global_init ? in->global_init[gi] : nullptr);
      c.len.push_back(in->global_len[gi]);
      c.base.push_back(gb);
      gb += in->global_len[gi];
      gi++;
    } else {
      c.gdata.push_back(nullptr);
      c.len.push_back((uint64_t)m.decl_len);
      c.base.push_back(lb);
      lb += (uint64_t)m.decl_len;
    }
  }
  return c;
}

// Worker threads of the library, started on first use (one fewer than the
// host's cores) and kept for the life of the process, so that a search pays
// no thread start-up per kernel.  A process forked after they started gets a
// pool of its own.
class Pool {
 public:
  explicit Pool(unsigned n) : pid_(getpid()) {
    for (unsigned i = 0; i < n; i++) std::thread([this] { loop(); }).detach();
    size_ = n;
  }
  unsigned size() const { return size_; }
  pid_t pid() const { return pid_; }
  void submit(std::function<void()> f) {
    {
      std::lock_guard<std::mutex> lk(mu_);
      q_.push_back(std::move(f));
    }
    cv_.notify_one();
  }

 private:
  void loop() {
    for (;;) {
      std::function<void()> f;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return !q_.empty(); });
        f = std::move(q_.front());
        q_.pop_front();
      }
      f();
    }
  }
  std::mutex mu_;
  std::condition_variable cv_;
  std::deque<std::function<void()>> q_;
  unsigned size_ = 0;
  pid_t pid_;
};

Pool &pool() {
  static std::mutex mu;
  static Pool *p = nullptr;  // never destroyed: its threads outlive static destructors
  std::lock_guard<std::mutex> lk(mu);
  if (!p || p->pid() != getpid()) {
    const unsigned hw = std::max(2u, std::thread::hardware_concurrency());
    p = new Pool(hw - 1);
  }
  return *p;
}

}  // namespace

struct FeatureJob {
  size_t n = 0;
  std::function<void(size_t)> one;  // features of candidate i
  std::atomic<size_t> next{0}, finished{0};
  std::atomic<unsigned> active{0};
  std::atomic<bool> cancelled{false}, failed{false};
  std::string error;
  std::mutex mu;
  std::condition_variable cv;

  // takes candidates until none is left; the last thread out wakes the waiter
  void work() {
    active.fetch_add(1);
    for (;;) {
      const size_t i = next.fetch_add(1);
      if (i >= n || cancelled.load(std::memory_order_relaxed)) break;
      try {
        one(i);
      } catch (...) {
        std::lock_guard<std::mutex> lk(mu);
        if (!failed.exchange(true)) error = "feature extraction failed (host memory)";
      }
      finished.fetch_add(1);
    }
    std::lock_guard<std::mutex> lk(mu);
    active.fetch_sub(1);
    cv.notify_all();
  }
  bool done() const { return finished.load() == n; }
};

std::shared_ptr<FeatureJob> features_start(const rc_bytecode *const *bcs, const uint32_t *groups,
                                           const uint32_t *group_size, const rc_input *inputs, size_t n,
                                           float *out, unsigned participants, bool caller_helps) {
  auto cands = std::make_shared<std::vector<Cand>>();
  cands->reserve(n);
  for (size_t i = 0; i < n; i++) cands->push_back(make_cand(bcs[i], groups[i], group_size[i], &inputs[i]));
  auto job = std::make_shared<FeatureJob>();
  job->n = n;
  job->one = [cands, out](size_t i) { features_one((*cands)[i], out + i * RC_N_FEATURES); };
  // one thread per 8 candidates at most: handing a candidate to a thread
  // costs about as much as a few candidates' features
  Pool &P = pool();
  unsigned nt = participants ? participants : std::max<unsigned>(1, (unsigned)std::min<size_t>(n / 8, P.size() + 1));
  nt = (unsigned)std::min<size_t>(nt, std::max<size_t>(n, 1));
  const unsigned workers = std::min(P.size(), caller_helps ? nt - 1 : std::max(nt, 1u));
  for (unsigned w = 0; w < workers; w++) P.submit([job] { job->work(); });
  return job;
}

bool features_finished(const FeatureJob &j) { return j.done(); }

void features_cancel(FeatureJob &j) { j.cancelled.store(true); }

void features_wait(FeatureJob &j) {
  j.work();  // the caller's share (nothing left when the workers took it all)
  std::unique_lock<std::mutex> lk(j.mu);
  j.cv.wait(lk, [&] { return j.active.load() == 0 && (j.done() || j.cancelled.load()); });
  if (j.failed.load()) throw j.error;
}

}  // namespace rc

extern "C" {

int rc_features(const rc_bytecode *bc, uint32_t groups, uint32_t group_size, const rc_input *in, float *out) {
  return rc_features_batch(&bc, &groups, &group_size, in, 1, out, 1);
}

int rc_features_batch(const rc_bytecode *const *bcs, const uint32_t *groups, const uint32_t *group_size,
                      const rc_input *inputs, size_t n, float *out, int n_threads) {
  using namespace rc;
  if (n && (!bcs || !groups || !group_size || !inputs || !out)) {
    set_last_error("null argument");
    return RC_E_INVALID;
  }
  try {
    auto job = features_start(bcs, groups, group_size, inputs, n, out, n_threads > 0 ? (unsigned)n_threads : 0u,
                              true);
    features_wait(*job);
  } catch (const std::string &e) {
    set_last_error(e);
    return RC_E_INVALID;
  } catch (const std::bad_alloc &) {
    set_last_error("out of host memory");
    return RC_E_NOMEM;
  }
  return RC_OK;
}

}  // extern "C"
