// ORACLE (test infrastructure only): plain sequential race checker.
//
// Only the test suite, __graft_entry__.smoke() and bench.py's CPU baseline
// leg may build, load or call this file.  It shares no code with the GPU
// path.  It is written for obviousness, not speed: threads run one after the
// other, every shared access of an interval goes into one list (grouped by
// cell with a sort that keeps their order within a cell), and conflicts are
// classified by looking at the logged accesses of each cell directly.
//
// What it computes (Distefano & Dubreil, Sec. 4 "Concrete Semantics" and the
// race Definition that closes it):
//   * thread-local rules of Sec. 4 for v:=e, a[v]:=e, v:=a[v], assert,
//     assume and barrier, with ⊥ for out-of-bounds accesses (Table 1's
//     bounds premise) and failed asserts, ⊤ for a failed assume;
//   * global semantics of Sec. 4: all threads of the kernel run to the same
//     barrier (the barrier-release rule), the end of the kernel being an
//     implicit barrier;
//   * the race rule of Sec. 4 / Sec. 1: a barrier interval is racy when the
//     shared state it produces is not the same for every schedule; several
//     threads writing one value to a cell is benign.
// Readings where the paper is silent (one canonical run instead of every
// schedule, per-thread last writes, read/write conflicts, witnesses, commit
// order, arithmetic) are the ones listed in the project's design notes; each
// is restated next to the code that implements it below.
//
// Work-group-scoped barriers (OpenCL's barrier, against the paper's
// kernel-wide one of Sec. 2 / Sec. 4): the same lock-step run (round k runs
// every group's k-th interval, which is one legal schedule when a barrier
// only waits for its own group), but the barrier-release rule is applied to
// each work-group on its own -- groups may stop at different barriers, and
// a group whose work-items all exited is finished while others go on -- and,
// since no barrier orders work-items of different groups, every global cell
// is also classified over the whole run between groups (run_cross_group).
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "kl_frontend.hpp"

namespace orc {

enum Cls : uint32_t {
  C_WW_RACE = 1, C_WW_BENIGN = 2, C_RW_RACE = 3,
  C_XG_WW_RACE = 4, C_XG_WW_BENIGN = 5, C_XG_RW_RACE = 6,
  C_OOB = 16, C_ASSERT = 17, C_DIVERGENCE = 18
};
enum Status : int32_t {
  ST_RACE_FREE = 0, ST_RACY = 1, ST_OOB = 2, ST_ASSERT = 3, ST_DIVERGENCE = 4
};

struct Record {  // 10 x u32, field order fixed so reports compare bytewise
  uint32_t interval, space, wg, addr, cls, t_a, t_b, n_readers, n_writers, n_accesses;
};

struct Report {
  int32_t status = ST_RACE_FREE;
  uint32_t n_intervals = 0;
  uint64_t n_access = 0, n_global = 0, n_local = 0;
  uint64_t max_acc = 0, max_wr = 0;  // most accesses / writes of one thread in one interval
  std::vector<Record> records;
  std::vector<int32_t> final_global;
  // trace mode: every performed shared access as (interval, gtid, space, wg,
  // addr, write, site, value: stored or loaded); site k is the k-th
  // load/store command of the kernel in text order, sites[k] = (write,
  // memory object)
  std::vector<uint32_t> trace;
  std::vector<uint32_t> sites;
};

struct Access {
  uint32_t gtid;
  bool write;
  int32_t value;  // value written, or value the read observed
};

// A shared cell: (space, work-group for local memory, flat address in space).
using Cell = std::tuple<uint32_t, uint32_t, uint32_t>;

enum TStatus { RUNNING, AT_BARRIER, EXITED, DEAD };
struct Thread {
  int node;  // node to execute next (AT_BARRIER: the barrier node)
  TStatus st;
};

// One logged access: its cell, the order it was logged in, what it did.
struct Logged {
  uint32_t space, wg, addr, order;
  Access a;
};

struct Checker {
  Program prog;
  Cfg cfg;
  uint32_t G, S;
  std::vector<int64_t> mem_len;   // per memory object
  std::vector<uint64_t> mem_base; // flat base inside its space
  uint64_t global_total = 0, local_total = 0;
  std::vector<int32_t> global_snap;  // committed global memory
  std::vector<int32_t> local_snap;   // committed local memory, G x local_total
  std::vector<Thread> th;
  // Named private variables, work-item major (N x n_named).  The front end's
  // temporaries (one per array read inside an expression) are written by
  // their load just before the statement that reads them and never live
  // across a barrier, so a work-item runs on a scratch copy of all
  // cfg.n_vars and only the named ones are kept between intervals.
  uint32_t n_named = 0;
  std::vector<int32_t> vars, scratch;
  Report rep;
  bool group_scope = false;
  std::map<uint32_t, std::vector<Access>> whole_run;  // group scope: every access to each global cell
  // Address sharding (for instances too large to log whole): shard p of P
  // logs and classifies only the cells with cell_hash % P == p; for every
  // other cell it keeps just the write to commit (the highest writer's last
  // one), so the run itself is the full run.  Only shard 0 reports errors.
  // The union of the P reports' race records, in report order, with shard
  // 0's error records is the unsharded report.
  uint32_t shard = 0, n_shards = 1;
  // the write to commit of each of other shards' cells: local cells in a map,
  // global cells in arrays indexed by address (with the list of those touched)
  std::map<Cell, std::pair<uint32_t, int32_t>> pending;
  std::vector<uint32_t> pend_writer, pend_touched;
  std::vector<int32_t> pend_value;
  bool mine(const Cell &c) const {
    if (n_shards == 1) return true;
    const uint32_t h = std::get<2>(c) * 0x9E3779B1u ^ std::get<1>(c) * 0x85EBCA77u ^ std::get<0>(c);
    return h % n_shards == shard;
  }
  std::vector<int32_t> initial_global;                // global memory before the run
  bool tracing = false;
  std::vector<uint32_t> site_of;                       // CFG node -> site ordinal (trace mode)

  // per interval: every logged access in the order it happened (grouped by
  // cell at the interval's end, keeping that order within a cell)
  std::vector<Logged> log;
  std::vector<Record> errors;

  int32_t committed(const Cell &c) const {
    if (std::get<0>(c) == 0) return global_snap[std::get<2>(c)];
    return local_snap[(uint64_t)std::get<1>(c) * local_total + std::get<2>(c)];
  }
  void commit_cell(const Cell &c, int32_t v) {
    if (std::get<0>(c) == 0) global_snap[std::get<2>(c)] = v;
    else local_snap[(uint64_t)std::get<1>(c) * local_total + std::get<2>(c)] = v;
  }

  // Choose the successor of node k: one successor is taken as is; several
  // successors are assume-guarded alternatives, of which the one whose
  // condition holds is taken.  None holding means the path has no
  // continuation (⊤), returned as -1.
  int next_node(int k, const Env &env) const {
    const Node &n = cfg.nodes[k];
    if (n.succ.size() == 1) return n.succ[0];
    for (int s : n.succ) {
      const Node &c = cfg.nodes[s];
      if (eval(*c.val, env) != 0) return s;
    }
    return -1;
  }

  // Run one thread from its current node to a barrier, exit or abort.
  // Reads see the thread's own latest write of this interval if it made one,
  // else the value committed at the last barrier (delayed visibility).
  void run_thread(uint32_t gtid, uint32_t interval) {
    Thread &t = th[gtid];
    const uint32_t wg = gtid / S, tid = gtid % S;
    int32_t *const kept = vars.data() + (uint64_t)gtid * n_named;
    int32_t *const my_vars = scratch.data();
    std::copy(kept, kept + n_named, my_vars);
    struct KeepNamed {  // copy the named variables back however the run ends
      int32_t *from, *to;
      uint32_t n;
      ~KeepNamed() { std::copy(from, from + n, to); }
    } keep_named{my_vars, kept, n_named};
    Env env{my_vars, tid, wg, S, G, &mem_len};
    std::map<Cell, int32_t> own;  // this thread's writes in this interval
    uint64_t nacc = 0, nwr = 0;
    struct Tally {  // record this thread's counts however the run ends
      Report &r; uint64_t &a, &w;
      ~Tally() { r.max_acc = std::max(r.max_acc, a); r.max_wr = std::max(r.max_wr, w); }
    } tally{rep, nacc, nwr};
    int k = t.node;
    if (t.st == AT_BARRIER) {  // resume after the barrier it waited at
      t.st = RUNNING;
      k = next_node(k, env);
      if (k < 0) { t.st = DEAD; return; }
    }
    for (;;) {
      const Node &n = cfg.nodes[k];
      switch (n.kind) {
        case N_START:
        case N_NOP:
          break;
        case N_EXIT:
          t.st = EXITED;
          t.node = k;
          return;
        case N_BARRIER:
          t.st = AT_BARRIER;
          t.node = k;
          return;
        case N_ASSIGN:
          my_vars[n.var] = eval(*n.val, env);
          break;
        case N_ASSUME:
          if (eval(*n.val, env) == 0) { t.st = DEAD; return; }  // ⊤
          break;
        case N_ASSERT:
          if (eval(*n.val, env) == 0) {  // ⊥
            errors.push_back({interval, 0, 0, 0, C_ASSERT, gtid, (uint32_t)n.id, 0, 0, 0});
            t.st = DEAD;
            return;
          }
          break;
        case N_LOAD:
        case N_STORE: {
          const Mem &m = prog.mems[n.mem];
          int32_t idx = eval(*n.idx, env);
          int32_t val = 0;
          if (n.kind == N_STORE) val = eval(*n.val, env);
          if (idx < 0 || (int64_t)idx >= mem_len[n.mem]) {  // ⊥: out of bounds
            errors.push_back({interval, (uint32_t)m.space, m.space ? wg : 0u, (uint32_t)idx,
                              C_OOB, gtid, (uint32_t)n.mem, 0, 0, 0});
            t.st = DEAD;
            return;
          }
          Cell c{(uint32_t)m.space, m.space ? wg : 0u, (uint32_t)(mem_base[n.mem] + (uint64_t)idx)};
          const size_t at = rep.trace.size();
          if (tracing)
            rep.trace.insert(rep.trace.end(), {interval, gtid, std::get<0>(c), std::get<1>(c), std::get<2>(c),
                                               n.kind == N_STORE ? 1u : 0u, site_of[k], (uint32_t)val});
          if (n.kind == N_STORE) {
            own[c] = val;
            if (mine(c)) {
              log.push_back({std::get<0>(c), std::get<1>(c), std::get<2>(c), (uint32_t)log.size(), {gtid, true, val}});
            } else if (std::get<0>(c) == 0) {  // another shard's global cell: only what the commit needs
              const uint32_t addr = std::get<2>(c);
              if (pend_writer[addr] == 0xFFFFFFFFu) pend_touched.push_back(addr);
              if (pend_writer[addr] == 0xFFFFFFFFu || gtid >= pend_writer[addr]) {
                pend_writer[addr] = gtid;
                pend_value[addr] = val;
              }
            } else {  // another shard's local cell
              auto it = pending.find(c);
              if (it == pending.end() || gtid >= it->second.first) pending[c] = {gtid, val};
            }
          } else {
            auto it = own.find(c);
            int32_t v = it != own.end() ? it->second : committed(c);
            if (tracing) rep.trace[at + 7] = (uint32_t)v;
            if (mine(c))
              log.push_back({std::get<0>(c), std::get<1>(c), std::get<2>(c), (uint32_t)log.size(), {gtid, false, v}});
            my_vars[n.var] = v;
          }
          rep.n_access++;
          nacc++;
          if (n.kind == N_STORE) nwr++;
          if (m.space == 0) rep.n_global++;
          else rep.n_local++;
          break;
        }
      }
      k = next_node(k, env);
      if (k < 0) { t.st = DEAD; return; }
    }
  }

  // Classify the accesses of one cell in one interval.
  //  * WW: take each writer thread's LAST write to the cell.  Two writers
  //    whose last values differ: WW_RACE, witness (smallest writer, smallest
  //    writer whose last value differs from it).  Two or more writers, all
  //    last values equal: WW_BENIGN, witness (two smallest writers).
  //  * RW: a read by thread r that observed o conflicts with a write of
  //    value v != o by another thread j.  Witness: the lexicographically
  //    smallest such (r, j).
  void classify_cell(uint32_t interval, const Cell &c, const std::vector<Access> &acc) {
    std::map<uint32_t, std::vector<int32_t>> writes, reads;  // per thread, program order
    for (const Access &a : acc) (a.write ? writes : reads)[a.gtid].push_back(a.value);
    Record base{interval, std::get<0>(c), std::get<1>(c), std::get<2>(c), 0, 0, 0,
                (uint32_t)reads.size(), (uint32_t)writes.size(), (uint32_t)acc.size()};
    if (writes.size() >= 2) {
      uint32_t w1 = writes.begin()->first;
      int32_t l1 = writes.begin()->second.back();
      bool race = false;
      uint32_t tb = 0;
      for (auto &w : writes) {
        if (w.second.back() != l1) { race = true; tb = w.first; break; }
      }
      Record r = base;
      if (race) { r.cls = C_WW_RACE; r.t_a = w1; r.t_b = tb; }
      else { r.cls = C_WW_BENIGN; r.t_a = w1; r.t_b = std::next(writes.begin())->first; }
      rep.records.push_back(r);
    }
    if (!reads.empty() && !writes.empty()) {
      // conflict(r, j) <=> some observed o of r and some written v of j differ
      // <=> not (r observed exactly one value c and j wrote only c).
      std::map<uint32_t, std::set<int32_t>> wset;
      for (auto &w : writes) wset[w.first] = std::set<int32_t>(w.second.begin(), w.second.end());
      bool found = false;
      uint32_t best_r = 0, best_j = 0;
      for (auto &rd : reads) {  // ascending reader
        std::set<int32_t> obs(rd.second.begin(), rd.second.end());
        for (auto &w : wset) {  // ascending writer
          if (w.first == rd.first) continue;
          bool same = obs.size() == 1 && w.second.size() == 1 && *obs.begin() == *w.second.begin();
          if (!same) { found = true; best_j = w.first; break; }
        }
        if (found) { best_r = rd.first; break; }
      }
      if (found) {
        Record r = base;
        r.cls = C_RW_RACE;
        r.t_a = best_r;
        r.t_b = best_j;
        rep.records.push_back(r);
      }
    }
  }

  // Group scope: classify each global cell over the whole run between
  // work-items of different groups (no barrier orders them).
  //  * XG WW: writers in two or more groups.  XG_WW_BENIGN when every write
  //    to the cell stored one value, else XG_WW_RACE; witness (smallest
  //    writer, largest writer).
  //  * XG RW: a reader and a writer in different groups, unless the cell
  //    held one value all along: its value before the run, every value
  //    written and every value the reads observed are one and the same (a
  //    read by another group may come before or after any write).
  //    Witness, from the smallest/largest reader r0/r1 and writer w0/w1:
  //    (r0, w0) if their groups differ, else (r0, w1) if those differ, else
  //    (r1, w0).
  //  Counts: n_readers = reads, n_writers = writes, n_accesses = both.
  void run_cross_group() {
    for (auto &kv : whole_run) {
      std::set<uint32_t> wgw, wgr;
      std::set<int32_t> written, seen;
      uint32_t w0 = 0, w1 = 0, r0 = 0, r1 = 0, nrd = 0, nwr = 0;
      for (const Access &a : kv.second) {
        if (a.write) {
          if (!nwr || a.gtid < w0) w0 = a.gtid;
          if (!nwr || a.gtid > w1) w1 = a.gtid;
          nwr++;
          wgw.insert(a.gtid / S);
          written.insert(a.value);
        } else {
          if (!nrd || a.gtid < r0) r0 = a.gtid;
          if (!nrd || a.gtid > r1) r1 = a.gtid;
          nrd++;
          wgr.insert(a.gtid / S);
          seen.insert(a.value);
        }
      }
      Record base{0xFFFFFFFFu, 0, 0, kv.first, 0, 0, 0, nrd, nwr, nrd + nwr};
      if (wgw.size() >= 2) {
        Record r = base;
        r.cls = written.size() == 1 ? C_XG_WW_BENIGN : C_XG_WW_RACE;
        r.t_a = w0;
        r.t_b = w1;
        rep.records.push_back(r);
      }
      const bool cross = !wgw.empty() && !wgr.empty() &&
                         !(wgw.size() == 1 && wgr.size() == 1 && *wgw.begin() == *wgr.begin());
      std::set<int32_t> all = written;
      all.insert(seen.begin(), seen.end());
      all.insert(initial_global[kv.first]);
      if (cross && all.size() >= 2) {
        Record r = base;
        r.cls = C_XG_RW_RACE;
        if (r0 / S != w0 / S) { r.t_a = r0; r.t_b = w0; }
        else if (r0 / S != w1 / S) { r.t_a = r0; r.t_b = w1; }
        else { r.t_a = r1; r.t_b = w0; }
        rep.records.push_back(r);
      }
    }
  }

  // Group scope: the barrier-release rule per work-group.  Returns whether
  // some group waits at a barrier (the run goes on); adds DIVERGENCE records
  // (wg = the group) for every group whose live work-items stopped at two
  // or more points, and sets diverged.
  bool group_agreement(uint32_t interval, std::vector<char> &done, bool &diverged) {
    bool any_barrier = false;
    for (uint32_t wg = 0; wg < G; wg++) {
      if (done[wg]) continue;
      std::map<uint32_t, std::pair<uint32_t, uint32_t>> stops;  // stop id -> (min gtid, count)
      bool waits = false;
      for (uint32_t t = 0; t < S; t++) {
        const uint32_t g = wg * S + t;
        uint32_t id;
        if (th[g].st == AT_BARRIER) { id = (uint32_t)cfg.nodes[th[g].node].id; waits = true; }
        else if (th[g].st == EXITED) id = 0xFFFFFFFFu;  // exited in this round: the group was not done
        else continue;
        auto it = stops.find(id);
        if (it == stops.end()) stops[id] = {g, 1};
        else it->second.second++;
      }
      if (stops.size() >= 2) {
        diverged = true;
        for (auto &s2 : stops)
          errors.push_back({interval, 0, wg, 0, C_DIVERGENCE, s2.second.first, s2.first, 0, 0, s2.second.second});
      }
      if (!waits) done[wg] = 1;  // every live work-item exited: the group is finished
      any_barrier |= waits;
    }
    return any_barrier;
  }

  void run(bool reverse) {
    const uint32_t N = G * S;
    th.assign(N, Thread{cfg.start, RUNNING});
    n_named = (uint32_t)prog.vars.size();
    vars.assign((uint64_t)N * n_named, 0);
    scratch.assign(std::max<int>(cfg.n_vars, 1), 0);
    std::vector<char> done(G, 0);  // group scope: groups whose work-items all exited
    if (tracing) {  // CFG nodes are created in text order, so their ids order the sites
      site_of.assign(cfg.nodes.size(), 0xFFFFFFFFu);
      for (size_t k = 0; k < cfg.nodes.size(); k++) {
        const Node &nd = cfg.nodes[k];
        if (nd.kind != N_LOAD && nd.kind != N_STORE) continue;
        site_of[k] = (uint32_t)(rep.sites.size() / 2);
        rep.sites.push_back(nd.kind == N_STORE ? 1u : 0u);
        rep.sites.push_back((uint32_t)nd.mem);
      }
    }
    if (group_scope) initial_global = global_snap;
    if (n_shards > 1) {
      pend_writer.assign(global_total, 0xFFFFFFFFu);
      pend_value.assign(global_total, 0);
    }
    for (uint32_t interval = 0;; interval++) {
      log.clear();
      errors.clear();
      for (uint32_t i = 0; i < N; i++) {
        uint32_t g = reverse ? N - 1 - i : i;
        if (th[g].st == RUNNING || th[g].st == AT_BARRIER) run_thread(g, interval);
      }
      rep.n_intervals = interval + 1;
      // group the interval's accesses by cell, keeping their order within a
      // cell (a thread's accesses stay in program order); then, cell by cell
      // in (space, wg, addr) order: classify it, add it to the whole-run
      // table (group scope), and commit it -- each written cell takes the
      // last write of its highest-gtid writer (the schedule that runs threads
      // in gtid order).  Committing here, before the barrier agreement below,
      // changes nothing: that reads no memory.
      std::sort(log.begin(), log.end(), [](const Logged &x, const Logged &y) {
        return std::tie(x.space, x.wg, x.addr, x.order) < std::tie(y.space, y.wg, y.addr, y.order);
      });
      std::vector<Access> acc;
      for (size_t i = 0; i < log.size();) {
        size_t j = i;
        acc.clear();
        for (; j < log.size() && log[j].space == log[i].space && log[j].wg == log[i].wg && log[j].addr == log[i].addr;
             j++)
          acc.push_back(log[j].a);
        const Cell c{log[i].space, log[i].wg, log[i].addr};
        i = j;
        classify_cell(interval, c, acc);
        if (group_scope && std::get<0>(c) == 0) {
          auto &v = whole_run[std::get<2>(c)];
          v.insert(v.end(), acc.begin(), acc.end());
        }
        bool any = false;
        uint32_t top = 0;
        for (const Access &a : acc)
          if (a.write && (!any || a.gtid > top)) { top = a.gtid; any = true; }
        if (!any) continue;
        int32_t v = 0;
        for (const Access &a : acc)  // a thread's accesses sit in program order
          if (a.write && a.gtid == top) v = a.value;
        commit_cell(c, v);
      }
      log.clear();
      for (auto &kv : pending) commit_cell(kv.first, kv.second.second);
      pending.clear();
      for (uint32_t addr : pend_touched) {
        global_snap[addr] = pend_value[addr];
        pend_writer[addr] = 0xFFFFFFFFu;
      }
      pend_touched.clear();
      // barrier agreement (Sec. 4 barrier-release rule): every thread that
      // is still alive must stop at the same barrier, or all must exit
      // (group scope: within each work-group).
      std::map<uint32_t, std::pair<uint32_t, uint32_t>> stops;  // stop id -> (min gtid, count)
      bool any_barrier = false, group_div = false;
      if (group_scope) any_barrier = group_agreement(interval, done, group_div);
      for (uint32_t g = 0; g < N && !group_scope; g++) {
        uint32_t id;
        // a thread that reached exit stops at the implicit final barrier;
        // once one has, the run ends, so no earlier exits are still around
        if (th[g].st == AT_BARRIER) { id = (uint32_t)cfg.nodes[th[g].node].id; any_barrier = true; }
        else if (th[g].st == EXITED) id = 0xFFFFFFFFu;
        else continue;
        auto it = stops.find(id);
        if (it == stops.end()) stops[id] = {g, 1};
        else it->second.second++;
      }
      bool diverged = stops.size() >= 2 || group_div;
      if (stops.size() >= 2) {
        for (auto &s : stops)
          errors.push_back({interval, 0, 0, 0, C_DIVERGENCE, s.second.first, s.first, 0, 0, s.second.second});
      }
      std::sort(errors.begin(), errors.end(), [](const Record &a, const Record &b) {
        return std::tie(a.cls, a.t_a) < std::tie(b.cls, b.t_a);
      });
      interval_errors.insert(interval_errors.end(), errors.begin(), errors.end());
      if (diverged || !any_barrier) break;
    }
    // report: race records already sorted by (interval, space, wg, addr, cls);
    // group scope: the cross-group records of the whole run (interval
    // 0xFFFFFFFF) by (addr, cls); error records follow, sorted by
    // (interval, kind, gtid).
    if (group_scope) run_cross_group();
    bool racy = false, div = false, as = false, oob = false;
    for (auto &r : rep.records)
      racy |= (r.cls == C_WW_RACE || r.cls == C_RW_RACE || r.cls == C_XG_WW_RACE || r.cls == C_XG_RW_RACE);
    for (auto &e : interval_errors) {
      if (shard != 0) break;  // shard 0 reports the errors
      div |= e.cls == C_DIVERGENCE;
      as |= e.cls == C_ASSERT;
      oob |= e.cls == C_OOB;
      rep.records.push_back(e);
    }
    rep.status = racy ? ST_RACY : div ? ST_DIVERGENCE : as ? ST_ASSERT : oob ? ST_OOB : ST_RACE_FREE;
    rep.final_global = global_snap;
  }

  std::vector<Record> interval_errors;
};

}  // namespace orc

// ------------------------------------------------------------------ C API
using namespace orc;

struct OracleHandle {
  Report rep;
};

extern "C" {

// Run the checker.  global_len/global_init give one int32 array per `global`
// declaration, in declaration order.  mode bit 0 runs the threads of every
// interval in descending gtid order (the report must not change); bit 1
// takes barriers as work-group scoped; bit 2 records the access trace;
// bits 8-19 / 20-31 give the shard p and the shard count P (0: unsharded)
// of an address-sharded run.
// Returns 0 on success, 1 on a parse error (message in err), 2 on a bad
// launch shape or input.
int oracle_check(const char *src, uint32_t groups, uint32_t group_size, uint32_t n_global,
                 const uint64_t *global_len, const int32_t *const *global_init, int mode,
                 void **out, char *err, size_t err_len) {
  *out = nullptr;
  try {
    Checker ck;
    ck.prog = Parser(src).parse();
    ck.cfg = CfgBuilder(ck.prog).build();
    ck.G = groups;
    ck.S = group_size;
    if (groups == 0 || group_size == 0 || (uint64_t)groups * group_size > (1ull << 26)) {
      snprintf(err, err_len, "bad launch shape");
      return 2;
    }
    uint32_t gi = 0;
    for (auto &m : ck.prog.mems) {
      if (m.space == 0) {
        if (gi >= n_global) { snprintf(err, err_len, "missing global input"); return 2; }
        ck.mem_len.push_back((int64_t)global_len[gi]);
        ck.mem_base.push_back(ck.global_total);
        ck.global_total += global_len[gi];
        gi++;
      } else {
        ck.mem_len.push_back(m.decl_len);
        ck.mem_base.push_back(ck.local_total);
        ck.local_total += (uint64_t)m.decl_len;
      }
    }
    if (gi != n_global) { snprintf(err, err_len, "global input count mismatch"); return 2; }
    ck.global_snap.assign(ck.global_total, 0);
    gi = 0;
    for (size_t i = 0; i < ck.prog.mems.size(); i++) {
      if (ck.prog.mems[i].space != 0) continue;
      for (uint64_t j = 0; j < global_len[gi]; j++) ck.global_snap[ck.mem_base[i] + j] = global_init[gi][j];
      gi++;
    }
    ck.local_snap.assign((uint64_t)groups * ck.local_total, 0);
    ck.group_scope = (mode & 2) != 0;
    ck.tracing = (mode & 4) != 0;
    const uint32_t shards = ((uint32_t)mode >> 20) & 0xFFFu;
    if (shards > 1) {
      ck.n_shards = shards;
      ck.shard = ((uint32_t)mode >> 8) & 0xFFFu;
      if (ck.shard >= shards) { snprintf(err, err_len, "bad shard"); return 2; }
    }
    ck.run((mode & 1) != 0);
    auto *h = new OracleHandle{std::move(ck.rep)};
    *out = h;
    return 0;
  } catch (const ParseError &e) {
    snprintf(err, err_len, "%s", e.what());
    return 1;
  } catch (const std::exception &e) {
    snprintf(err, err_len, "%s", e.what());
    return 2;
  }
}

int32_t oracle_status(void *h) { return ((OracleHandle *)h)->rep.status; }
uint32_t oracle_n_intervals(void *h) { return ((OracleHandle *)h)->rep.n_intervals; }
uint64_t oracle_n_access(void *h) { return ((OracleHandle *)h)->rep.n_access; }
uint64_t oracle_n_global(void *h) { return ((OracleHandle *)h)->rep.n_global; }
uint64_t oracle_n_local(void *h) { return ((OracleHandle *)h)->rep.n_local; }
uint64_t oracle_max_acc(void *h) { return ((OracleHandle *)h)->rep.max_acc; }
uint64_t oracle_max_wr(void *h) { return ((OracleHandle *)h)->rep.max_wr; }
uint64_t oracle_n_records(void *h) { return ((OracleHandle *)h)->rep.records.size(); }
const void *oracle_records(void *h) { return ((OracleHandle *)h)->rep.records.data(); }
uint64_t oracle_final_len(void *h) { return ((OracleHandle *)h)->rep.final_global.size(); }
const int32_t *oracle_final(void *h) { return ((OracleHandle *)h)->rep.final_global.data(); }
uint64_t oracle_trace_len(void *h) { return ((OracleHandle *)h)->rep.trace.size() / 8; }
const uint32_t *oracle_trace(void *h) { return ((OracleHandle *)h)->rep.trace.data(); }
uint64_t oracle_n_sites(void *h) { return ((OracleHandle *)h)->rep.sites.size() / 2; }
const uint32_t *oracle_sites(void *h) { return ((OracleHandle *)h)->rep.sites.data(); }
void oracle_free(void *h) { delete (OracleHandle *)h; }

}  // extern "C"
