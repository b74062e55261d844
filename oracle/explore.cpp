// ORACLE PIN (test infrastructure only): brute-force interleaving explorer.
//
// Only the test suite may build or call this file.  It gives the oracle
// something to be checked against that is not the oracle itself: the
// global semantics of Sec. 4 (Distefano & Dubreil) taken literally.  Every
// thread reads and writes one truly shared memory, any thread may take the
// next step, and the shared state reached when all threads meet at a barrier
// (or at the implicit barrier at exit) is collected over EVERY schedule.
// A kernel is racy in the sense of Sec. 4's Definition when two schedules
// reach different shared states there.
//
// Private commands commute with everything other threads do, so a thread's
// private commands are run eagerly and only its shared accesses (one per
// command, by construction of the CFG) are interleaved.  States are memoised,
// which keeps tiny kernels (2-4 threads, a handful of accesses) exhaustive.
//
// For each interval it reports how many distinct shared states all schedules
// reach at its closing barrier and whether some schedule makes some thread
// read a value different from what that thread reads when it runs first and
// alone from the same interval start (schedule-dependent reads).
#include <cstdint>
#include <cstdio>
#include <set>
#include <string>
#include <vector>

#include "kl_frontend.hpp"

namespace orc {
namespace ex {

enum { RUN = 0, BAR = 1, EXT = 2, DED = 3 };

struct TState {
  int node;
  int st;
  int reads;  // reads done in the current interval
  std::vector<int32_t> vars;
  bool operator<(const TState &o) const {
    if (node != o.node) return node < o.node;
    if (st != o.st) return st < o.st;
    if (reads != o.reads) return reads < o.reads;
    return vars < o.vars;
  }
  bool operator==(const TState &o) const {
    return node == o.node && st == o.st && reads == o.reads && vars == o.vars;
  }
};

struct GState {
  std::vector<TState> th;
  std::vector<int32_t> gmem, lmem;
  bool operator<(const GState &o) const {
    if (!(th == o.th)) return th < o.th;
    if (gmem != o.gmem) return gmem < o.gmem;
    return lmem < o.lmem;
  }
};

struct Explorer {
  Program prog;
  Cfg cfg;
  uint32_t G, S, N;
  std::vector<int64_t> mem_len;
  std::vector<uint64_t> mem_base;
  uint64_t local_total = 0;
  uint64_t max_states;
  uint64_t visited_total = 0;
  bool overflow = false;

  Env env_of(const GState &s, uint32_t g) const {
    return Env{s.th[g].vars.data(), g % S, g / S, S, G, &mem_len};
  }

  int next_node(int k, const Env &env) const {
    const Node &n = cfg.nodes[k];
    if (n.succ.size() == 1) return n.succ[0];
    for (int s : n.succ)
      if (eval(*cfg.nodes[s].val, env) != 0) return s;
    return -1;
  }

  // Advance thread g through private commands until it is about to make a
  // shared access (node = that LOAD/STORE, st = RUN) or it stops.
  void normalize(GState &s, uint32_t g) const {
    TState &t = s.th[g];
    while (t.st == RUN) {
      const Node &n = cfg.nodes[t.node];
      Env env = env_of(s, g);
      switch (n.kind) {
        case N_LOAD:
        case N_STORE:
          return;
        case N_EXIT: t.st = EXT; return;
        case N_BARRIER: t.st = BAR; return;
        case N_ASSIGN: t.vars[n.var] = eval(*n.val, env); break;
        case N_ASSUME:
          if (eval(*n.val, env) == 0) { t.st = DED; return; }
          break;
        case N_ASSERT:
          if (eval(*n.val, env) == 0) { t.st = DED; return; }
          break;
        default: break;
      }
      int k = next_node(t.node, env);
      if (k < 0) { t.st = DED; return; }
      t.node = k;
    }
  }

  // Perform thread g's pending shared access on the shared memory; returns
  // the value a read observed (or INT64_MIN for a write or an abort).
  int64_t step_access(GState &s, uint32_t g) const {
    TState &t = s.th[g];
    const Node &n = cfg.nodes[t.node];
    Env env = env_of(s, g);
    const Mem &m = prog.mems[n.mem];
    int32_t idx = eval(*n.idx, env);
    int32_t val = n.kind == N_STORE ? eval(*n.val, env) : 0;
    int64_t observed = INT64_MIN;
    if (idx < 0 || (int64_t)idx >= mem_len[n.mem]) {
      t.st = DED;
      return observed;
    }
    uint64_t a = mem_base[n.mem] + (uint64_t)idx;
    int32_t *cell = m.space == 0 ? &s.gmem[a] : &s.lmem[(uint64_t)(g / S) * local_total + a];
    if (n.kind == N_STORE) {
      *cell = val;
    } else {
      t.vars[n.var] = *cell;
      observed = *cell;
      t.reads++;
    }
    int k = next_node(t.node, env);
    if (k < 0) { t.st = DED; return observed; }
    t.node = k;
    normalize(s, g);
    return observed;
  }

  // Reads thread g makes when it runs alone from interval-start state s.
  std::vector<int32_t> solo_trace(const GState &s, uint32_t g) const {
    GState c = s;
    std::vector<int32_t> tr;
    while (c.th[g].st == RUN) {
      int64_t o = step_access(c, g);
      if (o != INT64_MIN) tr.push_back((int32_t)o);
    }
    return tr;
  }

  // All shared states at the end of the interval that starts at `start`.
  void explore_interval(const GState &start, std::set<GState> &ends, bool &deviated) {
    std::vector<std::vector<int32_t>> solo(N);
    for (uint32_t g = 0; g < N; g++) solo[g] = solo_trace(start, g);
    std::set<GState> seen;
    std::vector<GState> stack{start};
    while (!stack.empty()) {
      GState s = std::move(stack.back());
      stack.pop_back();
      if (!seen.insert(s).second) continue;
      if (++visited_total > max_states) { overflow = true; return; }
      bool any = false;
      for (uint32_t g = 0; g < N; g++) {
        if (s.th[g].st != RUN) continue;
        any = true;
        GState c = s;
        int r = c.th[g].reads;
        int64_t o = step_access(c, g);
        if (o != INT64_MIN && (r >= (int)solo[g].size() || solo[g][r] != (int32_t)o)) deviated = true;
        stack.push_back(std::move(c));
      }
      if (!any) ends.insert(s);
    }
  }
};

}  // namespace ex
}  // namespace orc

using namespace orc;
using namespace orc::ex;

struct ExploreResult {
  // pair mode: per interval, per pair (i < j) in (i, j) order, the distinct
  // shared states reached when only i and j run from the interval's start
  // (all other work-items frozen) | (a read of i or j depends on the
  // schedule) << 31; empty for an interval that starts from several states
  std::vector<std::vector<uint32_t>> pairs;
  std::vector<uint32_t> n_end_states;  // per interval: distinct shared states at its barrier
  std::vector<uint8_t> deviated;       // per interval: some read depends on the schedule
  std::vector<uint32_t> n_final;       // distinct final global memories (over all schedules)
  std::vector<int32_t> finals;         // those memories, concatenated
  int diverged = 0;                    // some schedule stops at mismatched barriers
  int overflow = 0;
};

extern "C" {

// Explore every schedule of a tiny instance.  Returns 0 on success, 1 parse
// error, 2 bad input.  max_states bounds the total work; on overflow the
// result has overflow = 1 and must not be used.
static int explore_impl(const char *src, uint32_t groups, uint32_t group_size, uint32_t n_global,
                        const uint64_t *global_len, const int32_t *const *global_init, uint64_t max_states,
                        bool pairs, void **out, char *err, size_t err_len) {
  *out = nullptr;
  try {
    Explorer ex;
    ex.prog = Parser(src).parse();
    ex.cfg = CfgBuilder(ex.prog).build();
    ex.G = groups;
    ex.S = group_size;
    ex.N = groups * group_size;
    ex.max_states = max_states;
    if (ex.N == 0 || ex.N > 16) { snprintf(err, err_len, "explorer handles 1..16 threads"); return 2; }
    uint64_t gtotal = 0;
    uint32_t gi = 0;
    for (auto &m : ex.prog.mems) {
      if (m.space == 0) {
        if (gi >= n_global) { snprintf(err, err_len, "missing global input"); return 2; }
        ex.mem_len.push_back((int64_t)global_len[gi]);
        ex.mem_base.push_back(gtotal);
        gtotal += global_len[gi++];
      } else {
        ex.mem_len.push_back(m.decl_len);
        ex.mem_base.push_back(ex.local_total);
        ex.local_total += (uint64_t)m.decl_len;
      }
    }
    GState init;
    init.gmem.assign(gtotal, 0);
    gi = 0;
    for (size_t i = 0; i < ex.prog.mems.size(); i++) {
      if (ex.prog.mems[i].space != 0) continue;
      for (uint64_t j = 0; j < global_len[gi]; j++) init.gmem[ex.mem_base[i] + j] = global_init[gi][j];
      gi++;
    }
    init.lmem.assign((uint64_t)groups * ex.local_total, 0);
    init.th.assign(ex.N, TState{ex.cfg.start, RUN, 0, std::vector<int32_t>(ex.cfg.n_vars, 0)});
    for (uint32_t g = 0; g < ex.N; g++) ex.normalize(init, g);

    auto *res = new ExploreResult();
    std::set<GState> frontier{init};
    std::set<std::vector<int32_t>> finals;
    while (!frontier.empty() && !ex.overflow) {
      if (pairs) {  // the interleaving product of every two work-items, from a unique start
        std::vector<uint32_t> pv;
        if (frontier.size() == 1) {
          const GState &s0 = *frontier.begin();
          for (uint32_t i = 0; i < ex.N; i++)
            for (uint32_t j = i + 1; j < ex.N; j++) {
              GState s = s0;
              for (uint32_t g = 0; g < ex.N; g++)
                if (g != i && g != j) s.th[g].st = DED;
              std::set<GState> pe;
              bool pd = false;
              ex.explore_interval(s, pe, pd);
              std::set<std::pair<std::vector<int32_t>, std::vector<int32_t>>> mem;
              for (const GState &e : pe) mem.insert({e.gmem, e.lmem});
              pv.push_back((uint32_t)mem.size() | (pd ? 0x80000000u : 0u));
            }
        }
        res->pairs.push_back(pv);
      }
      std::set<GState> ends;
      bool dev = false;
      for (const GState &s : frontier) ex.explore_interval(s, ends, dev);
      std::set<std::pair<std::vector<int32_t>, std::vector<int32_t>>> shared;
      std::set<GState> next;
      for (const GState &e : ends) {
        shared.insert({e.gmem, e.lmem});
        // barrier release: every live thread waits at the same barrier
        int bar = -2;
        bool exited = false, mixed = false;
        for (auto &t : e.th) {
          if (t.st == BAR) {
            int id = ex.cfg.nodes[t.node].id;
            if (bar == -2) bar = id;
            else if (bar != id) mixed = true;
          } else if (t.st == EXT) {
            exited = true;
          }
        }
        if (mixed || (bar != -2 && exited)) { res->diverged = 1; continue; }
        if (bar == -2) { finals.insert(e.gmem); continue; }
        GState r = e;
        for (uint32_t g = 0; g < ex.N; g++) {
          TState &t = r.th[g];
          t.reads = 0;
          if (t.st != BAR) continue;
          t.st = RUN;
          int k = ex.next_node(t.node, ex.env_of(r, g));
          if (k < 0) { t.st = DED; continue; }
          t.node = k;
          ex.normalize(r, g);
        }
        next.insert(r);
      }
      res->n_end_states.push_back((uint32_t)shared.size());
      res->deviated.push_back(dev ? 1 : 0);
      frontier.swap(next);
    }
    for (auto &f : finals) res->finals.insert(res->finals.end(), f.begin(), f.end());
    res->n_final.push_back((uint32_t)finals.size());
    res->overflow = ex.overflow ? 1 : 0;
    *out = res;
    return 0;
  } catch (const ParseError &e) {
    snprintf(err, err_len, "%s", e.what());
    return 1;
  } catch (const std::exception &e) {
    snprintf(err, err_len, "%s", e.what());
    return 2;
  }
}

int explore_check(const char *src, uint32_t groups, uint32_t group_size, uint32_t n_global,
                  const uint64_t *global_len, const int32_t *const *global_init,
                  uint64_t max_states, void **out, char *err, size_t err_len) {
  return explore_impl(src, groups, group_size, n_global, global_len, global_init, max_states, false, out, err,
                      err_len);
}

// explore_check plus, for every interval that starts from one state, the
// interleaving product of every pair of work-items (see ExploreResult::pairs)
int explore_pairs_check(const char *src, uint32_t groups, uint32_t group_size, uint32_t n_global,
                        const uint64_t *global_len, const int32_t *const *global_init,
                        uint64_t max_states, void **out, char *err, size_t err_len) {
  return explore_impl(src, groups, group_size, n_global, global_len, global_init, max_states, true, out, err,
                      err_len);
}

uint32_t explore_n_pairs(void *h, uint32_t k) { return (uint32_t)((ExploreResult *)h)->pairs[k].size(); }
const uint32_t *explore_pairs(void *h, uint32_t k) { return ((ExploreResult *)h)->pairs[k].data(); }

uint32_t explore_n_intervals(void *h) { return (uint32_t)((ExploreResult *)h)->n_end_states.size(); }
uint32_t explore_end_states(void *h, uint32_t k) { return ((ExploreResult *)h)->n_end_states[k]; }
int explore_deviated(void *h, uint32_t k) { return ((ExploreResult *)h)->deviated[k]; }
uint32_t explore_n_final(void *h) { return ((ExploreResult *)h)->n_final[0]; }
const int32_t *explore_finals(void *h) { return ((ExploreResult *)h)->finals.data(); }
int explore_diverged(void *h) { return ((ExploreResult *)h)->diverged; }
int explore_overflow(void *h) { return ((ExploreResult *)h)->overflow; }
void explore_free(void *h) { delete (ExploreResult *)h; }

}  // extern "C"
