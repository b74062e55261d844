// Host runtime and C ABI: instance set-up, the barrier-interval loop, the
// barrier agreement check, report assembly, device workspaces and timing.
//
// Per barrier interval (Distefano & Dubreil, Sec. 4): run every live
// work-item to its next barrier or exit (interpreter kernel), classify the
// interval's logged accesses and commit its writes (sort + segmented
// classification, or the shadow owner table path), then apply the barrier
// release rule: all work-items that are still alive must stop at the same
// barrier, or all must exit; anything else is reported as divergence and
// ends the run.  The end of the kernel is an implicit barrier, so the last
// interval is classified too.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <sys/stat.h>
#include <chrono>
#include <new>
#include <stdexcept>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#include "racecheck.h"
#include "device.cuh"
#include "jit.h"
#include "candidate_features.h"

namespace rc {
// The two-work-item pre-filter (prove.cpp).
void prove_analyze(const Program &p, uint32_t groups, uint32_t group_size, const std::vector<uint32_t> &lens,
                   rc_prove_result *out, std::vector<uint8_t> *priv, uint64_t enum_budget);
bool prove_lengths(const Program &p, const rc_input *in, std::vector<uint32_t> &lens);

namespace {

thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};
std::mutex g_mu;
int g_strategy = 0;
// interval kernels: 0 automatic, 1 bytecode interpreter, 2 compiled intervals
int g_engine = 0;
// automatic engine: compiled intervals from this many work-items on (one
// NVRTC compile, a fraction of a second, per program and launch shape)
constexpr uint64_t kJitAutoItems = 1ull << 17;

struct Fail {
  int code;
  std::string msg;
};

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      throw Fail{RC_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};      \
  } while (0)

// ---------------------------------------------------------------- workspace
struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
  template <class T>
  T *get(size_t n) {
    size_t bytes = std::max<size_t>(n * sizeof(T), 256);
    if (bytes > cap) {
      if (p) CK(cudaFree(p));
      p = nullptr;
      cap = 0;
      size_t want = bytes + bytes / 4;
      if (cudaMalloc(&p, want) != cudaSuccess) {
        cudaGetLastError();
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
          cudaGetLastError();
          throw Fail{RC_E_CAPACITY, "device allocation of " + std::to_string(bytes) + " bytes failed"};
        }
        want = bytes;
      }
      cap = want;
    }
    return static_cast<T *>(p);
  }
  template <class T>
  T *as() {
    return static_cast<T *>(p);
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

struct HostBuf {
  void *p = nullptr;
  size_t cap = 0;
  template <class T>
  T *as() {
    return static_cast<T *>(p);
  }
  template <class T>
  T *get(size_t n) {
    size_t bytes = std::max<size_t>(n * sizeof(T), 256);
    if (bytes > cap) {
      if (p) cudaFreeHost(p);
      p = nullptr;
      CK(cudaMallocHost(&p, bytes));
      cap = bytes;
    }
    return static_cast<T *>(p);
  }
};

struct Workspace {
  DevBuf code, mems, snap, regs, pc, st, ow, loga, logb, head, runidx, sum, khead, keyidx, nrec,
      recoff, out, scan, errs, stats, owner, owcnt, compact, ctacnt, ctaoff, sortscr, reckern,
      bdesc, bcode, bmems, btask, bkbase, bkgt, bklt, berrk, shared_acc, bround, big, bigres, nbig, xg, xgcnt,
      xgn, xgoff, xgtmp, xgout, rstat, rivoff, rbar;
  HostBuf hstats, hround, hdesc, hsmall, hstage, hrank;
  HostBuf hrecs[2], hreck[2];  // batch race records and their instances, alternate rounds
  DevBuf brounds;  // resident batch: intervals per instance, rounds, last tag
  DevBuf cellres;  // per-cell classification results between the classifier and the emitter
  DevBuf cstart;   // first summary of each cell
  DevBuf rankx;  // ranked search: features and scores of the candidates
  DevBuf stage;  // one-CTA checks: bytecode, memory table and snapshot in one block
  cudaStream_t bstream = nullptr;
  cudaStream_t cstream = nullptr;  // shadow-path classification beside the next interval
  cudaEvent_t sev[2] = {nullptr, nullptr};  // stats of an interval (by parity) reached the host
  bool configured = false, batch_configured = false;
  uint32_t epoch = 0;
  uint64_t owner_hi = 0;  // owner-table words that may hold a tag; the rest are zero
  void release_all() {
    for (DevBuf *b : {&code, &mems, &snap, &regs, &pc, &st, &ow, &loga, &logb, &head, &runidx, &sum,
                      &khead, &keyidx, &nrec, &recoff, &out, &scan, &errs, &stats, &owner,
                      &owcnt, &compact, &ctacnt, &ctaoff, &sortscr, &reckern, &bdesc, &bcode,
                      &bmems, &btask, &bkbase, &bkgt, &bklt, &berrk, &shared_acc, &bround, &big,
                      &bigres, &nbig, &xg, &xgcnt, &xgn, &xgoff, &xgtmp, &xgout, &rstat, &rivoff, &rbar, &stage,
                      &cellres, &cstart})
      b->release();
    epoch = 0;
    owner_hi = 0;
  }
};
Workspace g_ws;

// ---------------------------------------------------------------- profiling
struct Prof {
  bool on = false;
  uint64_t launches[3] = {0, 0, 0};
  double ms[3] = {0, 0, 0};
  double bytes[3] = {0, 0, 0};
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};
Prof g_prof;

void prof_events() {
  if (!g_prof.ev[0])
    for (auto &e : g_prof.ev) CK(cudaEventCreate(&e));
}

// ---------------------------------------------------------------- autotuner
// Classification strategy per size class.  Both strategies are exact, so
// an undecided class simply alternates them on successive intervals (or
// batch rounds), timing each interval per million accesses; after two
// samples of each the cheaper one is kept and written to a JSON cache.
// Batches also get a block shape (timed like the strategy) and a log
// capacity: the warp slices start at the compiler's static bound per
// interval (always enough), the fullest slice of each call is recorded, and
// later calls of the class allocate twice the largest fill seen; a call
// whose slices overflow that is checked again at the static bound, which
// the class then keeps.
struct Tuner {
  // block shapes of the batch interpreter (threads per CTA)
  static constexpr uint32_t kShapes[3] = {128, 256, 512};
  struct Entry {
    int best = 0;
    double cost[3] = {0, 0, 0};
    int n[3] = {0, 0, 0};
    uint32_t threads = 0;  // decided block shape (batches), 0 = not yet
    double scost[3] = {0, 0, 0};
    int sn[3] = {0, 0, 0};
    uint32_t log_pm = 0;   // batches: log capacity in permille of the static bound, 0 = not yet
    uint32_t fill_pm = 0;  // the fullest slice seen, in permille of the static bound
  };
  bool loaded = false;
  bool persist = true;
  std::string path;
  std::map<std::string, Entry> entries;

  static std::string default_path() {
    if (const char *e = std::getenv("RC_TUNE_CACHE")) return e;
    if (const char *x = std::getenv("XDG_CACHE_HOME")) return std::string(x) + "/racecheck_autotune.json";
    if (const char *h = std::getenv("HOME")) return std::string(h) + "/.cache/racecheck_autotune.json";
    return "";
  }
  void load() {
    if (loaded) return;
    loaded = true;
    if (path.empty()) path = default_path();
    if (!persist || path.empty()) return;
    FILE *f = std::fopen(path.c_str(), "rb");
    if (!f) return;
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
    std::fclose(f);
    // entries look like  "single:N18:B7": {"best": 2, ...}
    for (size_t p = 0; (p = text.find('"', p)) != std::string::npos;) {
      const size_t q = text.find('"', p + 1);
      if (q == std::string::npos) break;
      const std::string key = text.substr(p + 1, q - p - 1);
      p = q + 1;
      if (key.rfind("single:", 0) != 0 && key.rfind("batch:", 0) != 0) continue;
      const size_t b = text.find("\"best\":", q);
      const size_t close = text.find('}', q);
      if (b == std::string::npos || b > close) continue;
      const int best = std::atoi(text.c_str() + b + 7);
      if (best == 1 || best == 2) entries[key].best = best;
      const size_t th = text.find("\"threads\":", q);
      if (th != std::string::npos && th < close) {
        const uint32_t v = (uint32_t)std::atoi(text.c_str() + th + 10);
        if (v == 128 || v == 256 || v == 512) entries[key].threads = v;
      }
      const size_t lp = text.find("\"log_permille\":", q);
      if (lp != std::string::npos && lp < close) {
        const int v = std::atoi(text.c_str() + lp + 15);
        if (v >= 1 && v <= 1000) entries[key].log_pm = (uint32_t)v;
      }
    }
  }
  void save() {
    if (!persist || path.empty()) return;
    const size_t slash = path.rfind('/');
    if (slash != std::string::npos) {  // best effort: create the cache folder
      const std::string dir = path.substr(0, slash);
      mkdir(dir.c_str(), 0755);
    }
    const std::string tmp = path + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return;
    std::fprintf(f, "{\n  \"racecheck_autotune\": 1,\n  \"entries\": {");
    bool first = true;
    for (auto &kv : entries) {
      if (!kv.second.best) continue;
      const Entry &e = kv.second;
      std::fprintf(f, "%s\n    \"%s\": {\"best\": %d, \"ms_per_maccess_sort\": %.6g, \"ms_per_maccess_shadow\": %.6g",
                   first ? "" : ",", kv.first.c_str(), e.best, e.n[1] ? e.cost[1] / e.n[1] : 0.0,
                   e.n[2] ? e.cost[2] / e.n[2] : 0.0);
      if (e.threads) std::fprintf(f, ", \"threads\": %u", e.threads);
      if (e.log_pm) std::fprintf(f, ", \"log_permille\": %u, \"fill_permille\": %u", e.log_pm, e.fill_pm);
      std::fprintf(f, "}");
      first = false;
    }
    std::fprintf(f, "\n  }\n}\n");
    std::fclose(f);
    std::rename(tmp.c_str(), path.c_str());
  }
  int choose(const std::string &key) {
    load();
    Entry &e = entries[key];
    if (e.best) return e.best;
    return e.n[1] <= e.n[2] ? 1 : 2;
  }
  bool decided(const std::string &key) {
    load();
    return entries[key].best != 0;
  }
  // batches: once the strategy is decided, each block shape is timed on two
  // rounds and the fastest kept (per million accesses)
  uint32_t choose_threads(const std::string &key) {
    load();
    Entry &e = entries[key];
    if (e.threads) return e.threads;
    if (!e.best) return 256;
    int k = 0;
    for (int j = 1; j < 3; j++)
      if (e.sn[j] < e.sn[k]) k = j;
    return kShapes[k];
  }
  bool threads_decided(const std::string &key) {
    load();
    return entries[key].threads != 0;
  }
  void record_threads(const std::string &key, uint32_t threads, double ms, uint64_t accesses) {
    Entry &e = entries[key];
    if (e.threads || !e.best || accesses == 0) return;
    const int k = threads == 128 ? 0 : threads == 256 ? 1 : 2;
    e.scost[k] += ms * 1e6 / (double)accesses;
    e.sn[k]++;
    if (e.sn[0] >= 2 && e.sn[1] >= 2 && e.sn[2] >= 2) {
      int b = 0;
      for (int j = 1; j < 3; j++)
        if (e.scost[j] / e.sn[j] < e.scost[b] / e.sn[b]) b = j;
      e.threads = kShapes[b];
      save();
    }
  }
  // batches: log capacity, permille of the static bound
  uint32_t log_permille(const std::string &key) {
    load();
    const uint32_t v = entries[key].log_pm;
    return v ? v : 1000u;
  }
  // the fullest slice of a completed call (permille of the static bound)
  void record_fill(const std::string &key, uint32_t fill_pm) {
    Entry &e = entries[key];
    e.fill_pm = std::max(e.fill_pm, std::min(fill_pm, 1000u));
    const uint32_t want = std::min<uint32_t>(1000u, std::max<uint32_t>(2 * e.fill_pm, 16u));
    if (e.log_pm == 0 || want > e.log_pm) {
      e.log_pm = want;
      save();
    }
  }
  // a call overflowed its slices at the tuned capacity: the static bound from now on
  void record_overflow(const std::string &key) {
    Entry &e = entries[key];
    e.log_pm = 1000;
    e.fill_pm = 1000;
    save();
  }
  void record(const std::string &key, int strategy, double ms, uint64_t accesses) {
    Entry &e = entries[key];
    if (e.best || accesses == 0 || strategy < 1 || strategy > 2) return;
    e.cost[strategy] += ms * 1e6 / (double)accesses;
    e.n[strategy]++;
    if (e.n[1] >= 2 && e.n[2] >= 2) {
      e.best = e.cost[1] / e.n[1] <= e.cost[2] / e.n[2] ? 1 : 2;
      save();
    }
  }
};
Tuner g_tuner;
cudaEvent_t g_tev[2] = {nullptr, nullptr};

void tuner_events() {
  if (!g_tev[0])
    for (auto &e : g_tev) CK(cudaEventCreate(&e));
}

uint32_t bits_of(uint64_t v) {
  uint32_t b = 0;
  while (v) {
    b++;
    v >>= 1;
  }
  return b;
}

std::string single_key(uint64_t N, uint64_t bound) {
  return "single:N" + std::to_string(bits_of(N)) + ":B" + std::to_string(bits_of(bound));
}
std::string batch_key(uint64_t tasks, uint64_t bound) {
  return "batch:T" + std::to_string(bits_of(tasks)) + ":B" + std::to_string(bits_of(bound));
}

// stats block layout (uint32 words)
enum : uint32_t { ST_LOGGED = 0, ST_ACC = 2, ST_FLAGS = 6, ST_ERRCNT = 7, ST_SCRATCH = 8, ST_GDIV = 10, ST_STOPS = 12 };
// The two stats buffers (by interval parity) sit stat_words = ST_STOPS +
// 2 * (n_barriers + 1) words apart, and each holds 64-bit counters at ST_ACC
// and ST_SCRATCH: ST_STOPS must be even so both buffers keep them 8-byte aligned.
static_assert(ST_STOPS % 2 == 0 && ST_ACC % 2 == 0 && ST_SCRATCH % 2 == 0 && ST_LOGGED % 2 == 0,
              "64-bit stats words need 8-byte alignment");

uint32_t bitwidth(uint64_t v) {  // bits needed to represent values < v (v >= 1)
  uint32_t b = 0;
  while (b < 64 && (v - 1) >> b) b++;
  return std::max<uint32_t>(b, 1);
}

// Exhaustive exploration of each interval before the canonical run takes it
// (rc_explore): results by interval.
struct ExploreRun {
  uint64_t max_states;
  uint32_t max_intervals;
  bool pairs;  // the interleaving product of every two work-items instead of all of them
  std::vector<ExploreResult> results;
  std::vector<std::vector<uint32_t>> pair_results;
};

struct Instance {
  const Program *p;
  uint32_t G, S;
  uint64_t N;
  const rc_input *in;
  cudaStream_t s;
  ExploreRun *explore = nullptr;
};

struct Layout {
  std::vector<MemInfo> mems;
  uint64_t GT = 0, LT = 0, keys = 0;
};

Layout make_layout(const Program &p, const rc_input *in, uint32_t G) {
  Layout L;
  uint32_t gi = 0;
  for (const MemDecl &m : p.mems) {
    MemInfo mi{};
    mi.space = m.space;
    if (m.space == 0) {
      uint64_t len = in->global_len[gi++];
      if (len > 0x7FFFFFFFull) throw Fail{RC_E_INVALID, "global array longer than 2^31-1"};
      mi.len = (uint32_t)len;
      mi.base = (uint32_t)L.GT;
      L.GT += len;
    } else {
      mi.len = (uint32_t)m.decl_len;
      mi.base = (uint32_t)L.LT;
      L.LT += (uint64_t)m.decl_len;
    }
    if (L.GT >= 0xFFFFFFFFull || L.LT >= 0xFFFFFFFFull) throw Fail{RC_E_INVALID, "memory too large"};
    L.mems.push_back(mi);
  }
  L.keys = L.GT + (uint64_t)G * L.LT;
  if (L.keys >= 0xFFFFFFFFull) throw Fail{RC_E_INVALID, "global + local cells must stay below 2^32"};
  return L;
}

// Classify records already sorted by (cell, work-item): run reduce, per-cell
// classification with commit, and ordered emission of the records.
// A growable malloc'd array of records: a batch instance's race records,
// handed to its report without another copy (realloc of a large block
// remaps its pages instead of copying them).
struct RecList {
  OutRec *p = nullptr;
  size_t n = 0, cap = 0;
  RecList() = default;
  RecList(const RecList &) = delete;
  RecList &operator=(const RecList &) = delete;
  RecList(RecList &&o) noexcept : p(o.p), n(o.n), cap(o.cap) {
    o.p = nullptr;
    o.n = o.cap = 0;
  }
  ~RecList() { std::free(p); }
  void append(const OutRec *src, size_t k) {
    if (!k) return;
    if (n + k > cap) {
      const size_t c = std::max<size_t>({n + k, 2 * cap, 64});
      OutRec *q = static_cast<OutRec *>(std::realloc(p, c * sizeof(OutRec)));
      if (!q) throw Fail{RC_E_NOMEM, "record list allocation failed"};
      p = q;
      cap = c;
    }
    std::memcpy(p + n, src, k * sizeof(OutRec));
    n += k;
  }
  OutRec *release() {
    OutRec *q = p;
    p = nullptr;
    n = cap = 0;
    return q;
  }
};

struct RecordSink;
struct BatchMap {  // cell space of a batch: instance first cells and sizes (device)
  uint32_t n = 0;
  const uint64_t *kbase = nullptr;
  const uint32_t *kGT = nullptr, *kLT = nullptr;
  RecordSink *sink = nullptr;  // receives every record, for its instance's list
};

// A batch round's race records, in cell order (the instances' cells lie end
// to end, so each instance's records form one run; kernel_of names each
// record's instance), appended to the instances' lists run by run.
void distribute_records(const OutRec *rr, const uint32_t *kernel_of, uint64_t n, std::vector<RecList> &races) {
  for (uint64_t i = 0; i < n;) {
    uint64_t j = i + 1;
    while (j < n && kernel_of[j] == kernel_of[i]) j++;
    races[kernel_of[i]].append(rr + i, j - i);
    i = j;
  }
}

// Appends each batch round's race records to the instances' lists on a
// worker thread while the device classifies the next round.  Two page-
// locked buffer pairs alternate; a round's job starts once the previous
// one has ended, so the lists grow in round order, and the buffers a round
// fills were last read by the job two rounds back, already joined.
struct RecordSink {
  std::vector<RecList> &races;
  HostBuf *recs, *kern;  // [2] each, kept in the workspace
  uint32_t next = 0;
  std::thread job;
  std::exception_ptr err;
  RecordSink(std::vector<RecList> &r, HostBuf *rb, HostBuf *kb) : races(r), recs(rb), kern(kb) {}
  RecordSink(const RecordSink &) = delete;
  RecordSink &operator=(const RecordSink &) = delete;
  ~RecordSink() {
    if (job.joinable()) job.join();
  }
  // waits for the running job; rethrows its failure
  void join() {
    if (job.joinable()) job.join();
    if (err) {
      std::exception_ptr e = err;
      err = nullptr;
      std::rethrow_exception(e);
    }
  }
  // the buffers for the next round's n records
  OutRec *records(uint64_t n) { return recs[next & 1].get<OutRec>(n); }
  uint32_t *kernels(uint64_t n) { return kern[next & 1].get<uint32_t>(n); }
  // the next round's n records have arrived in its buffers
  void submit(uint64_t n) {
    join();
    const OutRec *r = recs[next & 1].as<OutRec>();
    const uint32_t *k = kern[next & 1].as<uint32_t>();
    next++;
    try {
      job = std::thread([this, r, k, n] {
        try {
          distribute_records(r, k, n, races);
        } catch (...) {
          err = std::current_exception();
        }
      });
    } catch (const std::system_error &) {  // no thread to be had: the same work on this one
      distribute_records(r, k, n, races);
    }
  }
};

void classify_run(Workspace &W, const LogRec *sorted, uint64_t n, uint32_t interval, const Layout &L,
                  int32_t *snap, uint32_t *hstats, std::vector<OutRec> &races, cudaStream_t s,
                  const BatchMap *bm = nullptr) {
  // Summaries, cells and records number at most n, so every step runs over n
  // entries: key heads and record counts past the real ends are zero (set
  // here), and the kernels that read summaries take their exact number from
  // device memory; the host reads one count, the number of records to emit.
  uint32_t *tmp = W.scan.get<uint32_t>(std::max(sort_tmp_words(n), scan_tmp_words(n)));
  uint32_t *head = W.head.get<uint32_t>(n), *runidx = W.runidx.get<uint32_t>(n);
  launch_run_heads(sorted, n, head, s);
  scan_exclusive(head, runidx, n, tmp, s);
  Summary *sum = W.sum.get<Summary>(n);
  uint32_t *khead = W.khead.get<uint32_t>(n), *keyidx = W.keyidx.get<uint32_t>(n);
  uint32_t *counts = W.nbig.get<uint32_t>(3);  // [0] large cells, [1] summaries, [2] cells
  CK(cudaMemsetAsync(khead, 0, n * 4, s));
  CK(cudaMemsetAsync(counts, 0, 12, s));
  launch_run_reduce(sorted, n, head, runidx, sum, khead, counts + 1, s);
  scan_exclusive(khead, keyidx, n, tmp, s);
  uint32_t *nrec = W.nrec.get<uint32_t>(n), *recoff = W.recoff.get<uint32_t>(n);
  CK(cudaMemsetAsync(nrec, 0, n * 4, s));
  ClassifyArgs ca{interval, (uint32_t)L.GT, (uint32_t)std::max<uint64_t>(L.LT, 1), snap};
  if (bm) {
    ca.n_kernels = bm->n;
    ca.kbase = bm->kbase;
    ca.kGT = bm->kGT;
    ca.kLT = bm->kLT;
  }
  ca.big = W.big.get<uint32_t>(big_cells_cap(n));
  ca.bigres = W.bigres.get<CellResult>(big_cells_cap(n));
  ca.cellres = W.cellres.get<CellResult>(n);
  ca.nbig = counts;
  ca.nsum = counts + 1;
  ca.ncell = counts + 2;
  ca.cstart = W.cstart.get<uint32_t>(n);
  launch_cell_starts(khead, keyidx, n, ca, s);
  launch_key_classify(sum, n, nrec, ca, s);
  launch_big_classify(sum, n, keyidx, nrec, ca, s);
  scan_exclusive(nrec, recoff, n, tmp, s);
  CK(cudaMemcpyAsync(hstats, recoff + n - 1, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hstats + 1, nrec + n - 1, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const uint64_t nrecs = (uint64_t)hstats[0] + hstats[1];
  if (nrecs == 0) return;
  OutRec *out = W.out.get<OutRec>(nrecs);
  if (bm) ca.rec_kernel = W.reckern.get<uint32_t>(nrecs);
  launch_key_emit(sum, n, nrec, recoff, out, ca, s);
  launch_big_emit(sum, n, keyidx, nrec, recoff, out, ca, s);
  if (bm) {  // through page-locked buffers into the instances' lists (on the sink's thread)
    OutRec *hr = bm->sink->records(nrecs);
    uint32_t *hk = bm->sink->kernels(nrecs);
    CK(cudaMemcpyAsync(hr, out, nrecs * sizeof(OutRec), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hk, ca.rec_kernel, nrecs * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    bm->sink->submit(nrecs);
    return;
  }
  size_t old = races.size();
  races.resize(old + nrecs);
  CK(cudaMemcpyAsync(races.data() + old, out, nrecs * sizeof(OutRec), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
}

// Sort path: the whole interval log is made dense, sorted and classified.
void classify_sorted(Workspace &W, LogRec *log, uint32_t n_slices, uint64_t slice, const uint32_t *count,
                     uint64_t keys, uint64_t N, uint32_t interval, const Layout &L, int32_t *snap,
                     uint32_t *hstats, std::vector<OutRec> &races, cudaStream_t s) {
  uint32_t *offs = W.ctaoff.get<uint32_t>(n_slices);
  uint32_t *tmp = W.scan.get<uint32_t>(scan_tmp_words(n_slices));
  scan_exclusive(count, offs, n_slices, tmp, s);
  CK(cudaMemcpyAsync(hstats, offs + n_slices - 1, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hstats + 1, count + n_slices - 1, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const uint64_t n = (uint64_t)hstats[0] + hstats[1];
  if (n == 0) return;
  LogRec *dense = W.logb.get<LogRec>(n);
  launch_densify(log, n_slices, slice, count, offs, dense, s);
  tmp = W.scan.get<uint32_t>(std::max(sort_tmp_words(n), scan_tmp_words(n)));
  LogRec *sorted = sort_log(dense, log, n, bitwidth(N), bitwidth(keys) + bitwidth(N), tmp, s);
  classify_run(W, sorted, n, interval, L, snap, hstats, races, s);
}

// Owner table of 4 words per cell (see shadow_claim); words tagged with an
// older tag count as empty, so the table is cleared only when it is
// (re)allocated or the 6-bit tag wraps.
// The table keeps the size of the largest instance (or batch) seen, which
// can be gigabytes; only its first W.owner_hi words can hold tags, so a
// clear covers those and no more.
uint32_t *shadow_table(Workspace &W, uint64_t keys, cudaStream_t s) {
  const size_t before = W.owner.cap;
  uint32_t *t = W.owner.get<uint32_t>(4 * keys);
  if (W.owner.cap != before) {  // a new buffer
    CK(cudaMemsetAsync(t, 0, W.owner.cap, s));
    W.epoch = 0;
    W.owner_hi = 0;
  } else if (W.epoch == 0 && W.owner_hi) {
    CK(cudaMemsetAsync(t, 0, W.owner_hi * 4, s));
    W.owner_hi = 0;
  }
  W.owner_hi = std::max<uint64_t>(W.owner_hi, 4 * keys);
  return t;
}

// next interval tag; when the 6-bit tag wraps, the words in use are cleared
// and `extent` (the running instance's words) becomes the range in use
uint32_t shadow_next_tag(Workspace &W, cudaStream_t s, uint64_t extent) {
  if (W.epoch >= 63) {
    CK(cudaMemsetAsync(W.owner.p, 0, W.owner_hi * 4, s));
    W.epoch = 0;
    W.owner_hi = extent;
  }
  return ++W.epoch;
}

// Shadow path, device half: every written cell takes its highest writer's
// last write, committed from that work-item's own-write table, and the
// records of cells that need the exact classification (two or more writers,
// or one writer and another reader) are compacted into W.logb; the number
// of compacted records lands in *dcount (64-bit).
void shadow_launch(Workspace &W, const LogRec *log, uint32_t n_slices, uint64_t slice, const uint32_t *count,
                   uint64_t N, int32_t *snap, const uint32_t *owner, uint32_t tag, const uint2 *ow,
                   const uint32_t *ow_count, uint32_t *dcount, cudaStream_t s) {
  launch_shadow_commit(ow, ow_count, N, (uint32_t)N, owner, tag, snap, s);
  unsigned long long *cnt = reinterpret_cast<unsigned long long *>(dcount);
  CK(cudaMemsetAsync(cnt, 0, 8, s));
  LogRec *shared = W.logb.get<LogRec>((uint64_t)n_slices * slice);
  launch_shadow_compact(log, n_slices, slice, count, owner, tag, shared, cnt, s);
}

// Shadow path, host half: the m compacted records are sorted and classified
// (no commits: shadow_launch made them all).  Reads only W.logb and the
// classification's own buffers, so it may run on another stream while the
// next interval runs.
void shadow_finish(Workspace &W, uint64_t m, uint64_t keys, uint64_t N, uint32_t interval, const Layout &L,
                   uint32_t *hstats, std::vector<OutRec> &races, cudaStream_t s) {
  if (m == 0) return;
  LogRec *shared = W.logb.as<LogRec>();
  uint32_t *tmp = W.scan.get<uint32_t>(std::max(sort_tmp_words(m), scan_tmp_words(m)));
  LogRec *other = W.compact.get<LogRec>(m);
  LogRec *sorted = sort_log(shared, other, m, bitwidth(N), bitwidth(keys) + bitwidth(N), tmp, s);
  classify_run(W, sorted, m, interval, L, nullptr, hstats, races, s);
}

// The stream the shadow path classifies on while the next interval runs:
// the highest priority, so that the classification's blocks are scheduled
// as soon as the interval kernel's blocks leave room.
cudaStream_t classify_stream(Workspace &W) {
  if (!W.cstream) {
    int least = 0, greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CK(cudaStreamCreateWithPriority(&W.cstream, cudaStreamNonBlocking, greatest));
  }
  return W.cstream;
}

// Report of one instance from nr race records (already in cell order) and
// the error records, which follow them.  owned: null, or a malloc'd array
// that already holds the races and then the errors and becomes the
// report's (no copy).
rc_report *make_report_core(const OutRec *races, size_t nr, const std::vector<OutRec> &errors, OutRec *owned,
                            uint32_t n_intervals, uint64_t acc_g, uint64_t acc_l, uint64_t logged, uint64_t GT,
                            const int32_t *final_dev, cudaStream_t s) {
  rc_report *rep = static_cast<rc_report *>(std::calloc(1, sizeof(rc_report)));
  if (!rep) {
    std::free(owned);
    throw Fail{RC_E_NOMEM, "report allocation failed"};
  }
  rep->n_intervals = n_intervals;
  rep->n_global = acc_g;
  rep->n_local = acc_l;
  rep->n_access = acc_g + acc_l;
  rep->n_logged = logged;
  bool racy = false, div = false, as = false, oob = false;
  for (size_t i = 0; i < nr; i++) {
    const uint32_t c = races[i].cls;
    racy |= c == CLS_WW_RACE || c == CLS_RW_RACE || c == CLS_XG_WW_RACE || c == CLS_XG_RW_RACE;
  }
  for (const OutRec &x : errors) {
    div |= x.cls == CLS_DIVERGENCE;
    as |= x.cls == CLS_ASSERT;
    oob |= x.cls == CLS_OOB;
  }
  rep->status = racy ? RC_RACY : div ? RC_ERROR_DIVERGENCE : as ? RC_ERROR_ASSERT : oob ? RC_ERROR_OOB : RC_RACE_FREE;
  rep->n_records = nr + errors.size();
  static_assert(sizeof(rc_record) == sizeof(OutRec), "record layout");
  if (owned) {
    rep->records = reinterpret_cast<rc_record *>(owned);
  } else if (rep->n_records) {
    rep->records = static_cast<rc_record *>(std::malloc(rep->n_records * sizeof(rc_record)));
    if (!rep->records) {
      std::free(rep);
      throw Fail{RC_E_NOMEM, "report allocation failed"};
    }
    if (nr) std::memcpy(rep->records, races, nr * sizeof(OutRec));
    if (!errors.empty()) std::memcpy(rep->records + nr, errors.data(), errors.size() * sizeof(OutRec));
  }
  rep->final_len = GT;
  if (final_dev && GT) {
    rep->final_global = static_cast<int32_t *>(std::malloc(GT * 4));
    if (!rep->final_global) {
      std::free(rep->records);
      std::free(rep);
      throw Fail{RC_E_NOMEM, "report allocation failed"};
    }
    CK(cudaMemcpyAsync(rep->final_global, final_dev, GT * 4, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  return rep;
}

// Report of one instance: race records (already in cell order), error
// records, counters, status (Sec. 4: racy iff a WW or RW race record) and,
// if asked, the final global memory read from the device snapshot.
rc_report *make_report(const std::vector<OutRec> &races, const std::vector<OutRec> &errors, uint32_t n_intervals,
                       uint64_t acc_g, uint64_t acc_l, uint64_t logged, uint64_t GT, const int32_t *final_dev,
                       cudaStream_t s) {
  return make_report_core(races.data(), races.size(), errors, nullptr, n_intervals, acc_g, acc_l, logged, GT,
                          final_dev, s);
}

// The same from a batch instance's record list, whose array the report takes.
rc_report *make_report(RecList &races, const std::vector<OutRec> &errors, uint32_t n_intervals, uint64_t acc_g,
                       uint64_t acc_l, uint64_t logged, uint64_t GT, const int32_t *final_dev, cudaStream_t s) {
  const size_t nr = races.n;
  races.append(errors.data(), errors.size());
  OutRec *arr = races.release();
  return make_report_core(arr, nr, errors, arr, n_intervals, acc_g, acc_l, logged, GT, final_dev, s);
}

// Stop points of one interval -> divergence records (Sec. 4 barrier-release
// rule: every live work-item must wait at the same barrier, or all exit).
// Returns true when the run goes on to another interval.
bool barrier_agreement(uint32_t interval, uint32_t n_barriers, const uint32_t *stop_min, const uint32_t *stop_cnt,
                       std::vector<OutRec> &errors) {
  uint32_t n_points = 0;
  bool any_barrier = false;
  for (uint32_t k = 0; k <= n_barriers; k++) {
    if (!stop_cnt[k]) continue;
    n_points++;
    if (k < n_barriers) any_barrier = true;
  }
  if (n_points >= 2) {
    std::vector<OutRec> dv;
    for (uint32_t k = 0; k <= n_barriers; k++) {
      if (!stop_cnt[k]) continue;
      dv.push_back(OutRec{interval, 0, 0, 0, CLS_DIVERGENCE, stop_min[k], k < n_barriers ? k : 0xFFFFFFFFu, 0, 0,
                          stop_cnt[k]});
    }
    std::sort(dv.begin(), dv.end(), [](const OutRec &x, const OutRec &y) { return x.t_a < y.t_a; });
    errors.insert(errors.end(), dv.begin(), dv.end());  // after this interval's OOB/ASSERT (class order)
    return false;
  }
  return any_barrier;
}

// Resident run of one instance (see interp.cu): every interval in one
// cooperative launch, then the exact classification of the compacted records
// interval by interval (their commits were made in-kernel).  Returns null
// when the instance cannot be resident or the run had to stop early (the
// record buffer or the interval table filled up); the caller then checks it
// interval by interval from the initial state.
constexpr uint32_t kResidentMaxIntervals = 4096;

// A device-usable address of page-locked host memory (null for pageable or
// device memory): kernels can read such memory directly over the CPU-GPU
// link, which on this part outruns a copy-engine transfer.
const int32_t *device_view(const int32_t *host) {
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, host) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (pa.type != cudaMemoryTypeHost || !pa.devicePointer) return nullptr;
  return static_cast<const int32_t *>(pa.devicePointer);
}

// The bytecode with CTL_PRIV on every access the pre-filter proves private
// for this launch shape and these input lengths (cached on the program).
const std::vector<Insn> &private_code(const Program &P, uint32_t G, uint32_t S, const rc_input *in) {
  std::vector<uint32_t> lens;
  if (!prove_lengths(P, in, lens)) throw Fail{RC_E_INVALID, "input count differs from the kernel's global declarations"};
  Program::PrivateCode &c = P.priv;
  if (!(c.valid && c.G == G && c.S == S && c.lens == lens)) {
    rc_prove_result r;
    std::vector<uint8_t> flags;
    prove_analyze(P, G, S, lens, &r, &flags, 0);  // the cheap analysis: it runs per launch shape
    c.code = P.code;
    c.n_private = 0;
    for (size_t k = 0; k < flags.size(); k++)
      if (flags[k]) {
        c.code[k].ctl |= CTL_PRIV;
        c.n_private++;
      }
    c.G = G;
    c.S = S;
    c.lens = lens;
    c.valid = true;
  }
  return c.code;
}

rc_report *run_resident(Workspace &W, const Instance &I, const Layout &L, const InterpArgs &base, size_t base_smem,
                        uint32_t *owner, int32_t *snap, OutRec *errs, uint32_t *hscratch, cudaStream_t s,
                        const JitKernel *jk) {
  const Program &P = *I.p;
  static int coop = -1;
  if (coop < 0) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  }
  if (!coop) return nullptr;
  // intervals of bounded work only (the grid barrier's wait is bounded too)
  if (P.max_access_per_interval > 4096) return nullptr;
  // the most own-write slots that still let every work-group be resident
  const int nsm = sm_count();
  int slots = -1;
  size_t smem = 0;
  const size_t max_dyn = jk ? kMaxSmemPerBlock - jk->static_smem : interp_max_dynamic_smem();
  for (int sl = (int)std::min<uint64_t>(8, P.max_write_per_interval); sl >= 0; sl--) {
    const size_t sm = base_smem + (size_t)sl * I.S * 8;
    if (sm > max_dyn) continue;
    const int per_sm = jk ? jit_blocks_per_sm(*jk, I.S, sm) : interp_resident_blocks_per_sm((uint32_t)P.code.size(), I.S, sm);
    if ((uint64_t)per_sm * nsm >= I.G) {
      slots = sl;
      smem = sm;
      break;
    }
  }
  if (slots < 0) return nullptr;
  const uint32_t nstops = P.n_barriers + 1;
  // device words: [0,1] logged accesses (u64), [2] unused, [3] error count,
  // [4,5] intervals run / last tag, [6,7] flags by interval parity, [8,9] compacted records
  // (u64), [10..13] access counters (2 x u64), then two stop tables (smallest work-item, count)
  // by interval parity
  enum : uint32_t { R_LOGGED = 0, R_BAR = 0, R_ERRS = 3, R_INFO = 4, R_FLAGS = 6, R_TOTAL = 8, R_ACC = 10, R_STOPS = 14 };
  const size_t words = R_STOPS + 4 * nstops;
  uint32_t *d = W.rstat.get<uint32_t>(words);
  CK(cudaMemsetAsync(d, 0, words * 4, s));
  unsigned *bar = W.rbar.get<unsigned>(kGridBarWords);
  CK(cudaMemsetAsync(bar, 0, kGridBarWords * 4, s));
  CK(cudaMemsetAsync(d + R_STOPS, 0xFF, 2 * nstops * 4, s));
  unsigned long long *ivoff = W.rivoff.get<unsigned long long>(kResidentMaxIntervals + 1);
  CK(cudaMemsetAsync(ivoff, 0, 8, s));
  const uint64_t acc_cap = std::max<uint64_t>((uint64_t)base.warps_per_cta * I.G * base.warp_slice, 1u << 16);
  LogRec *acc = W.logb.get<LogRec>(acc_cap);

  InterpArgs a = base;
  a.interval = 0;
  a.tag = shadow_next_tag(W, s, 4 * L.keys);
  a.owner = owner;
  a.ow_slots = (uint32_t)slots;
  a.errs = errs;
  a.err_count = d + R_ERRS;
  a.stop_min = d + R_STOPS;
  a.stop_cnt = d + R_STOPS + 2 * nstops;
  a.acc = reinterpret_cast<unsigned long long *>(d + R_ACC);
  a.logged = reinterpret_cast<unsigned long long *>(d + R_LOGGED);
  a.flags = d + R_FLAGS;
  a.proceed = nullptr;
  a.group_div = nullptr;
  a.commit = snap;
  a.grid_bar = bar;
  a.acc_out = acc;
  a.acc_total = reinterpret_cast<unsigned long long *>(d + R_TOTAL);
  a.acc_cap = acc_cap;
  a.iv_off = ivoff;
  a.max_intervals = kResidentMaxIntervals;
  a.run_info = d + R_INFO;
  // an in-kernel wrap clears this instance's words; the host clears the rest
  // of the range in use after the run (below)
  a.owner_words = 4 * L.keys;
  a.barrier_limit_ns = 20000000000ull;
  if (g_prof.on) CK(cudaEventRecord(g_prof.ev[0], s));
  const cudaError_t e = jk ? launch_jit_resident(*jk, a, I.G, smem, s) : launch_interp_resident(a, I.G, smem, s);
  if (e == cudaErrorCooperativeLaunchTooLarge) {
    cudaGetLastError();
    return nullptr;
  }
  CK(e);
  if (g_prof.on) CK(cudaEventRecord(g_prof.ev[1], s));
  std::vector<uint32_t> h(words);
  CK(cudaMemcpyAsync(h.data(), d, words * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&h[R_BAR + 2], bar + 2, 4, cudaMemcpyDeviceToHost, s));  // the barrier's timeout word
  // the first record offsets come back with the same synchronisation
  constexpr uint32_t kOffHead = 64;
  std::vector<unsigned long long> off(kOffHead);
  CK(cudaMemcpyAsync(off.data(), ivoff, kOffHead * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  W.epoch = h[R_INFO + 1];  // the owner-table tag of the last interval
  if (h[R_INFO] && a.tag + h[R_INFO] - 1 > 63 && W.owner_hi > 4 * L.keys) {
    // the tag wrapped in-kernel: words past this instance's cells still hold
    // tags of the earlier epoch, which later calls would meet again
    CK(cudaMemsetAsync(owner + 4 * L.keys, 0, (W.owner_hi - 4 * L.keys) * 4, s));
    W.owner_hi = 4 * L.keys;
  }
  const uint32_t flags = h[R_FLAGS] | h[R_FLAGS + 1];
  if (h[R_BAR + 2]) throw Fail{RC_E_TIMEOUT, "a grid barrier of the resident run timed out"};
  if (flags & (FLAG_LOG_FULL | FLAG_OW_FULL | FLAG_ERR_FULL))
    throw Fail{RC_E_CAPACITY, "interval log, own-write table or error log overflowed"};
  if (flags & FLAG_ACC_FULL) return nullptr;
  const uint32_t n_run = h[R_INFO];
  if (n_run == 0) throw Fail{RC_E_CUDA, "the resident run reported no interval"};
  const uint32_t last = n_run - 1;
  const uint64_t acc_g = *reinterpret_cast<const uint64_t *>(&h[R_ACC]);
  const uint64_t acc_l = *reinterpret_cast<const uint64_t *>(&h[R_ACC + 2]);
  const uint64_t logged = *reinterpret_cast<const uint64_t *>(&h[R_LOGGED]);
  if (g_prof.on) {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, g_prof.ev[0], g_prof.ev[1]));
    g_prof.launches[0]++;
    g_prof.ms[0] += ms;
    g_prof.bytes[0] += 12.0 * (double)acc_g;
  }
  // error records by (interval, class, work-item); the divergence records of
  // the last interval's barrier agreement follow
  std::vector<OutRec> races, errors(std::min<uint32_t>(h[R_ERRS], base.err_cap));
  if (!errors.empty()) {
    CK(cudaMemcpyAsync(errors.data(), errs, errors.size() * sizeof(OutRec), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::sort(errors.begin(), errors.end(), [](const OutRec &x, const OutRec &y) {
      return x.interval != y.interval ? x.interval < y.interval : x.cls != y.cls ? x.cls < y.cls : x.t_a < y.t_a;
    });
  }
  const uint32_t *smin = &h[R_STOPS + (last & 1u) * nstops], *scnt = &h[R_STOPS + 2 * nstops + (last & 1u) * nstops];
  if (barrier_agreement(last, P.n_barriers, smin, scnt, errors)) return nullptr;  // stopped at the interval cap
  // the compacted records, classified interval by interval without commits
  if (n_run + 1 > kOffHead) {
    off.resize(n_run + 1);
    CK(cudaMemcpyAsync(off.data(), ivoff, (n_run + 1) * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  if (g_prof.on) CK(cudaEventRecord(g_prof.ev[2], s));
  for (uint32_t k = 0; k < n_run; k++) {
    const uint64_t m = off[k + 1] - off[k];
    if (!m) continue;
    uint32_t *tmp = W.scan.get<uint32_t>(std::max(sort_tmp_words(m), scan_tmp_words(m)));
    LogRec *other = W.compact.get<LogRec>(m);
    LogRec *sorted = sort_log(acc + off[k], other, m, bitwidth(I.N), bitwidth(L.keys) + bitwidth(I.N), tmp, s);
    classify_run(W, sorted, m, k, L, nullptr, hscratch, races, s);
  }
  if (g_prof.on) {
    CK(cudaEventRecord(g_prof.ev[3], s));
    CK(cudaEventSynchronize(g_prof.ev[3]));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, g_prof.ev[2], g_prof.ev[3]));
    g_prof.launches[1]++;
    g_prof.ms[1] += ms;
    g_prof.bytes[1] += 12.0 * (double)acc_g;
  }
  return make_report(races, errors, n_run, acc_g, acc_l, logged, L.GT, (I.in->flags & RC_WANT_FINAL_MEMORY) ? snap : nullptr,
                     s);
}

// One-CTA check of a small instance (interp.cu, small_check_kernel): every
// interval, its classification and barrier agreement in one launch, results
// written to page-locked host memory.  Returns null when the instance does
// not fit it (too many work-items, records or barriers) or the run had to
// stop early (more records than the CTA sorts, the interval cap); the
// caller then checks it another way from the initial state.  The snapshot
// must hold the inputs and the bytecode (without private flags: the CTA
// classifies from the full log) must be uploaded.
// One global input array of len int32 values into dst: pinned host memory
// read by a copy kernel over the CPU-GPU link, other memory by
// cudaMemcpyAsync.
void upload_global(const int32_t *src, int32_t *dst, uint64_t len, bool on_device, cudaStream_t s) {
  const int32_t *mapped = on_device ? nullptr : device_view(src);
  if (mapped) {  // pinned host memory: the SMs read it over the CPU-GPU link
    launch_copy_words(mapped, dst, len, s);
    CK(cudaGetLastError());
  } else {
    CK(cudaMemcpyAsync(dst, src, len * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  }
}

// The snapshot of an instance's start: the global inputs and zeroed local
// memory.
void load_inputs(const Instance &I, const Layout &L, int32_t *snap, cudaStream_t s) {
  const Program &P = *I.p;
  uint32_t gi = 0;
  for (size_t m = 0; m < P.mems.size(); m++) {
    if (P.mems[m].space != 0) continue;
    const uint64_t len = I.in->global_len[gi];
    if (len) {
      if (!I.in->global_init || !I.in->global_init[gi]) throw Fail{RC_E_INVALID, "missing global input"};
      upload_global(I.in->global_init[gi], snap + L.mems[m].base, len, I.in->on_device, s);
    }
    gi++;
  }
  if (L.keys > L.GT) CK(cudaMemsetAsync(snap + L.GT, 0, (L.keys - L.GT) * 4, s));
}

bool small_fits(const Program &P, uint64_t N) {
  const uint64_t B = std::max<uint64_t>(P.max_access_per_interval, 1);
  const uint32_t T = (uint32_t)std::max<uint64_t>(32, (N + 31) / 32 * 32);
  return N <= kSmallMaxItems && (uint64_t)T * B <= kSmallCap && P.n_barriers + 1 <= kSmallMaxStops &&
         small_check_smem((uint32_t)P.mems.size(), P.n_regs, T, 0, kSmallCap, 0) <= kMaxSmemPerBlock - 4096;
}

rc_report *run_small(Workspace &W, const Instance &I, const Layout &L, int32_t *snap, const Insn *dcode,
                     const MemInfo *dmems, cudaStream_t s) {
  const Program &P = *I.p;
  const uint32_t N = (uint32_t)I.N, RS = std::max<uint32_t>(32, (N + 31) / 32 * 32);
  const uint64_t B = std::max<uint64_t>(P.max_access_per_interval, 1);
  const uint64_t capw = std::max<uint64_t>(P.max_write_per_interval, 1);
  const uint32_t cap = (uint32_t)std::min<uint64_t>(kSmallCap, (uint64_t)RS * B);
  const size_t budget = kMaxSmemPerBlock - 4096;
  uint32_t slots = 0;
  while (slots < 8 && slots < capw &&
         small_check_smem((uint32_t)P.mems.size(), P.n_regs, RS, slots + 1, cap, 0) <= budget)
    slots++;
  // the snapshot in shared memory first (the interpreter's reads wait on it),
  // then the sort's records and summaries, as far as they fit
  const bool smem_snap = L.keys <= (1u << 20) &&
      small_check_smem((uint32_t)P.mems.size(), P.n_regs, RS, slots, cap, (uint32_t)L.keys) <= budget;
  size_t smem = small_check_smem((uint32_t)P.mems.size(), P.n_regs, RS, slots, cap, smem_snap ? (uint32_t)L.keys : 0);
  const size_t log_b = (size_t)RS * B * sizeof(LogRec);
  const bool smem_log = smem + log_b <= budget;
  if (smem_log) smem += log_b;
  const bool smem_scratch = smem + (size_t)cap * (sizeof(LogRec) + sizeof(Summary)) <= budget;
  if (smem_scratch) smem += (size_t)cap * (sizeof(LogRec) + sizeof(Summary));
  // the sort: counting over (cell, work-item) when the pairs are few, else bitonic
  const uint64_t pairs = L.keys * RS;
  const bool bins = smem_scratch && pairs <= kSmallBins && smem + pairs * 4 <= budget;
  if (bins) smem += pairs * 4;
  const uint32_t out_cap = 16 * kSmallCap, err_cap = N + kSmallMaxStops;
  SmallArgs a{};
  InterpArgs &A = a.A;
  A.code = dcode;
  A.mems = dmems;
  A.n_insn = (uint32_t)P.code.size();
  A.n_regs = P.n_regs;
  A.n_mems = (uint32_t)P.mems.size();
  A.n_barriers = P.n_barriers;
  A.S = I.S;
  A.G = I.G;
  A.GT = (uint32_t)L.GT;
  A.LT = (uint32_t)L.LT;
  A.snap = snap;
  A.commit = snap;
  A.ow = W.ow.get<uint2>(capw * RS);
  A.capw = (uint32_t)std::min<uint64_t>(capw, 0xFFFFFFFFu);
  A.ow_stride = RS;
  A.ow_slots = slots;
  A.warps_per_cta = RS / 32;
  A.warp_slice = 32 * B;
  A.log = W.loga.get<LogRec>((uint64_t)RS * B);
  A.errs = W.errs.get<OutRec>(err_cap);
  A.err_cap = err_cap;
  uint32_t *cnt = W.rstat.get<uint32_t>(1);
  A.err_count = cnt;
  if (!smem_scratch) {
    a.sorted = W.compact.get<LogRec>(cap);
    a.sum = W.sum.get<Summary>(cap);
  }
  a.cap = cap;
  a.out_cap = out_cap;
  a.max_intervals = kResidentMaxIntervals;
  a.n_items = N;
  a.reg_stride = RS;
  a.smem_scratch = smem_scratch ? 1u : 0u;
  a.smem_snap = smem_snap ? 1u : 0u;
  a.smem_log = smem_log ? 1u : 0u;
  a.bins = bins ? (uint32_t)pairs : 0u;
  a.n_cells = (uint32_t)L.keys;
  unsigned char *h = W.hsmall.get<unsigned char>(64 + (size_t)(out_cap + err_cap) * sizeof(OutRec));
  unsigned char *hd = nullptr;
  CK(cudaHostGetDevicePointer(reinterpret_cast<void **>(&hd), h, 0));
  a.res = reinterpret_cast<unsigned long long *>(hd);
  a.host_out = reinterpret_cast<OutRec *>(hd + 64);
  a.host_err = a.host_out + out_cap;
  a.out = W.out.get<OutRec>(out_cap);
  CK(cudaMemsetAsync(cnt, 0, 4, s));
  if (g_prof.on) CK(cudaEventRecord(g_prof.ev[0], s));
  CK(launch_small_check(a, 1024, smem, s));
  if (g_prof.on) CK(cudaEventRecord(g_prof.ev[1], s));
  CK(cudaStreamSynchronize(s));
  const unsigned long long *res = reinterpret_cast<const unsigned long long *>(h);
  const uint32_t flags = (uint32_t)(res[3] >> 32), n_intervals = (uint32_t)res[3];
  if (flags & (FLAG_LOG_FULL | FLAG_OW_FULL | FLAG_ERR_FULL))
    throw Fail{RC_E_CAPACITY, "interval log, own-write table or error log overflowed"};
  if (flags) return nullptr;  // more records or intervals than the CTA takes
  if (g_prof.on) {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, g_prof.ev[0], g_prof.ev[1]));
    g_prof.launches[0]++;
    g_prof.ms[0] += ms;
    g_prof.bytes[0] += 12.0 * (double)res[0];
  }
  const OutRec *ho = reinterpret_cast<const OutRec *>(h + 64);
  std::vector<OutRec> races(ho, ho + res[4]);
  std::vector<OutRec> errors(ho + out_cap, ho + out_cap + res[5]);
  std::sort(errors.begin(), errors.end(), [](const OutRec &x, const OutRec &y) {
    return x.interval != y.interval ? x.interval < y.interval : x.cls != y.cls ? x.cls < y.cls : x.t_a < y.t_a;
  });
  return make_report(races, errors, n_intervals, res[0], res[1], res[2], L.GT,
                     (I.in->flags & RC_WANT_FINAL_MEMORY) ? snap : nullptr, s);
}

rc_report *run_instance(const Instance &I) {
  Workspace &W = g_ws;
  const Program &P = *I.p;
  cudaStream_t s = I.s;
  if (!W.configured) {
    CK(interp_configure());
    W.configured = true;
  }
  Layout L = make_layout(P, I.in, I.G);
  const uint64_t N = I.N;
  // work-group-scoped barriers: per-group stop points in shared memory, a
  // cross-group table over the global cells
  const bool group = (I.in->flags & RC_GROUP_BARRIERS) != 0;
  if (group && 2 * L.GT >= 0xFFFFFFFFull) throw Fail{RC_E_CAPACITY, "too many global cells for group scope"};
  // small instances: one CTA, one launch (strategy 0 and 4), with the plain
  // bytecode (the CTA classifies from the full log) and none of the other
  // paths' set-up (no pre-filter, owner table or work-item state)
  if ((g_strategy == 0 || g_strategy == 4) && !group && !I.explore && g_engine != 2 && small_fits(P, N)) {
    // bytecode, memory table and (host) inputs packed into one page-locked
    // block and sent with one copy; the snapshot is the block's tail
    const size_t code_b = P.code.size() * sizeof(Insn), mems_b = std::max<size_t>(L.mems.size(), 1) * sizeof(MemInfo);
    const size_t snap_off = (code_b + mems_b + 15) & ~(size_t)15, total = snap_off + std::max<uint64_t>(L.keys, 1) * 4;
    unsigned char *hb = W.hstage.get<unsigned char>(total);
    unsigned char *db = W.stage.get<unsigned char>(total);
    std::memcpy(hb, P.code.data(), code_b);
    if (!L.mems.empty()) std::memcpy(hb + code_b, L.mems.data(), L.mems.size() * sizeof(MemInfo));
    int32_t *hsnap = reinterpret_cast<int32_t *>(hb + snap_off);
    bool packed = !I.in->on_device;  // host inputs (pinned or not) are copied into the block
    if (packed) {
      uint32_t gi = 0;
      for (size_t m = 0; m < P.mems.size(); m++) {
        if (P.mems[m].space != 0) continue;
        const uint64_t len = I.in->global_len[gi];
        if (len) {
          if (!I.in->global_init || !I.in->global_init[gi]) throw Fail{RC_E_INVALID, "missing global input"};
          std::memcpy(hsnap + L.mems[m].base, I.in->global_init[gi], len * 4);
        }
        gi++;
      }
      if (L.keys > L.GT) std::memset(hsnap + L.GT, 0, (L.keys - L.GT) * 4);
    }
    CK(cudaMemcpyAsync(db, hb, packed ? total : snap_off, cudaMemcpyHostToDevice, s));
    CK(interp_upload_code(reinterpret_cast<const Insn *>(hb), (uint32_t)P.code.size(), s));
    int32_t *snap = reinterpret_cast<int32_t *>(db + snap_off);
    if (!packed) load_inputs(I, L, snap, s);
    rc_report *r = run_small(W, I, L, snap, reinterpret_cast<const Insn *>(db),
                             reinterpret_cast<const MemInfo *>(db + code_b), s);
    if (r) return r;  // else (too many records or intervals): the other paths, from the start
  }
  // own-write slots in shared memory: as many as fit (up to 8) while keeping
  // at least two CTAs, or 2048 threads, per SM
  const size_t base_smem = interp_smem_bytes((uint32_t)P.mems.size(), P.n_regs, I.S, 0) +
                           (group ? 8ull * (P.n_barriers + 1) : 0);
  if (base_smem > interp_max_dynamic_smem())
    throw Fail{RC_E_INVALID, "kernel too large for shared memory at this group size"};
  const uint32_t ctas_per_sm = std::max<uint32_t>(2, 2048 / I.S);
  const size_t budget = std::min<size_t>(interp_max_dynamic_smem(), 224 * 1024 / ctas_per_sm - 1024);
  uint32_t ow_slots = 0;
  while (ow_slots < 8 && ow_slots < P.max_write_per_interval &&
         base_smem + (size_t)(ow_slots + 1) * I.S * 8 <= budget)
    ow_slots++;
  const size_t smem = base_smem + (size_t)ow_slots * I.S * 8;
  const uint32_t wpc = (I.S + 31) / 32;               // warps per work-group
  const uint32_t n_slices = I.G * wpc;                 // one log slice per warp
  const uint64_t slice = 32ull * std::max<uint64_t>(P.max_access_per_interval, 1);
  const uint64_t cap = (uint64_t)n_slices * slice;     // >= N * bound: the log cannot overflow
  const uint64_t capw = std::max<uint64_t>(P.max_write_per_interval, 1);
  if (cap >= 0xFFFFFFFFull) throw Fail{RC_E_CAPACITY, "interval log bound exceeds 2^32 records"};
  // the sort path also needs a summary and index arrays per record; when that
  // would not fit, every interval takes the shadow path (only the records of
  // shared written cells are sorted)
  const uint64_t mem_budget = (uint64_t)200 << 30;
  const uint64_t base_need = cap * sizeof(LogRec) * 2 + N * (capw * 8 + 4ull * P.n_regs + 12) + L.keys * 20;
  const bool sort_fits = base_need + cap * (sizeof(Summary) + 24) <= mem_budget;
  if (base_need > mem_budget) throw Fail{RC_E_CAPACITY, "instance needs more than 200 GiB of workspace"};
  // strategy 3 (resident) runs like 0 when the instance cannot be resident
  const int asked = g_strategy == 3 || g_strategy == 4 ? 0 : g_strategy;
  const int fixed_strategy = asked ? asked : (sort_fits ? 0 : 2);
  if (fixed_strategy == 1 && !sort_fits) throw Fail{RC_E_CAPACITY, "the sort path does not fit this instance"};

  // ---- set-up: program, memory snapshot, work-item state
  Insn *dcode = W.code.get<Insn>(P.code.size());
  MemInfo *dmems = W.mems.get<MemInfo>(std::max<size_t>(L.mems.size(), 1));
  auto upload_code = [&](const std::vector<Insn> &c) {
    CK(cudaMemcpyAsync(dcode, c.data(), c.size() * sizeof(Insn), cudaMemcpyHostToDevice, s));
    CK(interp_upload_code(c.data(), (uint32_t)c.size(), s));
  };
  // resident run: every work-group on the GPU at once (one cooperative
  // launch runs all intervals), shadow owner table, full warps
  const bool resident_wanted =
      (g_strategy == 0 || g_strategy == 3 || g_strategy == 4) && !group && !I.explore && I.S % 32 == 0;
  // accesses the pre-filter proves private skip the log wherever commits come
  // from the owner table (resident runs, the shadow strategy throughout);
  // the full sort commits from the log, the cross-group table and the
  // explorer read it
  const bool prefilter = !group && !I.explore && !(I.in->flags & RC_LOG_EVERY_ACCESS);
  const std::vector<Insn> *pcode =
      prefilter && (resident_wanted || fixed_strategy == 2) ? &private_code(P, I.G, I.S, I.in) : nullptr;
  const std::vector<Insn> &interval_code = pcode && fixed_strategy == 2 ? *pcode : P.code;
  upload_code(pcode && resident_wanted ? *pcode : interval_code);
  // compiled intervals: one kernel per program, launch shape and mode (cached)
  const bool jit = !group && !I.explore && g_engine != 1 && (g_engine == 2 || N >= kJitAutoItems);
  JitKernel jk_res, jk_iv;
  bool have_res = false, have_iv = false;
  // the compiled interval kernel runs a work-group of 512 or more work-items
  // (a multiple of 256) as CTAs of 256: the same registers per SM, four
  // independent CTAs instead of one, so one CTA's tail overlaps the others'
  // work
  const uint32_t iv_split = !group && I.S >= 512 && I.S % 256 == 0 ? I.S / 256 : 1;
  const uint32_t iv_threads = I.S / iv_split;
  const size_t iv_smem = interp_smem_bytes((uint32_t)P.mems.size(), P.n_regs, iv_threads, ow_slots) +
                         (group ? 8ull * (P.n_barriers + 1) : 0);
  if (jit) {
    std::string why;
    if (!jit_available(&why)) {
      if (g_engine == 2) throw Fail{RC_E_INVALID, "compiled intervals unavailable: " + why};
    } else {
      try {
        const uint32_t nsm = (uint32_t)sm_count();
        const uint32_t per_sm = (I.G + nsm - 1) / nsm;  // CTAs each SM must hold for a resident run
        if (resident_wanted && (uint64_t)per_sm * I.S <= 2048) {
          JitShape sh;
          sh.resident = true;
          sh.threads = I.S;
          sh.min_blocks = std::min<uint32_t>(per_sm, 32);  // 32: the most CTAs an SM holds
          jk_res = jit_kernel(P, pcode ? *pcode : P.code, sh);
          have_res = true;
        }
        JitShape sh;
        sh.threads = iv_threads;
        // 1024 threads per SM: up to 64 registers a thread (a 32-register
        // bound, two 1024-thread CTAs per SM, measured 6.26 against 5.99 ms
        // per interval on the 2^26-work-item stress program)
        sh.min_blocks = std::min<uint32_t>(std::max<uint32_t>(1, 1024 / iv_threads), 32);
        jk_iv = jit_kernel(P, interval_code, sh);
        have_iv = iv_smem <= kMaxSmemPerBlock - jk_iv.static_smem;
      } catch (const JitError &e) {
        throw Fail{RC_E_CUDA, e.msg};
      }
    }
  }
  if (!L.mems.empty())
    CK(cudaMemcpyAsync(dmems, L.mems.data(), L.mems.size() * sizeof(MemInfo), cudaMemcpyHostToDevice, s));
  int32_t *snap = W.snap.get<int32_t>(std::max<uint64_t>(L.keys, 1));
  auto load_snapshot = [&]() { load_inputs(I, L, snap, s); };
  load_snapshot();
  int32_t *regs = W.regs.get<int32_t>(N * P.n_regs);
  uint32_t *pc = W.pc.get<uint32_t>(N), *st = W.st.get<uint32_t>(N);
  // work-item state starts at zero; a resident run sets its own up in-kernel
  auto clear_state = [&]() {
    CK(cudaMemsetAsync(regs, 0, N * P.n_regs * 4, s));
    CK(cudaMemsetAsync(pc, 0, N * 4, s));
    CK(cudaMemsetAsync(st, 0, N * 4, s));
  };
  uint2 *ow = W.ow.get<uint2>(N * capw);
  LogRec *log = W.loga.get<LogRec>(cap);
  const uint32_t err_cap = (uint32_t)std::min<uint64_t>(N, 1u << 24);
  // two of everything an interval reports (by interval parity), so the next
  // interval can be queued while the host reads this one's
  OutRec *errs2 = W.errs.get<OutRec>(2ull * err_cap);
  const uint32_t nstops = P.n_barriers + 1;
  const size_t stat_words = ST_STOPS + 2 * nstops;
  uint32_t *dstats2 = W.stats.get<uint32_t>(2 * stat_words + 2);
  uint32_t *gate = dstats2 + 2 * stat_words;  // gate[parity]: the speculatively queued interval may run
  uint32_t *hstats2 = W.hstats.get<uint32_t>(2 * stat_words + 8);
  uint32_t *hscratch = hstats2 + 2 * stat_words;
  if (!W.sev[0])
    for (auto &e : W.sev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));

  const std::string tkey = single_key(N, P.max_access_per_interval);
  uint32_t *owner = nullptr;
  if (fixed_strategy != 1 || resident_wanted) owner = shadow_table(W, L.keys, s);
  if (!fixed_strategy) tuner_events();
  uint32_t *warp_count = W.ctacnt.get<uint32_t>(n_slices);
  uint32_t *ow_cnt = W.owcnt.get<uint32_t>(N);

  XgCell *xg = nullptr;
  uint2 *xgcnt = nullptr;
  if (group) {
    xg = W.xg.get<XgCell>(std::max<uint64_t>(L.GT, 1));
    xgcnt = W.xgcnt.get<uint2>(std::max<uint64_t>(L.GT, 1));
    launch_xg_init(xg, xgcnt, snap, L.GT, s);
    CK(cudaGetLastError());
  }

  InterpArgs base{};
  base.code = dcode;
  base.mems = dmems;
  for (size_t k = 0; k < L.mems.size() && k < kInlineMems; k++) base.mem_inline[k] = L.mems[k];
  base.n_insn = (uint32_t)P.code.size();
  base.n_regs = P.n_regs;
  base.n_mems = (uint32_t)P.mems.size();
  base.n_barriers = P.n_barriers;
  base.S = I.S;
  base.G = I.G;
  base.group0 = 0;
  base.split = 1;
  base.GT = (uint32_t)L.GT;
  base.LT = (uint32_t)L.LT;
  base.snap = snap;
  base.regs = regs;
  base.pc = pc;
  base.st = st;
  base.ow = ow;
  base.capw = (uint32_t)std::min<uint64_t>(capw, 0xFFFFFFFFu);
  base.ow_stride = (uint32_t)N;
  base.ow_slots = ow_slots;
  base.log = log;
  base.warp_count = warp_count;
  base.warps_per_cta = wpc;
  base.warp_slice = slice;
  base.err_cap = err_cap;
  base.ow_count = ow_cnt;
  if (resident_wanted) {
    rc_report *r = run_resident(W, I, L, base, base_smem, owner, snap, errs2, hscratch, s,
                                have_res ? &jk_res : nullptr);
    if (r) return r;
    load_snapshot();  // the resident run stopped early: start over interval by interval
    if (pcode && &interval_code != pcode) upload_code(interval_code);
  }
  clear_state();
  auto dbuf = [&](uint32_t k) { return dstats2 + (k & 1) * stat_words; };
  auto hbuf = [&](uint32_t k) { return hstats2 + (k & 1) * stat_words; };
  // one interval's interpreter launch (gated: runs only if gate[k & 1] is set on the device)
  auto enqueue_interp = [&](uint32_t k, int strategy, uint32_t tag, bool gated, bool timed) {
    if (I.explore && k < I.explore->max_intervals) {  // every schedule of interval k, from this state
      CK(cudaStreamSynchronize(s));
      ExploreInput e{};
      e.code = dcode;
      e.mems = dmems;
      e.n_insn = (uint32_t)P.code.size();
      e.N = (uint32_t)N;
      e.S = I.S;
      e.n_regs = P.n_regs;
      e.cells = (uint32_t)L.keys;
      e.GT = (uint32_t)L.GT;
      e.LT = (uint32_t)L.LT;
      e.interval = k;
      e.max_access = (uint32_t)std::min<uint64_t>(P.max_access_per_interval, 1u << 20);
      e.snap = snap;
      e.regs = regs;
      e.pc = pc;
      e.st = st;
      try {
        if (I.explore->pairs) {
          std::vector<uint32_t> pv;
          I.explore->results.push_back(explore_interval(e, I.explore->max_states, s, &pv));
          I.explore->pair_results.push_back(std::move(pv));
        } else {
          I.explore->results.push_back(explore_interval(e, I.explore->max_states, s));
        }
      } catch (const ExploreError &x) {
        throw Fail{RC_E_CUDA, x.msg};
      }
    }
    uint32_t *d = dbuf(k);
    CK(cudaMemsetAsync(d, 0, ST_STOPS * 4, s));  // counters, flags, error count, scratch
    CK(cudaMemsetAsync(d + ST_STOPS, 0xFF, nstops * 4, s));
    CK(cudaMemsetAsync(d + ST_STOPS + nstops, 0, nstops * 4, s));
    InterpArgs a = base;
    a.interval = k;
    a.errs = errs2 + (uint64_t)(k & 1) * err_cap;
    a.err_count = d + ST_ERRCNT;
    a.stop_min = d + ST_STOPS;
    a.stop_cnt = d + ST_STOPS + nstops;
    a.acc = reinterpret_cast<unsigned long long *>(d + ST_ACC);
    a.logged = reinterpret_cast<unsigned long long *>(d + ST_LOGGED);
    a.flags = d + ST_FLAGS;
    a.owner = strategy == 2 ? owner : nullptr;
    a.tag = tag;
    a.proceed = gated ? gate + (k & 1) : nullptr;
    a.group_div = group ? d + ST_GDIV : nullptr;
    if (timed) CK(cudaEventRecord(g_tev[0], s));
    if (g_prof.on) CK(cudaEventRecord(g_prof.ev[0], s));
    if (have_iv) {
      a.split = iv_split;
      a.warps_per_cta = (iv_threads + 31) / 32;  // a partial warp when a group is not whole warps
      try {
        launch_jit(jk_iv, a, I.G, iv_smem, s);
      } catch (const JitError &e) {
        throw Fail{RC_E_CUDA, e.msg};
      }
    } else {
      launch_interp(a, I.G, smem, s);
    }
    CK(cudaGetLastError());
    if (g_prof.on) {
      CK(cudaEventRecord(g_prof.ev[1], s));
      CK(cudaEventRecord(g_prof.ev[2], s));
    }
  };
  // the work after the interpreter that needs nothing from the host, then the stats read
  auto enqueue_post = [&](uint32_t k, int strategy, uint32_t tag) {
    if (group) {
      launch_xg_update(log, n_slices, slice, warp_count, L.GT, xg, xgcnt, s);
      CK(cudaGetLastError());
    }
    if (strategy == 2)
      shadow_launch(W, log, n_slices, slice, warp_count, N, snap, owner, tag, ow, ow_cnt, dbuf(k) + ST_SCRATCH, s);
    CK(cudaMemcpyAsync(hbuf(k), dbuf(k), stat_words * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(W.sev[k & 1], s));
  };

  std::vector<OutRec> races, errors;
  uint64_t tot_g = 0, tot_l = 0, tot_logged = 0;
  uint32_t interval = 0;
  int strategy = fixed_strategy ? fixed_strategy : g_tuner.choose(tkey);
  bool timed = !fixed_strategy && !g_tuner.decided(tkey);  // autotuner sample of this interval
  uint32_t tag = strategy == 2 ? shadow_next_tag(W, s, 4 * L.keys) : 0;
  enqueue_interp(0, strategy, tag, false, timed);
  enqueue_post(0, strategy, tag);
  for (;; interval++) {
    // Speculation: when this interval and the next take the shadow path and
    // nothing is being timed, the next interval's interpreter is queued now,
    // behind a gate the device sets only if this interval overflowed nothing
    // and its barrier agreement lets the run go on -- exactly the case in
    // which the host would launch it unchanged.  The shadow path commits
    // every written cell before the gate, so the exact classification of
    // this interval's shared cells then runs on a second stream beside the
    // next interval.
    bool next_queued = false;
    uint32_t next_tag = 0;
    if (strategy == 2 && !timed && !g_prof.on && !I.explore && !group) {
      const int ns = fixed_strategy ? fixed_strategy : g_tuner.choose(tkey);
      if (ns == 2 && (fixed_strategy || g_tuner.decided(tkey))) {
        next_tag = shadow_next_tag(W, s, 4 * L.keys);
        uint32_t *d = dbuf(interval);
        launch_interval_gate(d + ST_FLAGS, d + ST_STOPS + nstops, P.n_barriers, gate + ((interval + 1) & 1), s);
        enqueue_interp(interval + 1, 2, next_tag, true, false);
        next_queued = true;
      }
    }
    CK(cudaEventSynchronize(W.sev[interval & 1]));
    const uint32_t *h = hbuf(interval);
    const uint32_t flags = h[ST_FLAGS];
    if (flags) throw Fail{RC_E_CAPACITY, "interval log, own-write table or error log overflowed"};
    const uint64_t acc_g = *reinterpret_cast<const uint64_t *>(h + ST_ACC);
    const uint64_t acc_l = *reinterpret_cast<const uint64_t *>(h + ST_ACC + 2);
    tot_logged += *reinterpret_cast<const uint64_t *>(h + ST_LOGGED);
    const uint64_t m = *reinterpret_cast<const uint64_t *>(h + ST_SCRATCH);
    std::vector<uint32_t> stop_min(h + ST_STOPS, h + ST_STOPS + nstops);
    std::vector<uint32_t> stop_cnt(h + ST_STOPS + nstops, h + ST_STOPS + 2 * nstops);
    const uint32_t nerr = std::min(h[ST_ERRCNT], err_cap);
    tot_g += acc_g;
    tot_l += acc_l;
    if (g_prof.on) {
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, g_prof.ev[0], g_prof.ev[1]));
      g_prof.launches[0]++;
      g_prof.ms[0] += ms;
      g_prof.bytes[0] += 12.0 * (double)acc_g;
    }
    // ---- classification + commit
    if (strategy == 2) {
      cudaStream_t cs = s;
      if (next_queued && m) {  // beside the next interval (the compaction is done: its stats arrived)
        cs = classify_stream(W);
        CK(cudaStreamWaitEvent(cs, W.sev[interval & 1], 0));
      }
      shadow_finish(W, m, L.keys, N, interval, L, hscratch, races, cs);
    } else {
      classify_sorted(W, log, n_slices, slice, warp_count, L.keys, N, interval, L, snap, hscratch, races, s);
    }
    if (g_prof.on) {
      CK(cudaEventRecord(g_prof.ev[3], s));
      CK(cudaEventSynchronize(g_prof.ev[3]));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, g_prof.ev[2], g_prof.ev[3]));
      g_prof.launches[1]++;
      g_prof.ms[1] += ms;
      g_prof.bytes[1] += 12.0 * (double)acc_g;
    }
    if (timed) {  // autotuner sample: this interval's time per access
      CK(cudaEventRecord(g_tev[1], s));
      CK(cudaEventSynchronize(g_tev[1]));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, g_tev[0], g_tev[1]));
      g_tuner.record(tkey, strategy, ms, acc_g + acc_l);
    }
    // ---- error records of this interval
    if (nerr) {
      std::vector<OutRec> e(nerr);
      CK(cudaMemcpyAsync(e.data(), errs2 + (uint64_t)(interval & 1) * err_cap, nerr * sizeof(OutRec),
                         cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      std::sort(e.begin(), e.end(), [](const OutRec &x, const OutRec &y) {
        return x.cls != y.cls ? x.cls < y.cls : x.t_a < y.t_a;
      });
      errors.insert(errors.end(), e.begin(), e.end());
    }
    // ---- barrier agreement (barrier-release rule of Sec. 4; group scope:
    // each group checked it on the device and wrote its DIVERGENCE records)
    if (group) {
      bool any_barrier = false;
      for (uint32_t k = 0; k < P.n_barriers; k++) any_barrier |= stop_cnt[k] != 0;
      if (h[ST_GDIV] || !any_barrier) break;
    } else if (!barrier_agreement(interval, P.n_barriers, stop_min.data(), stop_cnt.data(), errors)) {
      break;
    }
    if (next_queued) {  // the gate opened: the next interval is already running
      tag = next_tag;
      enqueue_post(interval + 1, 2, tag);
      continue;
    }
    // the next interval starts after this one's classification
    strategy = fixed_strategy ? fixed_strategy : g_tuner.choose(tkey);
    timed = !fixed_strategy && !g_tuner.decided(tkey);
    if (strategy == 2) tag = next_queued ? next_tag : shadow_next_tag(W, s, 4 * L.keys);  // a closed gate used no claims
    else tag = 0;
    enqueue_interp(interval + 1, strategy, tag, false, timed);
    enqueue_post(interval + 1, strategy, tag);
  }

  if (group && L.GT) {  // cross-group records of the whole run, in cell order
    uint32_t *nrec = W.xgn.get<uint32_t>(L.GT), *offs = W.xgoff.get<uint32_t>(L.GT);
    uint32_t *tmp = W.xgtmp.get<uint32_t>(scan_tmp_words(L.GT));
    launch_xg_count(xg, L.GT, I.S, nrec, s);
    scan_exclusive(nrec, offs, L.GT, tmp, s);
    CK(cudaGetLastError());
    uint32_t tail[2] = {0, 0};
    CK(cudaMemcpyAsync(&tail[0], offs + L.GT - 1, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&tail[1], nrec + L.GT - 1, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const uint64_t total = (uint64_t)tail[0] + tail[1];
    if (total) {
      OutRec *out = W.xgout.get<OutRec>(total);
      launch_xg_emit(xg, xgcnt, L.GT, I.S, nrec, offs, out, s);
      CK(cudaGetLastError());
      const size_t at = races.size();
      races.resize(at + total);
      CK(cudaMemcpyAsync(races.data() + at, out, total * sizeof(OutRec), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
  }
  return make_report(races, errors, interval + 1, tot_g, tot_l, tot_logged, L.GT,
                     (I.in->flags & RC_WANT_FINAL_MEMORY) ? snap : nullptr, s);
}

// ---------------------------------------------------------------- batches
struct BatchItem {
  const Program *p;
  uint32_t G, S;
  uint64_t N;
  const rc_input *in;
  Layout L;
  uint64_t B, capw, warps, bytes;
};

BatchItem plan_item(const rc_bytecode *bc, uint32_t G, uint32_t S, const rc_input *in) {
  BatchItem it;
  it.p = &bc->prog;
  it.G = G;
  it.S = S;
  it.N = (uint64_t)G * S;
  it.in = in;
  it.L = make_layout(bc->prog, in, G);
  it.B = std::max<uint64_t>(bc->prog.max_access_per_interval, 1);
  it.capw = std::max<uint64_t>(bc->prog.max_write_per_interval, 1);
  it.warps = (it.N + 31) / 32;
  // cells (snapshot + owner table), registers/state/own writes, two logs
  it.bytes = it.L.keys * 20 + it.N * (4ull * bc->prog.n_regs + 12 + 8 * it.capw) + it.warps * 32 * it.B * 32;
  return it;
}

// Check instances [0, n) of `items` together.  Lock-step rounds: every round
// runs one barrier interval of every instance still active, in one
// persistent interpreter launch (a captured graph with the commit), then the
// compaction, the host's barrier agreement and one classification over the
// shared cell space (on shadow rounds beside the next round's graph).  Resident (strategy 3): every round in one
// cooperative launch (batch.cu, batch_resident_kernel), then the
// classification of each round's compacted records.  Returns false when a
// resident run could not finish (not every CTA resident, the record buffer
// or the round cap reached): the caller checks the batch again in lock-step.
bool run_batch(const std::vector<BatchItem> &items, cudaStream_t s, int strategy, rc_report **out) {
  Workspace &W = g_ws;
  // profiling, kind 2: the host's own work of the call (set-up before the
  // first round, reports after the last classification), wall clock
  using Clock = std::chrono::steady_clock;
  const Clock::time_point t_start = Clock::now();
  double host_ms = 0;
  auto ms_since = [](Clock::time_point t) {
    return std::chrono::duration<double, std::milli>(Clock::now() - t).count();
  };
  auto host_done = [&](Clock::time_point t_reports) {
    if (!g_prof.on) return;
    g_prof.launches[2]++;
    g_prof.ms[2] += host_ms + ms_since(t_reports);
  };
  if (!W.batch_configured) {
    CK(batch_configure());
    W.batch_configured = true;
  }
  const uint32_t n = (uint32_t)items.size();
  std::vector<BatchDesc> desc(n);
  std::vector<Insn> code;
  std::vector<MemInfo> mems;
  std::vector<uint32_t> task_kernel;
  std::vector<uint64_t> kbase(n);
  std::vector<uint32_t> kGT(n), kLT(n);
  uint64_t keys = 0, regs = 0, state = 0, owe = 0, logrecs = 0;
  uint32_t stops = 0, max_regs = kBuiltinRegs, max_writes = 1;
  uint64_t maxN = 1;
  // the size class (warp tasks and the static bound per task) and its log
  // capacity: slices of 32 x ceil(bound x log_pm / 1000) records
  uint64_t tasks_all = 0, bound_recs = 0;
  for (const BatchItem &it : items) {
    tasks_all += it.warps;
    bound_recs += it.warps * 32 * it.B;
  }
  const std::string tkey = batch_key(tasks_all, bound_recs / std::max<uint64_t>(tasks_all, 1) / 32);
  const uint32_t log_pm = g_tuner.log_permille(tkey);
  for (uint32_t k = 0; k < n; k++) {
    const BatchItem &it = items[k];
    BatchDesc &D = desc[k];
    D.code_off = (uint32_t)code.size();
    code.insert(code.end(), it.p->code.begin(), it.p->code.end());
    D.mems_off = (uint32_t)mems.size();
    mems.insert(mems.end(), it.L.mems.begin(), it.L.mems.end());
    D.n_regs = it.p->n_regs;
    D.n_barriers = it.p->n_barriers;
    D.S = it.S;
    D.G = it.G;
    D.GT = (uint32_t)it.L.GT;
    D.LT = (uint32_t)it.L.LT;
    D.capw = (uint32_t)std::min<uint64_t>(it.capw, 0xFFFFFFFFu);
    D.stop_off = stops;
    D.task_off = (uint32_t)task_kernel.size();
    D.active = 1;
    D.N = it.N;
    D.key_base = keys;
    D.reg_off = regs;
    D.state_off = state;
    D.ow_off = owe;
    D.slice = 32 * std::max<uint64_t>(1, (it.B * log_pm + 999) / 1000);
    D.slice_off = logrecs;
    kbase[k] = keys;
    kGT[k] = D.GT;
    kLT[k] = D.LT;
    task_kernel.insert(task_kernel.end(), it.warps, k);
    keys += it.L.keys;
    regs += it.N * it.p->n_regs;
    state += it.N;
    owe += it.N * it.capw;
    logrecs += it.warps * D.slice;
    stops += it.p->n_barriers + 1;
    max_regs = std::max(max_regs, it.p->n_regs);
    max_writes = (uint32_t)std::max<uint64_t>(max_writes, it.capw);
    maxN = std::max(maxN, it.N);
  }
  const uint32_t n_tasks = (uint32_t)task_kernel.size();
  // device copies
  BatchDesc *ddesc = W.bdesc.get<BatchDesc>(n);
  Insn *dcode = W.bcode.get<Insn>(code.size());
  MemInfo *dmems = W.bmems.get<MemInfo>(std::max<size_t>(mems.size(), 1));
  uint32_t *dtask = W.btask.get<uint32_t>(n_tasks);
  uint64_t *dkbase = W.bkbase.get<uint64_t>(n);
  uint32_t *dkgt = W.bkgt.get<uint32_t>(n), *dklt = W.bklt.get<uint32_t>(n);
  CK(cudaMemcpyAsync(dcode, code.data(), code.size() * sizeof(Insn), cudaMemcpyHostToDevice, s));
  if (!mems.empty()) CK(cudaMemcpyAsync(dmems, mems.data(), mems.size() * sizeof(MemInfo), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dtask, task_kernel.data(), n_tasks * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dkbase, kbase.data(), n * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dkgt, kGT.data(), n * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dklt, kLT.data(), n * 4, cudaMemcpyHostToDevice, s));
  int32_t *snap = W.snap.get<int32_t>(std::max<uint64_t>(keys, 1));
  for (uint32_t k = 0; k < n; k++) {  // inputs, then zeroed local memory
    const BatchItem &it = items[k];
    uint32_t gi = 0;
    for (size_t m = 0; m < it.p->mems.size(); m++) {
      if (it.p->mems[m].space != 0) continue;
      const uint64_t len = it.in->global_len[gi];
      if (len) {
        if (!it.in->global_init || !it.in->global_init[gi]) throw Fail{RC_E_INVALID, "missing global input"};
        upload_global(it.in->global_init[gi], snap + kbase[k] + it.L.mems[m].base, len, it.in->on_device, s);
      }
      gi++;
    }
    if (it.L.keys > it.L.GT) CK(cudaMemsetAsync(snap + kbase[k] + it.L.GT, 0, (it.L.keys - it.L.GT) * 4, s));
  }
  int32_t *dregs = W.regs.get<int32_t>(std::max<uint64_t>(regs, 1));
  uint32_t *dpc = W.pc.get<uint32_t>(state), *dst = W.st.get<uint32_t>(state), *dowc = W.owcnt.get<uint32_t>(state);
  CK(cudaMemsetAsync(dregs, 0, regs * 4, s));
  CK(cudaMemsetAsync(dpc, 0, state * 4, s));
  CK(cudaMemsetAsync(dst, 0, state * 4, s));
  uint2 *dow = W.ow.get<uint2>(std::max<uint64_t>(owe, 1));
  LogRec *dlog = W.loga.get<LogRec>(std::max<uint64_t>(logrecs, 1));
  uint32_t *dwc = W.ctacnt.get<uint32_t>(n_tasks);
  const uint32_t err_cap = (uint32_t)std::min<uint64_t>(state, 1u << 26);
  OutRec *derrs = W.errs.get<OutRec>(err_cap);
  uint32_t *derrk = W.berrk.get<uint32_t>(err_cap);
  // stats: [0..1] acc is separate; words: flags, err_count, next_task, pad, compact count (2), stops...
  const size_t stat_words = 8 + 2 * (size_t)stops;
  uint32_t *dstats = W.stats.get<uint32_t>(stat_words);
  uint32_t *hstats = W.hstats.get<uint32_t>(stat_words + 8);
  unsigned long long *dacc = reinterpret_cast<unsigned long long *>(W.shared_acc.get<uint64_t>(2ull * n));
  CK(cudaMemsetAsync(dacc, 0, 16ull * n, s));
  uint32_t *owner = strategy != 1 ? shadow_table(W, keys, s) : W.owner.get<uint32_t>(4);
  if (!strategy) tuner_events();
  // block shapes: CTAs of 128, 256 or 512 threads, 1024 threads per SM; own-write
  // slots in shared memory (up to 8) within the SM's 200 KB shared among them
  if (batch_smem_bytes(max_regs, 0, 512) > kMaxSmemPerBlock)
    throw Fail{RC_E_INVALID, "batch needs too many registers per work-item"};
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
  uint32_t *dround = W.bround.get<uint32_t>(4);
  uint32_t *hround = W.hround.get<uint32_t>(4);
  BatchDesc *hdesc = W.hdesc.get<BatchDesc>(n);

  BatchArgs a{};
  a.desc = ddesc;
  a.task_kernel = dtask;
  a.n_tasks = n_tasks;
  a.next_task = dstats + 2;
  a.code = dcode;
  a.mems = dmems;
  a.max_regs = max_regs;
  a.round = dround;
  a.snap = snap;
  a.regs = dregs;
  a.pc = dpc;
  a.st = dst;
  a.ow_count = dowc;
  a.ow = dow;
  a.log = dlog;
  a.warp_count = dwc;
  a.errs = derrs;
  a.err_kernel = derrk;
  a.err_count = dstats + 1;
  a.err_cap = err_cap;
  a.stop_min = dstats + 8;
  a.stop_cnt = dstats + 8 + stops;
  a.acc = dacc;
  a.flags = dstats;
  a.owner = owner;
  a.fill_max = dstats + 6;
  unsigned long long *cnt = reinterpret_cast<unsigned long long *>(dstats + 4);
  host_ms = ms_since(t_start);
  if (strategy == 3) {
    // ---- resident run: every round in one cooperative launch
    const uint32_t threads = g_tuner.threads_decided(tkey) ? g_tuner.choose_threads(tkey) : 256u;
    const uint32_t ctas_per_sm = 1024 / threads;
    uint32_t ow_slots = 0;
    while (ow_slots < 8 && ow_slots < max_writes &&
           batch_smem_bytes(max_regs, ow_slots + 1, threads) <= 200 * 1024 / ctas_per_sm)
      ow_slots++;
    const size_t smem = batch_smem_bytes(max_regs, ow_slots, threads);
    if (smem + 256 > kMaxSmemPerBlock) return false;  // room for the grid barrier's static bytes
    const int per_sm = batch_resident_blocks_per_sm(threads, smem);
    if (per_sm <= 0) return false;
    const uint32_t warps_per_cta = threads / 32;
    const uint32_t grid = std::max<uint32_t>(
        1, std::min<uint32_t>((n_tasks + warps_per_cta - 1) / warps_per_cta, (uint32_t)sms * (uint32_t)per_sm));
    // compacted records of every round: twice one round's slice capacity, at
    // least 4 Mi records, at most 2^31 (32 GiB); a run that needs more starts
    // over in lock-step
    const uint64_t acc_cap = std::min<uint64_t>(std::max<uint64_t>(2 * bound_recs, 1ull << 22), 1ull << 31);
    LogRec *acc_out = W.logb.get<LogRec>(acc_cap);
    uint32_t *owner_r = owner;  // the shadow table (strategy 3 is not the sort path)
    const uint32_t tag0 = shadow_next_tag(W, s, 4 * keys);
    unsigned *bar = W.rbar.get<unsigned>(kGridBarWords);
    unsigned long long *ivoff = W.rivoff.get<unsigned long long>(kResidentMaxIntervals + 1);
    uint32_t *irounds = W.brounds.get<uint32_t>(n + 2);
    CK(cudaMemsetAsync(dstats, 0, 8 * 4, s));
    CK(cudaMemsetAsync(dstats + 8, 0xFF, stops * 4, s));
    CK(cudaMemsetAsync(dstats + 8 + stops, 0, stops * 4, s));
    CK(cudaMemsetAsync(bar, 0, kGridBarWords * 4, s));
    CK(cudaMemsetAsync(ivoff, 0, 8, s));
    CK(cudaMemsetAsync(dround, 0, 16, s));
    CK(cudaMemsetAsync(irounds, 0, (n + 2) * 4, s));
    CK(cudaMemcpyAsync(ddesc, desc.data(), n * sizeof(BatchDesc), cudaMemcpyHostToDevice, s));
    BatchArgs ar = a;
    ar.owner = owner_r;
    ar.ow_slots = ow_slots;
    ar.grid_bar = bar;
    ar.barrier_limit_ns = 20000000000ull;
    ar.acc_out = acc_out;
    ar.acc_total = cnt;
    ar.iv_off = ivoff;
    ar.acc_cap = acc_cap;
    ar.owner_words = 4 * keys;
    ar.n_inst = n;
    ar.max_rounds = kResidentMaxIntervals;
    ar.tag0 = tag0;
    ar.n_active = dround;
    ar.inst_rounds = irounds;
    if (g_prof.on) CK(cudaEventRecord(g_prof.ev[0], s));
    const cudaError_t e = launch_batch_resident(ar, grid, threads, smem, s);
    if (e == cudaErrorCooperativeLaunchTooLarge) {
      cudaGetLastError();
      return false;
    }
    CK(e);
    if (g_prof.on) CK(cudaEventRecord(g_prof.ev[1], s));
    std::vector<uint32_t> hr(n + 2), hs(8);
    std::vector<uint64_t> acc(2ull * n);
    uint32_t timed_out = 0;
    CK(cudaMemcpyAsync(hs.data(), dstats, 8 * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hr.data(), irounds, (n + 2) * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(acc.data(), dacc, 16ull * n, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&timed_out, bar + 2, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const uint32_t rounds = hr[n];
    if (rounds) {
      W.epoch = hr[n + 1];  // the owner-table tag of the last round
      if (tag0 + rounds - 1 > 63 && W.owner_hi > 4 * keys) {
        // the tag wrapped in-kernel: words past this batch's cells still hold
        // tags of the earlier epoch, which later calls would meet again
        CK(cudaMemsetAsync(owner_r + 4 * keys, 0, (W.owner_hi - 4 * keys) * 4, s));
        W.owner_hi = 4 * keys;
      }
    }
    if (timed_out) throw Fail{RC_E_TIMEOUT, "a grid barrier of the resident batch timed out"};
    if ((hs[0] & FLAG_LOG_FULL) && log_pm < 1000) {  // the tuned log capacity was too small
      g_tuner.record_overflow(tkey);
      return false;
    }
    if (hs[0] & (FLAG_LOG_FULL | FLAG_OW_FULL | FLAG_ERR_FULL))
      throw Fail{RC_E_CAPACITY, "batch log, own-write table or error log overflowed"};
    if (hs[0] & FLAG_ACC_FULL) return false;
    if (rounds == 0) throw Fail{RC_E_CUDA, "the resident batch reported no round"};
    for (uint32_t k = 0; k < n; k++)
      if (hr[k] == 0) return false;  // still active at the round cap
    g_tuner.record_fill(tkey, (uint32_t)(((uint64_t)hs[6] * log_pm + 999) / 1000));
    if (g_prof.on) {
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, g_prof.ev[0], g_prof.ev[1]));
      g_prof.launches[0]++;
      g_prof.ms[0] += ms;
      CK(cudaEventRecord(g_prof.ev[2], s));
    }
    // errors by (interval, class, work-item) per instance: the lock-step order
    std::vector<RecList> races(n);
    std::vector<std::vector<OutRec>> errors(n);
    RecordSink sink(races, W.hrecs, W.hreck);
    const uint32_t nerr = std::min(hs[1], err_cap);
    if (nerr) {
      std::vector<OutRec> ev(nerr);
      std::vector<uint32_t> ek(nerr);
      CK(cudaMemcpyAsync(ev.data(), derrs, nerr * sizeof(OutRec), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(ek.data(), derrk, nerr * 4, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (uint32_t i = 0; i < nerr; i++) errors[ek[i]].push_back(ev[i]);
      for (auto &v : errors)
        std::sort(v.begin(), v.end(), [](const OutRec &x, const OutRec &y) {
          return x.interval != y.interval ? x.interval < y.interval : x.cls != y.cls ? x.cls < y.cls : x.t_a < y.t_a;
        });
    }
    // the compacted records, classified round by round (commits were made in-kernel)
    std::vector<unsigned long long> off(rounds + 1);
    CK(cudaMemcpyAsync(off.data(), ivoff, (rounds + 1) * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<OutRec> rr;
    for (uint32_t r = 0; r < rounds; r++) {
      const uint64_t m = off[r + 1] - off[r];
      if (!m) continue;
      rr.clear();
      uint32_t *tmp = W.scan.get<uint32_t>(std::max(sort_tmp_words(m), scan_tmp_words(m)));
      LogRec *other = W.compact.get<LogRec>(m);
      LogRec *sorted = sort_log(acc_out + off[r], other, m, bitwidth(maxN), bitwidth(keys) + bitwidth(maxN), tmp, s);
      Layout none;
      BatchMap bm{n, dkbase, dkgt, dklt, &sink};
      classify_run(W, sorted, m, r, none, nullptr, hstats + stat_words, rr, s, &bm);
    }
    if (g_prof.on) {
      CK(cudaEventRecord(g_prof.ev[3], s));
      CK(cudaEventSynchronize(g_prof.ev[3]));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, g_prof.ev[2], g_prof.ev[3]));
      g_prof.launches[1]++;
      g_prof.ms[1] += ms;
    }
    sink.join();  // every round's records are in the lists
    const Clock::time_point t_reports = Clock::now();
    for (uint32_t k = 0; k < n; k++) {
      const BatchItem &it = items[k];
      out[k] = make_report(races[k], errors[k], hr[k], acc[2 * k], acc[2 * k + 1], acc[2 * k] + acc[2 * k + 1],
                           it.L.GT, (it.in->flags & RC_WANT_FINAL_MEMORY) ? snap + kbase[k] : nullptr, s);
    }
    host_done(t_reports);
    return true;
  }
  LogRec *picked = W.logb.get<LogRec>(std::max<uint64_t>(logrecs, 1));

  // One round's fixed launch sequence -- stat resets, the persistent
  // interpreter, the owner-table commit and the compaction of the records to
  // classify -- is captured once into a CUDA graph and replayed every round;
  // the round number, tag and path come from device memory.
  if (!W.bstream) CK(cudaStreamCreateWithFlags(&W.bstream, cudaStreamNonBlocking));
  cudaStream_t bs = W.bstream;
  {
    cudaEvent_t ready;
    CK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    CK(cudaEventRecord(ready, s));  // inputs and set-up issued on the caller's stream
    CK(cudaStreamWaitEvent(bs, ready, 0));
    CK(cudaEventDestroy(ready));
  }
  // one graph per block shape, captured the first time a round takes it
  struct Graphs {
    cudaGraph_t g[3] = {nullptr, nullptr, nullptr};
    cudaGraphExec_t e[3] = {nullptr, nullptr, nullptr};
    ~Graphs() {
      for (int k = 0; k < 3; k++) {
        if (e[k]) cudaGraphExecDestroy(e[k]);
        if (g[k]) cudaGraphDestroy(g[k]);
      }
    }
  } graphs;
  auto graph_for = [&](uint32_t threads) -> cudaGraphExec_t {
    const int k = threads == 128 ? 0 : threads == 256 ? 1 : 2;
    if (graphs.e[k]) return graphs.e[k];
    const uint32_t ctas_per_sm = 1024 / threads;
    const size_t budget = 200 * 1024 / ctas_per_sm;
    uint32_t ow_slots = 0;
    while (ow_slots < 8 && ow_slots < max_writes && batch_smem_bytes(max_regs, ow_slots + 1, threads) <= budget)
      ow_slots++;
    const size_t smem = batch_smem_bytes(max_regs, ow_slots, threads);
    const uint32_t warps_per_cta = threads / 32;
    const uint32_t grid = std::max<uint32_t>(
        1, std::min<uint32_t>((n_tasks + warps_per_cta - 1) / warps_per_cta, (uint32_t)sms * ctas_per_sm));
    BatchArgs ak = a;
    ak.ow_slots = ow_slots;
    CK(cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(dstats, 0, 8 * 4, bs);
    cudaMemsetAsync(dstats + 8, 0xFF, stops * 4, bs);
    cudaMemsetAsync(dstats + 8 + stops, 0, stops * 4, bs);
    launch_batch_interp(ak, grid, threads, smem, bs);
    launch_batch_commit(ak, bs);
    CK(cudaStreamEndCapture(bs, &graphs.g[k]));
    CK(cudaGraphInstantiate(&graphs.e[k], graphs.g[k], 0));
    return graphs.e[k];
  };

  // One round: the descriptors and round words uploaded, then the graph.
  auto launch_round = [&](uint32_t round, int strat, uint32_t threads, bool timed) {
    std::memcpy(hdesc, desc.data(), n * sizeof(BatchDesc));
    hround[0] = round;
    hround[1] = strat == 2 ? shadow_next_tag(W, bs, 4 * keys) : 0;
    hround[2] = strat == 2 ? 1u : 0u;
    CK(cudaMemcpyAsync(ddesc, hdesc, n * sizeof(BatchDesc), cudaMemcpyHostToDevice, bs));
    CK(cudaMemcpyAsync(dround, hround, 16, cudaMemcpyHostToDevice, bs));
    if (timed) CK(cudaEventRecord(g_tev[0], bs));
    if (g_prof.on) CK(cudaEventRecord(g_prof.ev[0], bs));
    CK(cudaGraphLaunch(graph_for(threads), bs));
    for (int q = 0; q < 2; q++) count_launch();  // kernels replayed by the graph
  };

  std::vector<RecList> races(n);
  std::vector<std::vector<OutRec>> errors(n);
  RecordSink sink(races, W.hrecs, W.hreck);
  std::vector<uint32_t> n_intervals(n, 0);
  uint32_t active = n, fill_seen = 0;
  std::vector<uint64_t> acc(2ull * n), prev(2ull * n, 0);
  std::vector<OutRec> rr;
  int strat = 0;
  uint32_t threads = 256;
  bool tuning = false, shape_tuning = false, launched = false;
  for (uint32_t round = 0; active; round++) {
    if (!launched) {
      strat = strategy ? strategy : g_tuner.choose(tkey);
      tuning = !strategy && !g_tuner.decided(tkey);
      // block shape: the tuner's (tried in turn once the strategy is decided), 256 with a fixed strategy
      threads = strategy ? 256u : g_tuner.choose_threads(tkey);
      shape_tuning = !strategy && !tuning && !g_tuner.threads_decided(tkey);
      launch_round(round, strat, threads, tuning || shape_tuning);
    }
    launched = false;
    // the round's compaction of the records to classify (queued after the
    // previous round's classification, which read the same buffer, ended)
    launch_batch_compact(a, picked, cnt, bs);
    if (g_prof.on) CK(cudaEventRecord(g_prof.ev[1], bs));
    CK(cudaMemcpyAsync(hstats, dstats, stat_words * 4, cudaMemcpyDeviceToHost, bs));
    CK(cudaMemcpyAsync(acc.data(), dacc, 16ull * n, cudaMemcpyDeviceToHost, bs));
    CK(cudaStreamSynchronize(bs));
    if ((hstats[0] & FLAG_LOG_FULL) && log_pm < 1000) {  // the tuned log capacity was too small
      g_tuner.record_overflow(tkey);
      return false;
    }
    if (hstats[0]) throw Fail{RC_E_CAPACITY, "batch log, own-write table or error log overflowed"};
    fill_seen = std::max(fill_seen, hstats[6]);
    if (g_prof.on) {
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, g_prof.ev[0], g_prof.ev[1]));
      g_prof.launches[0]++;
      g_prof.ms[0] += ms;
      CK(cudaEventRecord(g_prof.ev[2], bs));
    }
    const uint64_t m = *reinterpret_cast<const uint64_t *>(hstats + 4);
    // ---- error records of the round (the next round's launch reuses the buffer)
    const uint32_t nerr = std::min(hstats[1], err_cap);
    if (nerr) {
      std::vector<OutRec> e(nerr);
      std::vector<uint32_t> ek(nerr);
      CK(cudaMemcpyAsync(e.data(), derrs, nerr * sizeof(OutRec), cudaMemcpyDeviceToHost, bs));
      CK(cudaMemcpyAsync(ek.data(), derrk, nerr * 4, cudaMemcpyDeviceToHost, bs));
      CK(cudaStreamSynchronize(bs));
      std::vector<std::vector<OutRec>> per(n);
      for (uint32_t i = 0; i < nerr; i++) per[ek[i]].push_back(e[i]);
      for (uint32_t k = 0; k < n; k++) {
        if (per[k].empty()) continue;
        std::sort(per[k].begin(), per[k].end(), [](const OutRec &x, const OutRec &y) {
          return x.cls != y.cls ? x.cls < y.cls : x.t_a < y.t_a;
        });
        errors[k].insert(errors[k].end(), per[k].begin(), per[k].end());
      }
    }
    // ---- per-instance barrier agreement
    for (uint32_t k = 0; k < n; k++) {
      if (!desc[k].active) continue;
      const uint32_t *smin = hstats + 8 + desc[k].stop_off, *scnt = hstats + 8 + stops + desc[k].stop_off;
      if (!barrier_agreement(round, desc[k].n_barriers, smin, scnt, errors[k])) {
        desc[k].active = 0;
        n_intervals[k] = round + 1;
        active--;
      }
    }
    // ---- the next round beside this one's classification: a shadow round
    // committed every written cell in its graph (highest writer), so the
    // next round needs nothing from the classification; not while a round
    // is timed for the autotuner or profiled
    cudaStream_t cs = bs;
    if (strat == 2 && m && active && !tuning && !shape_tuning && !g_prof.on) {
      const int ns = strategy ? strategy : g_tuner.choose(tkey);
      const uint32_t nth = strategy ? 256u : g_tuner.choose_threads(tkey);
      if (strategy || (g_tuner.decided(tkey) && g_tuner.threads_decided(tkey))) {
        launch_round(round + 1, ns, nth, false);
        launched = true;
        cs = classify_stream(W);  // the compaction it reads is complete: the host waited for it
      }
    }
    // ---- exact classification of the picked records over the shared cell space
    rr.clear();
    if (m) {
      uint32_t *tmp = W.scan.get<uint32_t>(std::max(sort_tmp_words(m), scan_tmp_words(m)));
      LogRec *other = W.compact.get<LogRec>(m);
      LogRec *sorted = sort_log(picked, other, m, bitwidth(maxN), bitwidth(keys) + bitwidth(maxN), tmp, cs);
      Layout none;
      BatchMap bm{n, dkbase, dkgt, dklt, &sink};
      // shadow rounds: the commits were all made in the graph
      classify_run(W, sorted, m, round, none, strat == 2 ? nullptr : snap, hstats + stat_words, rr, cs, &bm);
    }
    if (g_prof.on) {
      CK(cudaEventRecord(g_prof.ev[3], bs));
      CK(cudaEventSynchronize(g_prof.ev[3]));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, g_prof.ev[2], g_prof.ev[3]));
      g_prof.launches[1]++;
      g_prof.ms[1] += ms;
    }
    if (tuning || shape_tuning) {
      CK(cudaEventRecord(g_tev[1], bs));
      CK(cudaEventSynchronize(g_tev[1]));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, g_tev[0], g_tev[1]));
      uint64_t done = 0;
      for (size_t q = 0; q < acc.size(); q++) done += acc[q] - prev[q];
      if (tuning) g_tuner.record(tkey, strat, ms, done);
      else g_tuner.record_threads(tkey, threads, ms, done);
    }
    prev = acc;
    if (launched) {  // the round already running
      strat = strategy ? strategy : g_tuner.choose(tkey);
      threads = strategy ? 256u : g_tuner.choose_threads(tkey);
      tuning = shape_tuning = false;
    }
  }
  g_tuner.record_fill(tkey, (uint32_t)(((uint64_t)fill_seen * log_pm + 999) / 1000));
  sink.join();  // every round's records are in the lists
  const Clock::time_point t_reports = Clock::now();
  s = bs;  // final memories are read on the batch stream
  for (uint32_t k = 0; k < n; k++) {
    const BatchItem &it = items[k];
    // batches log every access (no private accesses)
    out[k] = make_report(races[k], errors[k], n_intervals[k], acc[2 * k], acc[2 * k + 1],
                         acc[2 * k] + acc[2 * k + 1], it.L.GT,
                         (it.in->flags & RC_WANT_FINAL_MEMORY) ? snap + kbase[k] : nullptr, s);
  }
  host_done(t_reports);
  return true;
}

void check_args(const rc_bytecode *bc, uint32_t groups, uint32_t group_size, const rc_input *in) {
  if (!bc || !in) throw Fail{RC_E_INVALID, "null bytecode or input"};
  if (groups == 0 || group_size == 0 || group_size > 1024) throw Fail{RC_E_INVALID, "bad launch shape"};
  if ((uint64_t)groups * group_size > (1ull << 26)) throw Fail{RC_E_INVALID, "more than 2^26 work-items"};
  if (in->n_global != bc->prog.n_global) throw Fail{RC_E_INVALID, "input count differs from the kernel's global declarations"};
  if (in->n_global && !in->global_len) throw Fail{RC_E_INVALID, "missing global lengths"};
}

int fail_code(const Fail &f) {
  g_last_error = f.msg;
  return f.code;
}

}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void set_last_error(const std::string &msg) { g_last_error = msg; }

}  // namespace rc

using namespace rc;

extern "C" {

int rc_compile(const char *src, size_t len, rc_bytecode **out, char *err, size_t err_len) {
  if (!out || !src) return RC_E_INVALID;
  *out = nullptr;
  try {
    rc_bytecode *b = new rc_bytecode{compile_program(std::string(src, len))};
    *out = b;
    return RC_OK;
  } catch (const CompileError &e) {
    g_last_error = e.msg;
    if (err && err_len) std::snprintf(err, err_len, "%s", e.msg.c_str());
    return RC_E_PARSE;
  } catch (const std::bad_alloc &) {
    return RC_E_NOMEM;
  }
}

int rc_bytecode_info_get(const rc_bytecode *bc, rc_bytecode_info *info) {
  if (!bc || !info) return RC_E_INVALID;
  const Program &p = bc->prog;
  std::memset(info, 0, sizeof(*info));
  info->n_insn = (uint32_t)p.code.size();
  info->n_regs = p.n_regs;
  info->n_vars = p.n_vars;
  info->n_mems = (uint32_t)p.mems.size();
  info->n_global = p.n_global;
  info->n_barriers = p.n_barriers;
  info->n_asserts = p.n_asserts;
  uint64_t lc = 0;
  for (const MemDecl &m : p.mems)
    if (m.space == 1) lc += (uint64_t)m.decl_len;
  info->local_cells = (uint32_t)std::min<uint64_t>(lc, 0xFFFFFFFFu);
  info->max_access_per_interval = p.max_access_per_interval;
  info->max_write_per_interval = p.max_write_per_interval;
  return RC_OK;
}

int rc_check(const rc_bytecode *bc, uint32_t groups, uint32_t group_size, const rc_input *in,
             rc_report **out) {
  if (!out) return RC_E_INVALID;
  *out = nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  try {
    check_args(bc, groups, group_size, in);
    if (g_prof.on) prof_events();
    Instance I{&bc->prog, groups, group_size, (uint64_t)groups * group_size, in,
               static_cast<cudaStream_t>(in->cuda_stream)};
    *out = run_instance(I);
    return RC_OK;
  } catch (const Fail &f) {
    return fail_code(f);
  } catch (const std::bad_alloc &) {
    g_last_error = "host allocation failed";
    return RC_E_NOMEM;
  }
}

int rc_explore(const rc_bytecode *bc, uint32_t groups, uint32_t group_size, const rc_input *in, uint64_t max_states,
               rc_explore_interval *out, uint32_t max_intervals, uint32_t *n_out) {
  if (!out || !n_out) return RC_E_INVALID;
  *n_out = 0;
  std::lock_guard<std::mutex> lk(g_mu);
  try {
    check_args(bc, groups, group_size, in);
    if (in->flags & RC_GROUP_BARRIERS) throw Fail{RC_E_INVALID, "the explorer takes kernel-wide barriers only"};
    if ((uint64_t)groups * group_size > 16) throw Fail{RC_E_INVALID, "the explorer takes at most 16 work-items"};
    Layout L = make_layout(bc->prog, in, groups);
    if (L.keys > 4096) throw Fail{RC_E_INVALID, "the explorer takes at most 4096 cells"};
    if (bc->prog.n_regs > 64) throw Fail{RC_E_INVALID, "the explorer takes at most 64 registers"};
    ExploreRun ex{max_states ? max_states : 1000000, max_intervals, false, {}, {}};
    Instance I{&bc->prog, groups, group_size, (uint64_t)groups * group_size, in,
               static_cast<cudaStream_t>(in->cuda_stream), &ex};
    rc_report *r = run_instance(I);
    rc_report_free(r);
    for (size_t k = 0; k < ex.results.size(); k++) {
      out[k].interval = (uint32_t)k;
      out[k].n_end_states = ex.results[k].n_end_states;
      out[k].deviated = ex.results[k].deviated;
      out[k].complete = ex.results[k].complete;
      out[k].n_states = ex.results[k].n_states;
    }
    *n_out = (uint32_t)ex.results.size();
    return RC_OK;
  } catch (const Fail &f) {
    return fail_code(f);
  } catch (const std::bad_alloc &) {
    g_last_error = "host allocation failed";
    return RC_E_NOMEM;
  }
}

int rc_explore_pairs(const rc_bytecode *bc, uint32_t groups, uint32_t group_size, const rc_input *in,
                     uint64_t max_states, rc_pair_interval *out, uint32_t max_intervals, uint32_t *n_out,
                     uint32_t *pair_detail) {
  if (!out || !n_out) return RC_E_INVALID;
  *n_out = 0;
  std::lock_guard<std::mutex> lk(g_mu);
  try {
    check_args(bc, groups, group_size, in);
    if (in->flags & RC_GROUP_BARRIERS) throw Fail{RC_E_INVALID, "the explorer takes kernel-wide barriers only"};
    const uint64_t N = (uint64_t)groups * group_size;
    if (N > 256) throw Fail{RC_E_INVALID, "the pair explorer takes at most 256 work-items"};
    Layout L = make_layout(bc->prog, in, groups);
    if (L.keys > 4096) throw Fail{RC_E_INVALID, "the explorer takes at most 4096 cells"};
    if (bc->prog.n_regs > 64) throw Fail{RC_E_INVALID, "the explorer takes at most 64 registers"};
    ExploreRun ex{max_states ? max_states : 1000000, max_intervals, true, {}, {}};
    Instance I{&bc->prog, groups, group_size, N, in, static_cast<cudaStream_t>(in->cuda_stream), &ex};
    rc_report *r = run_instance(I);
    rc_report_free(r);
    const uint32_t P = (uint32_t)(N * (N - 1) / 2);
    for (size_t k = 0; k < ex.results.size(); k++) {
      const std::vector<uint32_t> &pv = ex.pair_results[k];
      rc_pair_interval &o = out[k];
      o.interval = (uint32_t)k;
      o.n_pairs = P;
      o.n_racy = o.n_deviated = 0;
      o.first_i = o.first_j = 0xFFFFFFFFu;
      o.complete = ex.results[k].complete;
      o.reserved = 0;
      o.n_states = ex.results[k].n_states;
      uint32_t p = 0;
      for (uint32_t i = 0; i < N; i++)
        for (uint32_t j = i + 1; j < N; j++, p++) {
          const uint32_t v = p < pv.size() ? pv[p] : 0;
          if ((v & 0x7FFFFFFFu) >= 2) {
            if (!o.n_racy) {
              o.first_i = i;
              o.first_j = j;
            }
            o.n_racy++;
          }
          if (v >> 31) o.n_deviated++;
          if (pair_detail) pair_detail[k * P + p] = v;
        }
    }
    *n_out = (uint32_t)ex.results.size();
    return RC_OK;
  } catch (const Fail &f) {
    return fail_code(f);
  } catch (const std::bad_alloc &) {
    g_last_error = "host allocation failed";
    return RC_E_NOMEM;
  }
}

int rc_search(const rc_bytecode *const *bcs, const uint32_t *groups, const uint32_t *group_size,
              const rc_input *inputs, size_t n, const float *scores, uint32_t max_checks, rc_search_result *res,
              rc_report **found) {
  if (!res || (n && (!bcs || !groups || !group_size || !inputs))) return RC_E_INVALID;
  res->first = -1;
  res->checks = 0;
  res->seconds = 0;
  if (found) *found = nullptr;
  // candidates in descending score (ties keep their order), or as given
  std::vector<size_t> order(n);
  for (size_t i = 0; i < n; i++) order[i] = i;
  if (scores)
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return scores[a] > scores[b]; });
  const size_t limit = max_checks ? std::min<size_t>(n, max_checks) : n;
  std::lock_guard<std::mutex> lk(g_mu);
  try {
    if (g_prof.on) prof_events();
    const auto t0 = std::chrono::steady_clock::now();
    for (size_t k = 0; k < limit; k++) {
      const size_t i = order[k];
      check_args(bcs[i], groups[i], group_size[i], &inputs[i]);
      Instance I{&bcs[i]->prog, groups[i], group_size[i], (uint64_t)groups[i] * group_size[i], &inputs[i],
                 static_cast<cudaStream_t>(inputs[i].cuda_stream)};
      rc_report *r = run_instance(I);
      res->checks++;
      if (r->status == RC_RACY) {
        res->first = (int64_t)i;
        if (found) *found = r;
        else rc_report_free(r);
        break;
      }
      rc_report_free(r);
    }
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return RC_OK;
  } catch (const Fail &f) {
    return fail_code(f);
  } catch (const std::bad_alloc &) {
    g_last_error = "host allocation failed";
    return RC_E_NOMEM;
  }
}

int rc_search_ranked(rc_mlp *model, const rc_bytecode *const *bcs, const uint32_t *groups,
                     const uint32_t *group_size, const rc_input *inputs, size_t n, uint32_t max_checks,
                     uint32_t flags, rc_ranked_result *res, rc_report **found) {
  if (!res || (n && (!bcs || !groups || !group_size || !inputs)) || (flags & ~RC_RANK_OVERLAP)) return RC_E_INVALID;
  *res = rc_ranked_result{-1, 0, 0, 0, 0, 0, 0};
  if (found) *found = nullptr;
  if (n == 0) return RC_OK;
  using clock = std::chrono::steady_clock;
  const auto t0 = clock::now();
  const auto secs = [](clock::time_point a, clock::time_point b) { return std::chrono::duration<double>(b - a).count(); };
  std::lock_guard<std::mutex> lk(g_mu);
  Workspace &W = g_ws;
  std::shared_ptr<FeatureJob> job;
  try {
    for (size_t i = 0; i < n; i++) {
      check_args(bcs[i], groups[i], group_size[i], &inputs[i]);
      if (inputs[i].on_device) throw Fail{RC_E_INVALID, "ranked search reads host inputs only"};
    }
    float *X = W.hrank.get<float>(n * RC_N_FEATURES + n);  // features, then scores
    float *score = X + n * RC_N_FEATURES;
    const size_t limit = max_checks ? std::min<size_t>(n, max_checks) : n;
    std::vector<uint8_t> checked(n, 0);
    // one exact check; true when it is racy (the search ends)
    const auto check = [&](size_t i) {
      const auto c0 = clock::now();
      Instance I{&bcs[i]->prog, groups[i], group_size[i], (uint64_t)groups[i] * group_size[i], &inputs[i],
                 static_cast<cudaStream_t>(inputs[i].cuda_stream)};
      rc_report *r = run_instance(I);
      checked[i] = 1;
      res->checks++;
      res->check_seconds += secs(c0, clock::now());
      if (r->status == RC_RACY) {
        res->first = (int64_t)i;
        if (found) *found = r;
        else rc_report_free(r);
        return true;
      }
      rc_report_free(r);
      return false;
    };
    const bool overlap = flags & RC_RANK_OVERLAP;
    try {
      job = features_start(bcs, groups, group_size, inputs, n, X, 0, !overlap);
    } catch (const std::string &e) {
      throw Fail{RC_E_INVALID, e};
    }
    // the job writes into X until features_wait returns: wait on every way out
    struct Waiter {
      std::shared_ptr<FeatureJob> &j;
      ~Waiter() {
        if (j) {
          features_cancel(*j);
          try {
            features_wait(*j);
          } catch (...) {
          }
        }
      }
    } waiter{job};
    if (g_prof.on) prof_events();
    bool racy = false;
    if (overlap)
      for (size_t i = 0; i < limit && !racy && !features_finished(*job); i++) racy = check(i);
    res->checks_unranked = res->checks;
    if (racy) features_cancel(*job);  // candidates in progress still finish
    try {
      features_wait(*job);
    } catch (const std::string &e) {
      if (!racy) throw Fail{RC_E_NOMEM, e};
    }
    job.reset();
    if (!racy) {
      const auto f1 = clock::now();
      res->features_seconds = secs(t0, f1);
      if (model) {
        cudaStream_t s = static_cast<cudaStream_t>(inputs[0].cuda_stream);
        float *dx = W.rankx.get<float>(n * RC_N_FEATURES + n);
        CK(cudaMemcpyAsync(dx, X, n * RC_N_FEATURES * sizeof(float), cudaMemcpyHostToDevice, s));
        const int e = rc_mlp_forward(model, dx, n, dx + n * RC_N_FEATURES, s);
        if (e != RC_OK) throw Fail{e, "scoring the candidates failed: " + g_last_error};
        CK(cudaMemcpyAsync(score, dx + n * RC_N_FEATURES, n * sizeof(float), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
      } else {
        for (size_t i = 0; i < n; i++) {
          const float *f = X + i * RC_N_FEATURES;
          // products by powers of two are exact and a division is never
          // fused: the same float on every host and in numpy
          score[i] = 4.0f * f[108] + 2.0f * f[107] + (f[104] + f[105]) / 10.0f;
        }
      }
      std::vector<size_t> order(n);
      for (size_t i = 0; i < n; i++) order[i] = i;
      std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return score[a] > score[b]; });
      res->scoring_seconds = secs(f1, clock::now());
      for (size_t k = 0; k < n && res->checks < limit && !racy; k++)
        if (!checked[order[k]]) racy = check(order[k]);
    } else {
      res->features_seconds = secs(t0, clock::now());
    }
    res->seconds = secs(t0, clock::now());
    return RC_OK;
  } catch (const Fail &f) {
    return fail_code(f);
  } catch (const std::bad_alloc &) {
    g_last_error = "host allocation failed";
    return RC_E_NOMEM;
  }
}

int rc_check_batch(const rc_bytecode *const *bcs, const uint32_t *groups, const uint32_t *group_size,
                   const rc_input *inputs, size_t n, rc_report **out) {
  if (!out || (n && (!bcs || !groups || !group_size || !inputs))) return RC_E_INVALID;
  for (size_t i = 0; i < n; i++) out[i] = nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  try {
    std::vector<BatchItem> items;
    items.reserve(n);
    for (size_t i = 0; i < n; i++) {
      check_args(bcs[i], groups[i], group_size[i], &inputs[i]);
      if (inputs[i].flags & RC_GROUP_BARRIERS)
        throw Fail{RC_E_INVALID, "batched checking takes kernel-wide barriers only"};
      items.push_back(plan_item(bcs[i], groups[i], group_size[i], &inputs[i]));
    }
    if (g_prof.on) prof_events();
    // sub-batches: instances in order while the cell space stays below 2^31
    // and the estimated workspace below the batch budget
    const uint64_t budget = (uint64_t)48 << 30;
    size_t i = 0;
    while (i < n) {
      size_t j = i;
      uint64_t cells = 0, bytes = 0;
      while (j < n && (j == i || (cells + items[j].L.keys < (1ull << 31) && bytes + items[j].bytes <= budget))) {
        cells += items[j].L.keys;
        bytes += items[j].bytes;
        j++;
      }
      if (cells >= (1ull << 31) || bytes > ((uint64_t)200 << 30)) throw Fail{RC_E_CAPACITY, "instance too large for a batch"};
      std::vector<BatchItem> sub(items.begin() + i, items.begin() + j);
      // strategies 1 and 2 fix the classification of lock-step rounds, 3 asks
      // for a resident run (lock-step when it cannot finish); 0 and 4 leave
      // the choice to the autotuner
      const cudaStream_t bs = static_cast<cudaStream_t>(inputs[i].cuda_stream);
      const int lockstep = g_strategy == 1 || g_strategy == 2 ? g_strategy : 0;
      bool done = g_strategy == 3 && run_batch(sub, bs, 3, out + i);
      // a run whose slices overflowed the tuned log capacity returns false and
      // goes again at the static bound, which the class keeps from then on
      for (int attempt = 0; !done && attempt < 2; attempt++) done = run_batch(sub, bs, lockstep, out + i);
      if (!done) throw Fail{RC_E_CAPACITY, "batch log overflowed at its static bound"};
      i = j;
    }
    return RC_OK;
  } catch (const Fail &f) {
    for (size_t i = 0; i < n; i++) {
      rc_report_free(out[i]);
      out[i] = nullptr;
    }
    return fail_code(f);
  } catch (const std::bad_alloc &) {
    for (size_t i = 0; i < n; i++) {
      rc_report_free(out[i]);
      out[i] = nullptr;
    }
    g_last_error = "host allocation failed";
    return RC_E_NOMEM;
  }
}

void rc_bytecode_free(rc_bytecode *bc) { delete bc; }

void rc_report_free(rc_report *rep) {
  if (!rep) return;
  std::free(rep->records);
  std::free(rep->final_global);
  std::free(rep);
}

const char *rc_strerror(int code) {
  switch (code) {
    case RC_OK: return "ok";
    case RC_E_PARSE: return "kernel source does not parse";
    case RC_E_INVALID: return "invalid argument, shape, input or bytecode";
    case RC_E_CAPACITY: return "instance exceeds device capacity";
    case RC_E_CUDA: return "CUDA runtime error";
    case RC_E_TIMEOUT: return "bounded device wait ran out";
    case RC_E_NOMEM: return "host out of memory";
    default: return "unknown error";
  }
}

const char *rc_last_error(void) { return g_last_error.c_str(); }

int rc_sort_accesses(const rc_access *in, rc_access *out, uint64_t n, uint32_t cell_bits, uint32_t item_bits,
                     void *cuda_stream) {
  static_assert(sizeof(rc_access) == sizeof(LogRec), "access record layout");
  if (n == 0) return RC_OK;
  if (!in || !out || item_bits > 31 || cell_bits + item_bits > 58 || n >= 0xFFFFFFFFull) {
    g_last_error = "rc_sort_accesses: bad pointers or sizes";
    return RC_E_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  try {
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    LogRec *scratch = g_ws.sortscr.get<LogRec>(n);
    uint32_t *tmp = g_ws.scan.get<uint32_t>(sort_tmp_words(n));
    sort_log_into(reinterpret_cast<const LogRec *>(in), reinterpret_cast<LogRec *>(out), scratch, n,
                  std::max<uint32_t>(item_bits, 1), cell_bits + std::max<uint32_t>(item_bits, 1), tmp, s);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    return RC_OK;
  } catch (const Fail &f) {
    return fail_code(f);
  }
}

int rc_diag_grid_barrier(uint32_t limit_us, int32_t *timed_out, double *seconds) {
  if (!timed_out || !seconds || limit_us == 0 || limit_us > 10000000u) return RC_E_INVALID;
  std::lock_guard<std::mutex> lk(g_mu);
  try {
    int dev = 0, coop = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) throw Fail{RC_E_CUDA, "cooperative launches are not supported"};
    unsigned *bar = g_ws.rbar.get<unsigned>(kGridBarWords);
    CK(cudaMemset(bar, 0, kGridBarWords * 4));
    const auto t0 = std::chrono::steady_clock::now();
    CK(launch_grid_barrier_probe(bar, (uint32_t)sm_count(), (unsigned long long)limit_us * 1000ull, nullptr));
    unsigned h[3] = {0, 0, 0};
    CK(cudaMemcpy(h, bar, 12, cudaMemcpyDeviceToHost));
    *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *timed_out = h[2] != 0;
    return RC_OK;
  } catch (const Fail &f) {
    return fail_code(f);
  }
}

int rc_release_workspace(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_ws.release_all();
  return RC_OK;
}

int rc_set_strategy(int strategy) {
  if (strategy < 0 || strategy > 4) return RC_E_INVALID;
  std::lock_guard<std::mutex> lk(g_mu);
  g_strategy = strategy;
  return RC_OK;
}

int rc_set_engine(int engine) {
  if (engine < 0 || engine > 2) return RC_E_INVALID;
  std::lock_guard<std::mutex> lk(g_mu);
  g_engine = engine;
  return RC_OK;
}

int rc_jit_compile(const rc_bytecode *bc, uint32_t groups, uint32_t group_size, const rc_input *in, int resident,
                   double *seconds, uint64_t *cubin_bytes) {
  try {
    check_args(bc, groups, group_size, in);
    std::string why;
    if (!jit_available(&why)) throw Fail{RC_E_INVALID, "compiled intervals unavailable: " + why};
    const std::vector<Insn> &code = private_code(bc->prog, groups, group_size, in);
    JitShape sh;
    sh.resident = resident != 0;
    sh.threads = group_size;
    sh.min_blocks = resident ? 2 : std::min<uint32_t>(std::max<uint32_t>(1, 1024 / group_size), 32);
    sh.load = false;
    const auto t0 = std::chrono::steady_clock::now();
    const JitKernel k = jit_kernel(bc->prog, code, sh);
    if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (cubin_bytes) *cubin_bytes = k.cubin_bytes;
    return RC_OK;
  } catch (const Fail &f) {
    return fail_code(f);
  } catch (const JitError &e) {
    g_last_error = e.msg;
    return RC_E_INVALID;
  } catch (const std::bad_alloc &) {
    g_last_error = "host allocation failed";
    return RC_E_NOMEM;
  }
}

int rc_jit_stats(uint64_t *compiles, double *seconds) {
  if (!compiles || !seconds) return RC_E_INVALID;
  jit_stats(compiles, seconds);
  return RC_OK;
}

int rc_autotune_config(const char *cache_path) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_tuner.entries.clear();
  g_tuner.loaded = false;
  g_tuner.persist = !(cache_path && cache_path[0] == 0);
  g_tuner.path = cache_path ? cache_path : "";
  return RC_OK;
}

int rc_autotune_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_tuner.entries.clear();
  g_tuner.loaded = true;  // do not re-read the file
  return RC_OK;
}

int rc_autotune_lookup(int kind, uint64_t a, uint64_t b) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_tuner.load();
  if (kind < 0 || kind > 3) return 0;
  const std::string key = kind == 0 ? single_key(a, b) : batch_key(a, b);
  auto it = g_tuner.entries.find(key);
  if (it == g_tuner.entries.end()) return 0;
  return kind == 3 ? (int)it->second.log_pm : kind == 2 ? (int)it->second.threads : it->second.best;
}

int rc_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_prof.on = on != 0;
  return RC_OK;
}

int rc_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (int k = 0; k < 3; k++) {
    g_prof.launches[k] = 0;
    g_prof.ms[k] = 0;
    g_prof.bytes[k] = 0;
  }
  return RC_OK;
}

uint64_t rc_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int rc_profile_get(int kind, uint64_t *launches, double *ms, double *bytes) {
  if (kind < 0 || kind > 2) return RC_E_INVALID;
  std::lock_guard<std::mutex> lk(g_mu);
  if (launches) *launches = g_prof.launches[kind];
  if (ms) *ms = g_prof.ms[kind];
  if (bytes) *bytes = g_prof.bytes[kind];
  return RC_OK;
}

}  // extern "C"
