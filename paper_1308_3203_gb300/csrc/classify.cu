// Race classification of one barrier interval from its access log sorted by
// (cell, work-item), and the commit of the interval's writes.
//
// Step 1 (run reduce): every run of records of one (cell, work-item) becomes
// a Summary: the range of values the work-item observed, the range it wrote,
// the value of its last write (highest sequence number) and its access count.
//
// Step 2 (per cell, over the summaries of that cell in work-item order):
//  * WW (Sec. 1 and the race rule of Sec. 4: differing values at a barrier
//    are a race, one common value is benign): each writer's LAST value
//    counts.  Two writers whose last values differ -> WW_RACE with witness
//    (smallest writer w1, smallest writer whose last value differs from
//    w1's); two or more writers, one value -> WW_BENIGN (w1, w2).
//  * RW: a read by r that observed o conflicts with a write by j != r of a
//    value v != o.  Witness: the lexicographically smallest (r, j).  A reader
//    r that observed one value c conflicts with the smallest writer j != r
//    that did not write c alone; one that observed several values conflicts
//    with the smallest writer j != r.  One forward pass over the writers
//    collects the few candidates this needs (w1, w2, the first two writers
//    differing from w1's value, the first writer after w2 differing from
//    w2's value); a second pass stops at the first reader with a conflict.
//  * commit: the cell takes the last write of its highest writer (the
//    schedule that runs work-items in id order).
#include "device.cuh"

namespace rc {
namespace {

constexpr int kThreads = 256;

__global__ void run_heads_kernel(const LogRec *r, uint64_t n, uint32_t *head) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t h = 1;
  if (i > 0) {
    const LogRec a = r[i - 1], b = r[i];
    h = (a.key != b.key || ((a.tw ^ b.tw) & 0x7FFFFFFFu) != 0) ? 1u : 0u;
  }
  head[i] = h;
}

__global__ void run_reduce_kernel(const LogRec *r, uint64_t n, const uint32_t *head,
                                  const uint32_t *runidx, Summary *sum, uint32_t *khead) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !head[i]) return;
  const LogRec f = r[i];
  const uint32_t g = f.tw & 0x7FFFFFFFu;
  Summary s;
  s.key = f.key;
  s.gtid = g;
  s.rmin = INT32_MAX;
  s.rmax = INT32_MIN;
  s.wmin = INT32_MAX;
  s.wmax = INT32_MIN;
  s.wlast = 0;
  uint32_t cnt = 0, flags = 0, lastseq = 0;
  for (uint64_t j = i; j < n; j++) {
    const LogRec x = r[j];
    if (x.key != f.key || (x.tw & 0x7FFFFFFFu) != g) break;
    cnt++;
    if (x.tw & 0x80000000u) {
      flags |= kMetaWrite;
      s.wmin = min(s.wmin, x.val);
      s.wmax = max(s.wmax, x.val);
      if (x.seq >= lastseq) {
        lastseq = x.seq;
        s.wlast = x.val;
      }
    } else {
      flags |= kMetaRead;
      s.rmin = min(s.rmin, x.val);
      s.rmax = max(s.rmax, x.val);
    }
  }
  s.meta = min(cnt, kMetaCount) | flags;
  const uint32_t k = runidx[i];
  sum[k] = s;
  khead[k] = (i == 0 || r[i - 1].key != f.key) ? 1u : 0u;
}

struct CellResult {
  uint32_t n_readers, n_writers, n_acc;
  uint32_t ww_cls, ww_a, ww_b;  // ww_cls 0 = none
  uint32_t rw_a, rw_b;          // rw_a kNone = none
  bool wrote;
  int32_t commit;
};

// uniform value of a range, or "mixed"
struct Uni {
  bool mixed;
  int32_t v;
};
__device__ __forceinline__ bool same(const Uni &a, const Uni &b) { return !a.mixed && !b.mixed && a.v == b.v; }

__device__ CellResult classify_cell(const Summary *sum, uint64_t b, uint64_t nsum) {
  CellResult c{};
  const uint32_t key = sum[b].key;
  uint32_t w1 = kNone, w2 = kNone, tb = kNone, d1 = kNone, d2 = kNone, e2 = kNone;
  Uni u1{true, 0}, u2{true, 0};
  int32_t l1 = 0;
  uint64_t e = b;
  for (; e < nsum && sum[e].key == key; e++) {  // pass 1: counts and writer candidates
    const Summary s = sum[e];
    c.n_acc += s.meta & kMetaCount;
    if (s.meta & kMetaRead) c.n_readers++;
    if (!(s.meta & kMetaWrite)) continue;
    c.n_writers++;
    const Uni u{s.wmin != s.wmax, s.wmin};
    if (w1 == kNone) {
      w1 = s.gtid;
      u1 = u;
      l1 = s.wlast;
    } else {
      if (w2 == kNone) {
        w2 = s.gtid;
        u2 = u;
      } else if (e2 == kNone && !same(u, u2)) {
        e2 = s.gtid;
      }
      if (tb == kNone && s.wlast != l1) tb = s.gtid;
      if (!u1.mixed && !same(u, u1)) {
        if (d1 == kNone) d1 = s.gtid;
        else if (d2 == kNone) d2 = s.gtid;
      }
    }
    c.wrote = true;
    c.commit = s.wlast;  // ascending order: ends with the highest writer
  }
  if (c.n_writers >= 2) {
    c.ww_cls = tb != kNone ? CLS_WW_RACE : CLS_WW_BENIGN;
    c.ww_a = w1;
    c.ww_b = tb != kNone ? tb : w2;
  }
  c.rw_a = kNone;
  if (c.n_writers > 0 && c.n_readers > 0) {
    for (uint64_t k = b; k < e; k++) {  // pass 2: first reader with a conflict
      const Summary s = sum[k];
      if (!(s.meta & kMetaRead)) continue;
      const uint32_t r = s.gtid;
      uint32_t j;
      if (s.rmin != s.rmax) {
        j = w1 != r ? w1 : w2;
      } else {
        const Uni o{false, s.rmin};
        if (!same(u1, o)) {
          if (w1 != r) j = w1;
          else if (w2 == kNone) j = kNone;
          else if (!same(u2, o)) j = w2;
          else j = e2;
        } else {
          j = d1 != r ? d1 : d2;
        }
      }
      if (j != kNone) {
        c.rw_a = r;
        c.rw_b = j;
        break;
      }
    }
  }
  return c;
}

__device__ __forceinline__ OutRec make_rec(const ClassifyArgs &a, uint32_t key, uint32_t cls, uint32_t ta,
                                           uint32_t tb, const CellResult &c, uint32_t p) {
  OutRec o;
  o.interval = a.interval;
  uint32_t GT = a.GT, LT = a.LT;
  if (a.n_kernels) {  // batch: find the instance owning the cell (binary search on first cells)
    uint32_t lo = 0, hi = a.n_kernels;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) / 2;
      if (a.kbase[mid] <= key) lo = mid;
      else hi = mid;
    }
    key -= (uint32_t)a.kbase[lo];
    GT = a.kGT[lo];
    LT = a.kLT[lo] ? a.kLT[lo] : 1;
    a.rec_kernel[p] = lo;
  }
  if (key < GT) {
    o.space = 0;
    o.wg = 0;
    o.addr = key;
  } else {
    const uint32_t l = key - GT;
    o.space = 1;
    o.wg = l / LT;
    o.addr = l % LT;
  }
  o.cls = cls;
  o.t_a = ta;
  o.t_b = tb;
  o.n_readers = c.n_readers;
  o.n_writers = c.n_writers;
  o.n_accesses = c.n_acc;
  return o;
}

__global__ void key_classify_kernel(const Summary *sum, uint64_t nsum, const uint32_t *khead,
                                    const uint32_t *keyidx, uint32_t *nrec, ClassifyArgs a) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsum || !khead[i]) return;
  const CellResult c = classify_cell(sum, i, nsum);
  if (c.wrote) a.snap[sum[i].key] = c.commit;
  nrec[keyidx[i]] = (c.ww_cls ? 1u : 0u) + (c.rw_a != kNone ? 1u : 0u);
}

__global__ void key_emit_kernel(const Summary *sum, uint64_t nsum, const uint32_t *khead,
                                const uint32_t *keyidx, const uint32_t *nrec, const uint32_t *recoff,
                                OutRec *out, ClassifyArgs a) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsum || !khead[i]) return;
  const uint32_t k = keyidx[i];
  if (nrec[k] == 0) return;
  const CellResult c = classify_cell(sum, i, nsum);
  uint32_t p = recoff[k];
  const uint32_t key = sum[i].key;
  if (c.ww_cls) {
    out[p] = make_rec(a, key, c.ww_cls, c.ww_a, c.ww_b, c, p);
    p++;
  }
  if (c.rw_a != kNone) out[p] = make_rec(a, key, CLS_RW_RACE, c.rw_a, c.rw_b, c, p);
}

unsigned blocks_for(uint64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

void launch_run_heads(const LogRec *r, uint64_t n, uint32_t *head, cudaStream_t s) {
  if (n) count_launch();
  if (n) run_heads_kernel<<<blocks_for(n), kThreads, 0, s>>>(r, n, head);
}
void launch_run_reduce(const LogRec *r, uint64_t n, const uint32_t *head, const uint32_t *runidx,
                       Summary *sum, uint32_t *khead, cudaStream_t s) {
  if (n) count_launch();
  if (n) run_reduce_kernel<<<blocks_for(n), kThreads, 0, s>>>(r, n, head, runidx, sum, khead);
}
void launch_key_classify(const Summary *sum, uint64_t nsum, const uint32_t *khead,
                         const uint32_t *keyidx, uint32_t *nrec, const ClassifyArgs &a,
                         cudaStream_t s) {
  if (nsum) count_launch();
  if (nsum) key_classify_kernel<<<blocks_for(nsum), kThreads, 0, s>>>(sum, nsum, khead, keyidx, nrec, a);
}
void launch_key_emit(const Summary *sum, uint64_t nsum, const uint32_t *khead,
                     const uint32_t *keyidx, const uint32_t *nrec, const uint32_t *recoff,
                     OutRec *out, const ClassifyArgs &a, cudaStream_t s) {
  if (nsum) count_launch();
  if (nsum)
    key_emit_kernel<<<blocks_for(nsum), kThreads, 0, s>>>(sum, nsum, khead, keyidx, nrec, recoff, out, a);
}

}  // namespace rc
