// Per-cell classification shared by the classification kernels
// (classify.cu) and the one-CTA check of small instances (interp.cu).
//
// A run of records of one (cell, work-item) becomes a Summary (summarize_run);
// classify_cell walks one cell's summaries in work-item order and applies the
// rules stated in classify.cu; emit_cell writes its records.
#pragma once
#include "device.cuh"

namespace rc {

// The Summary of the run of records of one (cell, work-item) that starts at
// r[i]: observed and written ranges, the value of the last write (highest
// sequence number: the records of a run need not be in program order), the
// access count.  *end = the first index past the run.
static __device__ __forceinline__ Summary summarize_run(const LogRec *r, uint64_t i, uint64_t n, uint64_t &end) {
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
  uint64_t j = i;
  for (; j < n; j++) {
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
  end = j;
  return s;
}

// uniform value of a range, or "mixed"
struct Uni {
  bool mixed;
  int32_t v;
};
static __device__ __forceinline__ bool same(const Uni &a, const Uni &b) { return !a.mixed && !b.mixed && a.v == b.v; }
static __device__ __forceinline__ Uni written(const Summary &s) { return Uni{s.wmin != s.wmax, s.wmin}; }

// What decides a cell's witnesses: the first two writers w1, w2 (their
// written ranges u1, u2, w1's last value l1); tb: first writer after w1
// whose last value differs from l1; d1, d2: first two writers after w1
// whose range is not w1's single value; e2: first writer after w2 whose
// range is not w2's single value.
struct CellVals {
  uint32_t w1, w2, tb, d1, d2, e2;
  Uni u1, u2;
  int32_t l1;
};

// The smallest writer j != r whose writes conflict with what reader s
// observed (kNone if none), from the cell's candidates.
static __device__ __forceinline__ uint32_t reader_conflict(const Summary &s, const CellVals &v) {
  const uint32_t r = s.gtid;
  if (s.rmin != s.rmax) return v.w1 != r ? v.w1 : v.w2;  // observed several values
  const Uni o{false, s.rmin};
  if (!same(v.u1, o)) {
    if (v.w1 != r) return v.w1;
    if (v.w2 == kNone) return kNone;
    return !same(v.u2, o) ? v.w2 : v.e2;
  }
  return v.d1 != r ? v.d1 : v.d2;
}

static __device__ __forceinline__ void set_ww(CellResult &c, const CellVals &v) {
  if (c.n_writers >= 2) {
    c.ww_cls = v.tb != kNone ? CLS_WW_RACE : CLS_WW_BENIGN;
    c.ww_a = v.w1;
    c.ww_b = v.tb != kNone ? v.tb : v.w2;
  }
}

// One thread walks the cell's summaries [b, end) in work-item order.
static __device__ CellResult classify_cell(const Summary *sum, uint64_t b, uint64_t nsum) {
  CellResult c{};
  const uint32_t key = sum[b].key;
  CellVals v{kNone, kNone, kNone, kNone, kNone, kNone, {true, 0}, {true, 0}, 0};
  uint64_t e = b;
  for (; e < nsum && sum[e].key == key; e++) {  // pass 1: counts and writer candidates
    const Summary s = sum[e];
    c.n_acc += s.meta & kMetaCount;
    if (s.meta & kMetaRead) c.n_readers++;
    if (!(s.meta & kMetaWrite)) continue;
    c.n_writers++;
    const Uni u = written(s);
    if (v.w1 == kNone) {
      v.w1 = s.gtid;
      v.u1 = u;
      v.l1 = s.wlast;
    } else {
      if (v.w2 == kNone) {
        v.w2 = s.gtid;
        v.u2 = u;
      } else if (v.e2 == kNone && !same(u, v.u2)) {
        v.e2 = s.gtid;
      }
      if (v.tb == kNone && s.wlast != v.l1) v.tb = s.gtid;
      if (!v.u1.mixed && !same(u, v.u1)) {
        if (v.d1 == kNone) v.d1 = s.gtid;
        else if (v.d2 == kNone) v.d2 = s.gtid;
      }
    }
    c.wrote = 1;
    c.commit = s.wlast;  // ascending order: ends with the highest writer
  }
  set_ww(c, v);
  c.rw_a = kNone;
  if (c.n_writers > 0 && c.n_readers > 0) {
    for (uint64_t k = b; k < e; k++) {  // pass 2: first reader with a conflict
      const Summary s = sum[k];
      if (!(s.meta & kMetaRead)) continue;
      const uint32_t j = reader_conflict(s, v);
      if (j != kNone) {
        c.rw_a = s.gtid;
        c.rw_b = j;
        break;
      }
    }
  }
  return c;
}

static __device__ __forceinline__ OutRec make_rec(const ClassifyArgs &a, uint32_t key, uint32_t cls, uint32_t ta,
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

static __device__ __forceinline__ void emit_cell(const ClassifyArgs &a, uint32_t key, const CellResult &c, uint32_t p,
                                          OutRec *out) {
  if (c.ww_cls) {
    out[p] = make_rec(a, key, c.ww_cls, c.ww_a, c.ww_b, c, p);
    p++;
  }
  if (c.rw_a != kNone) out[p] = make_rec(a, key, CLS_RW_RACE, c.rw_a, c.rw_b, c, p);
}

}  // namespace rc
