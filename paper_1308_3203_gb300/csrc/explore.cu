// Exhaustive interleavings of one barrier interval, on the GPU.
//
// Sec. 4's global rules let any work-item take the next step, and a kernel is
// racy when two schedules reach different shared states at a barrier (the
// Definition after the race rule).  The checker runs one canonical schedule
// with delayed visibility and flags conflicts conservatively; this explorer
// takes the checker's state at the start of an interval and runs EVERY
// schedule of that interval with one truly shared memory, so a flagged
// interval can be confirmed (several shared states reachable at its closing
// barrier, or a read that depends on the schedule) or shown schedule-
// independent.
//
// Private commands commute with the other work-items' steps, so a state keeps
// every work-item either stopped or at its next shared access, and a step is
// one work-item's access followed by its private commands up to the next one.
// The search is breadth-first over distinct states: each level expands every
// (state, work-item) pair in parallel, children are hashed, radix-sorted by
// hash and compared word by word with the earlier members of their hash
// group, and the unique ones form the next level.  States whose work-items
// have all stopped are the interval's end states; their shared memories are
// deduplicated the same way and counted.
//
// A state is [header: 2 words] + [per work-item: pc, status, reads, registers]
// + [cells].  In pair mode (the interleaving product of two work-items
// i < j, the fix the paper proposes at the end of Sec. 6) a state holds only
// the two work-items (header = (i, j)) and every pair is searched at once.
#include <algorithm>
#include <vector>

#include "device.cuh"
#include "semantics.cuh"

namespace rc {
namespace {

#define CK_EX(x)                                                          \
  do {                                                                    \
    cudaError_t e_ = (x);                                                 \
    if (e_ != cudaSuccess) throw ExploreError{cudaGetErrorString(e_)};    \
  } while (0)

// device array that grows on demand
template <class T>
struct DevArray {
  T *p = nullptr;
  size_t cap = 0;  // elements
  T *get(size_t n) {
    if (n > cap) {
      if (p) cudaFree(p);
      p = nullptr;
      cap = 0;
      const size_t want = std::max<size_t>(n + n / 4, 64);
      CK_EX(cudaMalloc(&p, want * sizeof(T)));
      cap = want;
    }
    return p;
  }
  // grow to n elements keeping the first `keep`
  T *grow(size_t n, size_t keep, cudaStream_t s) {
    if (n <= cap) return p;
    T *q = nullptr;
    const size_t want = n + n / 2;
    CK_EX(cudaMalloc(&q, want * sizeof(T)));
    if (keep) CK_EX(cudaMemcpyAsync(q, p, keep * sizeof(T), cudaMemcpyDeviceToDevice, s));
    CK_EX(cudaStreamSynchronize(s));
    if (p) cudaFree(p);
    p = q;
    cap = want;
    return p;
  }
  ~DevArray() {
    if (p) cudaFree(p);
  }
};

enum : uint32_t { EX_RUN = 0, EX_BAR = 1, EX_EXIT = 2, EX_DEAD = 3 };
constexpr uint32_t kExStepCap = 1u << 20;  // private instructions per step (constant-trip loops stay far below)

struct ExCtx {
  const uint4 *code;
  const MemInfo *mems;  // device copy of the layout (len, base, space)
  uint32_t n_insn, N, S, TS, GT, LT;
  uint32_t K;      // work-item slices per state: N, or 2 (pair mode)
  uint32_t C;      // cells
  uint32_t W;      // state words: 2 (header) + K * TS + C
  uint32_t E;      // end item words: 2 (header) + C
  bool pairs;      // header = the pair (i, j) of the slices, else (0, 0) and slice q is work-item q
  const int32_t *solo;  // [N][B] reads of each work-item alone from the start state
  const uint32_t *solo_len;
  uint32_t B;
  uint32_t *flags;      // bit 0: a read depended on the schedule, bit 1: a step ran past the cap
  uint32_t *pair_dev;   // pair mode: per pair, a read depended on the schedule
};

__device__ __forceinline__ uint32_t *slice(uint32_t *st, uint32_t q, const ExCtx &c) { return st + 2 + q * c.TS; }
__device__ __forceinline__ uint32_t wid(const uint32_t *st, uint32_t q, const ExCtx &c) { return c.pairs ? st[q] : q; }
__device__ __forceinline__ uint32_t pair_index(uint32_t i, uint32_t j, uint32_t N) {
  return i * (2 * N - i - 1) / 2 + (j - i - 1);
}

// Run the work-item in slice q through its private instructions until it is
// at a shared access or stops.
__device__ void ex_normalize(uint32_t *st, uint32_t q, const ExCtx &c) {
  uint32_t *t = slice(st, q, c);
  int32_t *reg = reinterpret_cast<int32_t *>(t + 3);
  for (uint32_t n = 0; t[1] == EX_RUN; n++) {
    if (n >= kExStepCap || t[0] >= c.n_insn) {
      atomicOr(c.flags, 2u);
      t[1] = EX_DEAD;
      return;
    }
    const uint4 raw = c.code[t[0]];
    const uint32_t d = (raw.x >> 8) & 0xFFu, ra = (raw.x >> 16) & 0xFFu, rb = raw.x >> 24;
    const int32_t imm = (int32_t)raw.y;
    const uint32_t ctl = raw.w, cls = (ctl >> CTL_CLASS_SHIFT) & 0xFu;
    const int32_t x = reg[ra], yr = reg[rb];
    switch (cls) {
      case CC_ALU: {
        const int32_t r = sem_alu(raw.x & 0xFFu, x, yr, imm);
        if (ctl & AL_WRITE) reg[d] = r;
        t[0] = sem_branch(ctl, r, imm) ? raw.z : t[0] + 1;
        break;
      }
      case CC_LD:
      case CC_ST:
        return;
      case CC_DIVMOD: reg[d] = sem_divmod(ctl, x, yr, imm); t[0]++; break;
      case CC_LOGIC: reg[d] = sem_logic(ctl, x, yr); t[0]++; break;
      case CC_SIZE: reg[d] = (int32_t)c.mems[ctl >> CTL_MEM_SHIFT].len; t[0]++; break;
      case CC_ASSUME:  // no continuation
      case CC_ASSERT:  // the work-item aborts
        if (x == 0) t[1] = EX_DEAD;
        t[0]++;
        break;
      case CC_BARRIER: t[1] = EX_BAR; return;
      default: t[1] = EX_EXIT; return;
    }
  }
}

// The work-item in slice q performs its pending access on the shared cells,
// then runs to its next one.  Returns true for a read, with the observed value.
__device__ bool ex_access(uint32_t *st, uint32_t q, const ExCtx &c, int32_t &observed) {
  uint32_t *t = slice(st, q, c);
  int32_t *reg = reinterpret_cast<int32_t *>(t + 3);
  int32_t *cells = reinterpret_cast<int32_t *>(st + 2 + c.K * c.TS);
  const uint4 raw = c.code[t[0]];
  const uint32_t d = (raw.x >> 8) & 0xFFu, ra = (raw.x >> 16) & 0xFFu, rb = raw.x >> 24;
  const uint32_t ctl = raw.w, cls = (ctl >> CTL_CLASS_SHIFT) & 0xFu;
  const MemInfo m = c.mems[ctl >> CTL_MEM_SHIFT];
  const int32_t idx = sem_index(reg[ra], (int32_t)raw.y, (int32_t)raw.z, ctl);
  if ((uint32_t)idx >= m.len) {  // out of bounds: the work-item stops, nothing is accessed
    t[1] = EX_DEAD;
    return false;
  }
  const uint32_t cell = (m.space ? c.GT + (uint32_t)reg[REG_WG] * c.LT : 0u) + m.base + (uint32_t)idx;
  bool read = false;
  if (cls == CC_LD) {
    reg[d] = cells[cell];
    observed = cells[cell];
    t[2]++;
    read = true;
  } else {
    cells[cell] = reg[rb];
  }
  t[0]++;
  ex_normalize(st, q, c);
  return read;
}

__device__ __forceinline__ void copy_words(uint32_t *dst, const uint32_t *src, uint32_t W) {
  for (uint32_t i = 0; i < W; i++) dst[i] = src[i];
}

// Full state from the checker's arrays: work-items at a barrier resume after
// it; registers 0..4 hold the built-ins.
__global__ void ex_start_kernel(ExCtx c, const int32_t *snap, const int32_t *regs, const uint32_t *pc,
                                const uint32_t *stv, uint32_t n_regs, uint32_t interval, uint32_t *out) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g == 0) out[0] = out[1] = 0;
  if (g < c.N) {
    uint32_t *t = slice(out, g, c);
    const uint32_t s = stv[g];
    t[0] = s == TS_BARRIER ? pc[g] + 1 : pc[g];
    t[1] = (s == TS_BARRIER || (s == TS_RUN && interval == 0)) ? EX_RUN : s == TS_EXIT ? EX_EXIT : EX_DEAD;
    t[2] = 0;
    int32_t *reg = reinterpret_cast<int32_t *>(t + 3);
    for (uint32_t r = 0; r < c.TS - 3; r++) reg[r] = r < n_regs ? regs[(uint64_t)r * c.N + g] : 0;
    reg[REG_TID] = (int32_t)(g % c.S);
    reg[REG_WG] = (int32_t)(g / c.S);
    reg[REG_GTID] = (int32_t)g;
    reg[REG_GSIZE] = (int32_t)c.S;
    reg[REG_NGROUPS] = (int32_t)(c.N / c.S);
  }
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < c.C; i += gridDim.x * blockDim.x)
    out[2 + c.N * c.TS + i] = (uint32_t)snap[i];
}

__global__ void ex_normalize_kernel(ExCtx c, uint32_t *st) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < c.N) ex_normalize(st, g, c);
}

// work-item g alone from the full start state: the reads it makes
__global__ void ex_solo_kernel(ExCtx c, const uint32_t *start, uint32_t *scratch, int32_t *solo, uint32_t *solo_len) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= c.N) return;
  uint32_t *st = scratch + (uint64_t)g * c.W;
  copy_words(st, start, c.W);
  uint32_t n = 0;
  while (slice(st, g, c)[1] == EX_RUN) {
    int32_t o = 0;
    if (ex_access(st, g, c, o)) {
      if (n < c.B) solo[(uint64_t)g * c.B + n] = o;
      n++;
    }
  }
  solo_len[g] = n;
}

// pair states: header (i, j), the two work-items' slices, the cells
__global__ void ex_pairs_kernel(ExCtx full, const uint32_t *start, ExCtx pc, const uint2 *pairs, uint32_t n_pairs,
                                uint32_t *out) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pairs) return;
  uint32_t *o = out + (uint64_t)p * pc.W;
  o[0] = pairs[p].x;
  o[1] = pairs[p].y;
  copy_words(o + 2, start + 2 + pairs[p].x * full.TS, full.TS);
  copy_words(o + 2 + pc.TS, start + 2 + pairs[p].y * full.TS, full.TS);
  copy_words(o + 2 + 2 * pc.TS, start + 2 + full.N * full.TS, full.C);
}

// a state whose work-items have all stopped is an end state: its header and
// cells go to the end pool, and it is marked finished (not a frontier state)
__device__ __forceinline__ void settle(uint32_t *st, const ExCtx &c, uint32_t *ends, unsigned long long *n_ends,
                                      uint64_t cap) {
  for (uint32_t q = 0; q < c.K; q++)
    if (slice(st, q, c)[1] == EX_RUN) return;
  const unsigned long long e = atomicAdd(n_ends, 1ull);
  if (e < cap) {
    uint32_t *o = ends + e * c.E;
    o[0] = st[0];
    o[1] = st[1];
    copy_words(o + 2, st + 2 + c.K * c.TS, c.C);
  }
  st[0] = 0xFFFFFFFFu;
}

__global__ void ex_settle_kernel(ExCtx c, uint32_t *states, uint64_t n, uint32_t *ends, unsigned long long *n_ends) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) settle(states + i * c.W, c, ends, n_ends, n);
}

// one thread per (frontier state, slice): the child where that work-item steps
__global__ void ex_expand_kernel(ExCtx c, const uint32_t *front, uint32_t n_front, uint32_t *kids,
                                 unsigned long long *n_kids, uint32_t *ends, unsigned long long *n_ends,
                                 uint64_t cap) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (uint64_t)n_front * c.K) return;
  const uint32_t f = (uint32_t)(i / c.K), q = (uint32_t)(i % c.K);
  const uint32_t *src = front + (uint64_t)f * c.W;
  if (src[2 + q * c.TS + 1] != EX_RUN) return;
  const unsigned long long k = atomicAdd(n_kids, 1ull);
  if (k >= cap) return;  // cannot happen: cap = n_front * K
  uint32_t *st = kids + k * c.W;
  copy_words(st, src, c.W);
  const uint32_t g = wid(st, q, c);
  const uint32_t r = slice(st, q, c)[2];
  int32_t o = 0;
  if (ex_access(st, q, c, o)) {
    if (r >= c.solo_len[g] || r >= c.B || c.solo[(uint64_t)g * c.B + r] != o) {
      atomicOr(c.flags, 1u);
      if (c.pairs) c.pair_dev[pair_index(st[0], st[1], c.N)] = 1;
    }
  }
  settle(st, c, ends, n_ends, cap);
}

// number of distinct end memories of each pair
__global__ void ex_pair_count_kernel(const uint32_t *ends, uint64_t n, uint32_t E, uint32_t N, uint32_t *count) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&count[pair_index(ends[i * E], ends[i * E + 1], N)], 1u);
}

// hash record per item of `words` words: (hash >> 32, hash & 0x7FFFFFFF, index); finished children
// (first word 0xFFFFFFFF) get the largest key and are dropped after the sort
__global__ void ex_hash_kernel(const uint32_t *items, uint64_t n, uint32_t words, bool skip_marked, LogRec *out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t *p = items + i * words;
  uint64_t h = 0x243F6A8885A308D3ull;
  for (uint32_t k = 0; k < words; k++) {
    h ^= p[k];
    h *= 0x9E3779B97F4A7C15ull;
    h ^= h >> 29;
  }
  if (skip_marked && p[0] == 0xFFFFFFFFu) h = ~0ull;
  else if ((h | 0x80000000ull) == ~0ull) h ^= 1ull << 32;  // keep the finished key for finished items only
  out[i] = LogRec{(uint32_t)(h >> 32), (uint32_t)(h & 0x7FFFFFFFu), (int32_t)i, 0};
}

__device__ __forceinline__ bool same_hash(const LogRec &a, const LogRec &b) { return a.key == b.key && a.tw == b.tw; }

// keep[i] = 1 for the first of each distinct item in hash order
__global__ void ex_unique_kernel(const LogRec *sorted, uint64_t n, const uint32_t *items, uint32_t words,
                                 uint32_t *keep) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const LogRec me = sorted[i];
  if (me.key == 0xFFFFFFFFu && me.tw == 0x7FFFFFFFu) {  // a finished child
    keep[i] = 0;
    return;
  }
  const uint32_t *a = items + (uint64_t)me.val * words;
  uint32_t k = 1;
  for (uint64_t j = i; j > 0 && same_hash(sorted[j - 1], me) && k; j--) {
    const uint32_t *b = items + (uint64_t)sorted[j - 1].val * words;
    bool eq = true;
    for (uint32_t w = 0; w < words && eq; w++) eq = a[w] == b[w];
    if (eq) k = 0;
  }
  keep[i] = k;
}

__global__ void ex_gather_kernel(const LogRec *sorted, uint64_t n, const uint32_t *keep, const uint32_t *pos,
                                 const uint32_t *items, uint32_t words, uint32_t *out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !keep[i]) return;
  copy_words(out + (uint64_t)pos[i] * words, items + (uint64_t)sorted[i].val * words, words);
}

unsigned nb(uint64_t n, unsigned t = 256) { return (unsigned)((n + t - 1) / t); }

struct ExBufs {
  DevArray<uint32_t> base, front, kids, ends, keep, pos, flags, scratch, solo_len, tmp, pcount, pdev;
  DevArray<int32_t> solo;
  DevArray<LogRec> ra, rb;
  DevArray<uint2> pairs;
  DevArray<unsigned long long> counts;
};

// Distinct items among items[0, n): they are written to the front of `out`
// (capacity n); returns how many.
uint64_t dedup(ExBufs &B, const uint32_t *items, uint64_t n, uint32_t words, bool skip_marked, uint32_t *out,
               cudaStream_t s) {
  if (n == 0) return 0;
  LogRec *a = B.ra.get(n), *b = B.rb.get(n);
  count_launch();
  ex_hash_kernel<<<nb(n), 256, 0, s>>>(items, n, words, skip_marked, a);
  uint32_t *tmp = B.tmp.get(std::max(sort_tmp_words(n), scan_tmp_words(n)));
  LogRec *sorted = sort_log(a, b, n, 31, 63, tmp, s);
  uint32_t *keep = B.keep.get(n), *pos = B.pos.get(n);
  count_launch();
  ex_unique_kernel<<<nb(n), 256, 0, s>>>(sorted, n, items, words, keep);
  scan_exclusive(keep, pos, n, tmp, s);
  uint32_t h[2];
  CK_EX(cudaMemcpyAsync(&h[0], pos + n - 1, 4, cudaMemcpyDeviceToHost, s));
  CK_EX(cudaMemcpyAsync(&h[1], keep + n - 1, 4, cudaMemcpyDeviceToHost, s));
  CK_EX(cudaStreamSynchronize(s));
  count_launch();
  ex_gather_kernel<<<nb(n), 256, 0, s>>>(sorted, n, keep, pos, items, words, out);
  return (uint64_t)h[0] + h[1];
}

}  // namespace

ExploreResult explore_interval(const ExploreInput &in, uint64_t max_states, cudaStream_t s,
                               std::vector<uint32_t> *pair_out) {
  static ExBufs B;
  ExploreResult res{};
  ExCtx full{};
  full.code = reinterpret_cast<const uint4 *>(in.code);
  full.mems = in.mems;
  full.n_insn = in.n_insn;
  full.N = in.N;
  full.S = in.S;
  full.TS = 3 + in.n_regs;
  full.GT = in.GT;
  full.LT = in.LT;
  full.K = in.N;
  full.C = in.cells;
  full.W = 2 + full.K * full.TS + full.C;
  full.E = 2 + full.C;
  full.B = std::max<uint32_t>(in.max_access, 1);
  full.flags = B.flags.get(1);
  CK_EX(cudaMemsetAsync(full.flags, 0, 4, s));
  uint32_t *base = B.base.get(full.W);
  count_launch();
  ex_start_kernel<<<nb(std::max(full.N, full.C)), 256, 0, s>>>(full, in.snap, in.regs, in.pc, in.st, in.n_regs,
                                                              in.interval, base);
  count_launch();
  ex_normalize_kernel<<<nb(full.N), 256, 0, s>>>(full, base);
  int32_t *solo = B.solo.get((uint64_t)full.N * full.B);
  uint32_t *solo_len = B.solo_len.get(full.N);
  uint32_t *scratch = B.scratch.get((uint64_t)full.N * full.W);
  count_launch();
  ex_solo_kernel<<<nb(full.N), 256, 0, s>>>(full, base, scratch, solo, solo_len);
  full.solo = solo;
  full.solo_len = solo_len;

  // the search runs on full states, or on the states of every pair (i < j)
  ExCtx c = full;
  uint64_t n_init = 1;
  const uint32_t P = in.N * (in.N - 1) / 2;
  if (pair_out) {
    c.pairs = true;
    c.K = 2;
    c.W = 2 + 2 * c.TS + c.C;
    c.pair_dev = B.pdev.get(std::max<uint32_t>(P, 1));
    CK_EX(cudaMemsetAsync(c.pair_dev, 0, std::max<uint32_t>(P, 1) * 4, s));
    std::vector<uint2> pr;
    pr.reserve(P);
    for (uint32_t i = 0; i < in.N; i++)
      for (uint32_t j = i + 1; j < in.N; j++) pr.push_back(make_uint2(i, j));
    uint2 *dpr = B.pairs.get(std::max<uint32_t>(P, 1));
    if (P) CK_EX(cudaMemcpyAsync(dpr, pr.data(), P * sizeof(uint2), cudaMemcpyHostToDevice, s));
    CK_EX(cudaStreamSynchronize(s));  // pr leaves scope
    n_init = P;
  }
  unsigned long long *cnt = B.counts.get(2);
  res.complete = 1;
  if (n_init == 0) {  // a single work-item has no pair
    pair_out->clear();
    res.n_states = 0;
    return res;
  }
  // level 0: the initial states, settled
  uint32_t *kids = B.kids.get(n_init * c.W);
  if (pair_out) {
    count_launch();
    ex_pairs_kernel<<<nb(n_init), 256, 0, s>>>(full, base, c, B.pairs.get(1), (uint32_t)n_init, kids);
  } else {
    CK_EX(cudaMemcpyAsync(kids, base, c.W * 4, cudaMemcpyDeviceToDevice, s));
  }
  uint32_t *ends = B.ends.get(n_init * c.E);
  CK_EX(cudaMemsetAsync(cnt, 0, 16, s));
  count_launch();
  ex_settle_kernel<<<nb(n_init), 256, 0, s>>>(c, kids, n_init, ends, cnt + 1);
  uint64_t nk = n_init, visited = 0, n_end_pool = 0;
  unsigned long long h[2];
  CK_EX(cudaMemcpyAsync(h, cnt, 16, cudaMemcpyDeviceToHost, s));
  CK_EX(cudaStreamSynchronize(s));
  uint64_t ne = std::min<uint64_t>(h[1], n_init);
  DevArray<uint32_t> endacc;  // the distinct end items so far
  for (;;) {
    // end items of this level join the pool (deduplicated as they come)
    if (ne) {
      uint32_t *acc = endacc.grow((n_end_pool + ne) * c.E, n_end_pool * c.E, s);
      CK_EX(cudaMemcpyAsync(acc + n_end_pool * c.E, ends, ne * c.E * 4, cudaMemcpyDeviceToDevice, s));
      uint32_t *tmpout = B.scratch.get((n_end_pool + ne) * c.E);
      n_end_pool = dedup(B, acc, n_end_pool + ne, c.E, false, tmpout, s);
      CK_EX(cudaMemcpyAsync(acc, tmpout, n_end_pool * c.E * 4, cudaMemcpyDeviceToDevice, s));
    }
    // the next level: distinct unfinished children
    uint32_t *front = B.front.get(std::max<uint64_t>(nk, 1) * c.W);
    const uint64_t n_front = dedup(B, kids, nk, c.W, true, front, s);
    visited += n_front;
    if (!n_front) break;
    if (visited > max_states) {
      res.complete = 0;
      break;
    }
    const uint64_t cap = n_front * c.K;
    if (cap * (c.W + c.E) * 4 > (uint64_t)8 << 30) {  // a level larger than 8 GiB of states: give up
      res.complete = 0;
      break;
    }
    kids = B.kids.get(cap * c.W);
    ends = B.ends.get(cap * c.E);
    CK_EX(cudaMemsetAsync(cnt, 0, 16, s));
    count_launch();
    ex_expand_kernel<<<nb(cap, 128), 128, 0, s>>>(c, front, (uint32_t)n_front, kids, cnt, ends, cnt + 1, cap);
    CK_EX(cudaMemcpyAsync(h, cnt, 16, cudaMemcpyDeviceToHost, s));
    CK_EX(cudaStreamSynchronize(s));
    nk = std::min<uint64_t>(h[0], cap);
    ne = std::min<uint64_t>(h[1], cap);
  }
  uint32_t fl = 0;
  CK_EX(cudaMemcpyAsync(&fl, full.flags, 4, cudaMemcpyDeviceToHost, s));
  if (pair_out) {  // per pair: distinct end memories | schedule-dependent read << 31
    uint32_t *pc = B.pcount.get(std::max<uint32_t>(P, 1));
    CK_EX(cudaMemsetAsync(pc, 0, P * 4, s));
    if (n_end_pool) {
      count_launch();
      ex_pair_count_kernel<<<nb(n_end_pool), 256, 0, s>>>(endacc.p, n_end_pool, c.E, in.N, pc);
    }
    std::vector<uint32_t> cntv(P), devv(P);
    CK_EX(cudaMemcpyAsync(cntv.data(), pc, P * 4, cudaMemcpyDeviceToHost, s));
    CK_EX(cudaMemcpyAsync(devv.data(), c.pair_dev, P * 4, cudaMemcpyDeviceToHost, s));
    CK_EX(cudaStreamSynchronize(s));
    pair_out->resize(P);
    for (uint32_t p = 0; p < P; p++) (*pair_out)[p] = cntv[p] | (devv[p] ? 0x80000000u : 0u);
  }
  CK_EX(cudaStreamSynchronize(s));
  res.n_end_states = (uint32_t)n_end_pool;
  res.deviated = (fl & 1u) ? 1 : 0;
  if (fl & 2u) res.complete = 0;
  res.n_states = visited;
  return res;
}

}  // namespace rc
