// Work-item interpreter: one CUDA thread per work-item, one CTA per
// work-group, one launch per barrier interval (or per range of groups), or
// one cooperative launch for every interval (resident runs).  The kernel
// body -- state set-up, stop points, counters, resident commits and
// compaction -- is interp_body (interp_kernel.cuh); this file supplies its
// bytecode-interpreting engine and the launchers.
#include "device.cuh"
#include "interp_kernel.cuh"
#include "classify_cell.cuh"

namespace rc {
namespace {

// Bytecode of the instance being checked when it fits (the warp fetches
// one instruction per step at a warp-uniform address: the constant cache's
// broadcast case).  Larger programs are read from global memory.
__constant__ uint4 c_code[kConstCodeInsns];

// Min-PC reconvergence: every iteration the warp executes the instruction
// at the smallest bytecode pc among its running lanes; lanes that are
// ahead (past a branch or a loop the others are still in) wait at their
// pc, so lanes that followed different paths meet again at the join point.
// The instruction is fetched and decoded once for the warp and every lane
// takes the same dispatch branch; only the side effects are predicated on
// the lane being at that pc.  Each warp appends to its own log slice: the
// ballot of the lanes that log in a step gives every lane its slot, and the
// slice fill level is a warp-uniform register (no atomics).
template <bool kConst, int kSnap>
struct InterpEngine {
  __device__ __forceinline__ uint32_t barrier_ordinal(const InterpArgs &A, uint32_t pc) const {
    return kConst ? c_code[pc].y : __ldg(reinterpret_cast<const uint4 *>(A.code) + pc).y;
  }

  __device__ __forceinline__ void run(const InterpArgs &A, IvState &s) const {
    const uint4 *__restrict__ code = reinterpret_cast<const uint4 *>(A.code);
    const uint32_t S = s.S, tid = s.tid, lanes = s.lanes, lane_lt = s.lane_lt;
    int32_t *const rf = s.rf;
#define REG(i) rf[(uint32_t)(i) * S + tid]
    for (;;) {
      const uint32_t minpc = __reduce_min_sync(lanes, s.running ? s.pc : kNone);
      if (minpc == kNone) break;
      const uint4 raw = kConst ? c_code[minpc] : __ldg(code + minpc);
      const bool act = s.running && s.pc == minpc;
      const uint32_t d = (raw.x >> 8) & 0xFFu, ra = (raw.x >> 16) & 0xFFu, rb = raw.x >> 24;
      const int32_t imm = (int32_t)raw.y;
      const uint32_t tgt = raw.z, ctl = raw.w;
      const uint32_t cls = (ctl >> CTL_CLASS_SHIFT) & 0xFu;
      const int32_t x = REG(ra);
      const int32_t yr = REG(rb);
      if (cls == CC_ALU) {  // arithmetic, moves, comparisons, branches
        // warp-uniform opcode; branch forms leave r != 0 when taken
        const int32_t r = sem_alu(raw.x & 0xFFu, x, yr, imm);
        if (act) {
          if (ctl & AL_WRITE) REG(d) = r;
          s.pc = sem_branch(ctl, r, imm) ? tgt : s.pc + 1;
        }
        continue;
      }
      if (cls == CC_LD || cls == CC_ST) {
        const uint32_t mem = ctl >> CTL_MEM_SHIFT;  // (LD/ST class: operand bits)
        const MemInfo m = s.mems[mem];
        const int32_t idx = sem_index(x, imm, (int32_t)tgt, ctl);
        const bool inb = (uint32_t)idx < m.len;
        // a private access (warp-uniform: one instruction) is counted but not logged
        const bool priv = (ctl & CTL_PRIV) != 0;
        const uint32_t performing = __ballot_sync(lanes, act && inb);
        const uint32_t logging = priv ? 0u : performing;
        const uint32_t slot_pos = s.wfill + __popc(logging & lane_lt);
        s.wfill += __popc(logging);
        if (!act) continue;
        s.pc++;
        if (!inb) {  // ⊥: out of bounds, the work-item stops
          out_of_bounds(A, s, m, mem, idx);
          s.st = TS_DEAD;
          s.running = false;
          continue;
        }
        // the lanes still here are exactly those in `performing`
        const int32_t v = shared_access<kSnap>(A, s, m, performing, cell_of(s, m, idx), cls == CC_ST, priv, yr,
                                               slot_pos);
        if (cls == CC_LD) REG(d) = v;
        continue;
      }
      if (!act) continue;
      s.pc++;
      switch (cls) {
        case CC_DIVMOD:
          REG(d) = sem_divmod(ctl, x, yr, imm);
          break;
        case CC_LOGIC:  // (x != 0) and / or (yr != 0)
          REG(d) = sem_logic(ctl, x, yr);
          break;
        case CC_SIZE:
          REG(d) = (int32_t)s.mems[ctl >> CTL_MEM_SHIFT].len;
          break;
        case CC_ASSUME:
          if (x == 0) {  // ⊤: no continuation
            s.st = TS_DEAD;
            s.running = false;
          }
          break;
        case CC_ASSERT:
          if (x == 0) {  // ⊥
            OutRec e{s.interval, 0, 0, 0, CLS_ASSERT, s.gtid, (uint32_t)imm, 0, 0, 0};
            append_err(A, e, s.flags);
            s.st = TS_DEAD;
            s.running = false;
          }
          break;
        case CC_BARRIER:
          s.st = TS_BARRIER;
          s.pc -= 1;  // remember the barrier itself
          s.running = false;
          break;
        default:  // CC_EXIT
          s.st = TS_EXIT;
          s.pc -= 1;
          s.running = false;
          break;
      }
    }
#undef REG
  }
};

template <bool kConst, bool kResident>
__global__ void __launch_bounds__(1024, 2) interp_kernel(InterpArgs A) {
  interp_body<kResident>(A, InterpEngine<kConst, kResident ? kSnapLdcg : kSnapLdg>{});
}

// Diagnostic: every CTA waits at a grid barrier that expects one more
// arrival than the launch has, so each wait must run out after limit_ns and
// report it in bar[2] (the status the host reads), leaving the context usable.
__global__ void grid_barrier_probe_kernel(unsigned *bar, unsigned long long limit_ns) {
  grid_sync(bar, gridDim.x + 1, limit_ns);
}

__global__ void interval_gate_kernel(const uint32_t *flags, const uint32_t *stop_cnt, uint32_t n_barriers,
                                     uint32_t *proceed) {
  uint32_t n_points = 0;
  bool any_barrier = false;
  for (uint32_t k = 0; k <= n_barriers; k++) {
    if (!stop_cnt[k]) continue;
    n_points++;
    if (k < n_barriers) any_barrier = true;
  }
  *proceed = (*flags == 0 && n_points == 1 && any_barrier) ? 1u : 0u;
}


// ---- one-CTA check of small instances
//
// Every work-item of a small instance (groups x group size <= 1024) in one
// CTA, every interval in one launch: the interpreter runs the interval (the
// same engine and access step as interp_kernel, owner table off), then the
// CTA classifies the interval itself -- its records gathered from the warp
// slices, sorted in shared memory by (cell, work-item), reduced to one
// Summary per (cell, work-item) and classified cell by cell by
// classify_cell, the sort path's rules -- commits each cell's value, writes
// the race records in report order, and applies the barrier-release rule to
// decide on the next interval.  The host makes one launch per check instead
// of a few dozen launches and synchronisations.

// block-wide exclusive scan of one value per thread (blockDim.x <= 1024);
// *total receives the sum (every thread)
__device__ __forceinline__ uint32_t cta_excl_scan(uint32_t v, uint32_t *sh, uint32_t &total) {
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5, nw = (blockDim.x + 31u) >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  __syncthreads();
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t q = lane < nw ? sh[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, q, o);
      if (lane >= (uint32_t)o) q += y;
    }
    if (lane < nw) sh[lane] = q;  // inclusive over warps
  }
  __syncthreads();
  total = sh[nw - 1];
  const uint32_t r = (w ? sh[w - 1] : 0u) + x - v;
  __syncthreads();
  return r;
}

// The warp whose log slice holds record i of the interval, the slices laid
// end to end (woff: each warp's first record; a warp without records has
// the next one's offset, so the largest w with woff[w] <= i is the holder).
__device__ __forceinline__ uint32_t slice_of(const uint32_t *woff, uint32_t nw, uint32_t i) {
  uint32_t lo = 0, hi = nw;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (woff[mid] <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <bool kConst>
__global__ void __launch_bounds__(1024, 1) small_check_kernel(SmallArgs P) {
  const InterpArgs &A = P.A;
  extern __shared__ __align__(16) unsigned char smem[];
  // T threads sort and classify; the first RS (the work-items, rounded up to
  // whole warps) also run the work-items: registers and own-write slots have
  // stride RS
  const uint32_t T = blockDim.x, t = threadIdx.x, N = P.n_items, S = A.S, RS = P.reg_stride;
  MemInfo *mems = reinterpret_cast<MemInfo *>(smem);
  int32_t *rf = reinterpret_cast<int32_t *>(mems + A.n_mems);           // [n_regs][RS]
  uint32_t *owk = reinterpret_cast<uint32_t *>(rf + A.n_regs * RS);      // [ow_slots][RS]
  int32_t *owv = reinterpret_cast<int32_t *>(owk + A.ow_slots * RS);     // [ow_slots][RS]
  // the snapshot in shared memory when it fits (reads then wait on no
  // global-memory latency), copied back to global memory at the end
  int32_t *ssnap = reinterpret_cast<int32_t *>((reinterpret_cast<uintptr_t>(owv + A.ow_slots * RS) + 15) &
                                               ~(uintptr_t)15);
  int32_t *snapp = P.smem_snap ? ssnap : A.commit;
  unsigned long long *keys = reinterpret_cast<unsigned long long *>(
      (reinterpret_cast<uintptr_t>(ssnap + (P.smem_snap ? P.n_cells : 0)) + 15) & ~(uintptr_t)15);  // [pow2 >= cap]
  uint32_t p2k = 1024;
  while (p2k < P.cap) p2k <<= 1;
  // the log's warp slices in shared memory after the keys when they fit
  uint4 *logp = P.smem_log ? reinterpret_cast<uint4 *>(keys + p2k) : reinterpret_cast<uint4 *>(A.log);
  // the sorted records and their summaries: after the keys in shared
  // memory when they fit, else in global memory
  LogRec *sorted = P.sorted;
  Summary *sum = P.sum;
  unsigned char *tail = P.smem_log ? reinterpret_cast<unsigned char *>(logp + (size_t)RS * (A.warp_slice / 32))
                                    : reinterpret_cast<unsigned char *>(keys + p2k);
  if (P.smem_scratch) {
    sorted = reinterpret_cast<LogRec *>(tail);
    sum = reinterpret_cast<Summary *>(sorted + P.cap);
    tail = reinterpret_cast<unsigned char *>(sum + P.cap);
  }
  uint32_t *cbin = reinterpret_cast<uint32_t *>(tail);  // [bins]: counting sort over (cell, work-item)
  __shared__ uint32_t s_stop_min[kSmallMaxStops], s_stop_cnt[kSmallMaxStops];
  __shared__ uint32_t s_fill[32], s_woff[32], s_scan[32];
  __shared__ unsigned long long s_acc[3];
  __shared__ uint32_t s_go, s_flags, s_nout, s_nsum;
  for (uint32_t k = t; k < A.n_mems; k += T) mems[k] = A.mems[k];
  if (P.smem_snap)
    for (uint32_t k = t; k < P.n_cells; k += T) ssnap[k] = A.snap[k];
  const bool item = t < N;
  const uint32_t wg = item ? t / S : 0u, tid = item ? t % S : 0u;
  if (item) {
    for (uint32_t r = kBuiltinRegs; r < A.n_regs; r++) rf[r * RS + t] = 0;
    rf[REG_TID * RS + t] = (int32_t)tid;
    rf[REG_WG * RS + t] = (int32_t)wg;
    rf[REG_GTID * RS + t] = (int32_t)t;
    rf[REG_GSIZE * RS + t] = (int32_t)S;
    rf[REG_NGROUPS * RS + t] = (int32_t)A.G;
  }
  if (t == 0) {
    s_acc[0] = s_acc[1] = s_acc[2] = 0;
    s_flags = 0;
    s_nout = 0;
  }
  uint32_t st = item ? (uint32_t)TS_RUN : (uint32_t)TS_DEAD, pc = 0;
  const uint32_t nstops = A.n_barriers + 1, warp = t >> 5, nwarps = (T + 31u) >> 5;
  const InterpEngine<kConst, kSnapPlain> E{};
  uint32_t interval = 0;
  for (;; interval++) {
    for (uint32_t k = t; k < nstops; k += T) {
      s_stop_min[k] = kNone;
      s_stop_cnt[k] = 0;
    }
    __syncthreads();
    const bool ran = st == TS_RUN;
    IvState s;
    s.snap = snapp;
    s.mems = mems;
    s.rf = rf;
    s.owk = owk;
    s.owv = owv;
    s.flags = &s_flags;
    s.wlog = logp + (uint64_t)warp * A.warp_slice;
    s.S = RS;  // register and own-write slot stride
    s.tid = t;
    s.gtid = t;
    s.wg = wg;
    s.lt = t;
    s.slots = A.ow_slots;
    s.lbase = A.GT + wg * A.LT;
    s.lanes = 0xFFFFFFFFu;
    s.lane_lt = (1u << (t & 31u)) - 1u;
    s.warp = warp;
    s.interval = interval;
    s.tag = 0;
    s.st = st;
    s.pc = pc;
    s.nloc = s.seq = s.nw = s.wfill = 0;
    s.bloom = 0;
    s.running = ran;
    E.run(A, s);
    st = s.st;
    pc = s.pc;
    // counters and stop points
    {
      const uint32_t sg = __reduce_add_sync(0xFFFFFFFFu, s.seq - s.nloc), sl = __reduce_add_sync(0xFFFFFFFFu, s.nloc);
      if ((t & 31u) == 0) {
        s_fill[warp] = s.wfill < A.warp_slice ? s.wfill : (uint32_t)A.warp_slice;
        if (sg) atomicAdd(&s_acc[0], (unsigned long long)sg);
        if (sl) atomicAdd(&s_acc[1], (unsigned long long)sl);
        if (s.wfill) atomicAdd(&s_acc[2], (unsigned long long)s.wfill);
      }
      if (st == TS_BARRIER || (st == TS_EXIT && ran)) {
        const uint32_t stop = st == TS_BARRIER ? E.barrier_ordinal(A, pc) : A.n_barriers;
        atomicMin(&s_stop_min[stop], t);
        atomicAdd(&s_stop_cnt[stop], 1u);
      }
    }
    __syncthreads();
    // ---- gather the interval's records: warp offsets, keys (cell, work-item, position)
    uint32_t M = 0;
    {
      if (t < 32) {
        const uint32_t v = t < nwarps ? s_fill[t] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
          if (t >= (uint32_t)o) x += y;
        }
        s_woff[t] = x - v;
        if (t == 31) s_scan[0] = x;
      }
      __syncthreads();
      M = s_scan[0];
      __syncthreads();
    }
    if (M > P.cap) {  // more records than the CTA sorts: the host checks the instance another way
      if (t == 0) s_flags |= FLAG_ACC_FULL;
      break;
    }
    if (P.bins) {
      // counting sort over (cell, work-item): one counter per pair in
      // shared memory; a record's position is its pair's offset plus its
      // rank among the pair's records (in atomic order: the summary takes a
      // work-item's last write by sequence number, not by position)
      for (uint32_t i = t; i < P.bins; i += T) cbin[i] = 0;
      __syncthreads();
      // every thread takes records of the interval (the slices of the few
      // warps that ran work-items, end to end), not only those warps
      for (uint32_t i = t; i < M; i += T) {
        const uint32_t w = slice_of(s_woff, nwarps, i);
        const uint4 r = logp[(uint64_t)w * A.warp_slice + (i - s_woff[w])];
        atomicAdd(&cbin[r.x * RS + (r.y & 0x7FFFFFFFu)], 1u);
      }
      __syncthreads();
      {
        const uint32_t per_b = (P.bins + T - 1) / T, blo = min(t * per_b, P.bins), bhi = min(blo + per_b, P.bins);
        uint32_t part = 0;
        for (uint32_t i = blo; i < bhi; i++) part += cbin[i];
        uint32_t tot = 0;
        uint32_t run = cta_excl_scan(part, s_scan, tot);
        for (uint32_t i = blo; i < bhi; i++) {
          const uint32_t c = cbin[i];
          cbin[i] = run;
          run += c;
        }
      }
      __syncthreads();
      for (uint32_t i = t; i < M; i += T) {
        const uint32_t w = slice_of(s_woff, nwarps, i);
        const uint4 r = logp[(uint64_t)w * A.warp_slice + (i - s_woff[w])];
        reinterpret_cast<uint4 *>(sorted)[atomicAdd(&cbin[r.x * RS + (r.y & 0x7FFFFFFFu)], 1u)] = r;
      }
      __syncthreads();
    } else {
      uint32_t P2 = T;  // sort length: a power of two, at least one key per thread
      while (P2 < M) P2 <<= 1;
      {  // key: cell (32 bits), work-item (10), warp (5), slot in the warp's slice (12)
        for (uint32_t i = t; i < M; i += T) {
          const uint32_t w = slice_of(s_woff, nwarps, i), j = i - s_woff[w];
          const uint4 r = logp[(uint64_t)w * A.warp_slice + j];
          keys[i] = ((unsigned long long)r.x << 27) | ((unsigned long long)(r.y & 0x3FFu) << 17) |
                    ((unsigned long long)w << 12) | j;
        }
        for (uint32_t j = M + t; j < P2; j += T) keys[j] = ~0ull;
      }
      __syncthreads();
      {  // bitonic sort (the keys are distinct): thread t holds keys t + q T in
         // registers; partners within a warp (distance < 32) by shuffles, the
         // others through shared memory
        const uint32_t Q = P2 / T;
        unsigned long long kq[kSmallCap / 1024];
  #pragma unroll
        for (uint32_t q = 0; q < kSmallCap / 1024; q++)
          if (q < Q) kq[q] = keys[t + q * T];
        for (uint32_t k = 2; k <= P2; k <<= 1)
          for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
  #pragma unroll
              for (uint32_t q = 0; q < kSmallCap / 1024; q++)
                if (q < Q) keys[t + q * T] = kq[q];
              __syncthreads();
  #pragma unroll
              for (uint32_t q = 0; q < kSmallCap / 1024; q++)
                if (q < Q) {
                  const uint32_t i = t + q * T;
                  const unsigned long long b = keys[i ^ j], a = kq[q];
                  kq[q] = (((i & j) == 0) == ((i & k) == 0)) ? min(a, b) : max(a, b);
                }
              __syncthreads();
            } else {
  #pragma unroll
              for (uint32_t q = 0; q < kSmallCap / 1024; q++)
                if (q < Q) {
                  const uint32_t i = t + q * T;
                  const unsigned long long b = __shfl_xor_sync(0xFFFFFFFFu, kq[q], (int)j), a = kq[q];
                  kq[q] = (((i & j) == 0) == ((i & k) == 0)) ? min(a, b) : max(a, b);
                }
            }
          }
  #pragma unroll
        for (uint32_t q = 0; q < kSmallCap / 1024; q++)
          if (q < Q) keys[t + q * T] = kq[q];
        __syncthreads();
      }
      // the sorted records
      for (uint32_t i = t; i < M; i += T) {
        const unsigned long long k = keys[i];
        sorted[i] = reinterpret_cast<const LogRec *>(logp)[(uint64_t)((k >> 12) & 31u) * A.warp_slice + (k & 0xFFFu)];
      }
      __syncthreads();
    }
    // one Summary per (cell, work-item) run of the sorted records
    const uint32_t per = (M + T - 1) / T, lo = min(t * per, M), hi = min(lo + per, M);
    uint32_t nh = 0;
    auto run_head = [&](uint32_t i) {
      return i == 0 || sorted[i].key != sorted[i - 1].key || ((sorted[i].tw ^ sorted[i - 1].tw) & 0x7FFFFFFFu) != 0;
    };
    for (uint32_t i = lo; i < hi; i++) nh += run_head(i) ? 1u : 0u;
    uint32_t nsum = 0;
    uint32_t ridx = cta_excl_scan(nh, s_scan, nsum);
    for (uint32_t i = lo; i < hi; i++) {
      if (!run_head(i)) continue;
      uint64_t end = 0;
      sum[ridx++] = summarize_run(sorted, i, M, end);
    }
    __syncthreads();
    // cells: classify, commit, count records; then emit in cell order
    ClassifyArgs ca{interval, A.GT, A.LT ? A.LT : 1u, nullptr};
    const uint32_t per2 = (nsum + T - 1) / T, lo2 = min(t * per2, nsum), hi2 = min(lo2 + per2, nsum);
    uint32_t nrec = 0;
    CellResult c1{};  // with one summary per thread, its cell's result waits here for the emit
    for (uint32_t k = lo2; k < hi2; k++) {
      if (k != 0 && sum[k].key == sum[k - 1].key) continue;
      const CellResult c = classify_cell(sum, k, nsum);
      if (c.wrote) snapp[sum[k].key] = c.commit;
      nrec += (c.ww_cls ? 1u : 0u) + (c.rw_a != kNone ? 1u : 0u);
      c1 = c;
    }
    uint32_t total = 0;
    uint32_t roff = cta_excl_scan(nrec, s_scan, total);
    const uint32_t base = s_nout;
    if (base + total > P.out_cap) {
      if (t == 0) s_flags |= FLAG_ACC_FULL;
      break;
    }
    for (uint32_t k = lo2; k < hi2 && nrec; k++) {
      if (k != 0 && sum[k].key == sum[k - 1].key) continue;
      const CellResult c = per2 == 1 ? c1 : classify_cell(sum, k, nsum);
      const uint32_t n = (c.ww_cls ? 1u : 0u) + (c.rw_a != kNone ? 1u : 0u);
      if (n) emit_cell(ca, sum[k].key, c, base + roff, P.out);
      roff += n;
    }
    __syncthreads();
    // ---- barrier agreement (the barrier-release rule of Sec. 4)
    if (t == 0) {
      s_nout = base + total;
      uint32_t points = 0;
      bool any_barrier = false;
      for (uint32_t k = 0; k < nstops; k++)
        if (s_stop_cnt[k]) {
          points++;
          any_barrier |= k < A.n_barriers;
        }
      if (points >= 2)
        for (uint32_t k = 0; k < nstops; k++)
          if (s_stop_cnt[k])
            append_err(A, OutRec{interval, 0, 0, 0, CLS_DIVERGENCE, s_stop_min[k], k < A.n_barriers ? k : kNone, 0,
                                 0, s_stop_cnt[k]}, &s_flags);
      if (points == 1 && any_barrier && interval + 1 >= P.max_intervals) s_flags |= FLAG_ACC_FULL;
      s_go = points == 1 && any_barrier && s_flags == 0;
    }
    __syncthreads();
    if (!s_go) break;
    if (st == TS_BARRIER) {
      st = TS_RUN;
      pc += 1;
    }
  }
  __syncthreads();
  if (P.smem_snap)  // the final memory
    for (uint32_t k = t; k < P.n_cells; k += T) A.commit[k] = ssnap[k];
  // results into page-locked host memory (one synchronisation for the host)
  const uint32_t nerr = min(*(volatile uint32_t *)A.err_count, A.err_cap), nout = s_nout;
  if (t == 0) {
    P.res[0] = s_acc[0];
    P.res[1] = s_acc[1];
    P.res[2] = s_acc[2];
    P.res[3] = (unsigned long long)(interval + 1) | ((unsigned long long)s_flags << 32);
    P.res[4] = nout;
    P.res[5] = nerr;
  }
  for (uint32_t i = t; i < nout; i += T) P.host_out[i] = P.out[i];
  for (uint32_t i = t; i < nerr; i += T) P.host_err[i] = A.errs[i];
}

}  // namespace

void launch_interval_gate(const uint32_t *flags, const uint32_t *stop_cnt, uint32_t n_barriers, uint32_t *proceed,
                          cudaStream_t s) {
  count_launch();
  interval_gate_kernel<<<1, 1, 0, s>>>(flags, stop_cnt, n_barriers, proceed);
}

size_t interp_smem_bytes(uint32_t n_mems, uint32_t n_regs, uint32_t S, uint32_t ow_slots) {
  return (size_t)n_mems * sizeof(MemInfo) + (size_t)n_regs * S * 4 + (size_t)ow_slots * S * 8;
}

size_t g_interp_static_smem = 0;

cudaError_t interp_configure() {
  const void *fns[4] = {(const void *)interp_kernel<true, false>, (const void *)interp_kernel<false, false>,
                        (const void *)interp_kernel<true, true>, (const void *)interp_kernel<false, true>};
  size_t st = 0;
  for (const void *f : fns) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    st = fa.sharedSizeBytes > st ? fa.sharedSizeBytes : st;
  }
  g_interp_static_smem = st;
  const int dyn = (int)(kMaxSmemPerBlock - g_interp_static_smem);
  for (const void *f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int interp_resident_blocks_per_sm(uint32_t n_insn, uint32_t S, size_t smem) {
  int nb = 0;
  const void *f = n_insn <= kConstCodeInsns ? (const void *)interp_kernel<true, true>
                                             : (const void *)interp_kernel<false, true>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, (int)S, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

cudaError_t launch_grid_barrier_probe(unsigned *bar, uint32_t n_blocks, unsigned long long limit_ns,
                                      cudaStream_t s) {
  count_launch();
  void *params[] = {&bar, &limit_ns};
  return cudaLaunchCooperativeKernel((const void *)grid_barrier_probe_kernel, dim3(n_blocks), dim3(64), params, 0,
                                     s);
}

cudaError_t launch_interp_resident(const InterpArgs &a, uint32_t n_groups, size_t smem, cudaStream_t s) {
  count_launch();
  InterpArgs arg = a;
  void *params[] = {&arg};
  const void *f = a.n_insn <= kConstCodeInsns ? (const void *)interp_kernel<true, true>
                                               : (const void *)interp_kernel<false, true>;
  return cudaLaunchCooperativeKernel(f, dim3(n_groups), dim3(a.S), params, smem, s);
}

size_t interp_max_dynamic_smem() { return kMaxSmemPerBlock - g_interp_static_smem; }

cudaError_t interp_upload_code(const Insn *host_code, uint32_t n_insn, cudaStream_t s) {
  if (n_insn > kConstCodeInsns) return cudaSuccess;
  return cudaMemcpyToSymbolAsync(c_code, host_code, (size_t)n_insn * sizeof(Insn), 0, cudaMemcpyHostToDevice, s);
}

void launch_interp(const InterpArgs &a, uint32_t n_groups, size_t smem, cudaStream_t s) {
  count_launch();
  if (a.n_insn <= kConstCodeInsns) interp_kernel<true, false><<<n_groups, a.S, smem, s>>>(a);
  else interp_kernel<false, false><<<n_groups, a.S, smem, s>>>(a);
}


size_t small_check_smem(uint32_t n_mems, uint32_t n_regs, uint32_t T, uint32_t ow_slots, uint32_t cap,
                        uint32_t snap_cells) {
  uint32_t p2 = 1024;  // the sort covers at least one key per thread of the 1024-thread CTA
  while (p2 < cap) p2 <<= 1;
  return (size_t)n_mems * sizeof(MemInfo) + (size_t)n_regs * T * 4 + (size_t)ow_slots * T * 8 + 16 +
         (size_t)snap_cells * 4 + 16 + (size_t)p2 * 8;
}

cudaError_t launch_small_check(const SmallArgs &a, uint32_t threads, size_t smem, cudaStream_t s) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(small_check_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kMaxSmemPerBlock - 4096));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(small_check_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(kMaxSmemPerBlock - 4096));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  count_launch();
  if (a.A.n_insn <= kConstCodeInsns) small_check_kernel<true><<<1, threads, smem, s>>>(a);
  else small_check_kernel<false><<<1, threads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace rc
