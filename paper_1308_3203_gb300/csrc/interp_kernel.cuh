// The body of the per-interval work-item kernel, shared by its two engines:
// the bytecode interpreter (interp.cu) and compiled intervals (a program's
// bytecode translated to straight-line code and compiled at run time, see
// jit.cu).  One CUDA thread per work-item, one CTA per work-group.
//
// Semantics (Distefano & Dubreil, Sec. 4, thread-local rules): each command
// updates the private stack (registers) or makes one shared access; assert
// false is an error (⊥), assume false ends the path (⊤), barrier suspends
// the work-item.  An access outside 0 <= index < size(a) is an error (Sec. 5,
// Table 1 bounds premise); the work-item stops and an OOB record is written.
//
// Shared reads see the work-item's own latest write to the cell in this
// interval if there is one, else the value committed at the last barrier
// (delayed visibility); shared writes go to the work-item's own-write table.
// Every access is counted and, unless the pre-filter proved it private (no
// other work-item touches its cells in the interval: CTL_PRIV), appended to
// its warp's slice of the interval's log as a 16-byte record.
//
// Resident runs: when every work-group of the instance fits on the GPU at
// once, one cooperative launch runs all intervals.  Registers stay in shared
// memory from one interval to the next; at each interval's end a bounded
// grid-wide barrier separates the interpretation from the commit (each
// work-item stores its last write to every cell whose highest writer it is,
// per the owner table: the value the sort path commits) and the compaction
// of the records that need the exact sort (appended for classification after
// the run), and a second barrier separates those from the next interval.
// Every CTA then reads the interval's stop points and flags and takes the
// same decision to go on or stop.
//
// An engine is a type with
//   __device__ void run(const InterpArgs &A, IvState &s) const
//     runs the work-item from s.pc until it stops (barrier, exit, abort);
//     s.running is true on entry for the work-items that run.  Every lane
//     of the work-group's warps calls it; on return s.st is the new status,
//     with s.pc at the barrier or exit instruction where it stopped, and
//     s.wfill is the warp's log fill level (warp-uniform).
//   __device__ uint32_t barrier_ordinal(const InterpArgs &A, uint32_t pc) const
//     the ordinal of the barrier instruction at pc.
// Accesses go through shared_access below, so both engines log, claim and
// read the same way.
#pragma once
#ifndef __CUDACC_RTC__
#include <cstdint>
#endif

#include "kernel_types.cuh"
#include "semantics.cuh"

namespace rc {

__device__ __forceinline__ uint64_t bloom_bit(uint32_t key) {
  return 1ull << ((key * 2654435761u) >> 26);
}

__device__ __forceinline__ void append_err(const InterpArgs &A, const OutRec &r, uint32_t *flags) {
  uint32_t pos = atomicAdd(A.err_count, 1u);
  if (pos < A.err_cap) A.errs[pos] = r;
  else atomicOr(flags, FLAG_ERR_FULL);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch (every CTA resident, so the
// wait ends unless a CTA left early).  Arrival is two-level: CTA b counts
// into sub-counter b mod 32 (each on its own 128-byte line), and the last
// arriver of each sub-counter into the top counter, so no single address
// takes more than 32 atomics (measured: 3.8 us per barrier for 1024 CTAs,
// 5.0 us with one counter).  After the CTA barrier thread 0 fences, arrives
// and waits for the generation to move, at most limit_ns of wall-clock time
// (resident runs: 20 s; an interval's work is bounded by the host's choice
// of resident runs, see run_resident); a CTA that gives up (or sees another
// give up) sets bar[2] and the call returns false, and the kernel then ends.
// bar (kGridBarWords, zero before the launch): [0] top arrivals, [1]
// generation, [2] timed out, [32 + 32 s] sub-counter s.
static __device__ __noinline__ bool grid_sync(unsigned *bar, unsigned nblocks, unsigned long long limit_ns) {
  __shared__ uint32_t s_ok;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = bar + 1;
    const unsigned g = *gen;
    uint32_t ok = 1;
    const unsigned sub = blockIdx.x & 31u;
    const unsigned n_sub = (nblocks - sub + 31u) / 32u;  // CTAs counting into this sub-counter
    unsigned *sc = bar + 32 + 32 * sub;
    bool release = false;
    if (atomicAdd(sc, 1u) == n_sub - 1) {  // the last of its sub-counter: reset it, arrive at the top
      atomicExch(sc, 0u);
      __threadfence();
      release = atomicAdd(bar, 1u) == (nblocks < 32u ? nblocks : 32u) - 1;
    }
    if (release) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*gen == g) {
        if (*(volatile unsigned *)(bar + 2) || global_ns() - t0 > limit_ns) {
          atomicExch(bar + 2, 1u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// How the access step reads committed values: read-only through the
// non-coherent cache (the snapshot does not change during an interval
// launch), through L2 (resident runs commit in-kernel), or plainly (a
// snapshot in shared memory).
enum SnapRead : int { kSnapLdg = 0, kSnapLdcg = 1, kSnapPlain = 2 };

// One work-item's state in one barrier interval, advanced by an engine.
struct IvState {
  const int32_t *snap;    // committed memory, indexed by cell
  const MemInfo *mems;    // the memory table (shared memory)
  int32_t *rf;            // registers [n_regs][S] (shared memory)
  uint32_t *owk;          // own-write slots in shared memory: keys [slots][S]
  int32_t *owv;           //   and values
  uint32_t *flags;        // this interval's flag word
  uint4 *wlog;            // the warp's log slice
  uint32_t S, tid, gtid, wg, lt, slots, lbase, lanes, lane_lt, warp, interval, tag;
  uint32_t st, pc;        // status and program counter
  uint32_t nloc, seq, nw; // local accesses, accesses, own-write entries this interval
  uint32_t wfill;         // records in the warp's slice (warp-uniform)
  uint64_t bloom;         // cells in the own-write table
  bool running;
};

// An out-of-bounds access (⊥): the OOB record; the caller stops the work-item.
__device__ __forceinline__ void out_of_bounds(const InterpArgs &A, const IvState &s, const MemInfo &m, uint32_t mem,
                                              int32_t idx) {
  OutRec e{s.interval, m.space, m.space ? s.wg : 0u, (uint32_t)idx, CLS_OOB, s.gtid, mem, 0, 0, 0};
  append_err(A, e, s.flags);
}

// One in-bounds shared access by this lane: `performing` = the lanes of the
// warp making an in-bounds access at this step (this one among them), key =
// its cell, v = the value stored (stores).  Claims the cell, looks the cell
// up in the own-write table (reads see the own latest write, else the
// committed value; writes update or add the entry), writes the log record
// at slot_pos unless the access is private, counts it.  Returns the value
// read or written.
template <int kSnap>
__device__ __forceinline__ int32_t shared_access(const InterpArgs &A, IvState &s, const MemInfo &m, uint32_t performing,
                                                 uint32_t key, bool store, bool priv, int32_t v, uint32_t slot_pos) {
  const uint32_t S = s.S, tid = s.tid, slots = s.slots, lt = s.lt;
  // a read's committed value is requested first, so that its latency
  // overlaps the claims and the own-write lookup (unused when the work-item
  // reads back its own write)
  int32_t committed = 0;
  if (!store)
    committed = kSnap == kSnapLdcg ? __ldcg(s.snap + key) : kSnap == kSnapLdg ? __ldg(s.snap + key) : s.snap[key];
  // a private access is counted but not logged, and only its stores claim
  // their cells (for the commit)
  if (A.owner && !(priv && !store)) shadow_claim_warp(A.owner, performing, key, store, s.tag, s.gtid, tid & 31u);
  // own-write table: the first `slots` distinct cells in shared memory, the rest in global
  const uint64_t bit = bloom_bit(key);
  int32_t slot = -1;
  if (s.bloom & bit) {
    const uint32_t ns = s.nw < slots ? s.nw : slots;
    for (uint32_t k = 0; k < ns; k++)
      if (s.owk[k * S + tid] == key) { slot = (int32_t)k; break; }
    if (slot < 0)
      for (uint32_t k = slots; k < s.nw; k++)
        if (A.ow[(uint64_t)k * A.ow_stride + lt].x == key) { slot = (int32_t)k; break; }
  }
  if (!store) {
    if (slot < 0) v = committed;
    else if ((uint32_t)slot < slots) v = s.owv[slot * S + tid];
    else v = (int32_t)A.ow[(uint64_t)slot * A.ow_stride + lt].y;
  } else {
    if (slot >= 0) {
      if ((uint32_t)slot < slots) s.owv[slot * S + tid] = v;
      else A.ow[(uint64_t)slot * A.ow_stride + lt].y = (uint32_t)v;
    } else if (s.nw < slots) {
      s.owk[s.nw * S + tid] = key;
      s.owv[s.nw * S + tid] = v;
      s.nw++;
      s.bloom |= bit;
    } else if (s.nw < A.capw) {
      A.ow[(uint64_t)s.nw * A.ow_stride + lt] = make_uint2(key, (uint32_t)v);
      s.nw++;
      s.bloom |= bit;
    } else {
      atomicOr(s.flags, FLAG_OW_FULL);
    }
  }
  if (!priv) {
    if (slot_pos < A.warp_slice)  // always true: the slice holds the static per-interval bound
      s.wlog[slot_pos] = make_uint4(key, s.gtid | (store ? 0x80000000u : 0u), (uint32_t)v, s.seq);
    else
      atomicOr(s.flags, FLAG_LOG_FULL);
  }
  s.seq++;
  s.nloc += m.space;
  return v;
}

// The cell of index idx of a memory object, for this work-item.
__device__ __forceinline__ uint32_t cell_of(const IvState &s, const MemInfo &m, int32_t idx) {
  return (m.space ? s.lbase : 0u) + m.base + (uint32_t)idx;
}

template <bool kResident, class Engine>
__device__ __forceinline__ void interp_body(const InterpArgs &A, const Engine &E) {
  if (!kResident && A.proceed && *A.proceed == 0) return;  // a closed gate: the host runs this interval later
  extern __shared__ __align__(16) unsigned char smem[];
  // Within an interval the work-items of a group do not interact (a read
  // sees the snapshot and the work-item's own writes), so a group may run as
  // `split` CTAs of consecutive work-items: T threads each, the register file
  // and own-write slots in shared memory with stride T.  Resident runs and
  // work-group-scoped barriers keep one CTA per group.
  const uint32_t T = blockDim.x, t = threadIdx.x;
  MemInfo *mems = reinterpret_cast<MemInfo *>(smem);
  int32_t *rf = reinterpret_cast<int32_t *>(mems + A.n_mems);  // [n_regs][T]
  uint32_t *owk = reinterpret_cast<uint32_t *>(rf + A.n_regs * T);  // [ow_slots][T] keys
  int32_t *owv = reinterpret_cast<int32_t *>(owk + A.ow_slots * T);  // [ow_slots][T] values

  const uint32_t S = A.S;
  const uint32_t split = kResident || A.split < 2 ? 1u : A.split;
  for (uint32_t k = t; k < A.n_mems; k += T) mems[k] = A.mems[k];

  const uint32_t wg = A.group0 + blockIdx.x / split;
  const uint32_t tid = (blockIdx.x % split) * T + t;  // the work-item's id in its group
  const uint32_t gtid = wg * S + tid;
  const uint64_t N = (uint64_t)A.G * S;
  const uint32_t lt = gtid - A.group0 * S;  // index in this launch's own-write table
  const uint32_t slots = A.ow_slots;
  // a resident run starts every work-item afresh (pc 0, registers 0); an
  // interval launch resumes the state the previous one saved
  uint32_t st = kResident ? (uint32_t)TS_RUN : A.st[gtid];
  uint32_t pc = kResident ? 0u : A.pc[gtid];
  if (st == TS_BARRIER) {  // resume after the barrier it waited at
    st = TS_RUN;
    pc += 1;
  }
  if (st == TS_RUN) {
    for (uint32_t r = kBuiltinRegs; r < A.n_regs; r++)
      rf[r * T + t] = kResident ? 0 : A.regs[(uint64_t)r * N + gtid];
    rf[REG_TID * T + t] = (int32_t)tid;
    rf[REG_WG * T + t] = (int32_t)wg;
    rf[REG_GTID * T + t] = (int32_t)gtid;
    rf[REG_GSIZE * T + t] = (int32_t)S;
    rf[REG_NGROUPS * T + t] = (int32_t)A.G;
  }
  // resident: the current interval and owner-table tag live in shared
  // memory (CTA-uniform), which keeps the interpreter's registers free
  __shared__ uint32_t s_iv[2];
  if (kResident && t == 0) {
    s_iv[0] = A.interval;
    s_iv[1] = A.tag;
  }
  __syncthreads();

  const uint32_t wbase = t & ~31u;
  const uint32_t lanes = T - wbase >= 32 ? 0xFFFFFFFFu : ((1u << (T - wbase)) - 1u);
  const uint32_t nstops = A.n_barriers + 1;
  const uint32_t warp = t >> 5;
  for (;;) {  // resident: one pass per barrier interval; otherwise a single pass
  const uint32_t interval = kResident ? s_iv[0] : A.interval;
  // resident runs raise an interval's flags in the word of its parity, so a
  // CTA still deciding on interval k never sees a flag of interval k + 1
  uint32_t *const flags = A.flags + (kResident ? (interval & 1u) : 0u);
  const bool ran = st == TS_RUN;
  IvState s;
  s.snap = A.snap;
  s.mems = mems;
  s.rf = rf;
  s.owk = owk;
  s.owv = owv;
  s.flags = flags;
  s.wlog = reinterpret_cast<uint4 *>(A.log) + ((uint64_t)blockIdx.x * A.warps_per_cta + warp) * A.warp_slice;
  s.S = T;  // register and own-write slot stride
  s.tid = t;
  s.gtid = gtid;
  s.wg = wg;
  s.lt = lt;
  s.slots = slots;
  s.lbase = A.GT + wg * A.LT;
  s.lanes = lanes;
  s.lane_lt = (1u << (t & 31u)) - 1u;
  s.warp = warp;
  s.interval = interval;
  s.tag = kResident ? s_iv[1] : A.tag;
  s.st = st;
  s.pc = pc;
  s.nloc = 0;
  s.seq = 0;
  s.nw = 0;
  s.wfill = 0;
  s.bloom = 0;
  s.running = ran;

  E.run(A, s);

  st = s.st;
  pc = s.pc;
  const uint32_t nloc = s.nloc, seq = s.seq, nw = s.nw, wfill = s.wfill;
  // Stop points (barrier ordinal, or n_barriers for the exit), reduced over
  // the CTA before they reach the kernel-wide table: every work-item of the
  // kernel reports one, and same-address atomics serialise in L2.  Each
  // warp folds its lanes by stop point; thread 0 folds the warps' entries.
  __shared__ uint32_t s_stop[32], s_min[32], s_cnt[32], s_acc[3][32];
  const bool stopping = st == TS_BARRIER || (st == TS_EXIT && ran);
  // resident runs alternate two stop tables by interval parity
  uint32_t *const stop_min = A.stop_min + (kResident ? (interval & 1u) * nstops : 0u);
  uint32_t *const stop_cnt = A.stop_cnt + (kResident ? (interval & 1u) * nstops : 0u);
  {
    // access counters of the warp (global, local)
    const uint32_t sg = __reduce_add_sync(lanes, seq - nloc), sl = __reduce_add_sync(lanes, nloc);
    if ((t & 31u) == 0) {
      s_acc[0][warp] = sg;
      s_acc[1][warp] = sl;
      s_acc[2][warp] = wfill;  // warp-uniform: this warp's records in the log
    }
    const uint32_t smask = __ballot_sync(lanes, stopping);
    const uint32_t lane = t & 31u;
    uint32_t stop = kNone, gmin = 0, gcnt = 0;
    if (stopping) {
      stop = st == TS_BARRIER ? E.barrier_ordinal(A, pc) : A.n_barriers;
      const uint32_t g = __match_any_sync(smask, stop);
      if (g != smask) {  // several stop points in this warp: each group reports its own
        if (lane == (uint32_t)(__ffs(g) - 1)) {
          atomicMin(&stop_min[stop], gtid);
          atomicAdd(&stop_cnt[stop], (uint32_t)__popc(g));
        }
        stop = kNone;
      }
      gmin = gtid;  // at the lowest stopping lane: the warp's smallest work-item
      gcnt = __popc(g);
    }
    const uint32_t leader = smask ? (uint32_t)(__ffs(smask) - 1) : 0u;
    if (lane == leader) {
      s_stop[warp] = smask ? stop : kNone;
      s_min[warp] = gmin;
      s_cnt[warp] = gcnt;
    }
  }
  __syncthreads();
  if (t == 0) {
    const uint32_t nwarps = (T + 31u) / 32u;
    unsigned long long cg = 0, cl = 0, cw = 0;
    for (uint32_t w = 0; w < nwarps; w++) {
      cg += s_acc[0][w];
      cl += s_acc[1][w];
      cw += s_acc[2][w];
    }
    if (cg) atomicAdd(&A.acc[0], cg);
    if (cl) atomicAdd(&A.acc[1], cl);
    if (cw && A.logged) atomicAdd(A.logged, cw);
    uint32_t cur = kNone, cmin = 0, ccnt = 0;
    for (uint32_t w = 0; w < nwarps; w++) {
      if (s_stop[w] == kNone) continue;
      if (s_stop[w] != cur) {
        if (cur != kNone) {
          atomicMin(&stop_min[cur], cmin);
          atomicAdd(&stop_cnt[cur], ccnt);
        }
        cur = s_stop[w];
        cmin = s_min[w];
        ccnt = 0;
      }
      ccnt += s_cnt[w];
    }
    if (cur != kNone) {
      atomicMin(&stop_min[cur], cmin);
      atomicAdd(&stop_cnt[cur], ccnt);
    }
  }
  if constexpr (kResident) {
    // ---- the interval's end: commit and compaction between two grid barriers
    if (!grid_sync(A.grid_bar, gridDim.x, A.barrier_limit_ns)) return;
    const uint32_t tag = s_iv[1];
    {
      const uint32_t hi = (tag << 26) | gtid;  // owner word of the cell's highest writer
      const uint32_t ns = nw < slots ? nw : slots;
      for (uint32_t k = 0; k < nw; k++) {
        uint32_t key;
        int32_t v;
        if (k < ns) {
          key = owk[k * T + t];
          v = owv[k * T + t];
        } else {
          const uint2 e = A.ow[(uint64_t)k * A.ow_stride + lt];
          key = e.x;
          v = (int32_t)e.y;
        }
        if (__ldcg(A.owner + 4ull * key) == hi) A.commit[key] = v;
      }
      compact_slice(s.wlog, wfill < A.warp_slice ? wfill : (uint32_t)A.warp_slice, A.owner, tag,
                    reinterpret_cast<uint4 *>(A.acc_out), A.acc_total, t & 31u, A.acc_cap, flags);
      if (blockIdx.x == 0)  // the next interval's stop table starts empty
        for (uint32_t k = t; k < nstops; k += blockDim.x) {
          A.stop_min[((interval + 1u) & 1u) * nstops + k] = kNone;
          A.stop_cnt[((interval + 1u) & 1u) * nstops + k] = 0;
        }
    }
    if (!grid_sync(A.grid_bar, gridDim.x, A.barrier_limit_ns)) return;
    __shared__ uint32_t s_go;
    if (t == 0) {  // every CTA reads the same final values: one decision for the grid
      uint32_t points = 0;
      bool any_barrier = false;
      for (uint32_t k = 0; k < nstops; k++)
        if (__ldcg(stop_cnt + k)) {
          points++;
          any_barrier |= k < A.n_barriers;
        }
      const uint32_t fl = __ldcg(flags);
      if (blockIdx.x == 0) {
        A.iv_off[interval + 1] = __ldcg(A.acc_total);
        A.run_info[0] = interval + 1;
        A.run_info[1] = tag;
      }
      s_go = fl == 0 && points == 1 && any_barrier && interval + 1 < A.max_intervals;
    }
    __syncthreads();
    if (!s_go) return;
    if (tag == 63) {  // the 6-bit tag wraps: clear the owner table first
      const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
      for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + t; i < A.owner_words; i += stride) A.owner[i] = 0;
      if (!grid_sync(A.grid_bar, gridDim.x, A.barrier_limit_ns)) return;
    }
    if (t == 0) {  // every thread read s_iv before the last __syncthreads
      s_iv[0] = interval + 1;
      s_iv[1] = tag == 63 ? 1u : tag + 1u;
    }
    __syncthreads();
    if (st == TS_BARRIER) {  // resume after the barrier it waited at
      st = TS_RUN;
      pc += 1;
    }
    continue;
  }
  A.st[gtid] = st;
  A.pc[gtid] = pc;
  A.ow_count[gtid] = nw;
  {  // spill the shared-memory own-write slots so the commit kernel sees every entry
    const uint32_t ns = nw < slots ? nw : slots;
    for (uint32_t k = 0; k < ns; k++)
      A.ow[(uint64_t)k * A.ow_stride + lt] = make_uint2(owk[k * T + t], (uint32_t)owv[k * T + t]);
  }
  if (st == TS_BARRIER) {
    for (uint32_t r = kBuiltinRegs; r < A.n_regs; r++) A.regs[(uint64_t)r * N + gtid] = rf[r * T + t];
  }
  if ((t & 31u) == 0)
    A.warp_count[(uint64_t)blockIdx.x * A.warps_per_cta + warp] = wfill < A.warp_slice ? wfill : (uint32_t)A.warp_slice;
  // Work-group-scoped barriers: the barrier-release rule within this group,
  // from its own stop points (smallest work-item, count) gathered in the
  // dynamic shared memory after the own-write slots (8 * (n_barriers + 1)
  // bytes the host adds in this mode).
  if (A.group_div) {  // uniform over the grid
    uint32_t *grp_min = reinterpret_cast<uint32_t *>(owv + slots * T), *grp_cnt = grp_min + (A.n_barriers + 1);
    for (uint32_t k = t; k <= A.n_barriers; k += blockDim.x) {
      grp_min[k] = kNone;
      grp_cnt[k] = 0;
    }
    __syncthreads();
    if (stopping) {
      const uint32_t stop = st == TS_BARRIER ? E.barrier_ordinal(A, pc) : A.n_barriers;
      atomicMin(&grp_min[stop], gtid);
      atomicAdd(&grp_cnt[stop], 1u);
    }
    __syncthreads();
    if (t == 0) {
      uint32_t points = 0;
      for (uint32_t k = 0; k <= A.n_barriers; k++) points += grp_cnt[k] != 0;
      if (points >= 2) {
        for (uint32_t k = 0; k <= A.n_barriers; k++)
          if (grp_cnt[k])
            append_err(A, OutRec{A.interval, 0, wg, 0, CLS_DIVERGENCE, grp_min[k], k < A.n_barriers ? k : kNone, 0,
                                 0, grp_cnt[k]}, A.flags);
        atomicAdd(A.group_div, 1u);
      }
    }
  }
  return;
  }  // the interval loop
}

}  // namespace rc
