// Work-item interpreter: one CUDA thread per work-item, one CTA per
// work-group, one launch per barrier interval (or per range of groups).
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
// its warp's slice of the interval's log -- a 16-byte store at the slot the
// ballot of the logging lanes gives it, no atomics.
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
#include "device.cuh"
#include "semantics.cuh"

namespace rc {
namespace {

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
__device__ __noinline__ bool grid_sync(unsigned *bar, unsigned nblocks, unsigned long long limit_ns) {
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

// Bytecode of the instance being checked when it fits (the warp fetches
// one instruction per step at a warp-uniform address: the constant cache's
// broadcast case).  Larger programs are read from global memory.
__constant__ uint4 c_code[kConstCodeInsns];

template <bool kConst, bool kResident>
__global__ void __launch_bounds__(1024, 2) interp_kernel(InterpArgs A) {
  if (!kResident && A.proceed && *A.proceed == 0) return;  // a closed gate: the host runs this interval later
  extern __shared__ __align__(16) unsigned char smem[];
  const uint4 *__restrict__ code = reinterpret_cast<const uint4 *>(A.code);
  MemInfo *mems = reinterpret_cast<MemInfo *>(smem);
  int32_t *rf = reinterpret_cast<int32_t *>(mems + A.n_mems);  // [n_regs][S]
  uint32_t *owk = reinterpret_cast<uint32_t *>(rf + A.n_regs * A.S);  // [ow_slots][S] keys
  int32_t *owv = reinterpret_cast<int32_t *>(owk + A.ow_slots * A.S);  // [ow_slots][S] values

  const uint32_t S = A.S;
  const uint32_t tid = threadIdx.x;
  for (uint32_t k = tid; k < A.n_mems; k += blockDim.x) mems[k] = A.mems[k];

  const uint32_t wg = A.group0 + blockIdx.x;
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
      rf[r * S + tid] = kResident ? 0 : A.regs[(uint64_t)r * N + gtid];
    rf[REG_TID * S + tid] = (int32_t)tid;
    rf[REG_WG * S + tid] = (int32_t)wg;
    rf[REG_GTID * S + tid] = (int32_t)gtid;
    rf[REG_GSIZE * S + tid] = (int32_t)S;
    rf[REG_NGROUPS * S + tid] = (int32_t)A.G;
  }
  // resident: the current interval and owner-table tag live in shared
  // memory (CTA-uniform), which keeps the interpreter's registers free
  __shared__ uint32_t s_iv[2];
  if (kResident && tid == 0) {
    s_iv[0] = A.interval;
    s_iv[1] = A.tag;
  }
  __syncthreads();

#define REG(i) rf[(uint32_t)(i) * S + tid]
#define INTERVAL (kResident ? s_iv[0] : A.interval)
#define TAG (kResident ? s_iv[1] : A.tag)
  const uint32_t lbase = A.GT + wg * A.LT;
  const uint32_t wbase = tid & ~31u;
  const uint32_t lanes = S - wbase >= 32 ? 0xFFFFFFFFu : ((1u << (S - wbase)) - 1u);
  const uint32_t nstops = A.n_barriers + 1;
  for (;;) {  // resident: one pass per barrier interval; otherwise a single pass
  // resident runs raise an interval's flags in the word of its parity, so a
  // CTA still deciding on interval k never sees a flag of interval k + 1
  uint32_t *const flags = A.flags + (kResident ? (INTERVAL & 1u) : 0u);
  uint32_t nloc = 0, seq = 0, nw = 0;  // global accesses = seq - nloc
  uint64_t bloom = 0;
  const bool ran = st == TS_RUN;
  bool running = ran;

  // Min-PC reconvergence: every iteration the warp executes the instruction
  // at the smallest bytecode pc among its running lanes; lanes that are
  // ahead (past a branch or a loop the others are still in) wait at their
  // pc, so lanes that followed different paths meet again at the join point.
  // The instruction is fetched and decoded once for the warp and every lane
  // takes the same dispatch branch; only the side effects are predicated on
  // the lane being at that pc.
  // Each warp appends to its own log slice: the ballot of the lanes that
  // log in a step gives every lane its slot, and the slice fill level is a
  // warp-uniform register (no atomics).
  const uint32_t warp = tid >> 5, lane_lt = (1u << (tid & 31u)) - 1u;
  uint4 *const wlog = reinterpret_cast<uint4 *>(A.log) +
                      ((uint64_t)blockIdx.x * A.warps_per_cta + warp) * A.warp_slice;
  uint32_t wfill = 0;

  for (;;) {
    const uint32_t minpc = __reduce_min_sync(lanes, running ? pc : kNone);
    if (minpc == kNone) break;
    const uint4 raw = kConst ? c_code[minpc] : __ldg(code + minpc);
    const bool act = running && pc == minpc;
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
        pc = sem_branch(ctl, r, imm) ? tgt : pc + 1;
      }
      continue;
    }
    if (cls == CC_LD || cls == CC_ST) {
      const MemInfo m = mems[ctl >> CTL_MEM_SHIFT];  // (LD/ST class: operand bits)
      const int32_t idx = sem_index(x, imm, (int32_t)tgt, ctl);
      const bool inb = (uint32_t)idx < m.len;
      // a private access (warp-uniform: one instruction) is counted but not
      // logged, and only its stores claim their cells (for the commit)
      const bool priv = (ctl & CTL_PRIV) != 0;
      const uint32_t performing = __ballot_sync(lanes, act && inb);
      const uint32_t logging = priv ? 0u : performing;
      const uint32_t slot_pos = wfill + __popc(logging & lane_lt);
      wfill += __popc(logging);
      if (!act) continue;
      pc++;
      if (!inb) {  // ⊥: out of bounds, the work-item stops
        OutRec e{INTERVAL, m.space, m.space ? wg : 0u, (uint32_t)idx, CLS_OOB, gtid,
                 ctl >> CTL_MEM_SHIFT, 0, 0, 0};
        append_err(A, e, flags);
        st = TS_DEAD;
        running = false;
        continue;
      }
      const uint32_t key = (m.space ? lbase : 0u) + m.base + (uint32_t)idx;
      // the lanes still here are exactly those in `performing`
      if (A.owner && !(priv && cls == CC_LD)) shadow_claim_warp(A.owner, performing, key, cls == CC_ST, TAG, gtid, tid & 31u);
      // own-write table: the first `slots` distinct cells in shared memory, the rest in global
      const uint64_t bit = bloom_bit(key);
      int32_t slot = -1;
      if (bloom & bit) {
        const uint32_t ns = nw < slots ? nw : slots;
        for (uint32_t k = 0; k < ns; k++)
          if (owk[k * S + tid] == key) { slot = (int32_t)k; break; }
        if (slot < 0)
          for (uint32_t k = slots; k < nw; k++)
            if (A.ow[(uint64_t)k * A.ow_stride + lt].x == key) { slot = (int32_t)k; break; }
      }
      int32_t v;
      if (cls == CC_LD) {
        if (slot < 0) v = kResident ? __ldcg(A.snap + key) : __ldg(A.snap + key);  // resident: committed in-kernel
        else if ((uint32_t)slot < slots) v = owv[slot * S + tid];
        else v = (int32_t)A.ow[(uint64_t)slot * A.ow_stride + lt].y;
        REG(d) = v;
      } else {
        v = yr;
        if (slot >= 0) {
          if ((uint32_t)slot < slots) owv[slot * S + tid] = v;
          else A.ow[(uint64_t)slot * A.ow_stride + lt].y = (uint32_t)v;
        } else if (nw < slots) {
          owk[nw * S + tid] = key;
          owv[nw * S + tid] = v;
          nw++;
          bloom |= bit;
        } else if (nw < A.capw) {
          A.ow[(uint64_t)nw * A.ow_stride + lt] = make_uint2(key, (uint32_t)v);
          nw++;
          bloom |= bit;
        } else {
          atomicOr(flags, FLAG_OW_FULL);
        }
      }
      if (!priv) {
        if (slot_pos < A.warp_slice)  // always true: the slice holds the static per-interval bound
          wlog[slot_pos] = make_uint4(key, gtid | (cls == CC_ST ? 0x80000000u : 0u), (uint32_t)v, seq);
        else
          atomicOr(flags, FLAG_LOG_FULL);
      }
      seq++;
      nloc += m.space;
      continue;
    }
    if (!act) continue;
    pc++;
    switch (cls) {
      case CC_DIVMOD:
        REG(d) = sem_divmod(ctl, x, yr, imm);
        break;
      case CC_LOGIC:  // (x != 0) and / or (yr != 0)
        REG(d) = sem_logic(ctl, x, yr);
        break;
      case CC_SIZE:
        REG(d) = (int32_t)mems[ctl >> CTL_MEM_SHIFT].len;
        break;
      case CC_ASSUME:
        if (x == 0) {  // ⊤: no continuation
          st = TS_DEAD;
          running = false;
        }
        break;
      case CC_ASSERT:
        if (x == 0) {  // ⊥
          OutRec e{INTERVAL, 0, 0, 0, CLS_ASSERT, gtid, (uint32_t)imm, 0, 0, 0};
          append_err(A, e, flags);
          st = TS_DEAD;
          running = false;
        }
        break;
      case CC_BARRIER:
        st = TS_BARRIER;
        pc -= 1;  // remember the barrier itself
        running = false;
        break;
      default:  // CC_EXIT
        st = TS_EXIT;
        pc -= 1;
        running = false;
        break;
    }
  }
#undef REG
  // Stop points (barrier ordinal, or n_barriers for the exit), reduced over
  // the CTA before they reach the kernel-wide table: every work-item of the
  // kernel reports one, and same-address atomics serialise in L2.  Each
  // warp folds its lanes by stop point; thread 0 folds the warps' entries.
  __shared__ uint32_t s_stop[32], s_min[32], s_cnt[32], s_acc[3][32];
  const bool stopping = st == TS_BARRIER || (st == TS_EXIT && ran);
  // resident runs alternate two stop tables by interval parity
  uint32_t *const stop_min = A.stop_min + (kResident ? (INTERVAL & 1u) * nstops : 0u);
  uint32_t *const stop_cnt = A.stop_cnt + (kResident ? (INTERVAL & 1u) * nstops : 0u);
  {
    // access counters of the warp (global, local)
    const uint32_t sg = __reduce_add_sync(lanes, seq - nloc), sl = __reduce_add_sync(lanes, nloc);
    if ((tid & 31u) == 0) {
      s_acc[0][warp] = sg;
      s_acc[1][warp] = sl;
      s_acc[2][warp] = wfill;  // warp-uniform: this warp's records in the log
    }
    const uint32_t smask = __ballot_sync(lanes, stopping);
    const uint32_t lane = tid & 31u;
    uint32_t stop = kNone, gmin = 0, gcnt = 0;
    if (stopping) {
      stop = st == TS_BARRIER ? (uint32_t)(kConst ? c_code[pc].y : __ldg(code + pc).y) : A.n_barriers;
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
  if (tid == 0) {
    const uint32_t nwarps = (S + 31u) / 32u;
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
    const uint32_t interval = s_iv[0], tag = s_iv[1];
    {
      const uint32_t hi = (tag << 26) | gtid;  // owner word of the cell's highest writer
      const uint32_t ns = nw < slots ? nw : slots;
      for (uint32_t k = 0; k < nw; k++) {
        uint32_t key;
        int32_t v;
        if (k < ns) {
          key = owk[k * S + tid];
          v = owv[k * S + tid];
        } else {
          const uint2 e = A.ow[(uint64_t)k * A.ow_stride + lt];
          key = e.x;
          v = (int32_t)e.y;
        }
        if (__ldcg(A.owner + 4ull * key) == hi) A.commit[key] = v;
      }
      compact_slice(wlog, wfill < A.warp_slice ? wfill : (uint32_t)A.warp_slice, A.owner, tag,
                    reinterpret_cast<uint4 *>(A.acc_out), A.acc_total, tid & 31u, A.acc_cap, flags);
      if (blockIdx.x == 0)  // the next interval's stop table starts empty
        for (uint32_t k = tid; k < nstops; k += blockDim.x) {
          A.stop_min[((interval + 1u) & 1u) * nstops + k] = kNone;
          A.stop_cnt[((interval + 1u) & 1u) * nstops + k] = 0;
        }
    }
    if (!grid_sync(A.grid_bar, gridDim.x, A.barrier_limit_ns)) return;
    __shared__ uint32_t s_go;
    if (tid == 0) {  // every CTA reads the same final values: one decision for the grid
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
      for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + tid; i < A.owner_words; i += stride) A.owner[i] = 0;
      if (!grid_sync(A.grid_bar, gridDim.x, A.barrier_limit_ns)) return;
    }
    if (tid == 0) {  // every thread read s_iv before the last __syncthreads
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
      A.ow[(uint64_t)k * A.ow_stride + lt] = make_uint2(owk[k * S + tid], (uint32_t)owv[k * S + tid]);
  }
  if (st == TS_BARRIER) {
    for (uint32_t r = kBuiltinRegs; r < A.n_regs; r++) A.regs[(uint64_t)r * N + gtid] = rf[r * S + tid];
  }
  if ((tid & 31u) == 0)
    A.warp_count[(uint64_t)blockIdx.x * A.warps_per_cta + warp] = wfill < A.warp_slice ? wfill : (uint32_t)A.warp_slice;
  // Work-group-scoped barriers: the barrier-release rule within this group,
  // from its own stop points (smallest work-item, count) gathered in the
  // dynamic shared memory after the own-write slots (8 * (n_barriers + 1)
  // bytes the host adds in this mode).
  if (A.group_div) {  // uniform over the grid
    uint32_t *grp_min = reinterpret_cast<uint32_t *>(owv + slots * S), *grp_cnt = grp_min + (A.n_barriers + 1);
    for (uint32_t k = tid; k <= A.n_barriers; k += blockDim.x) {
      grp_min[k] = kNone;
      grp_cnt[k] = 0;
    }
    __syncthreads();
    if (stopping) {
      const uint32_t stop = st == TS_BARRIER ? (uint32_t)(kConst ? c_code[pc].y : __ldg(code + pc).y) : A.n_barriers;
      atomicMin(&grp_min[stop], gtid);
      atomicAdd(&grp_cnt[stop], 1u);
    }
    __syncthreads();
    if (tid == 0) {
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
#undef INTERVAL
#undef TAG

// Diagnostic: every CTA waits at a grid barrier that expects one more
// arrival than the launch has, so each wait must run out after limit_ns and
// report it in bar[2] (the status the host reads), leaving the context usable.
__global__ void grid_barrier_probe_kernel(unsigned *bar, unsigned long long limit_ns) {
  grid_sync(bar, gridDim.x + 1, limit_ns);
}

__global__ void interval_gate_kernel(const uint32_t *flags, const unsigned long long *compacted,
                                     const uint32_t *stop_cnt, uint32_t n_barriers, uint32_t *proceed) {
  uint32_t n_points = 0;
  bool any_barrier = false;
  for (uint32_t k = 0; k <= n_barriers; k++) {
    if (!stop_cnt[k]) continue;
    n_points++;
    if (k < n_barriers) any_barrier = true;
  }
  *proceed = (*flags == 0 && *compacted == 0 && n_points == 1 && any_barrier) ? 1u : 0u;
}

}  // namespace

void launch_interval_gate(const uint32_t *flags, const unsigned long long *compacted, const uint32_t *stop_cnt,
                          uint32_t n_barriers, uint32_t *proceed, cudaStream_t s) {
  count_launch();
  interval_gate_kernel<<<1, 1, 0, s>>>(flags, compacted, stop_cnt, n_barriers, proceed);
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

}  // namespace rc
