// Batched checking: many kernel instances per launch.
//
// Every instance keeps its own bytecode, launch shape, cells, registers,
// own-write table and log slices; the device sees them through a table of
// descriptors.  Work is cut into warp tasks -- 32 consecutive work-items of
// one instance -- which a persistent grid pulls from an atomic counter, so
// instances of very different sizes balance across the GPU.  One launch runs
// one barrier interval of every instance that is still active (instances
// progress in lock-step rounds); classification then runs once over the
// shared cell space of the round, whose cells are the instances' cells laid
// end to end.  The interpreter step is the single-instance one (min-PC
// reconvergence, indexed LD/ST, ballot-ranked log appends, owner claims);
// see interp.cu for the semantics it implements.
#include "device.cuh"
#include "interp_kernel.cuh"  // grid_sync
#include "semantics.cuh"

namespace rc {
namespace {

__device__ __forceinline__ uint64_t bbloom(uint32_t key) { return 1ull << ((key * 2654435761u) >> 26); }

__device__ __forceinline__ void batch_err(const BatchArgs &A, uint32_t k, const OutRec &r) {
  const uint32_t pos = atomicAdd(A.err_count, 1u);
  if (pos < A.err_cap) {
    A.errs[pos] = r;
    A.err_kernel[pos] = k;
  } else {
    atomicOr(A.flags, FLAG_ERR_FULL);
  }
}

// Loads of state that changes between rounds.  A resident run keeps one
// launch across rounds, and a warp task may run on another SM than in the
// last round, whose L1 can still hold the old line: such loads go to L2.
template <bool kRes, class T>
__device__ __forceinline__ T ld_state(const T *p) {
  if constexpr (kRes) return __ldcg(p);
  else return *p;
}

// One warp task: one interval of 32 work-items of instance task_kernel[task]
// (rf/owk/owv: this CTA's shared register file and own-write slots).
// Returns how full the task's log slice got, in permille of its capacity
// (warp-uniform; 0 for a task with nothing to run).
template <uint32_t kBatchThreads, bool kRes>
__device__ __forceinline__ uint32_t batch_task(const BatchArgs &A, uint32_t task, uint32_t interval, uint32_t tag,
                                               uint32_t *owner, int32_t *rf, uint32_t *owk, int32_t *owv) {
  const uint32_t RS = kBatchThreads;  // register-file stride
  const uint32_t t = threadIdx.x, lane = t & 31u, lane_lt = (1u << lane) - 1u;
  const uint32_t slots = A.ow_slots;
#define REG(i) rf[(uint32_t)(i) * RS + t]
  const uint32_t k = A.task_kernel[task];
  const BatchDesc D = A.desc[k];
  if (!ld_state<kRes>(&A.desc[k].active)) return 0;  // finished instance: nothing to run, its slices stay unread
  const uint32_t lw = task - D.task_off;                 // warp of the instance
  const uint32_t gl = lw * 32 + lane;                    // instance-local work-item id
  const bool exists = (uint64_t)gl < D.N;
  const uint32_t lanes = __ballot_sync(0xFFFFFFFFu, exists);
  if (!exists) return 0;
  const uint32_t S = D.S, tid = gl % S, wg = gl / S;
  const uint32_t lbase = (uint32_t)D.key_base + D.GT + wg * D.LT;
  const uint4 *code = reinterpret_cast<const uint4 *>(A.code) + D.code_off;
  const uint4 *mems = reinterpret_cast<const uint4 *>(A.mems) + D.mems_off;
  uint32_t st = ld_state<kRes>(A.st + D.state_off + gl);
  uint32_t pc = ld_state<kRes>(A.pc + D.state_off + gl);
  if (st == TS_BARRIER) {
    st = TS_RUN;
    pc += 1;
  }
  const bool ran = st == TS_RUN;
  if (ran) {
    for (uint32_t r = kBuiltinRegs; r < D.n_regs; r++)
      REG(r) = ld_state<kRes>(A.regs + D.reg_off + (uint64_t)r * D.N + gl);
    REG(REG_TID) = (int32_t)tid;
    REG(REG_WG) = (int32_t)wg;
    REG(REG_GTID) = (int32_t)gl;
    REG(REG_GSIZE) = (int32_t)S;
    REG(REG_NGROUPS) = (int32_t)D.G;
  }
  __syncwarp(lanes);
  uint32_t nloc = 0, seq = 0, nw = 0, wfill = 0;
  uint64_t bloom = 0;
  bool running = ran;
  uint4 *const wlog = reinterpret_cast<uint4 *>(A.log) + D.slice_off + (uint64_t)lw * D.slice;
  uint2 *const ow = A.ow + D.ow_off;

  for (;;) {
    const uint32_t minpc = __reduce_min_sync(lanes, running ? pc : kNone);
    if (minpc == kNone) break;
    const uint4 raw = __ldg(code + minpc);
    const bool act = running && pc == minpc;
    const uint32_t d = (raw.x >> 8) & 0xFFu, ra = (raw.x >> 16) & 0xFFu, rb = raw.x >> 24;
    const int32_t imm = (int32_t)raw.y;
    const uint32_t tgt = raw.z, ctl = raw.w;
    const uint32_t cls = (ctl >> CTL_CLASS_SHIFT) & 0xFu;
    const int32_t x = REG(ra);
    const int32_t yr = REG(rb);
    if (cls == CC_ALU) {
      const int32_t r = sem_alu(raw.x & 0xFFu, x, yr, imm);
      if (act) {
        if (ctl & AL_WRITE) REG(d) = r;
        pc = sem_branch(ctl, r, imm) ? tgt : pc + 1;
      }
      continue;
    }
    if (cls == CC_LD || cls == CC_ST) {
      const uint4 mm = __ldg(mems + (ctl >> CTL_MEM_SHIFT));  // MemInfo: len, base, space
      const int32_t idx = sem_index(x, imm, (int32_t)tgt, ctl);
      const bool inb = (uint32_t)idx < mm.x;
      const uint32_t logging = __ballot_sync(lanes, act && inb);
      const uint32_t slot_pos = wfill + __popc(logging & lane_lt);
      wfill += __popc(logging);
      if (!act) continue;
      pc++;
      if (!inb) {
        OutRec e{interval, mm.z, mm.z ? wg : 0u, (uint32_t)idx, CLS_OOB, gl, ctl >> CTL_MEM_SHIFT, 0, 0, 0};
        batch_err(A, k, e);
        st = TS_DEAD;
        running = false;
        continue;
      }
      const uint32_t key = (mm.z ? lbase : (uint32_t)D.key_base) + mm.y + (uint32_t)idx;
      if (owner) shadow_claim_warp(owner, logging, key, cls == CC_ST, tag, gl, lane);  // lanes here = logging
      const uint64_t bit = bbloom(key);
      int32_t slot = -1;
      if (bloom & bit) {
        const uint32_t ns = nw < slots ? nw : slots;
        for (uint32_t q = 0; q < ns; q++)
          if (owk[q * RS + t] == key) { slot = (int32_t)q; break; }
        if (slot < 0)
          for (uint32_t q = slots; q < nw; q++)
            if (ow[(uint64_t)q * D.N + gl].x == key) { slot = (int32_t)q; break; }
      }
      int32_t v;
      if (cls == CC_LD) {
        // the committed value: read-only within a round launch; a resident
        // run commits between rounds in the same launch
        if (slot < 0) v = kRes ? __ldcg(A.snap + key) : __ldg(A.snap + key);
        else if ((uint32_t)slot < slots) v = owv[slot * RS + t];
        else v = (int32_t)ow[(uint64_t)slot * D.N + gl].y;
        REG(d) = v;
      } else {
        v = yr;
        if (slot >= 0) {
          if ((uint32_t)slot < slots) owv[slot * RS + t] = v;
          else ow[(uint64_t)slot * D.N + gl].y = (uint32_t)v;
        } else if (nw < slots) {
          owk[nw * RS + t] = key;
          owv[nw * RS + t] = v;
          nw++;
          bloom |= bit;
        } else if (nw < D.capw) {
          ow[(uint64_t)nw * D.N + gl] = make_uint2(key, (uint32_t)v);
          nw++;
          bloom |= bit;
        } else {
          atomicOr(A.flags, FLAG_OW_FULL);
        }
      }
      if (slot_pos < D.slice)
        wlog[slot_pos] = make_uint4(key, gl | (cls == CC_ST ? 0x80000000u : 0u), (uint32_t)v, seq);
      else
        atomicOr(A.flags, FLAG_LOG_FULL);
      seq++;
      nloc += mm.z;
      continue;
    }
    if (!act) continue;
    pc++;
    switch (cls) {
      case CC_DIVMOD:
        REG(d) = sem_divmod(ctl, x, yr, imm);
        break;
      case CC_LOGIC:
        REG(d) = sem_logic(ctl, x, yr);
        break;
      case CC_SIZE:
        REG(d) = (int32_t)__ldg(mems + (ctl >> CTL_MEM_SHIFT)).x;
        break;
      case CC_ASSUME:
        if (x == 0) {
          st = TS_DEAD;
          running = false;
        }
        break;
      case CC_ASSERT:
        if (x == 0) {
          OutRec e{interval, 0, 0, 0, CLS_ASSERT, gl, (uint32_t)imm, 0, 0, 0};
          batch_err(A, k, e);
          st = TS_DEAD;
          running = false;
        }
        break;
      case CC_BARRIER:
        st = TS_BARRIER;
        pc -= 1;
        running = false;
        break;
      default:
        st = TS_EXIT;
        pc -= 1;
        running = false;
        break;
    }
  }
  // ---- end of this warp task
  {  // stop points, one pair of atomics per group of lanes at the same one
    const bool stopping = st == TS_BARRIER || (st == TS_EXIT && ran);
    const uint32_t smask = __ballot_sync(lanes, stopping);
    if (stopping) {
      const uint32_t stop = st == TS_BARRIER ? (uint32_t)__ldg(code + pc).y : D.n_barriers;
      const uint32_t g = __match_any_sync(smask, stop);
      if (lane == (uint32_t)(__ffs(g) - 1)) {
        atomicMin(&A.stop_min[D.stop_off + stop], gl);
        atomicAdd(&A.stop_cnt[D.stop_off + stop], (uint32_t)__popc(g));
      }
    }
  }
  A.st[D.state_off + gl] = st;
  A.pc[D.state_off + gl] = pc;
  A.ow_count[D.state_off + gl] = nw;
  {
    const uint32_t ns = nw < slots ? nw : slots;
    for (uint32_t q = 0; q < ns; q++) ow[(uint64_t)q * D.N + gl] = make_uint2(owk[q * RS + t], (uint32_t)owv[q * RS + t]);
  }
  if (st == TS_BARRIER)
    for (uint32_t r = kBuiltinRegs; r < D.n_regs; r++) A.regs[D.reg_off + (uint64_t)r * D.N + gl] = REG(r);
  __syncwarp(lanes);
  const uint32_t sg = __reduce_add_sync(lanes, seq - nloc), sl = __reduce_add_sync(lanes, nloc);
  if (lane == __ffs(lanes) - 1) {
    if (sg) atomicAdd(&A.acc[2ull * k], (unsigned long long)sg);
    if (sl) atomicAdd(&A.acc[2ull * k + 1], (unsigned long long)sl);
    A.warp_count[task] = wfill < D.slice ? wfill : (uint32_t)D.slice;
  }
#undef REG
  return (uint32_t)(((wfill < D.slice ? wfill : D.slice) * 1000ull + D.slice - 1) / D.slice);
}

// the largest slice fill of this warp's tasks, one atomic per warp
__device__ __forceinline__ void report_fill(const BatchArgs &A, uint32_t fill_pm) {
  if ((threadIdx.x & 31u) == 0 && fill_pm) atomicMax(A.fill_max, fill_pm);
}

// Commits from the own-write tables of one warp task's lanes (instance-local
// work-items), by the owner table: every cell's highest writer commits its
// last write (the rule the classifier applies), so the next round needs
// nothing from the classification, which in a resident run comes after the
// launch and in lock-step rounds runs beside the next round.
template <bool kRes>
__device__ __forceinline__ void commit_task(const BatchArgs &A, uint32_t task, uint32_t tag, uint32_t lane) {
  const uint32_t k = A.task_kernel[task];
  const BatchDesc &D = A.desc[k];
  const uint32_t gl = (task - D.task_off) * 32 + lane;
  if ((uint64_t)gl >= D.N) return;
  const uint32_t nw = ld_state<kRes>(A.ow_count + D.state_off + gl);
  const uint32_t hi = (tag << 26) | gl;
  for (uint32_t q = 0; q < nw; q++) {
    const uint2 e = ld_state<kRes>(A.ow + D.ow_off + (uint64_t)q * D.N + gl);
    if (__ldcg(A.owner + 4ull * e.x) == hi) A.snap[e.x] = (int32_t)e.y;
  }
}

// Block shapes the autotuner chooses from: threads per CTA, always 1024
// threads (32 warps) per SM
template <uint32_t kBatchThreads>
__global__ void __launch_bounds__(kBatchThreads, 1024 / kBatchThreads) batch_interp_kernel(BatchArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  int32_t *rf = reinterpret_cast<int32_t *>(smem);                          // [max_regs][threads]
  uint32_t *owk = reinterpret_cast<uint32_t *>(rf + A.max_regs * kBatchThreads);  // [ow_slots][threads]
  int32_t *owv = reinterpret_cast<int32_t *>(owk + A.ow_slots * kBatchThreads);
  // round state lives in device memory so one captured launch serves every round
  const uint32_t interval = A.round[0], tag = A.round[1];
  uint32_t *const owner = A.round[2] ? A.owner : nullptr;
  uint32_t fill = 0;
  for (;;) {
    uint32_t task = 0;
    if ((threadIdx.x & 31u) == 0) task = atomicAdd(A.next_task, 1u);
    task = __shfl_sync(0xFFFFFFFFu, task, 0);
    if (task >= A.n_tasks) break;
    fill = max(fill, batch_task<kBatchThreads, false>(A, task, interval, tag, owner, rf, owk, owv));
  }
  report_fill(A, fill);
}

// Resident run: every round in one launch.  Round r (tag0 + r as the owner
// table's tag, cleared in-kernel when the 6-bit tag wraps):
//   1. warp tasks of the active instances from counter next_task[r & 1];
//   2. after a grid barrier, the commit of each cell's highest writer and the
//      compaction of the records of shared cells into acc_out (iv_off[r]
//      marks where the round's records start);
//   3. after another, each instance's barrier agreement (the rule of the
//      host's lock-step rounds): divergence records, the instance stops or
//      goes on, its stop table cleared for the next round;
//   4. after a third, every CTA reads the same count of instances still
//      active and ends when none is (or on an overflow, or at max_rounds).
template <uint32_t kBatchThreads>
__global__ void __launch_bounds__(kBatchThreads, 1024 / kBatchThreads) batch_resident_kernel(BatchArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  int32_t *rf = reinterpret_cast<int32_t *>(smem);
  uint32_t *owk = reinterpret_cast<uint32_t *>(rf + A.max_regs * kBatchThreads);
  int32_t *owv = reinterpret_cast<int32_t *>(owk + A.ow_slots * kBatchThreads);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = gridDim.x * (kBatchThreads / 32), gwarp = blockIdx.x * (kBatchThreads / 32) + (threadIdx.x >> 5);
  const uint32_t threads = gridDim.x * kBatchThreads, gthread = blockIdx.x * kBatchThreads + threadIdx.x;
  uint32_t tag = A.tag0;
  uint32_t fill = 0;
  for (uint32_t r = 0;; r++) {
    // ---- 1. the round's warp tasks
    for (;;) {
      uint32_t task = 0;
      if (lane == 0) task = atomicAdd(A.next_task + (r & 1u), 1u);
      task = __shfl_sync(0xFFFFFFFFu, task, 0);
      if (task >= A.n_tasks) break;
      fill = max(fill, batch_task<kBatchThreads, true>(A, task, r, tag, A.owner, rf, owk, owv));
    }
    if (!grid_sync(A.grid_bar, gridDim.x, A.barrier_limit_ns)) return;
    // ---- 2. commit and compaction (no task of this round is running)
    if (gthread == 0) {
      A.next_task[(r + 1u) & 1u] = 0;  // last used in round r - 1
      A.n_active[r & 1u] = 0;          // read before this round's tasks; counts round r + 2
    }
    for (uint32_t task = gwarp; task < A.n_tasks; task += warps) {
      const uint32_t k = A.task_kernel[task];
      if (!__ldcg(&A.desc[k].active)) continue;
      commit_task<true>(A, task, tag, lane);
      const BatchDesc &D = A.desc[k];
      compact_slice(reinterpret_cast<const uint4 *>(A.log) + D.slice_off + (uint64_t)(task - D.task_off) * D.slice,
                    __ldcg(A.warp_count + task), A.owner, tag, reinterpret_cast<uint4 *>(A.acc_out), A.acc_total,
                    lane, A.acc_cap, A.flags);
    }
    if (!grid_sync(A.grid_bar, gridDim.x, A.barrier_limit_ns)) return;
    // ---- 3. barrier agreement of every instance that ran this round
    if (gthread == 0) A.iv_off[r + 1] = __ldcg(A.acc_total);
    for (uint32_t k = gthread; k < A.n_inst; k += threads) {
      if (!__ldcg(&A.desc[k].active)) continue;
      const BatchDesc &D = A.desc[k];
      uint32_t *smin = A.stop_min + D.stop_off, *scnt = A.stop_cnt + D.stop_off;
      uint32_t points = 0;
      bool any_barrier = false;
      for (uint32_t j = 0; j <= D.n_barriers; j++)
        if (__ldcg(scnt + j)) {
          points++;
          any_barrier |= j < D.n_barriers;
        }
      bool go = points == 1 && any_barrier;
      if (points >= 2) {  // work-items stopped at different points: one record per point
        for (uint32_t j = 0; j <= D.n_barriers; j++) {
          const uint32_t c = __ldcg(scnt + j);
          if (c) batch_err(A, k, OutRec{r, 0, 0, 0, CLS_DIVERGENCE, __ldcg(smin + j),
                                        j < D.n_barriers ? j : 0xFFFFFFFFu, 0, 0, c});
        }
        go = false;
      }
      for (uint32_t j = 0; j <= D.n_barriers; j++) {
        smin[j] = kNone;
        scnt[j] = 0;
      }
      if (go) {
        atomicAdd(A.n_active + ((r + 1u) & 1u), 1u);
      } else {
        A.desc[k].active = 0;
        A.inst_rounds[k] = r + 1;
      }
    }
    if (!grid_sync(A.grid_bar, gridDim.x, A.barrier_limit_ns)) return;
    // ---- 4. one decision for the grid
    const uint32_t active = __ldcg(A.n_active + ((r + 1u) & 1u));
    const uint32_t fl = __ldcg(A.flags);
    if (active == 0 || fl || r + 1 >= A.max_rounds) {
      if (gthread == 0) {
        A.inst_rounds[A.n_inst] = r + 1;
        A.inst_rounds[A.n_inst + 1] = tag;
      }
      report_fill(A, fill);
      return;
    }
    if (tag == 63) {  // the 6-bit tag wraps: clear the batch's owner words first
      for (uint64_t i = gthread; i < A.owner_words; i += threads) A.owner[i] = 0;
      if (!grid_sync(A.grid_bar, gridDim.x, A.barrier_limit_ns)) return;
      tag = 1;
    } else {
      tag++;
    }
  }
}

// One warp per warp task: slices of inactive instances hold nothing this round.
__global__ void batch_compact_kernel(BatchArgs A, LogRec *out, unsigned long long *total) {
  const uint32_t task = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (task >= A.n_tasks) return;
  const uint32_t k = A.task_kernel[task];
  if (!A.desc[k].active) return;
  const BatchDesc &D = A.desc[k];
  compact_slice<8>(reinterpret_cast<const uint4 *>(A.log) + D.slice_off + (uint64_t)(task - D.task_off) * D.slice,
                   A.warp_count[task], A.round[2] ? A.owner : nullptr, A.round[1], reinterpret_cast<uint4 *>(out),
                   total, threadIdx.x & 31u);
}

// One thread per work-item of every active instance (task-major).
__global__ void batch_commit_kernel(BatchArgs A) {
  const uint32_t task = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (task >= A.n_tasks) return;
  if (!A.desc[A.task_kernel[task]].active) return;
  if (!A.round[2]) return;  // sort-path round: the classifier commits every cell
  commit_task<false>(A, task, A.round[1], threadIdx.x & 31u);
}

}  // namespace

size_t batch_smem_bytes(uint32_t max_regs, uint32_t ow_slots, uint32_t threads) {
  return ((size_t)max_regs + 2ull * ow_slots) * threads * 4;
}

cudaError_t batch_configure() {
  const void *fns[] = {(const void *)batch_interp_kernel<128>, (const void *)batch_interp_kernel<256>,
                       (const void *)batch_interp_kernel<512>, (const void *)batch_resident_kernel<128>,
                       (const void *)batch_resident_kernel<256>, (const void *)batch_resident_kernel<512>};
  for (const void *f : fns) {
    // the resident kernels hold a few static bytes (the grid barrier's flag)
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kMaxSmemPerBlock - fa.sharedSizeBytes));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_batch_resident(const BatchArgs &a, uint32_t grid, uint32_t threads, size_t smem, cudaStream_t s) {
  count_launch();
  BatchArgs arg = a;
  void *params[] = {&arg};
  const void *fn = threads == 128   ? (const void *)batch_resident_kernel<128>
                   : threads == 512 ? (const void *)batch_resident_kernel<512>
                                    : (const void *)batch_resident_kernel<256>;
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(threads), params, smem, s);
}

int batch_resident_blocks_per_sm(uint32_t threads, size_t smem) {
  const void *fn = threads == 128   ? (const void *)batch_resident_kernel<128>
                   : threads == 512 ? (const void *)batch_resident_kernel<512>
                                    : (const void *)batch_resident_kernel<256>;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, (int)threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

void launch_batch_interp(const BatchArgs &a, uint32_t grid, uint32_t threads, size_t smem, cudaStream_t s) {
  count_launch();
  if (threads == 128) batch_interp_kernel<128><<<grid, 128, smem, s>>>(a);
  else if (threads == 512) batch_interp_kernel<512><<<grid, 512, smem, s>>>(a);
  else batch_interp_kernel<256><<<grid, 256, smem, s>>>(a);
}

void launch_batch_compact(const BatchArgs &a, LogRec *out, unsigned long long *total, cudaStream_t s) {
  if (!a.n_tasks) return;
  count_launch();
  batch_compact_kernel<<<(a.n_tasks + 7) / 8, 256, 0, s>>>(a, out, total);
}

void launch_batch_commit(const BatchArgs &a, cudaStream_t s) {
  if (!a.n_tasks) return;
  count_launch();
  batch_commit_kernel<<<(a.n_tasks + 7) / 8, 256, 0, s>>>(a);
}

}  // namespace rc
