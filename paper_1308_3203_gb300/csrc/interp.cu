// Work-item interpreter: one CUDA thread per work-item, one CTA per
// work-group, one launch per barrier interval (or per range of groups), or
// one cooperative launch for every interval (resident runs).  The kernel
// body -- state set-up, stop points, counters, resident commits and
// compaction -- is interp_body (interp_kernel.cuh); this file supplies its
// bytecode-interpreting engine and the launchers.
#include "device.cuh"
#include "interp_kernel.cuh"

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
template <bool kConst, bool kResident>
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
        const int32_t v = shared_access<kResident>(A, s, m, performing, cell_of(s, m, idx), cls == CC_ST, priv, yr,
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
  interp_body<kResident>(A, InterpEngine<kConst, kResident>{});
}

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
