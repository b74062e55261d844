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
// Every access is appended to the interval's log with one warp-aggregated
// atomic per instruction and one 16-byte store per work-item.
#include <cooperative_groups.h>

#include "device.cuh"

namespace cg = cooperative_groups;

namespace rc {
namespace {

__device__ __forceinline__ int32_t idiv(int32_t a, int32_t b) {
  if (b == 0) return 0;
  if (a == INT32_MIN && b == -1) return INT32_MIN;  // 2^31 wraps
  return a / b;
}
__device__ __forceinline__ int32_t imod(int32_t a, int32_t b) {  // Euclidean, in [0, |b|)
  if (b == 0) return 0;
  int64_t m = b < 0 ? -(int64_t)b : (int64_t)b;
  int64_t r = (int64_t)a % m;
  if (r < 0) r += m;
  return (int32_t)r;
}
__device__ __forceinline__ uint64_t bloom_bit(uint32_t key) {
  return 1ull << ((key * 2654435761u) >> 26);
}

__device__ __forceinline__ void append_log(const InterpArgs &A, uint32_t key, uint32_t tw, int32_t v,
                                           uint32_t seq) {
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned long long base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(A.log_count, (unsigned long long)g.size());
  base = g.shfl(base, 0);
  unsigned long long pos = base + g.thread_rank();
  if (pos < A.log_cap) {
    reinterpret_cast<uint4 *>(A.log)[pos] = make_uint4(key, tw, (uint32_t)v, seq);
  } else {
    atomicOr(A.flags, FLAG_LOG_FULL);
  }
}

__device__ __forceinline__ void append_err(const InterpArgs &A, const OutRec &r) {
  uint32_t pos = atomicAdd(A.err_count, 1u);
  if (pos < A.err_cap) A.errs[pos] = r;
  else atomicOr(A.flags, FLAG_ERR_FULL);
}

__global__ void __launch_bounds__(1024) interp_kernel(InterpArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint2 *code = reinterpret_cast<uint2 *>(smem);
  MemInfo *mems = reinterpret_cast<MemInfo *>(code + A.n_insn);
  int32_t *rf = reinterpret_cast<int32_t *>(mems + A.n_mems);

  const uint32_t S = A.S;
  const uint32_t tid = threadIdx.x;
  for (uint32_t k = tid; k < A.n_insn; k += blockDim.x) code[k] = reinterpret_cast<const uint2 *>(A.code)[k];
  for (uint32_t k = tid; k < A.n_mems; k += blockDim.x) mems[k] = A.mems[k];

  const uint32_t wg = A.group0 + blockIdx.x;
  const uint32_t gtid = wg * S + tid;
  const uint64_t N = (uint64_t)A.G * S;
  const uint32_t lt = gtid - A.group0 * S;  // index in this launch's own-write table
  uint32_t st = A.st[gtid];
  uint32_t pc = A.pc[gtid];
  if (st == TS_BARRIER) {  // resume after the barrier it waited at
    st = TS_RUN;
    pc += 1;
  }
  if (st == TS_RUN) {
    for (uint32_t r = 0; r < A.n_regs; r++) rf[r * S + tid] = A.regs[(uint64_t)r * N + gtid];
  }
  __syncthreads();

#define REG(i) rf[(uint32_t)(i) * S + tid]
  uint32_t nglob = 0, nloc = 0, seq = 0, nw = 0, stop = kNone;
  uint64_t bloom = 0;
  const uint32_t lbase = A.GT + wg * A.LT;

  if (st == TS_RUN) {
    for (;;) {
      const uint2 raw = code[pc];
      const uint32_t op = raw.x & 0xFFu, d = (raw.x >> 8) & 0xFFu, ra = (raw.x >> 16) & 0xFFu,
                     rb = raw.x >> 24;
      const int32_t imm = (int32_t)raw.y;
      pc++;
      switch (op) {
        case OP_NOP: break;
        case OP_MOVI: REG(d) = imm; break;
        case OP_MOV: REG(d) = REG(ra); break;
        case OP_ADD: REG(d) = (int32_t)((uint32_t)REG(ra) + (uint32_t)REG(rb)); break;
        case OP_SUB: REG(d) = (int32_t)((uint32_t)REG(ra) - (uint32_t)REG(rb)); break;
        case OP_MUL: REG(d) = (int32_t)((uint32_t)REG(ra) * (uint32_t)REG(rb)); break;
        case OP_DIV: REG(d) = idiv(REG(ra), REG(rb)); break;
        case OP_MOD: REG(d) = imod(REG(ra), REG(rb)); break;
        case OP_ADDI: REG(d) = (int32_t)((uint32_t)REG(ra) + (uint32_t)imm); break;
        case OP_SUBI: REG(d) = (int32_t)((uint32_t)REG(ra) - (uint32_t)imm); break;
        case OP_MULI: REG(d) = (int32_t)((uint32_t)REG(ra) * (uint32_t)imm); break;
        case OP_DIVI: REG(d) = idiv(REG(ra), imm); break;
        case OP_MODI: REG(d) = imod(REG(ra), imm); break;
        case OP_RSUBI: REG(d) = (int32_t)((uint32_t)imm - (uint32_t)REG(ra)); break;
        case OP_LT: REG(d) = REG(ra) < REG(rb); break;
        case OP_LE: REG(d) = REG(ra) <= REG(rb); break;
        case OP_GT: REG(d) = REG(ra) > REG(rb); break;
        case OP_GE: REG(d) = REG(ra) >= REG(rb); break;
        case OP_EQ: REG(d) = REG(ra) == REG(rb); break;
        case OP_NE: REG(d) = REG(ra) != REG(rb); break;
        case OP_LTI: REG(d) = REG(ra) < imm; break;
        case OP_LEI: REG(d) = REG(ra) <= imm; break;
        case OP_GTI: REG(d) = REG(ra) > imm; break;
        case OP_GEI: REG(d) = REG(ra) >= imm; break;
        case OP_EQI: REG(d) = REG(ra) == imm; break;
        case OP_NEI: REG(d) = REG(ra) != imm; break;
        case OP_LAND: REG(d) = (REG(ra) != 0) && (REG(rb) != 0); break;
        case OP_LOR: REG(d) = (REG(ra) != 0) || (REG(rb) != 0); break;
        case OP_NEG: REG(d) = (int32_t)(0u - (uint32_t)REG(ra)); break;
        case OP_NOT: REG(d) = REG(ra) == 0; break;
        case OP_TID: REG(d) = (int32_t)tid; break;
        case OP_WG: REG(d) = (int32_t)wg; break;
        case OP_GTID: REG(d) = (int32_t)gtid; break;
        case OP_GSIZE: REG(d) = (int32_t)S; break;
        case OP_NGROUPS: REG(d) = (int32_t)A.G; break;
        case OP_SIZE: REG(d) = (int32_t)mems[imm].len; break;
        case OP_JMP: pc = (uint32_t)imm; break;
        case OP_BZ: if (REG(ra) == 0) pc = (uint32_t)imm; break;
        case OP_LD:
        case OP_ST: {
          const MemInfo m = mems[imm];
          const int32_t idx = REG(ra);
          if ((uint32_t)idx >= m.len) {  // ⊥: out of bounds, the work-item stops
            OutRec e{A.interval, m.space, m.space ? wg : 0u, (uint32_t)idx, CLS_OOB, gtid, (uint32_t)imm, 0, 0, 0};
            append_err(A, e);
            st = TS_DEAD;
            goto done;
          }
          const uint32_t key = (m.space ? lbase : 0u) + m.base + (uint32_t)idx;
          const uint64_t bit = bloom_bit(key);
          int32_t slot = -1;
          if (bloom & bit) {
            for (int32_t k = (int32_t)nw - 1; k >= 0; k--) {
              if (A.ow[(uint64_t)k * A.ow_stride + lt].x == key) { slot = k; break; }
            }
          }
          if (A.owner) shadow_claim(A.owner + 2ull * key + (op == OP_LD ? 1 : 0), A.epoch, gtid);
          if (op == OP_LD) {
            const int32_t v = slot >= 0 ? (int32_t)A.ow[(uint64_t)slot * A.ow_stride + lt].y : A.snap[key];
            REG(d) = v;
            append_log(A, key, gtid, v, seq++);
          } else {
            const int32_t v = REG(rb);
            if (slot >= 0) {
              A.ow[(uint64_t)slot * A.ow_stride + lt].y = (uint32_t)v;
            } else if (nw < A.capw) {
              A.ow[(uint64_t)nw * A.ow_stride + lt] = make_uint2(key, (uint32_t)v);
              nw++;
              bloom |= bit;
            } else {
              atomicOr(A.flags, FLAG_OW_FULL);
            }
            append_log(A, key, gtid | 0x80000000u, v, seq++);
          }
          if (m.space) nloc++;
          else nglob++;
          break;
        }
        case OP_ASSUME:
          if (REG(ra) == 0) { st = TS_DEAD; goto done; }  // ⊤: no continuation
          break;
        case OP_ASSERT:
          if (REG(ra) == 0) {  // ⊥
            OutRec e{A.interval, 0, 0, 0, CLS_ASSERT, gtid, (uint32_t)imm, 0, 0, 0};
            append_err(A, e);
            st = TS_DEAD;
            goto done;
          }
          break;
        case OP_BARRIER:
          st = TS_BARRIER;
          stop = (uint32_t)imm;
          pc -= 1;  // remember the barrier itself
          goto done;
        case OP_EXIT:
        default:
          st = TS_EXIT;
          stop = A.n_barriers;
          pc -= 1;
          goto done;
      }
    }
  }
done:
#undef REG
  if (stop != kNone) {
    atomicMin(&A.stop_min[stop], gtid);
    atomicAdd(&A.stop_cnt[stop], 1u);
  }
  A.st[gtid] = st;
  A.pc[gtid] = pc;
  A.ow_count[gtid] = nw;
  if (st == TS_BARRIER) {
    for (uint32_t r = 0; r < A.n_regs; r++) A.regs[(uint64_t)r * N + gtid] = rf[r * S + tid];
  }
  // access counters: one atomic per warp
  const uint32_t wbase = tid & ~31u;
  const uint32_t live = S - wbase >= 32 ? 0xFFFFFFFFu : ((1u << (S - wbase)) - 1u);
  __syncwarp(live);
  const uint32_t sg = __reduce_add_sync(live, nglob), sl = __reduce_add_sync(live, nloc);
  if ((tid & 31u) == 0) {
    if (sg) atomicAdd(&A.acc[0], (unsigned long long)sg);
    if (sl) atomicAdd(&A.acc[1], (unsigned long long)sl);
  }
}

}  // namespace

size_t interp_smem_bytes(uint32_t n_insn, uint32_t n_mems, uint32_t n_regs, uint32_t S) {
  return (size_t)n_insn * 8 + (size_t)n_mems * sizeof(MemInfo) + (size_t)n_regs * S * 4;
}

cudaError_t interp_configure() {
  return cudaFuncSetAttribute(interp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

void launch_interp(const InterpArgs &a, uint32_t n_groups, size_t smem, cudaStream_t s) {
  interp_kernel<<<n_groups, a.S, smem, s>>>(a);
}

}  // namespace rc
