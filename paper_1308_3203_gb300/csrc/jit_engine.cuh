// Engine of compiled intervals: the work-item runs a program's bytecode
// translated into one straight-line function (translate.cpp) instead of the
// interpreter's fetch-decode-dispatch loop.  Compiled at run time (NVRTC)
// together with the function; see jit.cu for the source it is part of.
//
// The translated function keeps the registers in a constant-indexed array
// (machine registers) and reaches shared memory through the hooks defined
// here, which take the same path as the interpreter's LD/ST step
// (shared_access: claims, own-write table, log record, counters).  Two
// things differ because lanes of a warp no longer step together:
//  * a hook is called by the lanes that reached it together (__activemask);
//    they rank their log slots by ballot as the interpreter's step does;
//  * the warp's log fill level is a shared-memory counter that each such
//    group advances with one atomic, so groups that diverged and reach log
//    appends at different times never take the same slot.
// A work-item's records still follow its program order (each of its
// appends takes a later slot), and the classifier orders records by cell,
// work-item and that order only, so reports do not depend on the engine.
#pragma once
#include "interp_kernel.cuh"

namespace rc {

template <bool kRes>
struct JitCtx {
  const InterpArgs &A;
  IvState &s;
  uint32_t *fill;  // the warp's log fill counter (shared memory)
};

// Log slot of this lane among `performing` (the calling lanes with an
// in-bounds access); every lane in `mask` (the calling lanes) takes part.
__device__ __forceinline__ uint32_t jit_log_slot(uint32_t *fill, uint32_t mask, uint32_t performing,
                                                 uint32_t lane, uint32_t lane_lt) {
  const uint32_t leader = (uint32_t)(__ffs(mask) - 1);
  uint32_t base = 0;
  if (lane == leader && performing) base = atomicAdd(fill, (uint32_t)__popc(performing));
  base = __shfl_sync(mask, base, (int)leader);
  return base + __popc(performing & lane_lt);
}

template <bool kPriv, bool kStore, bool kRes>
__device__ __forceinline__ bool jit_access(JitCtx<kRes> &cx, uint32_t mem, int32_t idx, int32_t &v) {
  IvState &s = cx.s;
  const uint32_t mask = __activemask();
  const MemInfo m = mem < kInlineMems ? cx.A.mem_inline[mem] : s.mems[mem];
  const bool inb = (uint32_t)idx < m.len;
  const uint32_t performing = __ballot_sync(mask, inb);
  const uint32_t slot = kPriv ? 0u : jit_log_slot(cx.fill, mask, performing, s.tid & 31u, s.lane_lt);
  if (!inb) {  // ⊥: the generated code stops the work-item
    out_of_bounds(cx.A, s, m, mem, idx);
    return false;
  }
  // inlined at every access site: one call shared by all sites measured
  // 10.5 against 6.2 ms per interval on the 2^26-work-item stress program
  v = shared_access<kRes ? kSnapLdcg : kSnapLdg>(cx.A, s, m, performing, cell_of(s, m, idx), kStore, kPriv, v, slot);
  return true;
}

template <bool kPriv, bool kRes>
__device__ __forceinline__ bool jit_load(JitCtx<kRes> &cx, uint32_t mem, int32_t idx, int32_t &out) {
  int32_t v = 0;
  if (!jit_access<kPriv, false>(cx, mem, idx, v)) return false;
  out = v;
  return true;
}

template <bool kPriv, bool kRes>
__device__ __forceinline__ bool jit_store(JitCtx<kRes> &cx, uint32_t mem, int32_t idx, int32_t val) {
  return jit_access<kPriv, true>(cx, mem, idx, val);
}

template <bool kRes>
__device__ __forceinline__ void jit_assert_fail(JitCtx<kRes> &cx, int32_t id) {
  OutRec e{cx.s.interval, 0, 0, 0, CLS_ASSERT, cx.s.gtid, (uint32_t)id, 0, 0, 0};
  append_err(cx.A, e, cx.s.flags);
}

// Prog: the compiled program, a type with kRegs (its register count) and
//   template <bool kRes> static void run(JitCtx<kRes> &, int32_t (&)[kRegs], uint32_t &pc, uint32_t &st)
// where pc is the instruction to resume at (0, or the one after a barrier)
// and, on return, st is the work-item's status with pc at the instruction
// after the barrier it stopped at (barriers), at the exit instruction, or at
// the instruction that stopped it.
template <bool kRes, class Prog>
struct JitEngine {
  __device__ __forceinline__ uint32_t barrier_ordinal(const InterpArgs &A, uint32_t pc) const {
    return __ldg(reinterpret_cast<const uint4 *>(A.code) + pc).y;
  }

  __device__ __forceinline__ void run(const InterpArgs &A, IvState &s) const {
    __shared__ uint32_t s_fill[32];
    const uint32_t S = s.S, tid = s.tid;
    if ((tid & 31u) == 0) s_fill[s.warp] = 0;
    __syncwarp(s.lanes);
    if (s.running) {
      int32_t r[Prog::kRegs];
#pragma unroll
      for (uint32_t k = 0; k < Prog::kRegs; k++) r[k] = s.rf[k * S + tid];
      JitCtx<kRes> cx{A, s, &s_fill[s.warp]};
      uint32_t pc = s.pc, st = TS_RUN;
      Prog::template run<kRes>(cx, r, pc, st);
#pragma unroll
      for (uint32_t k = 0; k < Prog::kRegs; k++) s.rf[k * S + tid] = r[k];
      // the state keeps the interpreter's convention: a waiting work-item's
      // pc is its barrier instruction
      s.pc = st == TS_BARRIER ? pc - 1 : pc;
      s.st = st;
      s.running = false;
    }
    __syncwarp(s.lanes);
    s.wfill = s_fill[s.warp];
  }
};

}  // namespace rc

// The translated function's hooks (see translate.cpp).
#define RC_JIT_FN template <bool kRes> __device__ __forceinline__
#define RC_JIT_CTX ::rc::JitCtx<kRes>
#define RC_LD(cx, site, mem, idx, out) ::rc::jit_load<rc_jit_private(site)>(cx, mem, idx, out)
#define RC_ST(cx, site, mem, idx, val) ::rc::jit_store<rc_jit_private(site)>(cx, mem, idx, val)
#define RC_SIZE(cx, mem) ((int32_t)((mem) < ::rc::kInlineMems ? (cx).A.mem_inline[mem] : (cx).s.mems[mem]).len)
#define RC_ASSERT_FAIL(cx, id) ::rc::jit_assert_fail(cx, id)
#define RC_AT_BARRIER(cx, id) ((void)0)
