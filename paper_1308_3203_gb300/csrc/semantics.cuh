// Per-work-item semantics of one bytecode instruction (Distefano & Dubreil,
// Sec. 4 thread-local rules, with the int32 arithmetic of the language):
// shared by every kernel that executes bytecode, so the canonical checker,
// the batched checker and the interleaving explorer compute the same thing.
#pragma once
#ifndef __CUDACC_RTC__
#include <cstdint>
#endif

#include "isa.h"

namespace rc {

// truncating division; x / 0 = 0, INT_MIN / -1 wraps to INT_MIN
__device__ __forceinline__ int32_t sem_div(int32_t a, int32_t b) {
  if (b == 0) return 0;
  if (a == INT32_MIN && b == -1) return INT32_MIN;
  return a / b;
}

// Euclidean remainder in [0, |b|); x % 0 = 0
__device__ __forceinline__ int32_t sem_mod(int32_t a, int32_t b) {
  if (b == 0) return 0;
  const uint32_t m = b < 0 ? 0u - (uint32_t)b : (uint32_t)b;
  if ((int32_t)m > 0) {
    const int32_t r = a % (int32_t)m;
    return r < 0 ? r + (int32_t)m : r;
  }
  return a & 0x7FFFFFFF;  // |b| = 2^31
}

// Result of an ALU-class instruction (arithmetic, moves, comparisons, and
// every branch form, whose result is nonzero when the branch is taken),
// x = REG(a), yr = REG(b).
__device__ __forceinline__ int32_t sem_alu(uint32_t op, int32_t x, int32_t yr, int32_t imm) {
  const uint32_t ux = (uint32_t)x, uy = (uint32_t)yr, ui = (uint32_t)imm;
  switch (op) {
    case OP_MOVI: return imm;
    case OP_MOV: return x;
    case OP_ADD: return (int32_t)(ux + uy);
    case OP_SUB: return (int32_t)(ux - uy);
    case OP_MUL: return (int32_t)(ux * uy);
    case OP_ADDI: return (int32_t)(ux + ui);
    case OP_MULI: return (int32_t)(ux * ui);
    case OP_ANDI: return x & imm;
    case OP_RSUBI: return (int32_t)(ui - ux);
    case OP_MADI: return (int32_t)(ux * ui + uy);
    case OP_NEG: return (int32_t)(0u - ux);
    case OP_NOT: return x == 0;
    case OP_LT: return x < yr;
    case OP_LE: return x <= yr;
    case OP_GT: return x > yr;
    case OP_GE: return x >= yr;
    case OP_EQ: return x == yr;
    case OP_NE: return x != yr;
    case OP_LTI: return x < imm;
    case OP_LEI: return x <= imm;
    case OP_GTI: return x > imm;
    case OP_GEI: return x >= imm;
    case OP_EQI: return x == imm;
    case OP_NEI: return x != imm;
    case OP_BZ: return x == 0;
    case OP_BFLTI: return !(x < imm);
    case OP_BFLEI: return !(x <= imm);
    case OP_BFGTI: return !(x > imm);
    case OP_BFGEI: return !(x >= imm);
    case OP_BFEQI: return x != imm;
    case OP_BFNEI: return x == imm;
    case OP_LOOP: return (int32_t)(ux + 1u);
    default: return 1;  // OP_JMP, OP_NOP
  }
}

// Does an ALU-class instruction with result r branch to its target?
__device__ __forceinline__ bool sem_branch(uint32_t ctl, int32_t r, int32_t imm) {
  const uint32_t mode = (ctl >> AL_MODE_SHIFT) & 3u;
  return mode == 2u || (mode == 1u && ((ctl & AL_LOOPCOND) ? r < imm : r != 0));
}

// Index of a load or store: x + imm + imm2, or ((x + imm) mod 2^k) + imm2
__device__ __forceinline__ int32_t sem_index(int32_t x, int32_t imm, int32_t imm2, uint32_t ctl) {
  uint32_t ui = (uint32_t)x + (uint32_t)imm;
  if (ctl & CTL_AM) ui &= ((2u << ((ctl >> CTL_K_SHIFT) & 0x1Fu)) - 1u) >> 1;  // 2^k - 1
  return (int32_t)(ui + (uint32_t)imm2);
}

// DIVMOD and LOGIC classes
__device__ __forceinline__ int32_t sem_divmod(uint32_t ctl, int32_t x, int32_t yr, int32_t imm) {
  const int32_t y = (ctl & DM_YIMM) ? imm : yr;
  return (ctl & DM_MOD) ? sem_mod(x, y) : sem_div(x, y);
}
__device__ __forceinline__ int32_t sem_logic(uint32_t ctl, int32_t x, int32_t yr) {
  return (ctl & 1u) ? ((x != 0) || (yr != 0)) : ((x != 0) && (yr != 0));
}

}  // namespace rc
