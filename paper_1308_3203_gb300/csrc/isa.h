// The bytecode's instruction set and the codes kernels and host share
// (opcodes, control-word bits, thread status, record classes).  Plain
// constants and one POD struct: this header is also compiled at run time
// (NVRTC) into the kernels of compiled intervals, where no host standard
// library is available; the fixed-width integer types then come from the
// code that includes it.
#pragma once
#ifndef __CUDACC_RTC__
#include <cstdint>
#endif

namespace rc {

enum Op : uint8_t {
  OP_NOP = 0,
  OP_MOVI,    // d = imm
  OP_MOV,     // d = a
  OP_ADD, OP_SUB, OP_MUL, OP_DIV, OP_MOD,          // d = a op b
  OP_ADDI, OP_MULI, OP_DIVI, OP_MODI,              // d = a op imm
  OP_ANDI,    // d = a & imm  (Euclidean modulus by a power of two, imm = 2^k - 1)
  OP_RSUBI,   // d = imm - a
  OP_LT, OP_LE, OP_GT, OP_GE, OP_EQ, OP_NE,        // d = (a op b)
  OP_LTI, OP_LEI, OP_GTI, OP_GEI, OP_EQI, OP_NEI,  // d = (a op imm)
  OP_LAND, OP_LOR,                                 // d = (a != 0) and/or (b != 0)
  OP_NEG, OP_NOT,                                  // d = -a, d = (a == 0)
  OP_TID, OP_WG, OP_GTID, OP_GSIZE, OP_NGROUPS,    // (not emitted: built-ins are registers 0..4)
  OP_SIZE,    // d = size(mem ctl.mem)
  OP_LD,      // d = mem[ctl.mem][index]   (one shared read; index: a + imm + imm2, or the mask form)
  OP_ST,      // mem[ctl.mem][index] = b   (one shared write)
  OP_JMP,     // pc = imm2
  OP_BZ,      // if a == 0: pc = imm2
  OP_BFLTI, OP_BFLEI, OP_BFGTI, OP_BFGEI, OP_BFEQI, OP_BFNEI,  // if !(a op imm): pc = imm2
  OP_LOOP,    // d = a + 1 (d == a); if d < imm: pc = imm2   (loop back edge)
  OP_MADI,    // d = a * imm + b
  OP_ASSUME,  // a == 0: the work-item retires silently (no continuation)
  OP_ASSERT,  // a == 0: the work-item aborts with an assertion record (id imm)
  OP_BARRIER, // stop at barrier imm
  OP_EXIT,    // reach the exit node
  OP_COUNT
};

// Registers 0..4 hold the built-ins tid, wg, gtid, gsize and ngroups; the
// interpreter sets them when a work-item starts an interval and the code
// only reads them.
enum : int { REG_TID = 0, REG_WG = 1, REG_GTID = 2, REG_GSIZE = 3, REG_NGROUPS = 4, kBuiltinRegs = 5 };

struct Insn {
  uint8_t op, d, a, b;  // opcode and register fields (always valid registers)
  int32_t imm;          // constant operand / offset / id
  int32_t imm2;         // jump target, or the second index constant of LD/ST
  uint32_t ctl;         // control word, see below
};

// Control word.  Everything except the operand fields (memory object and
// index addressing mode of LD/ST/SIZE) is a pure function of the opcode
// (predecode).  ALU-class instructions -- arithmetic, moves, comparisons and
// every branch form -- are evaluated by one branch-free formula with
// x = REG(a), yr = REG(b):
//   arith = (M*x*yr + P*x + Q*yr + C) & mask        (32-bit wrap)
//       P = imm if AL_PIMM else the small code P (0, +1, -1);  Q likewise (no imm)
//       C = 1 if AL_CONE, 0 if AL_PIMM or AL_MASKIMM, else imm
//       mask = imm if AL_MASKIMM else all ones
//   cmp  = ((x < y) & AL_LT | (x == y) & AL_EQ) ^ AL_INV,  y = imm if AL_YIMM else yr
//   r    = cmp if AL_CMP else arith;  REG(d) = r if AL_WRITE
//   next pc = imm2 if (mode == always) or (mode == cond and c), else pc + 1,
//       c = (arith < imm) if AL_LOOPCOND else cmp
enum : uint32_t {
  AL_P_SHIFT = 0,           // 2 bits: 0 -> 0, 1 -> +1, 2 -> -1
  AL_Q_SHIFT = 2,           // 2 bits, same code
  AL_M = 1u << 4,           // x * yr term
  AL_PIMM = 1u << 5,
  AL_MASKIMM = 1u << 6,
  AL_CONE = 1u << 7,
  AL_CMP = 1u << 8,
  AL_YIMM = 1u << 9,
  AL_LT = 1u << 10,
  AL_EQ = 1u << 11,
  AL_INV = 1u << 12,
  AL_WRITE = 1u << 13,
  AL_MODE_SHIFT = 14,       // 2 bits: 0 no branch, 1 conditional, 2 always
  AL_LOOPCOND = 1u << 18,   // (bits 16-17 of the ALU layout are unused)
  CTL_CLASS_SHIFT = 20,     // 4 bits, all classes
  // LD/ST operand bits
  CTL_AM = 1u << 0,         // index = ((REG(a) + imm) & (2^k - 1)) + imm2
  CTL_K_SHIFT = 1,          // 5 bits: k
  CTL_MEM_SHIFT = 24,       // 8 bits: memory object of LD/ST/SIZE
  CTL_PRIV = 1u << 6,       // LD/ST proven private for this launch shape (set per check, never compiled in):
                            // no other work-item touches its cells in its interval -- not logged, loads claim nothing
  // DIVMOD bits
  DM_MOD = 1u << 0,
  DM_YIMM = 1u << 1,
};
enum CtlClass : uint32_t {
  CC_ALU = 0, CC_LD, CC_ST, CC_DIVMOD, CC_SIZE, CC_LOGIC, CC_ASSUME, CC_ASSERT, CC_BARRIER, CC_EXIT
};
// Thread status codes kept in device state.
enum TStatus : uint32_t { TS_RUN = 0, TS_BARRIER = 1, TS_EXIT = 2, TS_DEAD = 3 };

// Record classes (values shared with the public header).
enum Cls : uint32_t {
  CLS_WW_RACE = 1, CLS_WW_BENIGN = 2, CLS_RW_RACE = 3,
  CLS_XG_WW_RACE = 4, CLS_XG_WW_BENIGN = 5, CLS_XG_RW_RACE = 6,
  CLS_OOB = 16, CLS_ASSERT = 17, CLS_DIVERGENCE = 18
};

static_assert(sizeof(Insn) == 16, "instruction must be 16 bytes");

}  // namespace rc
