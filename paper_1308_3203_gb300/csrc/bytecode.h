// Register bytecode executed by the work-item interpreter kernel.
//
// One instruction is 8 bytes: opcode, destination register, two source
// registers and a 32-bit immediate.  Every private variable of the kernel
// (Sec. 3, Locals) owns one register; expression temporaries take the
// registers above them.  LD and ST are the only instructions that touch
// shared memory, one access each, matching the paper's commands
// v := a[v] and a[v] := e (Sec. 3).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace rc {

enum Op : uint8_t {
  OP_NOP = 0,
  OP_MOVI,    // d = imm
  OP_MOV,     // d = a
  OP_ADD, OP_SUB, OP_MUL, OP_DIV, OP_MOD,          // d = a op b
  OP_ADDI, OP_SUBI, OP_MULI, OP_DIVI, OP_MODI,     // d = a op imm
  OP_RSUBI,   // d = imm - a
  OP_LT, OP_LE, OP_GT, OP_GE, OP_EQ, OP_NE,        // d = (a op b)
  OP_LTI, OP_LEI, OP_GTI, OP_GEI, OP_EQI, OP_NEI,  // d = (a op imm)
  OP_LAND, OP_LOR,                                 // d = (a != 0) and/or (b != 0)
  OP_NEG, OP_NOT,                                  // d = -a, d = (a == 0)
  OP_TID, OP_WG, OP_GTID, OP_GSIZE, OP_NGROUPS,    // d = built-in
  OP_SIZE,    // d = size(mem imm)
  OP_LD,      // d = mem[imm][a]          (one shared read)
  OP_ST,      // mem[imm][a] = b          (one shared write)
  OP_JMP,     // pc = imm
  OP_BZ,      // if a == 0: pc = imm
  OP_ASSUME,  // a == 0: the work-item retires silently (no continuation)
  OP_ASSERT,  // a == 0: the work-item aborts with an assertion record (id imm)
  OP_BARRIER, // stop at barrier imm
  OP_EXIT,    // reach the exit node
  OP_COUNT
};

struct Insn {
  uint8_t op, d, a, b;
  int32_t imm;
};
static_assert(sizeof(Insn) == 8, "instruction must be 8 bytes");

struct MemDecl {
  std::string name;
  uint32_t space;     // 0 global, 1 local (one copy per work-group)
  int64_t decl_len;   // local: declared length; global: -1 (length from the input)
};

// A compiled kernel (what rc_compile returns, behind an opaque handle).
struct Program {
  std::string name;
  std::vector<MemDecl> mems;
  std::vector<Insn> code;
  uint32_t n_vars = 0;   // named private variables
  uint32_t n_regs = 0;   // registers incl. temporaries
  uint32_t n_barriers = 0, n_asserts = 0;
  uint32_t n_global = 0; // number of global memory objects
  // static upper bounds per work-item per barrier interval (constant-trip
  // loops make these finite); used to size logs so they cannot overflow
  uint64_t max_access_per_interval = 0;
  uint64_t max_write_per_interval = 0;
};

// Thread status codes kept in device state.
enum TStatus : uint32_t { TS_RUN = 0, TS_BARRIER = 1, TS_EXIT = 2, TS_DEAD = 3 };

// Record classes (values shared with the public header).
enum Cls : uint32_t {
  CLS_WW_RACE = 1, CLS_WW_BENIGN = 2, CLS_RW_RACE = 3,
  CLS_OOB = 16, CLS_ASSERT = 17, CLS_DIVERGENCE = 18
};

// Compile kernel source; throws CompileError.
struct CompileError {
  std::string msg;
};
Program compile_program(const std::string &src);
// Structural validation of a program's bytecode; returns empty string when ok.
std::string validate_program(const Program &p);

}  // namespace rc
