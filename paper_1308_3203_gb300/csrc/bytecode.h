// Register bytecode executed by the work-item interpreter kernel.
//
// One instruction is 16 bytes: opcode, destination register, two source
// registers, a 32-bit constant and a 32-bit memory id or jump target.  Every private variable of the kernel
// (Sec. 3, Locals) owns one register; expression temporaries take the
// registers above them.  LD and ST are the only instructions that touch
// shared memory, one access each, matching the paper's commands
// v := a[v] and a[v] := e (Sec. 3).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "isa.h"

namespace rc {

// opcode-derived part of the control word; returns false for opcodes that
// may not appear in a program (or whose fields the formula cannot take)
bool predecode(const Insn &in, uint32_t &ctl);
// mask of the operand bits of an instruction's control word
uint32_t operand_bits(const Insn &in);

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
  // the bytecode with CTL_PRIV set on the private accesses of the last launch
  // shape and input lengths it was checked with (filled by the checker)
  struct PrivateCode {
    bool valid = false;
    uint32_t G = 0, S = 0, n_private = 0;
    std::vector<uint32_t> lens;
    std::vector<Insn> code;
  };
  mutable PrivateCode priv;
};

// Message for rc_last_error() on the calling thread.
void set_last_error(const std::string &msg);

// Compile kernel source; throws CompileError.
struct CompileError {
  std::string msg;
};
Program compile_program(const std::string &src);
// Structural validation of a program's bytecode; returns empty string when ok.
std::string validate_program(const Program &p);

}  // namespace rc

// The object behind the opaque rc_bytecode handle.
struct rc_bytecode {
  rc::Program prog;
};

