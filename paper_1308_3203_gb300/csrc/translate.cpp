// Translation of a compiled kernel into straight-line C++: one function that
// runs one work-item from a resume point to its next barrier, its exit or
// its end (the thread-local rules of Sec. 4 (Distefano & Dubreil), with the
// int32 arithmetic of the language), with the registers as a fixed-size
// array indexed by constants only and every jump a goto.
//
// The interpreter spends most of its issue slots on fetching, decoding and
// dispatching bytecode; a compiled function spends them on the program's own
// arithmetic.  The text compiles as CUDA C++ (the registers then live in
// machine registers) and as plain C++.  The code that includes it supplies
// the shared-memory side through these hooks:
//
//   RC_JIT_FN                       qualifiers of the generated function
//   RC_JIT_CTX                      the type of the context argument `cx`
//   RC_LD(cx, site, mem, idx, out)  one shared read, true when in bounds
//   RC_ST(cx, site, mem, idx, val)  one shared write, true when in bounds
//   RC_SIZE(cx, mem)                the length of a memory object
//   RC_ASSERT_FAIL(cx, id)          a failed assert (the work-item then stops)
//   RC_AT_BARRIER(cx, id)           the work-item stops at barrier id
//
// and includes semantics.cuh first (division, remainder and the index
// forms are the same functions the interpreter calls).  `site` numbers the
// kernel's loads and stores in bytecode order (rc_access_sites).  The
// function's status word takes the interpreter's values: TS_BARRIER (pc =
// the instruction after the barrier), TS_EXIT, TS_DEAD (a failed assume or
// assert, an out-of-bounds access).
#include <cinttypes>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "racecheck.h"
#include "bytecode.h"

namespace rc {

namespace {

void line(std::string &out, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
void line(std::string &out, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  out += buf;
  out += '\n';
}

const char *cmp_op(uint8_t op) {
  switch (op) {
    case OP_LT: case OP_LTI: return "<";
    case OP_LE: case OP_LEI: return "<=";
    case OP_GT: case OP_GTI: return ">";
    case OP_GE: case OP_GEI: return ">=";
    case OP_EQ: case OP_EQI: return "==";
    case OP_NE: case OP_NEI: return "!=";
    default: return nullptr;
  }
}

// the condition under which a branch-class instruction does NOT fall through
const char *branch_neg(uint8_t op) {
  switch (op) {
    case OP_BFLTI: return "<";
    case OP_BFLEI: return "<=";
    case OP_BFGTI: return ">";
    case OP_BFGEI: return ">=";
    case OP_BFEQI: return "==";
    case OP_BFNEI: return "!=";
    default: return nullptr;
  }
}

}  // namespace

std::string translate_program(const Program &p, const std::string &fn_name) {
  const uint32_t n = (uint32_t)p.code.size();
  std::vector<uint8_t> label(n + 1, 0), entry(n + 1, 0);
  entry[0] = label[0] = 1;
  std::vector<uint32_t> site(n, 0xFFFFFFFFu);
  uint32_t n_sites = 0;
  for (uint32_t k = 0; k < n; k++) {
    const Insn &in = p.code[k];
    switch (in.op) {
      case OP_JMP: case OP_BZ: case OP_LOOP:
      case OP_BFLTI: case OP_BFLEI: case OP_BFGTI: case OP_BFGEI: case OP_BFEQI: case OP_BFNEI:
        label[in.imm2] = 1;
        break;
      case OP_BARRIER:
        if (k + 1 < n) entry[k + 1] = label[k + 1] = 1;
        break;
      case OP_LD: case OP_ST:
        site[k] = n_sites++;
        break;
      default:
        break;
    }
  }
  std::string o;
  line(o, "// kernel %s: %u instructions, %u registers, %u shared-access sites", p.name.c_str(), n, p.n_regs,
       n_sites);
  line(o, "RC_JIT_FN void %s(RC_JIT_CTX &cx, int32_t (&r)[%u], uint32_t &pc, uint32_t &st) {", fn_name.c_str(),
       p.n_regs);
  line(o, "  (void)cx;");
  line(o, "  st = %u;", (unsigned)TS_RUN);
  line(o, "  switch (pc) {");
  for (uint32_t k = 0; k < n; k++)
    if (entry[k]) line(o, "    case %u: goto L%u;", k, k);
  line(o, "    default: st = %u; return;", (unsigned)TS_DEAD);
  line(o, "  }");
  auto R = [](uint32_t x) { return "r[" + std::to_string(x) + "]"; };
  for (uint32_t k = 0; k < n; k++) {
    const Insn &in = p.code[k];
    if (label[k]) line(o, "L%u:", k);
    const std::string d = R(in.d), a = R(in.a), b = R(in.b);
    const int32_t imm = in.imm, imm2 = in.imm2;
    const uint32_t mem = in.ctl >> CTL_MEM_SHIFT;
    char immb[32];
    std::snprintf(immb, sizeof immb, "(int32_t)%" PRId32 "LL", imm);  // INT32_MIN as a literal
    const std::string I = immb;
    const std::string U = "(uint32_t)";
    switch (in.op) {
      case OP_NOP: break;
      case OP_MOVI: line(o, "  %s = %s;", d.c_str(), I.c_str()); break;
      case OP_MOV: line(o, "  %s = %s;", d.c_str(), a.c_str()); break;
      case OP_ADD: line(o, "  %s = (int32_t)(%s%s + %s%s);", d.c_str(), U.c_str(), a.c_str(), U.c_str(), b.c_str()); break;
      case OP_SUB: line(o, "  %s = (int32_t)(%s%s - %s%s);", d.c_str(), U.c_str(), a.c_str(), U.c_str(), b.c_str()); break;
      case OP_MUL: line(o, "  %s = (int32_t)(%s%s * %s%s);", d.c_str(), U.c_str(), a.c_str(), U.c_str(), b.c_str()); break;
      case OP_ADDI: line(o, "  %s = (int32_t)(%s%s + %s%s);", d.c_str(), U.c_str(), a.c_str(), U.c_str(), I.c_str()); break;
      case OP_MULI: line(o, "  %s = (int32_t)(%s%s * %s%s);", d.c_str(), U.c_str(), a.c_str(), U.c_str(), I.c_str()); break;
      case OP_ANDI: line(o, "  %s = %s & %s;", d.c_str(), a.c_str(), I.c_str()); break;
      case OP_RSUBI: line(o, "  %s = (int32_t)(%s%s - %s%s);", d.c_str(), U.c_str(), I.c_str(), U.c_str(), a.c_str()); break;
      case OP_MADI:
        line(o, "  %s = (int32_t)(%s%s * %s%s + %s%s);", d.c_str(), U.c_str(), a.c_str(), U.c_str(), I.c_str(),
             U.c_str(), b.c_str());
        break;
      case OP_NEG: line(o, "  %s = (int32_t)(0u - %s%s);", d.c_str(), U.c_str(), a.c_str()); break;
      case OP_NOT: line(o, "  %s = %s == 0;", d.c_str(), a.c_str()); break;
      case OP_LT: case OP_LE: case OP_GT: case OP_GE: case OP_EQ: case OP_NE:
        line(o, "  %s = %s %s %s;", d.c_str(), a.c_str(), cmp_op(in.op), b.c_str());
        break;
      case OP_LTI: case OP_LEI: case OP_GTI: case OP_GEI: case OP_EQI: case OP_NEI:
        line(o, "  %s = %s %s %s;", d.c_str(), a.c_str(), cmp_op(in.op), I.c_str());
        break;
      case OP_LAND: line(o, "  %s = (%s != 0) && (%s != 0);", d.c_str(), a.c_str(), b.c_str()); break;
      case OP_LOR: line(o, "  %s = (%s != 0) || (%s != 0);", d.c_str(), a.c_str(), b.c_str()); break;
      case OP_DIV: line(o, "  %s = rc::sem_div(%s, %s);", d.c_str(), a.c_str(), b.c_str()); break;
      case OP_MOD: line(o, "  %s = rc::sem_mod(%s, %s);", d.c_str(), a.c_str(), b.c_str()); break;
      case OP_DIVI: line(o, "  %s = rc::sem_div(%s, %s);", d.c_str(), a.c_str(), I.c_str()); break;
      case OP_MODI: line(o, "  %s = rc::sem_mod(%s, %s);", d.c_str(), a.c_str(), I.c_str()); break;
      case OP_SIZE: line(o, "  %s = RC_SIZE(cx, %u);", d.c_str(), mem); break;
      case OP_LD:
      case OP_ST: {
        char ix[160];
        std::snprintf(ix, sizeof ix, "rc::sem_index(%s, %s, (int32_t)%" PRId32 "LL, %uu)", a.c_str(), I.c_str(), imm2,
                      in.ctl & (CTL_AM | (0x1Fu << CTL_K_SHIFT)));
        if (in.op == OP_LD)
          line(o, "  if (!RC_LD(cx, %u, %u, %s, %s)) { pc = %u; st = %u; return; }", site[k], mem, ix, d.c_str(), k,
               (unsigned)TS_DEAD);
        else
          line(o, "  if (!RC_ST(cx, %u, %u, %s, %s)) { pc = %u; st = %u; return; }", site[k], mem, ix, b.c_str(), k,
               (unsigned)TS_DEAD);
        break;
      }
      case OP_JMP: line(o, "  goto L%d;", imm2); break;
      case OP_BZ: line(o, "  if (%s == 0) goto L%d;", a.c_str(), imm2); break;
      case OP_BFLTI: case OP_BFLEI: case OP_BFGTI: case OP_BFGEI: case OP_BFEQI: case OP_BFNEI:
        line(o, "  if (!(%s %s %s)) goto L%d;", a.c_str(), branch_neg(in.op), I.c_str(), imm2);
        break;
      case OP_LOOP:
        line(o, "  %s = (int32_t)(%s%s + 1u);", d.c_str(), U.c_str(), a.c_str());
        line(o, "  if (%s < %s) goto L%d;", d.c_str(), I.c_str(), imm2);
        break;
      case OP_ASSUME: line(o, "  if (%s == 0) { pc = %u; st = %u; return; }", a.c_str(), k, (unsigned)TS_DEAD); break;
      case OP_ASSERT:
        line(o, "  if (%s == 0) { RC_ASSERT_FAIL(cx, %d); pc = %u; st = %u; return; }", a.c_str(), imm, k,
             (unsigned)TS_DEAD);
        break;
      case OP_BARRIER:
        line(o, "  RC_AT_BARRIER(cx, %d); pc = %u; st = %u; return;", imm, k + 1, (unsigned)TS_BARRIER);
        break;
      case OP_EXIT: line(o, "  pc = %u; st = %u; return;", k, (unsigned)TS_EXIT); break;
      default:
        throw CompileError{"cannot translate opcode " + std::to_string(in.op) + " at " + std::to_string(k)};
    }
  }
  line(o, "}");
  return o;
}

}  // namespace rc

extern "C" int rc_translate(const rc_bytecode *bc, const char *fn_name, char *buf, size_t cap, size_t *len) {
  using namespace rc;
  if (!bc || !fn_name || !len || (cap && !buf)) {
    set_last_error("null argument");
    return RC_E_INVALID;
  }
  const std::string name = fn_name;
  bool ok = !name.empty() && name.size() <= 128 && !(name[0] >= '0' && name[0] <= '9');
  for (char c : name) ok = ok && ((c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z') || (c >= '0' && c <= '9') || c == '_');
  if (!ok) {
    set_last_error("function name must be a C identifier");
    return RC_E_INVALID;
  }
  try {
    const std::string text = translate_program(bc->prog, name);
    *len = text.size();
    if (cap) {
      const size_t k = text.size() < cap - 1 ? text.size() : cap - 1;
      std::memcpy(buf, text.data(), k);
      buf[k] = '\0';
    }
    return RC_OK;
  } catch (const CompileError &e) {
    set_last_error(e.msg);
    return RC_E_INVALID;
  } catch (const std::bad_alloc &) {
    return RC_E_NOMEM;
  }
}
