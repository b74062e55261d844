// Host compiler: kernel source -> register bytecode (see bytecode.h).
//
// The language is the minimal OpenCL kernel language of Distefano & Dubreil,
// Sec. 3 (expressions e, booleans b, commands Comm; a kernel is a CFG from a
// unique start to a unique exit) with structured if/else and constant-trip
// for-loops as surface syntax.  Array reads inside an expression are emitted
// as one LD each, in evaluation order (left operand first, an index before
// the read that uses it), so each shared access is its own step; a store
// evaluates its index, then its value, then writes.
//
// Alongside code generation the compiler derives a static upper bound on the
// shared accesses (and on the writes) a work-item can make between two
// consecutive barriers.  Loop trip counts are literals, so the bound is
// finite; the runtime sizes its per-interval logs with it.
#include <algorithm>
#include <cctype>
#include <climits>
#include <cstring>
#include <map>
#include <memory>
#include <set>

#include "bytecode.h"

namespace rc {
namespace {

// ------------------------------------------------------------------ tokens
struct Token {
  enum Kind { END, NUM, NAME, PUNCT } kind;
  std::string s;
  uint64_t num = 0;
  int line = 0;
};

std::vector<Token> tokenize(const std::string &src) {
  std::vector<Token> t;
  int line = 1;
  for (size_t i = 0; i < src.size();) {
    unsigned char c = (unsigned char)src[i];
    if (c == '\n') { line++; i++; continue; }
    if (std::isspace(c)) { i++; continue; }
    if (c == '/' && i + 1 < src.size() && src[i + 1] == '/') {
      while (i < src.size() && src[i] != '\n') i++;
      continue;
    }
    Token k;
    k.line = line;
    if (std::isdigit(c)) {
      size_t j = i;
      uint64_t v = 0;
      for (; j < src.size() && std::isdigit((unsigned char)src[j]); j++) {
        v = v * 10 + (uint64_t)(src[j] - '0');
        if (v > 0xFFFFFFFFull) throw CompileError{"line " + std::to_string(line) + ": literal exceeds 32 bits"};
      }
      k.kind = Token::NUM;
      k.num = v;
      k.s = src.substr(i, j - i);
      i = j;
    } else if (std::isalpha(c) || c == '_') {
      size_t j = i;
      while (j < src.size() && (std::isalnum((unsigned char)src[j]) || src[j] == '_')) j++;
      k.kind = Token::NAME;
      k.s = src.substr(i, j - i);
      i = j;
    } else {
      static const char *pairs[] = {"<=", ">=", "==", "!=", "&&", "||", ".."};
      k.kind = Token::PUNCT;
      for (const char *p : pairs)
        if (src.compare(i, 2, p) == 0) k.s = p;
      if (k.s.empty()) {
        if (!std::strchr("+-*/%<>=!(){}[];,", (int)c) || c == 0)
          throw CompileError{"line " + std::to_string(line) + ": unexpected character '" + std::string(1, (char)c) + "'"};
        k.s = std::string(1, (char)c);
      }
      i += k.s.size();
    }
    t.push_back(k);
  }
  Token e;
  e.kind = Token::END;
  e.line = line;
  t.push_back(e);
  return t;
}

const std::set<std::string> &reserved() {
  static const std::set<std::string> r = {"kernel", "global", "local", "int", "barrier", "assume",
                                          "assert", "if", "else", "for", "in", "tid", "wg",
                                          "gtid", "gsize", "ngroups", "size"};
  return r;
}

// ------------------------------------------------------------------ expressions
struct Ex {
  enum K { CONST, VAR, LOAD, BUILTIN, SIZE, UN, BIN } k;
  int32_t c = 0;       // CONST
  int reg = -1;        // VAR
  int mem = -1;        // LOAD, SIZE
  Op op = OP_NOP;      // BUILTIN (OP_TID..), UN (OP_NEG/OP_NOT), BIN (reg-reg form)
  std::unique_ptr<Ex> l, r;
};
using ExP = std::unique_ptr<Ex>;

int count_loads(const Ex *e) {
  if (!e) return 0;
  return (e->k == Ex::LOAD ? 1 : 0) + count_loads(e->l.get()) + count_loads(e->r.get());
}

// ------------------------------------------------------------------ bounds
const int64_t NEG = INT64_MIN / 4;
const int64_t CAP = (int64_t)1 << 50;
int64_t sadd(int64_t a, int64_t b) {
  if (a <= NEG || b <= NEG) return NEG;
  return std::min(CAP, a + b);
}
int64_t smul(int64_t k, int64_t a) {  // k >= 0
  if (a <= NEG) return NEG;
  if (k == 0 || a == 0) return 0;
  if (a > CAP / k) return CAP;
  return k * a;
}

// max shared accesses on paths that: cross the piece with no barrier (thr),
// go from its start to a barrier inside it (ent), from a barrier inside it
// to its end (ext), between two barriers inside it (inn)
struct Bound {
  int64_t thr = 0, ent = NEG, ext = NEG, inn = NEG;
  static Bound accesses(int64_t k) { Bound b; b.thr = k; return b; }
  static Bound barrier() { Bound b; b.thr = NEG; b.ent = 0; b.ext = 0; return b; }
};
Bound seq(const Bound &p, const Bound &q) {
  Bound r;
  r.thr = sadd(p.thr, q.thr);
  r.ent = std::max(p.ent, sadd(p.thr, q.ent));
  r.ext = std::max(q.ext, sadd(p.ext, q.thr));
  r.inn = std::max({p.inn, q.inn, sadd(p.ext, q.ent)});
  return r;
}
Bound alt(const Bound &p, const Bound &q) {
  Bound r;
  r.thr = std::max(p.thr, q.thr);
  r.ent = std::max(p.ent, q.ent);
  r.ext = std::max(p.ext, q.ext);
  r.inn = std::max(p.inn, q.inn);
  return r;
}
Bound loop(const Bound &b, int64_t trips) {
  if (trips <= 0) return Bound();
  Bound r;
  r.thr = smul(trips, b.thr);
  int64_t pre = b.thr <= NEG ? 0 : smul(trips - 1, b.thr);
  r.ent = sadd(pre, b.ent);
  r.ext = sadd(b.ext, pre);
  r.inn = b.inn;
  if (trips >= 2) {
    int64_t mid = b.thr <= NEG ? 0 : smul(trips - 2, b.thr);
    r.inn = std::max(r.inn, sadd(sadd(b.ext, mid), b.ent));
  }
  return r;
}
int64_t worst(const Bound &b) { return std::max({b.thr, b.ent, b.ext, b.inn, (int64_t)0}); }

// ------------------------------------------------------------------ compiler
class Compiler {
 public:
  explicit Compiler(const std::string &src) : tk_(tokenize(src)) {}

  Program run() {
    word("kernel");
    p_.name = name();
    punct("(");
    if (!at(")")) {
      do declaration(); while (take(","));
    }
    punct(")");
    collect_vars();
    Bound acc, wr;
    block(acc, wr);
    if (tk_[i_].kind != Token::END) fail("text after the kernel body");
    emit(OP_EXIT, 0, 0, 0, 0);
    p_.n_vars = (uint32_t)vars_.size();
    p_.n_regs = (uint32_t)std::max<int>(max_reg_, 1);
    if (p_.n_regs > 255) fail("kernel needs more than 255 registers");
    p_.max_access_per_interval = (uint64_t)worst(acc);
    p_.max_write_per_interval = (uint64_t)worst(wr);
    return p_;
  }

 private:
  std::vector<Token> tk_;
  size_t i_ = 0;
  Program p_;
  std::map<std::string, int> mems_, vars_;
  std::vector<int> loops_;  // registers of enclosing loop variables
  int next_tmp_ = 0, max_reg_ = 0;

  [[noreturn]] void fail(const std::string &m) const {
    throw CompileError{"line " + std::to_string(tk_[i_].line) + ": " + m};
  }
  bool at(const char *s) const { return tk_[i_].kind == Token::PUNCT && tk_[i_].s == s; }
  bool at_word(const char *s) const { return tk_[i_].kind == Token::NAME && tk_[i_].s == s; }
  bool take(const char *s) {
    if (!at(s)) return false;
    i_++;
    return true;
  }
  void punct(const char *s) {
    if (!take(s)) fail(std::string("expected '") + s + "'");
  }
  void word(const char *s) {
    if (!at_word(s)) fail(std::string("expected '") + s + "'");
    i_++;
  }
  std::string name() {
    if (tk_[i_].kind != Token::NAME) fail("expected a name");
    if (reserved().count(tk_[i_].s)) fail("'" + tk_[i_].s + "' is reserved");
    return tk_[i_++].s;
  }
  uint64_t number() {
    if (tk_[i_].kind != Token::NUM) fail("expected a number");
    return tk_[i_++].num;
  }

  void declaration() {
    MemDecl m;
    if (at_word("global")) m.space = 0;
    else if (at_word("local")) m.space = 1;
    else fail("expected 'global' or 'local'");
    i_++;
    word("int");
    m.name = name();
    if (mems_.count(m.name)) fail("'" + m.name + "' declared twice");
    m.decl_len = m.space == 0 ? -1 : 1;
    if (take("[")) {
      if (m.space == 0) {
        if (!at("]")) fail("a global array takes its length from the input");
      } else {
        m.decl_len = (int64_t)number();
      }
      punct("]");
    }
    if (m.space == 0) p_.n_global++;
    mems_[m.name] = (int)p_.mems.size();
    p_.mems.push_back(m);
  }

  // every name in the body that is not reserved and not a memory object is
  // a private variable (implicitly declared, initially 0)
  static int builtin_reg(Op op) {
    switch (op) {
      case OP_TID: return REG_TID;
      case OP_WG: return REG_WG;
      case OP_GTID: return REG_GTID;
      case OP_GSIZE: return REG_GSIZE;
      default: return REG_NGROUPS;
    }
  }

  void collect_vars() {
    for (size_t j = i_; j < tk_.size(); j++) {
      const Token &t = tk_[j];
      if (t.kind != Token::NAME || reserved().count(t.s) || mems_.count(t.s)) continue;
      if (!vars_.count(t.s)) {
        int r = kBuiltinRegs + (int)vars_.size();
        vars_[t.s] = r;
      }
    }
    next_tmp_ = kBuiltinRegs + (int)vars_.size();
    max_reg_ = next_tmp_;
  }

  int tmp() {
    int r = next_tmp_++;
    max_reg_ = std::max(max_reg_, next_tmp_);
    return r;
  }
  bool is_tmp(int r) const { return r >= kBuiltinRegs + (int)vars_.size(); }
  void release(int r) {
    if (is_tmp(r) && r == next_tmp_ - 1) next_tmp_--;
  }

  int emit(Op op, int d, int a, int b, int32_t imm, int32_t imm2 = 0) {
    Insn in{(uint8_t)op, (uint8_t)d, (uint8_t)a, (uint8_t)b, imm, imm2, 0};
    p_.code.push_back(in);
    return (int)p_.code.size() - 1;
  }
  int here() const { return (int)p_.code.size(); }

  // ---- expression parsing (precedence climbing, C-like levels)
  ExP leaf(Ex::K k) {
    ExP e(new Ex());
    e->k = k;
    return e;
  }
  ExP bin(Op op, ExP l, ExP r) {
    ExP e = leaf(Ex::BIN);
    e->op = op;
    e->l = std::move(l);
    e->r = std::move(r);
    return e;
  }
  ExP expr() { return lor(); }
  ExP lor() {
    ExP l = land();
    while (take("||")) l = bin(OP_LOR, std::move(l), land());
    return l;
  }
  ExP land() {
    ExP l = equality();
    while (take("&&")) l = bin(OP_LAND, std::move(l), equality());
    return l;
  }
  ExP equality() {
    ExP l = relation();
    for (;;) {
      if (take("==")) l = bin(OP_EQ, std::move(l), relation());
      else if (take("!=")) l = bin(OP_NE, std::move(l), relation());
      else return l;
    }
  }
  ExP relation() {
    ExP l = additive();
    for (;;) {
      if (take("<")) l = bin(OP_LT, std::move(l), additive());
      else if (take("<=")) l = bin(OP_LE, std::move(l), additive());
      else if (take(">")) l = bin(OP_GT, std::move(l), additive());
      else if (take(">=")) l = bin(OP_GE, std::move(l), additive());
      else return l;
    }
  }
  ExP additive() {
    ExP l = term();
    for (;;) {
      if (take("+")) l = bin(OP_ADD, std::move(l), term());
      else if (take("-")) l = bin(OP_SUB, std::move(l), term());
      else return l;
    }
  }
  ExP term() {
    ExP l = unary();
    for (;;) {
      if (take("*")) l = bin(OP_MUL, std::move(l), unary());
      else if (take("/")) l = bin(OP_DIV, std::move(l), unary());
      else if (take("%")) l = bin(OP_MOD, std::move(l), unary());
      else return l;
    }
  }
  ExP unary() {
    if (take("-")) {
      ExP a = unary();
      if (a->k == Ex::CONST) {  // literal negation: -c is the constant 0 - c
        a->c = (int32_t)(0u - (uint32_t)a->c);
        return a;
      }
      ExP e = leaf(Ex::UN);
      e->op = OP_NEG;
      e->l = std::move(a);
      return e;
    }
    if (take("!")) {
      ExP e = leaf(Ex::UN);
      e->op = OP_NOT;
      e->l = unary();
      return e;
    }
    return primary();
  }
  ExP primary() {
    if (tk_[i_].kind == Token::NUM) {
      ExP e = leaf(Ex::CONST);
      e->c = (int32_t)(uint32_t)number();
      return e;
    }
    if (take("(")) {
      ExP e = expr();
      punct(")");
      return e;
    }
    static const std::pair<const char *, Op> builtins[] = {
        {"tid", OP_TID}, {"wg", OP_WG}, {"gtid", OP_GTID}, {"gsize", OP_GSIZE}, {"ngroups", OP_NGROUPS}};
    for (auto &b : builtins) {
      if (at_word(b.first)) {
        i_++;
        ExP e = leaf(Ex::BUILTIN);
        e->op = b.second;
        return e;
      }
    }
    if (at_word("size")) {
      i_++;
      punct("(");
      std::string n = name();
      auto m = mems_.find(n);
      if (m == mems_.end()) fail("size() of an undeclared array");
      punct(")");
      ExP e = leaf(Ex::SIZE);
      e->mem = m->second;
      return e;
    }
    std::string n = name();
    auto m = mems_.find(n);
    if (m != mems_.end()) {
      ExP e = leaf(Ex::LOAD);
      e->mem = m->second;
      if (take("[")) {
        e->l = expr();
        punct("]");
      } else {
        e->l = leaf(Ex::CONST);
      }
      return e;
    }
    if (at("[")) fail("'" + n + "' is not an array");
    ExP e = leaf(Ex::VAR);
    e->reg = vars_.at(n);
    return e;
  }

  // ---- expression code generation; returns the register holding the value.
  // dst >= 0 forces the result into dst (only the outermost operation writes it).
  static bool imm_form(Op op, Op &iop, bool swapped) {
    switch (op) {
      case OP_ADD: iop = OP_ADDI; return true;
      case OP_MUL: iop = OP_MULI; return true;
      case OP_SUB: iop = swapped ? OP_RSUBI : OP_ADDI; return true;  // a - c == a + (-c) mod 2^32
      case OP_DIV: if (swapped) return false; iop = OP_DIVI; return true;
      case OP_MOD: if (swapped) return false; iop = OP_MODI; return true;
      case OP_LT: iop = swapped ? OP_GTI : OP_LTI; return true;
      case OP_LE: iop = swapped ? OP_GEI : OP_LEI; return true;
      case OP_GT: iop = swapped ? OP_LTI : OP_GTI; return true;
      case OP_GE: iop = swapped ? OP_LEI : OP_GEI; return true;
      case OP_EQ: iop = OP_EQI; return true;
      case OP_NE: iop = OP_NEI; return true;
      default: return false;
    }
  }

  // Index of a shared access.  Constants around the index fold into the
  // LD/ST operands: `e + c` gives index = REG + c, and `c2 + (e + c1) % 2^k`
  // gives index = ((REG + c1) & (2^k - 1)) + c2 (the Euclidean modulus by a
  // power of two is that mask); the folded forms wrap exactly as the
  // expression does.
  struct Index {
    int32_t c1 = 0, c2 = 0;
    bool am = false;
    uint32_t k = 0;
    uint32_t ctl(uint32_t mem) const {
      return (am ? (CTL_AM | (k << CTL_K_SHIFT)) : 0u) | (mem << CTL_MEM_SHIFT);
    }
  };
  static bool split_const(const Ex *e, const Ex *&rest, int32_t &c) {
    if (e->k != Ex::BIN) return false;
    if (e->op == OP_ADD && e->r->k == Ex::CONST) { rest = e->l.get(); c = e->r->c; return true; }
    if (e->op == OP_ADD && e->l->k == Ex::CONST) { rest = e->r.get(); c = e->l->c; return true; }
    if (e->op == OP_SUB && e->r->k == Ex::CONST) {
      rest = e->l.get();
      c = (int32_t)(0u - (uint32_t)e->r->c);
      return true;
    }
    return false;
  }
  static bool pow2_mod(const Ex *e, uint32_t &k) {
    if (e->k != Ex::BIN || e->op != OP_MOD || e->r->k != Ex::CONST) return false;
    const uint32_t m = e->r->c < 0 ? 0u - (uint32_t)e->r->c : (uint32_t)e->r->c;
    if (m == 0 || (m & (m - 1)) != 0) return false;
    k = 0;
    while ((1u << k) != m) k++;
    return true;
  }
  int gen_index(const Ex *e, Index &ix) {
    ix = Index();
    const Ex *inner = e;
    int32_t c2 = 0;
    if (!split_const(e, inner, c2)) {
      inner = e;
      c2 = 0;
    }
    uint32_t k = 0;
    if (pow2_mod(inner, k)) {
      ix.am = true;
      ix.k = k;
      ix.c2 = c2;
      const Ex *base = inner->l.get();
      int32_t c1 = 0;
      if (!split_const(base, base, c1)) c1 = 0;
      ix.c1 = c1;
      return gen(base, -1);
    }
    ix.c1 = c2;
    return gen(inner, -1);
  }

  static bool is_mul_const(const Ex *e) {
    return e->k == Ex::BIN && e->op == OP_MUL && (e->r->k == Ex::CONST || e->l->k == Ex::CONST);
  }

  // Emit a branch taken when condition c is false; returns its index (the
  // caller patches imm2).  A comparison with a constant becomes one fused
  // compare-and-branch instruction.
  int branch_if_false(const Ex *c) {
    static const Op cmp[] = {OP_LT, OP_LE, OP_GT, OP_GE, OP_EQ, OP_NE};
    static const Op bf[] = {OP_BFLTI, OP_BFLEI, OP_BFGTI, OP_BFGEI, OP_BFEQI, OP_BFNEI};
    static const Op mirror[] = {OP_BFGTI, OP_BFGEI, OP_BFLTI, OP_BFLEI, OP_BFEQI, OP_BFNEI};
    if (c->k == Ex::BIN) {
      for (int k = 0; k < 6; k++) {
        if (c->op != cmp[k]) continue;
        if (c->r->k == Ex::CONST) {
          int ra = gen(c->l.get(), -1);
          release(ra);
          return emit(bf[k], 0, ra, 0, c->r->c);
        }
        if (c->l->k == Ex::CONST) {
          int rb = gen(c->r.get(), -1);
          release(rb);
          return emit(mirror[k], 0, rb, 0, c->l->c);
        }
      }
    }
    int r = gen(c, -1);
    release(r);
    return emit(OP_BZ, 0, r, 0, 0);
  }

  int gen(const Ex *e, int dst) {
    switch (e->k) {
      case Ex::CONST: {
        int d = dst >= 0 ? dst : tmp();
        emit(OP_MOVI, d, 0, 0, e->c);
        return d;
      }
      case Ex::VAR:
        if (dst >= 0 && dst != e->reg) {
          emit(OP_MOV, dst, e->reg, 0, 0);
          return dst;
        }
        return e->reg;
      case Ex::BUILTIN: {  // built-ins live in the fixed registers 0..kBuiltinRegs-1
        const int r = builtin_reg(e->op);
        if (dst >= 0 && dst != r) {
          emit(OP_MOV, dst, r, 0, 0);
          return dst;
        }
        return r;
      }
      case Ex::SIZE: {
        int d = dst >= 0 ? dst : tmp();
        int k = emit(OP_SIZE, d, 0, 0, 0, 0);
        p_.code[k].ctl = (uint32_t)e->mem << CTL_MEM_SHIFT;
        return d;
      }
      case Ex::LOAD: {
        Index ix;
        int ri = gen_index(e->l.get(), ix);
        release(ri);
        int d = dst >= 0 ? dst : tmp();
        int k = emit(OP_LD, d, ri, 0, ix.c1, ix.c2);
        p_.code[k].ctl = ix.ctl((uint32_t)e->mem);
        return d;
      }
      case Ex::UN: {
        int ra = gen(e->l.get(), -1);
        release(ra);
        int d = dst >= 0 ? dst : tmp();
        emit(e->op, d, ra, 0, 0);
        return d;
      }
      case Ex::BIN: {
        Op iop;
        // constant right operand (or constant left operand of a commutable op)
        if (e->r->k == Ex::CONST && imm_form(e->op, iop, false)) {
          int ra = gen(e->l.get(), -1);
          release(ra);
          int d = dst >= 0 ? dst : tmp();
          int32_t c = e->r->c;
          if (e->op == OP_SUB) c = (int32_t)(0u - (uint32_t)c);
          uint32_t m = c < 0 ? 0u - (uint32_t)c : (uint32_t)c;  // |c| (2^31 for INT_MIN)
          if (e->op == OP_MOD && m != 0 && (m & (m - 1)) == 0) {
            emit(OP_ANDI, d, ra, 0, (int32_t)(m - 1));  // Euclidean a mod 2^k == a & (2^k - 1)
          } else {
            emit(iop, d, ra, 0, c);
          }
          return d;
        }
        if (e->l->k == Ex::CONST && imm_form(e->op, iop, true)) {
          int rb = gen(e->r.get(), -1);
          release(rb);
          int d = dst >= 0 ? dst : tmp();
          emit(iop, d, rb, 0, e->l->c);
          return d;
        }
        if (e->op == OP_ADD) {  // e1 * c + e2 and e2 + e1 * c: one multiply-add
          const Ex *mul = nullptr, *other = nullptr;
          bool mul_first = false;
          if (is_mul_const(e->l.get())) { mul = e->l.get(); other = e->r.get(); mul_first = true; }
          else if (is_mul_const(e->r.get())) { mul = e->r.get(); other = e->l.get(); }
          if (mul) {
            const Ex *factor = mul->r->k == Ex::CONST ? mul->l.get() : mul->r.get();
            const int32_t c = mul->r->k == Ex::CONST ? mul->r->c : mul->l->c;
            int rx, ry;
            if (mul_first) { rx = gen(factor, -1); ry = gen(other, -1); }
            else { ry = gen(other, -1); rx = gen(factor, -1); }
            release(mul_first ? ry : rx);
            release(mul_first ? rx : ry);
            int d = dst >= 0 ? dst : tmp();
            emit(OP_MADI, d, rx, ry, c);
            return d;
          }
        }
        int ra = gen(e->l.get(), -1);
        int rb = gen(e->r.get(), -1);
        release(rb);
        release(ra);
        int d = dst >= 0 ? dst : tmp();
        emit(e->op, d, ra, rb, 0);
        return d;
      }
    }
    fail("internal: bad expression");
  }

  // ---- statements; each returns its access / write bounds
  void block(Bound &acc, Bound &wr) {
    punct("{");
    acc = Bound();
    wr = Bound();
    while (!at("}")) {
      if (tk_[i_].kind == Token::END) fail("missing '}'");
      Bound a, w;
      statement(a, w);
      acc = seq(acc, a);
      wr = seq(wr, w);
    }
    punct("}");
  }

  void body(Bound &acc, Bound &wr) {
    if (at("{")) block(acc, wr);
    else statement(acc, wr);
  }

  void statement(Bound &acc, Bound &wr) {
    acc = Bound();
    wr = Bound();
    if (at_word("barrier")) {
      i_++;
      punct(";");
      emit(OP_BARRIER, 0, 0, 0, (int32_t)p_.n_barriers++);
      acc = Bound::barrier();
      wr = Bound::barrier();
      return;
    }
    if (at_word("assume") || at_word("assert")) {
      bool is_assert = at_word("assert");
      i_++;
      punct("(");
      ExP c = expr();
      punct(")");
      punct(";");
      int r = gen(c.get(), -1);
      release(r);
      if (is_assert) emit(OP_ASSERT, 0, r, 0, (int32_t)p_.n_asserts++);
      else emit(OP_ASSUME, 0, r, 0, 0);
      acc = Bound::accesses(count_loads(c.get()));
      return;
    }
    if (at_word("if")) {
      i_++;
      punct("(");
      ExP c = expr();
      punct(")");
      int bz = branch_if_false(c.get());
      Bound ta, tw, ea, ew;
      body(ta, tw);
      if (at_word("else")) {
        i_++;
        int j = emit(OP_JMP, 0, 0, 0, 0);
        p_.code[bz].imm2 = here();
        body(ea, ew);
        p_.code[j].imm2 = here();
      } else {
        p_.code[bz].imm2 = here();
      }
      acc = seq(Bound::accesses(count_loads(c.get())), alt(ta, ea));
      wr = alt(tw, ew);
      return;
    }
    if (at_word("for")) {
      i_++;
      std::string v = name();
      if (mems_.count(v)) fail("a loop variable cannot be a memory object");
      int reg = vars_.at(v);
      for (int l : loops_)
        if (l == reg) fail("nested loop reuses '" + v + "'");
      word("in");
      bool nlo = take("-");
      int32_t lo = (int32_t)(uint32_t)number();
      if (nlo) lo = (int32_t)(0u - (uint32_t)lo);
      punct("..");
      bool nhi = take("-");
      int32_t hi = (int32_t)(uint32_t)number();
      if (nhi) hi = (int32_t)(0u - (uint32_t)hi);
      // v := lo; if !(v < hi) skip; body; v := v + 1; if (v < hi) repeat
      emit(OP_MOVI, reg, 0, 0, lo);
      int bz = emit(OP_BFLTI, 0, reg, 0, hi);
      int body_pc = here();
      loops_.push_back(reg);
      Bound ba, bw;
      block(ba, bw);
      loops_.pop_back();
      emit(OP_LOOP, reg, reg, 0, hi, body_pc);
      p_.code[bz].imm2 = here();
      int64_t trips = std::max<int64_t>(0, (int64_t)hi - (int64_t)lo);
      acc = loop(ba, trips);
      wr = loop(bw, trips);
      return;
    }
    if (at("{")) {
      block(acc, wr);
      return;
    }
    std::string n = name();
    auto m = mems_.find(n);
    if (m != mems_.end()) {  // store: index, then value, then the write
      ExP idx;
      if (take("[")) {
        idx = expr();
        punct("]");
      } else {
        idx = leaf(Ex::CONST);
      }
      punct("=");
      ExP val = expr();
      punct(";");
      Index ix;
      int ri = gen_index(idx.get(), ix);
      int rv = gen(val.get(), -1);
      release(rv);
      release(ri);
      int k = emit(OP_ST, 0, ri, rv, ix.c1, ix.c2);
      p_.code[k].ctl = ix.ctl((uint32_t)m->second);
      acc = Bound::accesses(count_loads(idx.get()) + count_loads(val.get()) + 1);
      wr = Bound::accesses(1);
      return;
    }
    if (at("[")) fail("'" + n + "' is not an array");
    int reg = vars_.at(n);
    for (int l : loops_)
      if (l == reg) fail("assignment to loop variable '" + n + "'");
    punct("=");
    ExP val = expr();
    punct(";");
    gen(val.get(), reg);
    acc = Bound::accesses(count_loads(val.get()));
  }
};

}  // namespace

bool predecode(const Insn &in, uint32_t &ctl) {
  enum : uint32_t { P0 = 0, P1 = 1u << AL_P_SHIFT, PM = 2u << AL_P_SHIFT, Q1 = 1u << AL_Q_SHIFT,
                    QM = 2u << AL_Q_SHIFT, W = AL_WRITE, COND = 1u << AL_MODE_SHIFT,
                    ALWAYS = 2u << AL_MODE_SHIFT };
  const uint32_t LTc = AL_CMP | AL_LT, EQc = AL_CMP | AL_EQ, I = AL_INV, Y = AL_YIMM;
  auto cls = [](CtlClass c, uint32_t extra = 0) { return extra | ((uint32_t)c << CTL_CLASS_SHIFT); };
  switch (in.op) {
    case OP_NOP: ctl = 0; return in.imm == 0;                       // arith = 0, not written
    case OP_MOVI: ctl = W; return true;                              // C = imm
    case OP_MOV: ctl = P1 | W; return in.imm == 0;                   // x
    case OP_ADD: ctl = P1 | Q1 | W; return in.imm == 0;
    case OP_SUB: ctl = P1 | QM | W; return in.imm == 0;
    case OP_MUL: ctl = AL_M | W; return in.imm == 0;
    case OP_ADDI: ctl = P1 | W; return true;                         // x + imm
    case OP_MULI: ctl = AL_PIMM | W; return true;                    // imm * x
    case OP_ANDI: ctl = P1 | AL_MASKIMM | W; return true;            // x & imm
    case OP_RSUBI: ctl = PM | W; return true;                        // -x + imm
    case OP_MADI: ctl = AL_PIMM | Q1 | W; return true;               // imm * x + yr
    case OP_NEG: ctl = PM | W; return in.imm == 0;
    case OP_LT: ctl = LTc | W; return true;
    case OP_LE: ctl = LTc | AL_EQ | W; return true;
    case OP_GT: ctl = LTc | AL_EQ | I | W; return true;
    case OP_GE: ctl = LTc | I | W; return true;
    case OP_EQ: ctl = EQc | W; return true;
    case OP_NE: ctl = EQc | I | W; return true;
    case OP_LTI: ctl = LTc | Y | W; return true;
    case OP_LEI: ctl = LTc | AL_EQ | Y | W; return true;
    case OP_GTI: ctl = LTc | AL_EQ | I | Y | W; return true;
    case OP_GEI: ctl = LTc | I | Y | W; return true;
    case OP_EQI: ctl = EQc | Y | W; return true;
    case OP_NEI: ctl = EQc | I | Y | W; return true;
    case OP_NOT: ctl = EQc | Y | W; return in.imm == 0;              // x == 0
    case OP_JMP: ctl = ALWAYS; return true;
    case OP_BZ: ctl = EQc | Y | COND; return in.imm == 0;             // taken if x == 0
    case OP_BFLTI: ctl = LTc | I | Y | COND; return true;             // taken if !(x < imm)
    case OP_BFLEI: ctl = LTc | AL_EQ | I | Y | COND; return true;     // taken if !(x <= imm)
    case OP_BFGTI: ctl = LTc | AL_EQ | Y | COND; return true;         // taken if !(x > imm)
    case OP_BFGEI: ctl = LTc | Y | COND; return true;                 // taken if !(x >= imm)
    case OP_BFEQI: ctl = EQc | I | Y | COND; return true;             // taken if !(x == imm)
    case OP_BFNEI: ctl = EQc | Y | COND; return true;                 // taken if !(x != imm)
    case OP_LOOP: ctl = P1 | AL_CONE | W | COND | AL_LOOPCOND; return in.d == in.a;  // d = a + 1; taken if d < imm
    case OP_LAND: ctl = cls(CC_LOGIC, 0); return true;
    case OP_LOR: ctl = cls(CC_LOGIC, 1); return true;
    case OP_DIV: ctl = cls(CC_DIVMOD, 0); return true;
    case OP_MOD: ctl = cls(CC_DIVMOD, DM_MOD); return true;
    case OP_DIVI: ctl = cls(CC_DIVMOD, DM_YIMM); return true;
    case OP_MODI: ctl = cls(CC_DIVMOD, DM_MOD | DM_YIMM); return true;
    case OP_SIZE: ctl = cls(CC_SIZE); return true;
    case OP_LD: ctl = cls(CC_LD); return true;
    case OP_ST: ctl = cls(CC_ST); return true;
    case OP_ASSUME: ctl = cls(CC_ASSUME); return true;
    case OP_ASSERT: ctl = cls(CC_ASSERT); return true;
    case OP_BARRIER: ctl = cls(CC_BARRIER); return true;
    case OP_EXIT: ctl = cls(CC_EXIT); return true;
    default: return false;  // built-in opcodes are registers now; anything else is invalid
  }
}

uint32_t operand_bits(const Insn &in) {
  if (in.op == OP_LD || in.op == OP_ST) return CTL_AM | (0x1Fu << CTL_K_SHIFT) | (0xFFu << CTL_MEM_SHIFT);
  if (in.op == OP_SIZE) return 0xFFu << CTL_MEM_SHIFT;
  return 0;
}

Program compile_program(const std::string &src) {
  Compiler c(src);
  Program p = c.run();
  for (Insn &in : p.code) {
    uint32_t base = 0;
    if (!predecode(in, base)) throw CompileError{"internal: cannot decode an emitted instruction"};
    in.ctl = base | (in.ctl & operand_bits(in));
  }
  std::string err = validate_program(p);
  if (!err.empty()) throw CompileError{"internal: " + err};
  return p;
}

std::string validate_program(const Program &p) {
  if (p.code.empty() || p.code.back().op != OP_EXIT) return "program must end with EXIT";
  if (p.n_regs == 0 || p.n_regs > 255) return "bad register count";
  if (p.code.size() > (1u << 20)) return "program longer than 2^20 instructions";
  const int n = (int)p.code.size();
  for (int k = 0; k < n; k++) {
    const Insn &in = p.code[k];
    uint32_t ctl = 0;
    if (in.op >= OP_COUNT || !predecode(in, ctl)) return "bad opcode at " + std::to_string(k);
    if (ctl != (in.ctl & ~operand_bits(in))) return "bad control word at " + std::to_string(k);
    const bool uses_mem = in.op == OP_LD || in.op == OP_ST || in.op == OP_SIZE;
    if (uses_mem && (in.ctl >> CTL_MEM_SHIFT) >= p.mems.size()) return "bad memory id at " + std::to_string(k);
    if (in.d >= p.n_regs || in.a >= p.n_regs || in.b >= p.n_regs) return "bad register at " + std::to_string(k);
    switch (in.op) {
      case OP_JMP:
      case OP_BZ:
      case OP_BFLTI: case OP_BFLEI: case OP_BFGTI: case OP_BFGEI: case OP_BFEQI: case OP_BFNEI:
      case OP_LOOP:
        if (in.imm2 < 0 || in.imm2 >= n) return "bad jump target at " + std::to_string(k);
        break;

      case OP_BARRIER:
        if (in.imm < 0 || (uint32_t)in.imm >= p.n_barriers) return "bad barrier id at " + std::to_string(k);
        break;
      case OP_ASSERT:
        if (in.imm < 0 || (uint32_t)in.imm >= p.n_asserts) return "bad assert id at " + std::to_string(k);
        break;
      default:
        break;
    }
  }
  if (p.mems.size() > 256) return "more than 256 memory objects";
  for (const MemDecl &m : p.mems) {
    if (m.space > 1) return "bad memory space";
    if (m.space == 1 && (m.decl_len < 0 || m.decl_len > (1 << 24))) return "bad local length";
  }
  return "";
}

}  // namespace rc
