// Kernel-language front end of the ORACLE (test infrastructure only).
//
// This file, oracle.cpp and explore.cpp form the sequential CPU reference
// checker.  Only the test suite, __graft_entry__.smoke() and bench.py's CPU
// baseline leg may build or call it.  It shares no code with the GPU path in
// paper_1308_3203_gb300/ (which has its own lexer, parser and bytecode
// compiler): a bug in one cannot hide in the other.
//
// Language (Distefano & Dubreil, Sec. 3, the grammar of expressions e,
// booleans b and commands Comm, plus the kernel tuple K(Args)):
//   e    ::= c | v | op(e..) | tid | size(v)      (+ wg, gtid, gsize, ngroups)
//   b    ::= e<e | e=e | b&&b | !b               (C-like comparison set)
//   Comm ::= v:=e | a[v]:=e | v:=a[v] | barrier | assume(b) | assert(b)
// Surface syntax adds `if/else` and constant-trip `for v in lo .. hi` which
// lower to assume-guarded CFG edges exactly as Sec. 3 presents a kernel: a
// control-flow graph of command nodes with unique start and exit nodes.
// Array reads that appear inside expressions (Fig. 1, Fig. 2) are lowered to
// one `v := a[e]` command each, left to right, before the command that uses
// them, so every CFG node performs at most one shared access.
#pragma once
#include <cctype>
#include <cstdint>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

namespace orc {

struct ParseError : std::runtime_error {
  explicit ParseError(const std::string &m) : std::runtime_error(m) {}
};

// ---------------------------------------------------------------- lexer
enum TokKind { T_EOF, T_INT, T_ID, T_SYM };
struct Tok {
  TokKind kind;
  std::string text;
  uint64_t ival;
  int line;
};

static std::vector<Tok> lex(const std::string &src) {
  std::vector<Tok> out;
  size_t i = 0;
  int line = 1;
  while (i < src.size()) {
    char c = src[i];
    if (c == '\n') { line++; i++; continue; }
    if (isspace((unsigned char)c)) { i++; continue; }
    if (c == '/' && i + 1 < src.size() && src[i + 1] == '/') {
      while (i < src.size() && src[i] != '\n') i++;
      continue;
    }
    if (isdigit((unsigned char)c)) {
      uint64_t v = 0;
      size_t j = i;
      while (j < src.size() && isdigit((unsigned char)src[j])) {
        v = v * 10 + (uint64_t)(src[j] - '0');
        if (v > 0xFFFFFFFFull) throw ParseError("integer literal too large at line " + std::to_string(line));
        j++;
      }
      out.push_back({T_INT, src.substr(i, j - i), v, line});
      i = j;
      continue;
    }
    if (isalpha((unsigned char)c) || c == '_') {
      size_t j = i;
      while (j < src.size() && (isalnum((unsigned char)src[j]) || src[j] == '_')) j++;
      out.push_back({T_ID, src.substr(i, j - i), 0, line});
      i = j;
      continue;
    }
    static const char *two[] = {"<=", ">=", "==", "!=", "&&", "||", ".."};
    bool matched = false;
    for (const char *t : two) {
      if (src.compare(i, 2, t) == 0) {
        out.push_back({T_SYM, t, 0, line});
        i += 2;
        matched = true;
        break;
      }
    }
    if (matched) continue;
    if (std::string("+-*/%<>=!(){}[];,").find(c) != std::string::npos) {
      out.push_back({T_SYM, std::string(1, c), 0, line});
      i++;
      continue;
    }
    throw ParseError(std::string("unexpected character '") + c + "' at line " + std::to_string(line));
  }
  out.push_back({T_EOF, "", 0, line});
  return out;
}

// ---------------------------------------------------------------- AST
enum ExprKind {
  E_CONST, E_VAR, E_LOAD, E_TID, E_WG, E_GTID, E_GSIZE, E_NGROUPS, E_SIZE,
  E_NEG, E_NOT, E_ADD, E_SUB, E_MUL, E_DIV, E_MOD, E_LT, E_LE, E_GT, E_GE,
  E_EQ, E_NE, E_AND, E_OR
};
struct Expr {
  ExprKind kind;
  int32_t value = 0;  // E_CONST
  int var = -1;       // E_VAR: private variable index
  int mem = -1;       // E_LOAD / E_SIZE: memory object index
  std::shared_ptr<Expr> a, b;
};
using ExprP = std::shared_ptr<Expr>;

enum StmtKind { S_ASSIGN, S_STORE, S_BARRIER, S_ASSUME, S_ASSERT, S_IF, S_FOR, S_BLOCK };
struct Stmt {
  StmtKind kind;
  int var = -1;                 // S_ASSIGN target, S_FOR loop variable
  int mem = -1;                 // S_STORE target memory object
  ExprP idx, val;               // S_STORE index/value, S_ASSIGN value, S_IF/ASSUME/ASSERT condition in val
  int32_t lo = 0, hi = 0;       // S_FOR bounds
  int id = -1;                  // barrier ordinal / assert ordinal (source order)
  std::vector<std::shared_ptr<Stmt>> body, els;
};
using StmtP = std::shared_ptr<Stmt>;

struct Mem {
  std::string name;
  int space;         // 0 = global, 1 = local (per work-group)
  int64_t decl_len;  // local: declared length; global: -1 (from the input)
};

struct Program {
  std::string name;
  std::vector<Mem> mems;
  std::vector<std::string> vars;  // private variables (implicitly declared)
  std::vector<StmtP> body;
  int n_barriers = 0, n_asserts = 0;
};

// ---------------------------------------------------------------- parser
class Parser {
 public:
  explicit Parser(const std::string &src) : toks_(lex(src)) {}

  Program parse() {
    expect_id("kernel");
    prog_.name = ident();
    expect("(");
    if (!is(")")) {
      do decl(); while (accept(","));
    }
    expect(")");
    prog_.body = block();
    if (peek().kind != T_EOF) fail("trailing text after kernel body");
    return prog_;
  }

 private:
  std::vector<Tok> toks_;
  size_t p_ = 0;
  Program prog_;
  std::map<std::string, int> memidx_, varidx_;
  std::vector<int> active_loops_;

  const Tok &peek() const { return toks_[p_]; }
  [[noreturn]] void fail(const std::string &m) const {
    throw ParseError(m + " at line " + std::to_string(peek().line));
  }
  bool is(const char *s) const { return peek().kind == T_SYM && peek().text == s; }
  bool is_id(const char *s) const { return peek().kind == T_ID && peek().text == s; }
  bool accept(const char *s) {
    if (is(s)) { p_++; return true; }
    return false;
  }
  void expect(const char *s) {
    if (!accept(s)) fail(std::string("expected '") + s + "'");
  }
  void expect_id(const char *s) {
    if (!is_id(s)) fail(std::string("expected '") + s + "'");
    p_++;
  }
  static bool keyword(const std::string &s) {
    static const char *kw[] = {"kernel", "global", "local", "int", "barrier", "assume", "assert",
                               "if", "else", "for", "in", "tid", "wg", "gtid", "gsize",
                               "ngroups", "size"};
    for (const char *k : kw)
      if (s == k) return true;
    return false;
  }
  std::string ident() {
    if (peek().kind != T_ID) fail("expected identifier");
    std::string s = peek().text;
    if (keyword(s)) fail("keyword '" + s + "' used as identifier");
    p_++;
    return s;
  }
  uint64_t intlit() {
    if (peek().kind != T_INT) fail("expected integer literal");
    return toks_[p_++].ival;
  }
  int32_t signed_int() {
    bool neg = accept("-");
    uint64_t v = intlit();
    uint32_t u = (uint32_t)v;
    if (neg) u = 0u - u;
    return (int32_t)u;
  }

  void decl() {
    int space;
    if (is_id("global")) space = 0;
    else if (is_id("local")) space = 1;
    else fail("expected 'global' or 'local'");
    p_++;
    expect_id("int");
    std::string name = ident();
    if (memidx_.count(name)) fail("duplicate declaration of '" + name + "'");
    int64_t len = space == 0 ? -1 : 1;
    if (accept("[")) {
      if (space == 0) {
        if (!is("]")) fail("global array length comes from the input, not the declaration");
      } else {
        len = (int64_t)intlit();
      }
      expect("]");
    }
    memidx_[name] = (int)prog_.mems.size();
    prog_.mems.push_back({name, space, len});
  }

  int var_index(const std::string &name) {
    auto it = varidx_.find(name);
    if (it != varidx_.end()) return it->second;
    int k = (int)prog_.vars.size();
    varidx_[name] = k;
    prog_.vars.push_back(name);
    return k;
  }

  std::vector<StmtP> block() {
    expect("{");
    std::vector<StmtP> out;
    while (!is("}")) {
      if (peek().kind == T_EOF) fail("unterminated block");
      out.push_back(stmt());
    }
    expect("}");
    return out;
  }

  std::vector<StmtP> stmt_or_block() {
    if (is("{")) return block();
    return {stmt()};
  }

  StmtP stmt() {
    auto s = std::make_shared<Stmt>();
    if (is_id("barrier")) {
      p_++;
      expect(";");
      s->kind = S_BARRIER;
      s->id = prog_.n_barriers++;
      return s;
    }
    if (is_id("assume") || is_id("assert")) {
      bool as = is_id("assert");
      p_++;
      expect("(");
      s->val = expr();
      expect(")");
      expect(";");
      s->kind = as ? S_ASSERT : S_ASSUME;
      if (as) s->id = prog_.n_asserts++;
      return s;
    }
    if (is_id("if")) {
      p_++;
      expect("(");
      s->val = expr();
      expect(")");
      s->kind = S_IF;
      s->body = stmt_or_block();
      if (is_id("else")) {
        p_++;
        s->els = stmt_or_block();
      }
      return s;
    }
    if (is_id("for")) {
      p_++;
      std::string v = ident();
      if (memidx_.count(v)) fail("loop variable '" + v + "' is a memory object");
      s->kind = S_FOR;
      s->var = var_index(v);
      for (int a : active_loops_)
        if (a == s->var) fail("nested loop reuses loop variable '" + v + "'");
      expect_id("in");
      s->lo = signed_int();
      expect("..");
      s->hi = signed_int();
      active_loops_.push_back(s->var);
      s->body = block();
      active_loops_.pop_back();
      return s;
    }
    if (is("{")) {
      s->kind = S_BLOCK;
      s->body = block();
      return s;
    }
    std::string name = ident();
    auto mi = memidx_.find(name);
    if (mi != memidx_.end()) {
      s->kind = S_STORE;
      s->mem = mi->second;
      if (accept("[")) {
        s->idx = expr();
        expect("]");
      } else {
        s->idx = cnst(0);
      }
      expect("=");
      s->val = expr();
      expect(";");
      return s;
    }
    if (is("[")) fail("'" + name + "' is not a declared array");
    s->kind = S_ASSIGN;
    s->var = var_index(name);
    for (int a : active_loops_)
      if (a == s->var) fail("assignment to loop variable '" + name + "'");
    expect("=");
    s->val = expr();
    expect(";");
    return s;
  }

  static ExprP cnst(int32_t v) {
    auto e = std::make_shared<Expr>();
    e->kind = E_CONST;
    e->value = v;
    return e;
  }
  static ExprP bin(ExprKind k, ExprP a, ExprP b) {
    auto e = std::make_shared<Expr>();
    e->kind = k;
    e->a = a;
    e->b = b;
    return e;
  }

  ExprP expr() { return orx(); }
  ExprP orx() {
    ExprP l = andx();
    while (accept("||")) l = bin(E_OR, l, andx());
    return l;
  }
  ExprP andx() {
    ExprP l = eqx();
    while (accept("&&")) l = bin(E_AND, l, eqx());
    return l;
  }
  ExprP eqx() {
    ExprP l = relx();
    for (;;) {
      if (accept("==")) l = bin(E_EQ, l, relx());
      else if (accept("!=")) l = bin(E_NE, l, relx());
      else return l;
    }
  }
  ExprP relx() {
    ExprP l = addx();
    for (;;) {
      if (accept("<=")) l = bin(E_LE, l, addx());
      else if (accept(">=")) l = bin(E_GE, l, addx());
      else if (accept("<")) l = bin(E_LT, l, addx());
      else if (accept(">")) l = bin(E_GT, l, addx());
      else return l;
    }
  }
  ExprP addx() {
    ExprP l = mulx();
    for (;;) {
      if (accept("+")) l = bin(E_ADD, l, mulx());
      else if (accept("-")) l = bin(E_SUB, l, mulx());
      else return l;
    }
  }
  ExprP mulx() {
    ExprP l = unary();
    for (;;) {
      if (accept("*")) l = bin(E_MUL, l, unary());
      else if (accept("/")) l = bin(E_DIV, l, unary());
      else if (accept("%")) l = bin(E_MOD, l, unary());
      else return l;
    }
  }
  ExprP unary() {
    if (accept("-")) return bin(E_NEG, unary(), nullptr);
    if (accept("!")) return bin(E_NOT, unary(), nullptr);
    return primary();
  }
  ExprP primary() {
    if (peek().kind == T_INT) return cnst((int32_t)(uint32_t)intlit());
    if (accept("(")) {
      ExprP e = expr();
      expect(")");
      return e;
    }
    auto e = std::make_shared<Expr>();
    static const std::pair<const char *, ExprKind> specials[] = {
        {"tid", E_TID}, {"wg", E_WG}, {"gtid", E_GTID}, {"gsize", E_GSIZE}, {"ngroups", E_NGROUPS}};
    for (auto &sp : specials) {
      if (is_id(sp.first)) {
        p_++;
        e->kind = sp.second;
        return e;
      }
    }
    if (is_id("size")) {
      p_++;
      expect("(");
      std::string n = ident();
      auto mi = memidx_.find(n);
      if (mi == memidx_.end()) fail("size() of undeclared array '" + n + "'");
      expect(")");
      e->kind = E_SIZE;
      e->mem = mi->second;
      return e;
    }
    std::string name = ident();
    auto mi = memidx_.find(name);
    if (mi != memidx_.end()) {
      e->kind = E_LOAD;
      e->mem = mi->second;
      if (accept("[")) {
        e->a = expr();
        expect("]");
      } else {
        e->a = cnst(0);
      }
      return e;
    }
    if (is("[")) fail("'" + name + "' is not a declared array");
    e->kind = E_VAR;
    e->var = var_index(name);
    return e;
  }
};

// ---------------------------------------------------------------- CFG
// One node per command of Comm (Sec. 3) plus START, EXIT and NOP join nodes.
// Expressions held by nodes are load-free: every shared read was lowered to
// its own LOAD node.
enum NodeKind { N_START, N_EXIT, N_NOP, N_ASSIGN, N_LOAD, N_STORE, N_BARRIER, N_ASSUME, N_ASSERT };
struct Node {
  Node(NodeKind k = N_NOP) : kind(k) {}
  NodeKind kind;
  int var = -1;       // ASSIGN / LOAD destination (private variable index)
  int mem = -1;       // LOAD / STORE memory object
  ExprP idx, val;     // LOAD index; STORE index+value; ASSIGN value; ASSUME/ASSERT condition
  int id = -1;        // barrier / assert ordinal
  std::vector<int> succ;
};

struct Cfg {
  std::vector<Node> nodes;
  int start = 0, exit = 1;
  int n_vars = 0;  // private variables incl. temporaries
};

class CfgBuilder {
 public:
  explicit CfgBuilder(const Program &p) : prog_(p) {}

  Cfg build() {
    cfg_.n_vars = (int)prog_.vars.size();
    cfg_.start = add({N_START});
    cfg_.exit = add({N_EXIT});
    int last = lower_list(prog_.body, cfg_.start);
    link(last, cfg_.exit);
    return cfg_;
  }

 private:
  const Program &prog_;
  Cfg cfg_;

  int add(Node n) {
    cfg_.nodes.push_back(n);
    return (int)cfg_.nodes.size() - 1;
  }
  void link(int from, int to) { cfg_.nodes[from].succ.push_back(to); }
  int fresh_temp() { return cfg_.n_vars++; }

  // Replace every array read in `e` by a fresh temporary, emitting one LOAD
  // node per read in evaluation order (left operand first, an index before
  // the read that uses it).  `cur` is the node the new chain hangs from.
  ExprP lower_loads(const ExprP &e, int &cur) {
    if (!e) return e;
    if (e->kind == E_LOAD) {
      ExprP idx = lower_loads(e->a, cur);
      Node n{N_LOAD};
      n.var = fresh_temp();
      n.mem = e->mem;
      n.idx = idx;
      int k = add(n);
      link(cur, k);
      cur = k;
      auto v = std::make_shared<Expr>();
      v->kind = E_VAR;
      v->var = n.var;
      return v;
    }
    auto c = std::make_shared<Expr>(*e);
    c->a = lower_loads(e->a, cur);
    c->b = lower_loads(e->b, cur);
    return c;
  }

  int lower_list(const std::vector<StmtP> &ss, int cur) {
    for (auto &s : ss) cur = lower_stmt(*s, cur);
    return cur;
  }

  static ExprP negate(const ExprP &b) {
    auto e = std::make_shared<Expr>();
    e->kind = E_NOT;
    e->a = b;
    return e;
  }

  int lower_stmt(const Stmt &s, int cur) {
    switch (s.kind) {
      case S_ASSIGN: {
        ExprP v = lower_loads(s.val, cur);
        Node n{N_ASSIGN};
        n.var = s.var;
        n.val = v;
        int k = add(n);
        link(cur, k);
        return k;
      }
      case S_STORE: {
        ExprP i = lower_loads(s.idx, cur);
        ExprP v = lower_loads(s.val, cur);
        Node n{N_STORE};
        n.mem = s.mem;
        n.idx = i;
        n.val = v;
        int k = add(n);
        link(cur, k);
        return k;
      }
      case S_BARRIER: {
        Node n{N_BARRIER};
        n.id = s.id;
        int k = add(n);
        link(cur, k);
        return k;
      }
      case S_ASSUME:
      case S_ASSERT: {
        ExprP b = lower_loads(s.val, cur);
        Node n{s.kind == S_ASSUME ? N_ASSUME : N_ASSERT};
        n.val = b;
        n.id = s.id;
        int k = add(n);
        link(cur, k);
        return k;
      }
      case S_BLOCK:
        return lower_list(s.body, cur);
      case S_IF: {
        // branch node with two assume-guarded successors (Sec. 3: control
        // flow as a relation between command nodes)
        ExprP b = lower_loads(s.val, cur);
        Node t{N_ASSUME};
        t.val = b;
        Node f{N_ASSUME};
        f.val = negate(b);
        int kt = add(t), kf = add(f);
        link(cur, kt);
        link(cur, kf);
        int endt = lower_list(s.body, kt);
        int endf = lower_list(s.els, kf);
        int join = add({N_NOP});
        link(endt, join);
        link(endf, join);
        return join;
      }
      case S_FOR: {
        // v := lo; head: [assume(v < hi); body; v := v + 1; -> head] | [assume(!(v < hi))]
        auto lo = std::make_shared<Expr>();
        lo->kind = E_CONST;
        lo->value = s.lo;
        Node init{N_ASSIGN};
        init.var = s.var;
        init.val = lo;
        int ki = add(init);
        link(cur, ki);
        int head = add({N_NOP});
        link(ki, head);
        auto vv = std::make_shared<Expr>();
        vv->kind = E_VAR;
        vv->var = s.var;
        auto hi = std::make_shared<Expr>();
        hi->kind = E_CONST;
        hi->value = s.hi;
        auto cond = std::make_shared<Expr>();
        cond->kind = E_LT;
        cond->a = vv;
        cond->b = hi;
        Node t{N_ASSUME};
        t.val = cond;
        Node f{N_ASSUME};
        f.val = negate(cond);
        int kt = add(t), kf = add(f);
        link(head, kt);
        link(head, kf);
        int endb = lower_list(s.body, kt);
        auto one = std::make_shared<Expr>();
        one->kind = E_CONST;
        one->value = 1;
        auto inc = std::make_shared<Expr>();
        inc->kind = E_ADD;
        inc->a = vv;
        inc->b = one;
        Node step{N_ASSIGN};
        step.var = s.var;
        step.val = inc;
        int ks = add(step);
        link(endb, ks);
        link(ks, head);
        return kf;
      }
    }
    throw ParseError("internal: unknown statement");
  }
};

// ---------------------------------------------------------------- arithmetic
// int32 two's-complement wrap; `/` truncates, `%` is Euclidean (result in
// [0, |m|)); division or modulus by zero yields 0; comparisons and logical
// operators yield 0 or 1.
struct Env {
  const int32_t *vars;  // the work-item's private variables
  uint32_t tid, wg, gsize, ngroups;
  const std::vector<int64_t> *mem_len;
};

static int32_t eval(const Expr &e, const Env &env) {
  auto A = [&]() { return eval(*e.a, env); };
  auto B = [&]() { return eval(*e.b, env); };
  switch (e.kind) {
    case E_CONST: return e.value;
    case E_VAR: return env.vars[e.var];
    case E_TID: return (int32_t)env.tid;
    case E_WG: return (int32_t)env.wg;
    case E_GTID: return (int32_t)(uint32_t)((uint64_t)env.wg * env.gsize + env.tid);
    case E_GSIZE: return (int32_t)env.gsize;
    case E_NGROUPS: return (int32_t)env.ngroups;
    case E_SIZE: return (int32_t)(uint32_t)(*env.mem_len)[e.mem];
    case E_NEG: return (int32_t)(0u - (uint32_t)A());
    case E_NOT: return A() == 0 ? 1 : 0;
    case E_ADD: { int32_t x = A(), y = B(); return (int32_t)((uint32_t)x + (uint32_t)y); }
    case E_SUB: { int32_t x = A(), y = B(); return (int32_t)((uint32_t)x - (uint32_t)y); }
    case E_MUL: { int32_t x = A(), y = B(); return (int32_t)((uint32_t)x * (uint32_t)y); }
    case E_DIV: {
      int64_t x = A(), y = B();
      if (y == 0) return 0;
      return (int32_t)(uint32_t)(uint64_t)(x / y);
    }
    case E_MOD: {
      int64_t x = A(), y = B();
      if (y == 0) return 0;
      int64_t m = y < 0 ? -y : y;
      int64_t r = x % m;
      if (r < 0) r += m;
      return (int32_t)r;
    }
    case E_LT: { int32_t x = A(), y = B(); return x < y; }
    case E_LE: { int32_t x = A(), y = B(); return x <= y; }
    case E_GT: { int32_t x = A(), y = B(); return x > y; }
    case E_GE: { int32_t x = A(), y = B(); return x >= y; }
    case E_EQ: { int32_t x = A(), y = B(); return x == y; }
    case E_NE: { int32_t x = A(), y = B(); return x != y; }
    case E_AND: { int32_t x = A(), y = B(); return (x != 0) && (y != 0); }
    case E_OR: { int32_t x = A(), y = B(); return (x != 0) || (y != 0); }
    case E_LOAD: break;
  }
  throw std::runtime_error("internal: load left in a lowered expression");
}

}  // namespace orc
