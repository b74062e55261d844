// Host harness for the kernel text rc_translate writes (test
// infrastructure): the generated functions run on the CPU, one work-item and
// one barrier interval per call, with every load answered from a list of
// values and every access, out-of-bounds access and failed assert written
// to an event list.  RC_JIT_TEXT names a file that holds the generated
// functions and, per function, one extern "C" wrapper (written by the test).
#include <cstdint>

#define __device__
#define __forceinline__ inline
#include "semantics.cuh"

namespace {

struct Ctx {
  const int32_t *load_vals;
  uint32_t n_load_vals, next_load;
  const int64_t *mem_len;
  uint32_t *ev;  // 5 words per event: kind (0 load, 1 store, 2 out of bounds, 3 assert), site, mem, index, value
  uint32_t cap, n_ev;
  int32_t barrier;
};

inline void push(Ctx &cx, uint32_t kind, uint32_t site, uint32_t mem, int32_t idx, int32_t val) {
  if (cx.n_ev < cx.cap) {
    uint32_t *e = cx.ev + 5ull * cx.n_ev;
    e[0] = kind;
    e[1] = site;
    e[2] = mem;
    e[3] = (uint32_t)idx;
    e[4] = (uint32_t)val;
  }
  cx.n_ev++;
}

inline bool in_bounds(const Ctx &cx, uint32_t mem, int32_t idx) { return idx >= 0 && (int64_t)idx < cx.mem_len[mem]; }

inline bool hk_ld(Ctx &cx, uint32_t site, uint32_t mem, int32_t idx, int32_t &out) {
  if (!in_bounds(cx, mem, idx)) {
    push(cx, 2, site, mem, idx, 0);
    return false;
  }
  const int32_t v = cx.next_load < cx.n_load_vals ? cx.load_vals[cx.next_load] : 0;
  cx.next_load++;
  push(cx, 0, site, mem, idx, v);
  out = v;
  return true;
}

inline bool hk_st(Ctx &cx, uint32_t site, uint32_t mem, int32_t idx, int32_t val) {
  if (!in_bounds(cx, mem, idx)) {
    push(cx, 2, site, mem, idx, 0);
    return false;
  }
  push(cx, 1, site, mem, idx, val);
  return true;
}

}  // namespace

#define RC_JIT_FN static
#define RC_JIT_CTX Ctx
#define RC_LD(cx, s, m, i, o) hk_ld(cx, s, m, i, o)
#define RC_ST(cx, s, m, i, v) hk_st(cx, s, m, i, v)
#define RC_SIZE(cx, m) ((int32_t)(uint32_t)(cx).mem_len[m])
#define RC_ASSERT_FAIL(cx, id) push(cx, 3, 0, 0, (id), 0)
#define RC_AT_BARRIER(cx, id) ((cx).barrier = (id))

// one wrapper per generated function:
//   int <name>_run(int32_t *regs, uint32_t *pc, uint32_t *st, const int32_t *load_vals,
//                  uint32_t n_load_vals, const int64_t *mem_len, uint32_t *ev, uint32_t cap,
//                  uint32_t *n_ev, int32_t *barrier)
#define RC_HARNESS_WRAPPER(name, nregs)                                                                       \
  extern "C" int name##_run(int32_t *regs, uint32_t *pc, uint32_t *st, const int32_t *load_vals,              \
                            uint32_t n_load_vals, const int64_t *mem_len, uint32_t *ev, uint32_t cap,         \
                            uint32_t *n_ev, int32_t *barrier) {                                               \
    Ctx cx{load_vals, n_load_vals, 0, mem_len, ev, cap, 0, -1};                                               \
    int32_t r[nregs];                                                                                         \
    for (int k = 0; k < (nregs); k++) r[k] = regs[k];                                                         \
    name(cx, r, *pc, *st);                                                                                    \
    for (int k = 0; k < (nregs); k++) regs[k] = r[k];                                                         \
    *n_ev = cx.n_ev;                                                                                          \
    *barrier = cx.barrier;                                                                                    \
    return cx.next_load == n_load_vals ? 0 : 1;                                                               \
  }

#include RC_JIT_TEXT
