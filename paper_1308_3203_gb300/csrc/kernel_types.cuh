// Device-side data layouts and helpers of the interpreter kernels: access
// log records, report records, the launch arguments of one interval, and the
// shadow owner table's claim and compaction steps.  Compiled into the
// library and, at run time (NVRTC), into the kernels of compiled intervals,
// so it uses no host standard library.
#pragma once
#ifndef __CUDACC_RTC__
#include <cstdint>
#endif

#include "isa.h"

namespace rc {

// One logged shared access (16 bytes, one vector store).
//   key  : flat cell index; global cells first (arrays in declared order),
//          then local cells, work-group major
//   tw   : global work-item id | (is_write << 31)
//   val  : value written, or value the read observed
//   seq  : position of the access in the work-item's interval (program order)
struct __align__(16) LogRec {
  uint32_t key, tw;
  int32_t val;
  uint32_t seq;
};

struct MemInfo {  // per memory object
  uint32_t len, base, space, pad;
};

// Everything one work-item did to one cell in one interval.
struct __align__(16) Summary {
  uint32_t key, gtid;
  int32_t rmin, rmax;   // observed values (reads)
  int32_t wmin, wmax;   // written values
  int32_t wlast;        // value of its last write (highest seq)
  uint32_t meta;        // accesses | has_read << 30 | has_write << 31
};

struct OutRec {  // report record, field order of rc_record
  uint32_t interval, space, wg, addr, cls, t_a, t_b, n_readers, n_writers, n_accesses;
};

constexpr uint32_t kNone = 0xFFFFFFFFu;
// device-side overflow / error flags of a run (InterpArgs::flags)
enum Flag : uint32_t { FLAG_LOG_FULL = 1, FLAG_OW_FULL = 2, FLAG_ERR_FULL = 4, FLAG_ACC_FULL = 16 };
constexpr uint32_t kMetaRead = 1u << 30, kMetaWrite = 1u << 31, kMetaCount = (1u << 30) - 1;

// Interpreter launch arguments (one launch runs one barrier interval for a
// contiguous range of work-groups).
struct InterpArgs {
  const Insn *code;
  const MemInfo *mems;
  uint32_t n_insn, n_regs, n_mems, n_barriers;
  uint32_t S, G, group0;   // block b runs (a part of) work-group group0 + b / split
  uint32_t split;          // CTAs per work-group (0 or 1: one CTA runs the whole group); the
                           // parts are consecutive work-items, blockDim.x = S / split each
  uint32_t GT, LT;         // global cells, local cells per group
  uint32_t interval;
  const int32_t *snap;     // committed memory, indexed by key
  int32_t *regs;           // [n_regs][N] registers of every work-item
  uint32_t *pc, *st;       // [N]
  uint2 *ow;               // own-write table [capw][ow_stride] (key, value); entries
  uint32_t capw, ow_stride; // below ow_slots live in shared memory during the run
  uint32_t ow_slots;
  LogRec *log;                    // one slice of warp_slice records per warp
  uint32_t *warp_count;           // [n_cta * warps_per_cta] records each warp logged
  uint32_t warps_per_cta;
  unsigned long long warp_slice;  // 32 * (static bound of accesses per interval)
  OutRec *errs;
  uint32_t *err_count;
  uint32_t err_cap;
  uint32_t *stop_min, *stop_cnt;  // [n_barriers + 1], last slot = exit
  unsigned long long *acc;        // [0] global accesses, [1] local accesses
  unsigned long long *logged;     // accesses written to the log (the rest are private: CTL_PRIV)
  uint32_t *flags;                // bit 0 log full, bit 1 own-write table full, bit 2 error log full
                                  // (resident runs: two words, by interval parity)
  uint32_t *ow_count;             // [N] own-write entries per work-item
  uint32_t *owner;                // shadow owner table (nullptr: not used)
  uint32_t tag;
  const uint32_t *proceed;        // non-null: the launch does nothing unless *proceed != 0
  uint32_t *group_div;            // non-null: work-group-scoped barriers; counts diverging groups,
                                  // whose DIVERGENCE records go to errs (needs 8 * (n_barriers + 1)
                                  // bytes of dynamic shared memory after the own-write slots)
  // Resident runs (one cooperative launch runs every interval):
  int32_t *commit;                // the snapshot the kernel commits to (== snap)
  unsigned *grid_bar;             // kGridBarWords, zero before the launch ([2]: timed out; see interp.cu)
  LogRec *acc_out;                // records of cells that need the exact sort, all intervals
  unsigned long long *acc_total;  // records in acc_out
  unsigned long long acc_cap;
  unsigned long long *iv_off;     // [max_intervals + 1]: first record of each interval in acc_out
  uint32_t max_intervals;
  uint32_t *run_info;             // [0] intervals run, [1] owner-table tag of the last one
  unsigned long long owner_words; // size of the owner table (cleared in-kernel when the tag wraps)
  unsigned long long barrier_limit_ns;  // longest wait at a grid barrier before the run gives up
  // the first kInlineMems entries of mems, in the launch arguments (compiled
  // intervals read them from the constant bank: the memory object of every
  // access is a constant there)
  MemInfo mem_inline[4];
};
constexpr uint32_t kInlineMems = 4;

// ---- shadow owner table (shadow.cu)
// Four 32-bit words per cell: [4k] max writer, [4k+1] min writer, [4k+2] max
// reader, [4k+3] min reader.  A word holds (tag << 26 | id) where id is the
// work-item (max words) or kIdMask - work-item (min words), so atomicMax
// keeps the largest / smallest work-item of the current interval.  The tag
// (1..63) grows every interval, so any word with an older tag counts as
// empty; the table is cleared when the tag wraps.  Claims are fire-and-forget
// reductions: no round trip on the interpreter's critical path.
constexpr uint32_t kIdMask = (1u << 26) - 1;
// Warp-aggregated claim, called by exactly the lanes in `mask` (lane
// `lane` claiming cell `key` for work-item `id`; ids grow by one per lane
// within a warp).  When every lane is on one cell (an index that does not
// depend on the work-item), the lowest lane issues the two reductions for
// the largest and smallest id: same-address reductions serialise in L2, and
// a cell that a whole warp touches would otherwise take 32 pairs.  Lanes on
// different cells claim their own.
__device__ __forceinline__ void shadow_claim_warp(uint32_t *owner, uint32_t mask, uint32_t key, bool write,
                                                  uint32_t tag, uint32_t id, uint32_t lane) {
  uint32_t *w = owner + 4ull * key + (write ? 0 : 2);
  if (__reduce_min_sync(mask, key) == __reduce_max_sync(mask, key)) {
    if (lane != (uint32_t)(__ffs(mask) - 1)) return;
    const uint32_t hi = 31u - __clz(mask);
    atomicMax(w, (tag << 26) | (id + (hi - lane)));
    atomicMax(w + 1, (tag << 26) | (kIdMask - id));
    return;
  }
  atomicMax(w, (tag << 26) | id);
  atomicMax(w + 1, (tag << 26) | (kIdMask - id));
}

// Cells that need the exact (sorted) classification: written by two or more
// work-items, or written by one and read by another.
__device__ __forceinline__ bool shadow_needs_exact(const uint32_t *owner, uint32_t key, uint32_t tag) {
  const uint4 o = __ldcg(reinterpret_cast<const uint4 *>(owner) + key);  // L2: written by other SMs' atomics
  if ((o.x >> 26) != tag) return false;  // nobody wrote the cell
  const uint32_t wmax = o.x & kIdMask, wmin = kIdMask - (o.y & kIdMask);
  if (wmax != wmin) return true;
  if ((o.z >> 26) != tag) return false;  // one writer, no reader
  const uint32_t rmax = o.z & kIdMask, rmin = kIdMask - (o.w & kIdMask);
  return rmax != wmax || rmin != wmax;
}

// One warp appends the records of its log slice src[0, n) that need the
// exact classification (all of them when owner is null) to out, at
// positions taken from *total.  Each lane holds kPer records in flight, so
// the owner-table lookups overlap, and the warp takes its positions with one
// atomic per 32 x kPer records; a work-item's records keep their slice
// order.  Positions at or past cap are not written and raise FLAG_ACC_FULL
// in *flags.  Called by all 32 lanes of a warp.  (Kernels that run it in a
// tight register budget, the resident ones, keep four per lane.)
template <int kPer = 4>
__device__ __forceinline__ void compact_slice(const uint4 *src, uint32_t n, const uint32_t *owner, uint32_t tag,
                                              uint4 *out, unsigned long long *total, uint32_t lane,
                                              unsigned long long cap = ~0ull, uint32_t *flags = nullptr) {
  const uint32_t lt = (1u << lane) - 1u;
  for (uint32_t base = 0; base < n; base += 32 * kPer) {
    uint4 r[kPer];
    bool need[kPer];
#pragma unroll
    for (int q = 0; q < kPer; q++) {
      const uint32_t i = base + q * 32 + lane;
      // through L2: a resident batch compacts slices another SM wrote in the same launch
      r[q] = i < n ? __ldcg(src + i) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int q = 0; q < kPer; q++)
      need[q] = base + q * 32 + lane < n && (!owner || shadow_needs_exact(owner, r[q].x, tag));
    uint32_t bal[kPer], tot = 0;
#pragma unroll
    for (int q = 0; q < kPer; q++) {
      bal[q] = __ballot_sync(0xFFFFFFFFu, need[q]);
      tot += __popc(bal[q]);
    }
    if (tot == 0) continue;
    unsigned long long pos = 0;
    if (lane == 0) pos = atomicAdd(total, (unsigned long long)tot);
    pos = __shfl_sync(0xFFFFFFFFu, pos, 0);
#pragma unroll
    for (int q = 0; q < kPer; q++) {
      if (need[q]) {
        const unsigned long long p = pos + __popc(bal[q] & lt);
        if (p < cap) out[p] = r[q];
        else atomicOr(flags, FLAG_ACC_FULL);
      }
      pos += __popc(bal[q]);
    }
  }
}

}  // namespace rc
