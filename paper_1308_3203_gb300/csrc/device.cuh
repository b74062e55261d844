// Device-side data layouts shared by the kernels of the checker.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "bytecode.h"

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
constexpr uint32_t kMetaRead = 1u << 30, kMetaWrite = 1u << 31, kMetaCount = (1u << 30) - 1;

// Interpreter launch arguments (one launch runs one barrier interval for a
// contiguous range of work-groups).
struct InterpArgs {
  const Insn *code;
  const MemInfo *mems;
  uint32_t n_insn, n_regs, n_mems, n_barriers;
  uint32_t S, G, group0;   // block b runs work-group group0 + b
  uint32_t GT, LT;         // global cells, local cells per group
  uint32_t interval;
  const int32_t *snap;     // committed memory, indexed by key
  int32_t *regs;           // [n_regs][N] registers of every work-item
  uint32_t *pc, *st;       // [N]
  uint2 *ow;               // own-write table [capw][ow_stride] (key, value)
  uint32_t capw, ow_stride;
  LogRec *log;
  unsigned long long *log_count;
  unsigned long long log_cap;
  OutRec *errs;
  uint32_t *err_count;
  uint32_t err_cap;
  uint32_t *stop_min, *stop_cnt;  // [n_barriers + 1], last slot = exit
  unsigned long long *acc;        // [0] global accesses, [1] local accesses
  uint32_t *flags;                // bit 0 log full, bit 1 own-write table full, bit 2 error log full
  uint32_t *ow_count;             // [N] own-write entries per work-item
  unsigned long long *owner;      // shadow owner table (nullptr: not used)
  uint32_t epoch;
};

// ---- shadow owner table (shadow.cu)
// Two 64-bit words per cell: [2*key] = writer, [2*key+1] = reader.  A word
// holds (epoch << 32 | gtid) of the only work-item that wrote (read) the cell
// in the current interval, (epoch << 32 | kNone) once two or more did, and
// anything with an older epoch means "nobody yet".
__device__ __forceinline__ void shadow_claim(unsigned long long *p, uint32_t epoch, uint32_t gtid) {
  const unsigned long long mine = ((unsigned long long)epoch << 32) | gtid;
  const unsigned long long shared = ((unsigned long long)epoch << 32) | 0xFFFFFFFFull;
  unsigned long long cur = *reinterpret_cast<volatile unsigned long long *>(p);
  for (int it = 0; it < 4; it++) {
    if ((uint32_t)(cur >> 32) != epoch) {
      const unsigned long long prev = atomicCAS(p, cur, mine);
      if (prev == cur) return;
      cur = prev;
      continue;
    }
    if ((uint32_t)cur == gtid || (uint32_t)cur == 0xFFFFFFFFu) return;
    break;
  }
  atomicExch(p, shared);
}

// Cells that need the exact (sorted) classification: written by two or more
// work-items, or written by one and read by another.
__device__ __forceinline__ bool shadow_needs_exact(const unsigned long long *owner, uint32_t key, uint32_t epoch) {
  const unsigned long long w = owner[2ull * key], r = owner[2ull * key + 1];
  if ((uint32_t)(w >> 32) != epoch) return false;
  const uint32_t wg = (uint32_t)w;
  if (wg == 0xFFFFFFFFu) return true;
  if ((uint32_t)(r >> 32) != epoch) return false;
  return (uint32_t)r != wg;
}

void launch_shadow_compact(const LogRec *log, uint64_t n, const unsigned long long *owner, uint32_t epoch,
                           LogRec *out, unsigned long long *count, cudaStream_t s);
void launch_shadow_commit(const uint2 *ow, const uint32_t *ow_count, uint64_t N, uint32_t ow_stride,
                          const unsigned long long *owner, uint32_t epoch, int32_t *snap, cudaStream_t s);

enum Flag : uint32_t { FLAG_LOG_FULL = 1, FLAG_OW_FULL = 2, FLAG_ERR_FULL = 4 };

void launch_interp(const InterpArgs &a, uint32_t n_groups, size_t smem, cudaStream_t s);
size_t interp_smem_bytes(uint32_t n_insn, uint32_t n_mems, uint32_t n_regs, uint32_t S);
cudaError_t interp_configure();

// ---- scan / sort (sort.cu)
// exclusive prefix sum of n uint32 values; tmp must hold scan_tmp_words(n)
size_t scan_tmp_words(uint64_t n);
void scan_exclusive(const uint32_t *in, uint32_t *out, uint64_t n, uint32_t *tmp, cudaStream_t s);
// stable LSD radix sort of n log records by (key << gbits | gtid) over
// `bits` key bits; returns the buffer holding the result (a or b)
size_t sort_tmp_words(uint64_t n);
LogRec *sort_log(LogRec *a, LogRec *b, uint64_t n, uint32_t gbits, uint32_t bits, uint32_t *tmp,
                 cudaStream_t s);

// ---- classification (classify.cu)
struct ClassifyArgs {
  uint32_t interval, GT, LT;
  int32_t *snap;  // committed memory, updated in place
};
void launch_run_heads(const LogRec *r, uint64_t n, uint32_t *head, cudaStream_t s);
void launch_run_reduce(const LogRec *r, uint64_t n, const uint32_t *head, const uint32_t *runidx,
                       Summary *sum, uint32_t *khead, cudaStream_t s);
void launch_key_classify(const Summary *sum, uint64_t nsum, const uint32_t *khead,
                         const uint32_t *keyidx, uint32_t *nrec, const ClassifyArgs &a,
                         cudaStream_t s);
void launch_key_emit(const Summary *sum, uint64_t nsum, const uint32_t *khead,
                     const uint32_t *keyidx, const uint32_t *nrec, const uint32_t *recoff,
                     OutRec *out, const ClassifyArgs &a, cudaStream_t s);

}  // namespace rc
