// Device-side data layouts shared by the kernels of the checker.
#pragma once
#include <cstdint>
#include <vector>
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
// device-side overflow / error flags of a run (InterpArgs::flags)
enum Flag : uint32_t { FLAG_LOG_FULL = 1, FLAG_OW_FULL = 2, FLAG_ERR_FULL = 4, FLAG_ACC_FULL = 16 };
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
};

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
// positions taken from *total.  Each lane holds four records in flight, so
// the owner-table lookups overlap, and the warp takes its positions with one
// atomic per 128 records; a work-item's records keep their slice order.
// Positions at or past cap are not written and raise FLAG_ACC_FULL in
// *flags.  Called by all 32 lanes of a warp.
__device__ __forceinline__ void compact_slice(const uint4 *src, uint32_t n, const uint32_t *owner, uint32_t tag,
                                              uint4 *out, unsigned long long *total, uint32_t lane,
                                              unsigned long long cap = ~0ull, uint32_t *flags = nullptr) {
  const uint32_t lt = (1u << lane) - 1u;
  for (uint32_t base = 0; base < n; base += 128) {
    uint4 r[4];
    bool need[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const uint32_t i = base + q * 32 + lane;
      r[q] = i < n ? src[i] : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int q = 0; q < 4; q++)
      need[q] = base + q * 32 + lane < n && (!owner || shadow_needs_exact(owner, r[q].x, tag));
    uint32_t bal[4], tot = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      bal[q] = __ballot_sync(0xFFFFFFFFu, need[q]);
      tot += __popc(bal[q]);
    }
    if (tot == 0) continue;
    unsigned long long pos = 0;
    if (lane == 0) pos = atomicAdd(total, (unsigned long long)tot);
    pos = __shfl_sync(0xFFFFFFFFu, pos, 0);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      if (need[q]) {
        const unsigned long long p = pos + __popc(bal[q] & lt);
        if (p < cap) out[p] = r[q];
        else atomicOr(flags, FLAG_ACC_FULL);
      }
      pos += __popc(bal[q]);
    }
  }
}

// log: n_slices warp slices of `slice` records, count[i] valid in slice i
void launch_shadow_compact(const LogRec *log, uint32_t n_slices, uint64_t slice, const uint32_t *count,
                           const uint32_t *owner, uint32_t tag, LogRec *out, unsigned long long *total,
                           cudaStream_t s);
void launch_shadow_commit(const uint2 *ow, const uint32_t *ow_count, uint64_t N, uint32_t ow_stride,
                          const uint32_t *owner, uint32_t tag, int32_t *snap, cudaStream_t s);
// n int32 values src -> dst by a kernel (src may be pinned host memory, read over the CPU-GPU link)
void launch_copy_words(const int32_t *src, int32_t *dst, uint64_t n, cudaStream_t s);
// copy the used part of every slice into one dense array (offs = exclusive scan of count)
void launch_densify(const LogRec *log, uint32_t n_slices, uint64_t slice, const uint32_t *count,
                    const uint32_t *offs, LogRec *out, cudaStream_t s);

// Kernels launched by the library since load (every launch site adds one).
void count_launch();
// streaming multiprocessors of the current device
int sm_count();

void launch_interp(const InterpArgs &a, uint32_t n_groups, size_t smem, cudaStream_t s);
// Resident run: every interval in one cooperative launch of n_groups CTAs
// (all resident at once; see interp.cu).  blocks_per_sm: how many CTAs of
// this shape fit on one SM.
cudaError_t launch_interp_resident(const InterpArgs &a, uint32_t n_groups, size_t smem, cudaStream_t s);
int interp_resident_blocks_per_sm(uint32_t n_insn, uint32_t S, size_t smem);
constexpr uint32_t kGridBarWords = 32 + 32 * 32;  // grid barrier: top counter, generation, flag, 32 sub-counters
// Diagnostic cooperative launch whose grid barrier cannot complete (bar: kGridBarWords zeroed words).
cudaError_t launch_grid_barrier_probe(unsigned *bar, uint32_t n_blocks, unsigned long long limit_ns, cudaStream_t s);
// Gate of a speculatively queued interval: *proceed = 1 iff the previous
// interval overflowed nothing, compacted no record for the exact sort, and
// its work-items all stopped at one barrier (the run goes on unchanged).
void launch_interval_gate(const uint32_t *flags, const unsigned long long *compacted, const uint32_t *stop_cnt,
                          uint32_t n_barriers, uint32_t *proceed, cudaStream_t s);
size_t interp_smem_bytes(uint32_t n_mems, uint32_t n_regs, uint32_t S, uint32_t ow_slots);
cudaError_t interp_configure();
constexpr uint32_t kConstCodeInsns = 4000;  // programs up to this size run from constant memory
// copy bytecode to constant memory (no-op for larger programs); stream-ordered
cudaError_t interp_upload_code(const Insn *host_code, uint32_t n_insn, cudaStream_t s);
constexpr size_t kMaxSmemPerBlock = 227 * 1024;  // opt-in shared memory per CTA on sm_103
size_t interp_max_dynamic_smem();  // valid after interp_configure()

// ---- work-group-scoped barriers: cross-group classification (xgroup.cu)
// One global cell over the whole run: smallest/largest writer and reader,
// smallest/largest value written, smallest/largest value observed (seeded
// with the cell's value before the run).  Counts (reads, writes) live apart.
struct __align__(16) XgCell {
  uint32_t wmin, wmax, rmin, rmax;
  int32_t vmin, vmax, omin, omax;
};
void launch_xg_init(XgCell *xg, uint2 *cnt, const int32_t *snap, uint64_t GT, cudaStream_t s);
// fold one interval's log (its warp slices) into the table
void launch_xg_update(const LogRec *log, uint32_t n_slices, uint64_t slice, const uint32_t *count, uint64_t GT,
                      XgCell *xg, uint2 *cnt, cudaStream_t s);
// records per cell (0-2), then the records at offs (exclusive scan of nrec)
void launch_xg_count(const XgCell *xg, uint64_t GT, uint32_t S, uint32_t *nrec, cudaStream_t s);
void launch_xg_emit(const XgCell *xg, const uint2 *cnt, uint64_t GT, uint32_t S, const uint32_t *nrec,
                    const uint32_t *offs, OutRec *out, cudaStream_t s);

// ---- batched checking (batch.cu)
struct BatchDesc {  // one instance of a batch
  uint32_t code_off, mems_off, n_regs, n_barriers;
  uint32_t S, G, GT, LT;
  uint32_t capw, stop_off, task_off, active;
  uint64_t N;          // work-items
  uint64_t key_base;   // first cell of the instance in the batch's cell space
  uint64_t reg_off;    // registers [n_regs][N] start here
  uint64_t state_off;  // pc / st / own-write counts start here
  uint64_t ow_off;     // own-write table [capw][N] starts here
  uint64_t slice_off;  // first log record of the instance's warp slices
  uint64_t slice;      // records per warp slice (32 * static bound)
};

struct BatchArgs {
  BatchDesc *desc;
  const uint32_t *task_kernel;  // warp task -> instance
  uint32_t n_tasks;
  uint32_t *next_task;          // persistent-grid task counter (zero before each launch)
  const Insn *code;             // all instances' bytecode, end to end
  const MemInfo *mems;          // all instances' memory tables
  uint32_t max_regs, ow_slots;
  const uint32_t *round;        // device: [0] interval, [1] owner-table tag, [2] shadow path on
  int32_t *snap;
  int32_t *regs;
  uint32_t *pc, *st, *ow_count;
  uint2 *ow;
  LogRec *log;
  uint32_t *warp_count;         // per warp task
  OutRec *errs;
  uint32_t *err_kernel, *err_count;
  uint32_t err_cap;
  uint32_t *stop_min, *stop_cnt;
  unsigned long long *acc;      // [2 * instances]: global, local accesses
  uint32_t *flags;
  uint32_t *owner;              // shadow owner table over the batch's cells
};

size_t batch_smem_bytes(uint32_t max_regs, uint32_t ow_slots);
cudaError_t batch_configure();
uint32_t batch_threads();
void launch_batch_interp(const BatchArgs &a, uint32_t grid, size_t smem, cudaStream_t s);
void launch_batch_compact(const BatchArgs &a, LogRec *out, unsigned long long *total, cudaStream_t s);
void launch_batch_commit(const BatchArgs &a, cudaStream_t s);

// ---- interleaving explorer (explore.cu)
// The checker's state at the start of one interval of a small instance.
struct ExploreInput {
  const Insn *code;
  const MemInfo *mems;  // device
  uint32_t n_insn, N, S, n_regs, cells, GT, LT, interval, max_access;
  const int32_t *snap, *regs;  // cells; registers [n_regs][N]
  const uint32_t *pc, *st;     // [N]
};
struct ExploreResult {
  uint32_t n_end_states;  // distinct shared memories at the interval's closing barrier
  uint32_t deviated;      // a read of some schedule differs from the work-item's solo run
  uint32_t complete;      // every schedule was explored within the budget
  uint64_t n_states;      // distinct states visited
};
struct ExploreError {
  const char *msg;
};
// Every schedule of the interval from that state (throws ExploreError on a
// CUDA failure).  With pair_out, the search covers every pair of work-items
// (i < j) alone instead (the others do not run), and pair_out receives per
// pair, in (i, j) order, its distinct end memories | (schedule-dependent
// read) << 31; n_end_states then counts distinct (pair, memory) items.
ExploreResult explore_interval(const ExploreInput &in, uint64_t max_states, cudaStream_t s,
                               std::vector<uint32_t> *pair_out = nullptr);

// ---- scan / sort (sort.cu)
// exclusive prefix sum of n uint32 values; tmp must hold scan_tmp_words(n)
size_t scan_tmp_words(uint64_t n);
void scan_exclusive(const uint32_t *in, uint32_t *out, uint64_t n, uint32_t *tmp, cudaStream_t s);
// stable LSD radix sort of n log records by (key << gbits | gtid) over
// `bits` key bits; returns the buffer holding the result (a or b)
size_t sort_tmp_words(uint64_t n);
LogRec *sort_log(LogRec *a, LogRec *b, uint64_t n, uint32_t gbits, uint32_t bits, uint32_t *tmp,
                 cudaStream_t s);
// same sort from `in` (not written) into `out`, ping-ponging through scratch (n records)
void sort_log_into(const LogRec *in, LogRec *out, LogRec *scratch, uint64_t n, uint32_t gbits, uint32_t bits,
                   uint32_t *tmp, cudaStream_t s);

// ---- classification (classify.cu)
// Classification of one cell: counts, WW class and witnesses, RW witnesses,
// and the value the cell commits.
struct CellResult {
  uint32_t n_readers, n_writers, n_acc;
  uint32_t ww_cls, ww_a, ww_b;  // ww_cls 0 = none
  uint32_t rw_a, rw_b;          // rw_a kNone = none
  uint32_t wrote;
  int32_t commit;
};

// Cells with more summaries than this are classified by a whole CTA.
constexpr uint32_t kBigCell = 64;

struct ClassifyArgs {
  uint32_t interval, GT, LT;
  int32_t *snap;  // committed memory, updated in place
  // cells above kBigCell summaries: head index of each, how many, their results
  uint32_t *big = nullptr, *nbig = nullptr;
  CellResult *bigres = nullptr;
  const uint32_t *nsum = nullptr;  // device: number of summaries (launches cover an upper bound)
  // batches: cells of several instances end to end; records name their instance
  uint32_t n_kernels = 0;
  const uint64_t *kbase = nullptr;  // sorted first cell of each instance
  const uint32_t *kGT = nullptr, *kLT = nullptr;
  uint32_t *rec_kernel = nullptr;   // instance of each emitted record
};
void launch_run_heads(const LogRec *r, uint64_t n, uint32_t *head, cudaStream_t s);
// also stores the number of summaries in *nsum (device)
void launch_run_reduce(const LogRec *r, uint64_t n, const uint32_t *head, const uint32_t *runidx,
                       Summary *sum, uint32_t *khead, uint32_t *nsum, cudaStream_t s);
void launch_key_classify(const Summary *sum, uint64_t nsum, const uint32_t *khead,
                         const uint32_t *keyidx, uint32_t *nrec, const ClassifyArgs &a,
                         cudaStream_t s);
void launch_key_emit(const Summary *sum, uint64_t nsum, const uint32_t *khead,
                     const uint32_t *keyidx, const uint32_t *nrec, const uint32_t *recoff,
                     OutRec *out, const ClassifyArgs &a, cudaStream_t s);
// the large cells key_classify set aside (a.big, a.nbig): results, commit, record counts
void launch_big_classify(const Summary *sum, uint64_t nsum, const uint32_t *keyidx, uint32_t *nrec,
                         const ClassifyArgs &a, cudaStream_t s);
void launch_big_emit(const Summary *sum, uint64_t nsum, const uint32_t *keyidx, const uint32_t *nrec,
                     const uint32_t *recoff, OutRec *out, const ClassifyArgs &a, cudaStream_t s);
// capacity of the large-cell list for nsum summaries
inline uint64_t big_cells_cap(uint64_t nsum) { return nsum / (kBigCell + 1) + 1; }

}  // namespace rc
