// Device-side data layouts shared by the kernels of the checker.
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "bytecode.h"
#include "kernel_types.cuh"

namespace rc {

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
// interval overflowed nothing and its work-items all stopped at one barrier
// (the run goes on unchanged; the shadow path has committed every written
// cell before the gate, so the exact classification of the previous
// interval's shared cells is not needed first).
void launch_interval_gate(const uint32_t *flags, const uint32_t *stop_cnt, uint32_t n_barriers, uint32_t *proceed,
                          cudaStream_t s);
size_t interp_smem_bytes(uint32_t n_mems, uint32_t n_regs, uint32_t S, uint32_t ow_slots);
cudaError_t interp_configure();
constexpr uint32_t kConstCodeInsns = 4000;  // programs up to this size run from constant memory
// copy bytecode to constant memory (no-op for larger programs); stream-ordered
cudaError_t interp_upload_code(const Insn *host_code, uint32_t n_insn, cudaStream_t s);
constexpr size_t kMaxSmemPerBlock = 227 * 1024;  // opt-in shared memory per CTA on sm_103
size_t interp_max_dynamic_smem();  // valid after interp_configure()

// ---- one-CTA check of small instances (interp.cu): every work-item in one
// CTA, every interval, its classification and barrier agreement in one launch
constexpr uint32_t kSmallMaxItems = 1024;  // groups x group size
constexpr uint32_t kSmallCap = 4096;       // records of one interval (sorted in shared memory)
constexpr uint32_t kSmallMaxStops = 64;    // barriers + 1
constexpr uint32_t kSmallBins = 16384;     // (cell, work-item) pairs the counting sort takes
struct SmallArgs {
  InterpArgs A;              // program, shape, snapshot (= commit), own-write spill, log slices, errors
  LogRec *sorted;            // [cap] the interval's records, sorted (global; unused with smem_scratch)
  Summary *sum;              // [cap] (likewise)
  OutRec *out;               // [out_cap] race records in report order
  uint32_t cap;              // records one interval may log (at most kSmallCap)
  uint32_t out_cap, max_intervals, n_items;
  uint32_t reg_stride;       // work-items rounded up to whole warps
  uint32_t smem_scratch;     // sorted records and summaries in shared memory
  uint32_t smem_snap;        // the snapshot in shared memory (n_cells cells)
  uint32_t smem_log;         // the warp slices of the log in shared memory
  uint32_t bins;             // cells x reg_stride counters in shared memory (counting sort), or 0 (bitonic)
  uint32_t n_cells;
  // page-locked host memory the kernel writes its results to: res [0] global,
  // [1] local, [2] logged accesses, [3] intervals | flags << 32, [4] race
  // records, [5] error records; then the records themselves
  unsigned long long *res;
  OutRec *host_out, *host_err;
};
size_t small_check_smem(uint32_t n_mems, uint32_t n_regs, uint32_t T, uint32_t ow_slots, uint32_t cap,
                        uint32_t snap_cells);
cudaError_t launch_small_check(const SmallArgs &a, uint32_t threads, size_t smem, cudaStream_t s);

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
  // resident runs: every round of the batch in one cooperative launch
  unsigned *grid_bar;           // kGridBarWords, zero before the launch
  unsigned long long barrier_limit_ns;
  LogRec *acc_out;              // records of shared cells, every round end to end
  unsigned long long *acc_total;  // records in acc_out
  unsigned long long *iv_off;   // [max_rounds + 1]: first record of each round
  unsigned long long acc_cap;
  uint64_t owner_words;         // owner-table words the batch's cells use (cleared in-kernel at a tag wrap)
  uint32_t n_inst, max_rounds, tag0;
  uint32_t *n_active;           // [2] instances active in the next round (by parity; zero before the launch)
  uint32_t *inst_rounds;        // [n_inst] intervals each instance ran; [n_inst] rounds, [n_inst + 1] last tag
  uint32_t *fill_max;           // largest fill of a warp task's log slice, in permille of its capacity
};

// block shapes of the batch interpreter: 128, 256 or 512 threads per CTA
size_t batch_smem_bytes(uint32_t max_regs, uint32_t ow_slots, uint32_t threads);
cudaError_t batch_configure();
void launch_batch_interp(const BatchArgs &a, uint32_t grid, uint32_t threads, size_t smem, cudaStream_t s);
// Every round of the batch in one cooperative launch of `grid` CTAs (all
// resident): the interpreter's round, then the commit of the owner table's
// highest writers and the compaction of the records of shared cells into
// acc_out, then each instance's barrier agreement, between grid barriers.
cudaError_t launch_batch_resident(const BatchArgs &a, uint32_t grid, uint32_t threads, size_t smem, cudaStream_t s);
// CTAs of the resident batch kernel one SM holds with this block shape and shared memory
int batch_resident_blocks_per_sm(uint32_t threads, size_t smem);
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
  // the other cells' results by cell index (written by the classifier for
  // cells with records, read by the emitter: one walk of each cell)
  CellResult *cellres = nullptr;
  const uint32_t *nsum = nullptr;  // device: number of summaries (launches cover an upper bound)
  uint32_t *cstart = nullptr;      // first summary of each cell, by cell index
  uint32_t *ncell = nullptr;       // device: number of cells
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
// a.cstart and *a.ncell from the cell heads and their exclusive scan
void launch_cell_starts(const uint32_t *khead, const uint32_t *keyidx, uint64_t n, const ClassifyArgs &a,
                        cudaStream_t s);
// one thread per cell; n bounds the number of cells
void launch_key_classify(const Summary *sum, uint64_t n, uint32_t *nrec, const ClassifyArgs &a, cudaStream_t s);
void launch_key_emit(const Summary *sum, uint64_t n, const uint32_t *nrec, const uint32_t *recoff, OutRec *out,
                     const ClassifyArgs &a, cudaStream_t s);
// the large cells key_classify set aside (a.big, a.nbig): results, commit, record counts
void launch_big_classify(const Summary *sum, uint64_t nsum, const uint32_t *keyidx, uint32_t *nrec,
                         const ClassifyArgs &a, cudaStream_t s);
void launch_big_emit(const Summary *sum, uint64_t nsum, const uint32_t *keyidx, const uint32_t *nrec,
                     const uint32_t *recoff, OutRec *out, const ClassifyArgs &a, cudaStream_t s);
// capacity of the large-cell list for nsum summaries
inline uint64_t big_cells_cap(uint64_t nsum) { return nsum / (kBigCell + 1) + 1; }

}  // namespace rc
