/*
 * racecheck.h - C ABI of the GB300 concrete race checker.
 *
 * The library runs every work-item of an instance of a kernel written in the
 * minimal OpenCL kernel language of Distefano & Dubreil, "Detecting Data
 * Races on OpenCL Kernels with Symbolic Execution" (Sec. 3: expressions,
 * booleans and commands v:=e, a[v]:=e, v:=a[v], barrier, assume, assert;
 * a kernel is a control-flow graph from a unique start to a unique exit),
 * under the concrete SIMD semantics of Sec. 4 (thread-local rules, barrier
 * release, the race rule and the Definition of a race), on one sm_103a GPU.
 * Each barrier interval's shared accesses are logged in device memory and
 * classified: several work-items writing the same value to a cell is benign
 * (Sec. 1; Sec. 4 after the race rule), differing values are a race.
 *
 * Conventions for every entry point:
 *  - return value: RC_OK (0) or an RC_E_* code; no exception crosses the ABI;
 *    rc_last_error() gives a message for the calling thread's last failure;
 *  - a race is a successful check (report status RC_RACY), not an error;
 *  - objects returned through out-pointers are owned by the library and are
 *    released with the matching rc_*_free; inputs are read during the call
 *    and never retained after it returns;
 *  - all device work runs on the caller's CUDA stream (rc_input.cuda_stream,
 *    NULL = legacy default stream); the call synchronises that stream before
 *    it returns;
 *  - the library keeps device workspaces between calls (grown on demand,
 *    released by rc_release_workspace); calls from several host threads are
 *    serialised internally.
 */
#ifndef RACECHECK_H
#define RACECHECK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes */
#define RC_OK 0
#define RC_E_PARSE 1     /* source text is not a valid kernel               */
#define RC_E_INVALID 2   /* bad argument, launch shape, input or bytecode   */
#define RC_E_CAPACITY 3  /* instance needs more device memory than allowed  */
#define RC_E_CUDA 4      /* a CUDA runtime call failed                      */
#define RC_E_TIMEOUT 5   /* a bounded device wait ran out                   */
#define RC_E_NOMEM 6     /* host allocation failed                          */

/* ---- report status (rc_report.status) */
#define RC_RACE_FREE 0        /* no race, no error                                  */
#define RC_RACY 1             /* at least one WW_RACE, RW_RACE, XG_WW_RACE or XG_RW_RACE record */
#define RC_ERROR_OOB 2        /* out-of-bounds access (Sec. 5 Table 1 premise), no race */
#define RC_ERROR_ASSERT 3     /* failed assert (Sec. 4 assert rule), no race        */
#define RC_ERROR_DIVERGENCE 4 /* work-items stopped at different barriers, no race  */

/* ---- record classes (rc_record.cls) */
#define RC_WW_RACE 1    /* two writers' last values in the interval differ       */
#define RC_WW_BENIGN 2  /* >= 2 writers, all last values equal (benign, Sec. 1)  */
#define RC_RW_RACE 3    /* a read observed o, another work-item wrote v != o     */
/* cross-group classes (RC_GROUP_BARRIERS only): one global cell over the whole run */
#define RC_XG_WW_RACE 4   /* writers in >= 2 work-groups, written values differ     */
#define RC_XG_WW_BENIGN 5 /* writers in >= 2 work-groups, one value written         */
#define RC_XG_RW_RACE 6   /* reader and writer in different work-groups, and the cell
                             did not hold one value all along                        */
#define RC_OOB 16       /* error: access outside 0 <= index < size(array)        */
#define RC_ASSERT_FAIL 17
#define RC_DIVERGENCE 18

/* Options for rc_input.flags */
#define RC_WANT_FINAL_MEMORY 1u /* fill rc_report.final_global            */
/* Work-group-scoped barriers (OpenCL's barrier; the paper's is kernel-wide,
 * Sec. 2 and the barrier-release rule of Sec. 4).  The run is the same
 * lock-step schedule (round k runs every group's k-th interval), but barrier
 * agreement holds per work-group: groups may wait at different barriers, and
 * a group whose work-items all exited is finished while others go on.  As no
 * barrier orders work-items of different groups, every global cell is also
 * classified over the whole run between groups (RC_XG_* records).  Only
 * rc_check and rc_search take it; rc_check_batch, rc_explore and
 * rc_explore_pairs return RC_E_INVALID. */
#define RC_GROUP_BARRIERS 2u
/* Log every shared access: the two-work-item pre-filter (rc_prove_private)
 * is not consulted, so no access is taken as private; every access is
 * written to its interval's log and claims its cell.  Same report (the
 * pre-filter only drops accesses that cannot change it), n_logged =
 * n_access. */
#define RC_LOG_EVERY_ACCESS 4u

typedef struct rc_bytecode rc_bytecode; /* opaque, library-owned */

/* Static facts about a compiled kernel. */
typedef struct {
  uint32_t n_insn;        /* bytecode instructions                          */
  uint32_t n_regs;        /* registers per work-item (variables + temps)    */
  uint32_t n_vars;        /* named private variables                        */
  uint32_t n_mems;        /* memory objects (global + local), declared order */
  uint32_t n_global;      /* global memory objects = inputs rc_check wants  */
  uint32_t n_barriers;    /* barrier statements                             */
  uint32_t n_asserts;     /* assert statements                              */
  uint32_t local_cells;   /* int32 cells of local memory per work-group     */
  uint64_t max_access_per_interval; /* static bound per work-item           */
  uint64_t max_write_per_interval;  /* static bound per work-item           */
} rc_bytecode_info;

/* Input of one instance.  global_len[i] / global_init[i] give the length
 * and the initial int32 contents of the i-th `global` declaration (declared
 * order).  on_device != 0: global_init pointers are device pointers;
 * otherwise host pointers (pageable or pinned).  cuda_stream is a
 * cudaStream_t or NULL. */
typedef struct {
  uint32_t n_global;
  const uint64_t *global_len;
  const int32_t *const *global_init;
  int on_device;
  void *cuda_stream;
  uint32_t flags;
} rc_input;

/* One report record: ten uint32 fields, fixed order.
 *  race records (cls 1..3): the cell (space 0 = global, 1 = local; wg = the
 *    work-group owning a local cell, 0 for global; addr = flat index in the
 *    space, arrays laid out in declared order), the barrier interval, the
 *    witness pair (t_a, t_b) of global work-item ids, distinct readers and
 *    writers, and the number of accesses to the cell in the interval;
 *  OOB: space/wg of the array, addr = the index (two's complement), t_a =
 *    the work-item, t_b = the array's declaration index;
 *  ASSERT_FAIL: t_a = the work-item, t_b = assert ordinal (source order);
 *  DIVERGENCE: one record per stop point, t_a = smallest work-item stopped
 *    there, t_b = barrier ordinal (0xFFFFFFFF = exit), n_accesses = how many
 *    work-items stopped there (RC_GROUP_BARRIERS: per diverging work-group,
 *    wg = the group);
 *  XG records (RC_GROUP_BARRIERS): interval = 0xFFFFFFFF (the whole run),
 *    space 0, wg 0, addr = the global cell; XG_WW_*: (t_a, t_b) = smallest
 *    and largest writer; XG_RW_RACE: from the smallest/largest reader r0/r1
 *    and writer w0/w1, (r0, w0) if their groups differ, else (r0, w1) if
 *    those differ, else (r1, w0); n_readers / n_writers = reads / writes of
 *    the cell in the run, n_accesses = both.
 * Race records come first, sorted by (interval, space, wg, addr, cls), then
 * the XG records by (addr, cls); error records follow, sorted by (interval,
 * cls, t_a). */
typedef struct {
  uint32_t interval, space, wg, addr, cls, t_a, t_b, n_readers, n_writers, n_accesses;
} rc_record;

typedef struct {
  int32_t status;         /* RC_RACE_FREE .. RC_ERROR_DIVERGENCE */
  uint32_t n_intervals;   /* barrier intervals executed          */
  uint64_t n_access;      /* shared accesses performed           */
  uint64_t n_global;      /* ... of which to global memory       */
  uint64_t n_local;       /* ... of which to local memory        */
  uint64_t n_records;
  rc_record *records;
  uint64_t final_len;     /* global cells (sum of global_len)    */
  int32_t *final_global;  /* final global memory, or NULL        */
  uint64_t n_logged;      /* accesses written to the interval    */
                          /* logs; the others were proved        */
                          /* private (no other work-item touches */
                          /* their cells in the interval) and    */
                          /* were counted, not logged            */
} rc_report;

/* Compile kernel source text (Sec. 3 grammar, see the package docs for the
 * surface syntax).  On RC_E_PARSE a message is written to err (if err_len >
 * 0).  *out receives a new bytecode object on success. */
int rc_compile(const char *src, size_t len, rc_bytecode **out, char *err, size_t err_len);

/* Fill *info with static facts about bc. */
int rc_bytecode_info_get(const rc_bytecode *bc, rc_bytecode_info *info);

/* Check one instance: groups x group_size work-items (1 <= group_size <=
 * 1024, groups * group_size <= 2^26) run bc on `in`.  *out receives a new
 * report.  Errors: RC_E_INVALID (shape, input count/lengths, local memory
 * too large), RC_E_CAPACITY, RC_E_CUDA. */
int rc_check(const rc_bytecode *bc, uint32_t groups, uint32_t group_size, const rc_input *in,
             rc_report **out);

/* Check n independent instances; out must hold n report pointers.  Reports
 * are identical to n rc_check calls.  On error no report is returned. */
int rc_check_batch(const rc_bytecode *const *bcs, const uint32_t *groups,
                   const uint32_t *group_size, const rc_input *inputs, size_t n,
                   rc_report **out);

void rc_bytecode_free(rc_bytecode *bc);
void rc_report_free(rc_report *rep);
const char *rc_strerror(int code);
const char *rc_last_error(void);

/* One shared access as the checker logs it (16 bytes):
 *   cell   flat cell index (global cells first, arrays in declared order,
 *          then local cells, work-group major)
 *   item   global work-item id in bits 0..30, 1 in bit 31 for a write
 *   value  value written, or value the read observed
 *   seq    position of the access in its work-item's barrier interval */
typedef struct {
  uint32_t cell, item;
  int32_t value;
  uint32_t seq;
} rc_access;

/* Sort n access records by (cell, work-item id), stably, on the device: the
 * first step of the exact classification of one barrier interval (records
 * of one cell become contiguous, and within a cell those of one work-item,
 * in input order).  in and out are device pointers to n records each, must
 * not overlap, and in is not modified.  cell_bits / item_bits: the cells are
 * below 2^cell_bits and the work-item ids below 2^item_bits (item_bits <= 31,
 * cell_bits + item_bits <= 58; fewer bits mean fewer 8-bit passes).  Runs on
 * cuda_stream and synchronises it.  Scratch memory comes from the library's
 * workspace (grown on demand).  Errors: RC_E_INVALID for bad sizes or null
 * pointers with n > 0, RC_E_CAPACITY, RC_E_CUDA. */
int rc_sort_accesses(const rc_access *in, rc_access *out, uint64_t n, uint32_t cell_bits, uint32_t item_bits,
                     void *cuda_stream);

/* rc_sort_accesses for callers that cannot allocate device memory.  The
 * paper has no counterpart: this is an engineering variant of the sort
 * above.  Callers that must not call cudaMalloc -- a process serving under a
 * device-memory budget it reserved in full at start-up, a real-time pipeline
 * that cannot take the device-wide synchronisation an allocation may cause,
 * a library that must not touch its host application's allocator -- get the
 * same sort with its scratch (ping-pong records, digit histograms) in one
 * fixed file-scope device array of about 4.3 MiB, which every GPU that loads
 * the library holds until the process exits.  This call allocates nothing:
 * no cudaMalloc, cudaFree or allocating library routine.
 *  - n may not exceed 2^18 records (RC_E_CAPACITY beyond that); other
 *    arguments and results are those of rc_sort_accesses.
 *  - The first call on each device, with that device current, is the
 *    set-up call: it looks up the device address of the array
 *    (cudaGetSymbolAddress), and under lazy module loading (CUDA's default)
 *    that is when the driver loads the module holding the array and creates
 *    the array on the device.  Make that first call (an n = 1 sort will do)
 *    before reserving the rest of the device budget and before any stream
 *    capture; later calls allocate nothing.
 *  - Errors also set rc_last_error(); a CUDA error already pending before
 *    the call is reported as RC_E_CUDA without running the sort.
 *  - All calls share the one array and it keeps the last call's contents;
 *    calls whose work overlaps on the GPU (other streams, other host
 *    threads) race on it and must be serialised by the caller. */
int rc_sort_accesses_noalloc(const rc_access *in, rc_access *out, uint64_t n, uint32_t cell_bits,
                             uint32_t item_bits, void *cuda_stream);

/* Release every device workspace the library holds. */
int rc_release_workspace(void);

/* Diagnostic of the resident runs' failure path: one cooperative launch
 * (a CTA per SM) waits at a grid-wide barrier that expects one arrival more
 * than the launch has, so every wait must give up after limit_us (1 .. 10^7)
 * microseconds.  *timed_out = 1 when the kernel reported the timeout (the
 * status a resident run turns into RC_E_TIMEOUT); *seconds = host time of
 * the call.  The device stays usable. */
int rc_diag_grid_barrier(uint32_t limit_us, int32_t *timed_out, double *seconds);

/* Classification strategy for later calls: 0 = automatic (one CTA for small
 * instances, else resident when possible, else size-based), 1 = radix sort
 * of the whole log + segmented scan, 2 = shadow-cell owner table + sort of
 * shared cells only, both one launch sequence per barrier interval; 3 =
 * resident: when every work-group fits on the GPU at once (and the group
 * size is a multiple of 32, barriers are kernel-wide), one cooperative
 * launch runs every interval with the owner table, committing in-kernel
 * between grid-wide barriers, and the shared cells' records are sorted
 * after the run; otherwise as 0; 4 = one CTA: when the instance has at most
 * 1024 work-items, at most 4096 logged accesses per interval (its static
 * bound) and at most 63 barriers, one launch of one CTA runs every
 * interval, sorts and classifies each interval's log in shared memory by
 * the same rules and applies the barrier-release rule, and writes the
 * report to page-locked host memory (kernel-wide barriers; the
 * interpreter); otherwise as 0.  Batches take 3 and 4 as 0.  Returns
 * RC_E_INVALID for other values. */
int rc_set_strategy(int strategy);

/* Engine of the interval kernels for later rc_check / rc_search calls:
 * 0 = automatic (compiled intervals for instances of at least 2^17
 * work-items when NVRTC can be loaded, else the interpreter), 1 = the
 * bytecode interpreter, 2 = compiled intervals (rc_check then returns
 * RC_E_INVALID when NVRTC cannot be loaded).  Compiled intervals translate
 * the program's bytecode into one straight-line function per program
 * (rc_translate) and compile it, with the interpreter's access, logging and
 * barrier steps, into an interval kernel of its own at run time (NVRTC,
 * sm_103a; cached per program, launch shape and mode).  Reports are the
 * same under both engines.  Work-group-scoped barriers, batches and the
 * explorers always interpret.  Returns RC_E_INVALID for other values. */
int rc_set_engine(int engine);

/* Compile the interval kernel of (bc, groups, group_size, in) -- the
 * pre-filter's private accesses for that launch shape included -- without
 * loading it (no GPU needed): a check of the generated source.  resident:
 * the kernel of one-launch runs instead of one launch per interval.
 * *seconds = compile time (0 when it was cached), *cubin_bytes = its size
 * (either may be NULL).  RC_E_INVALID when NVRTC cannot be loaded or the
 * compile fails (message in rc_last_error()). */
int rc_jit_compile(const rc_bytecode *bc, uint32_t groups, uint32_t group_size, const rc_input *in, int resident,
                   double *seconds, uint64_t *cubin_bytes);
/* Interval kernels compiled so far by this process and their total compile seconds. */
int rc_jit_stats(uint64_t *compiles, double *seconds);

/* Autotuner of the classification strategy (strategy 0 above).  Per size
 * class -- single instances by work-items and per-interval access bound,
 * batches by warp tasks and bound -- an undecided class alternates the two
 * exact strategies on successive intervals (or batch rounds), times each,
 * and keeps the cheaper one after two samples of each; a batch class then
 * times each block shape of the batch interpreter (128, 256, 512 threads per
 * CTA) on two rounds and keeps the fastest.  A batch class's log capacity:
 * the first call gives every warp's slice the program's static per-interval
 * bound (overflow impossible) and records the fullest slice; later calls of
 * the class allocate twice the largest fill seen (in permille of the bound,
 * at least 16); a call that overflows that capacity is checked again at the
 * bound, which the class keeps (the reports are the same either way).
 * Decisions persist in
 * a JSON file: cache_path, or NULL for the default ($RC_TUNE_CACHE, else
 * $XDG_CACHE_HOME/racecheck_autotune.json, else
 * ~/.cache/racecheck_autotune.json), or "" for no file. */
int rc_autotune_config(const char *cache_path);
/* Forget every decision held in memory (the cache file is not touched). */
int rc_autotune_reset(void);
/* Decision for a size class: kind 0 single (a = work-items, b = accesses per
 * work-item per interval bound), kind 1 batch (a = warp tasks, b = bound);
 * returns 1 (sort), 2 (shadow) or 0 if undecided.  Kind 2: the batch size
 * class's block shape -- threads per CTA of the batch interpreter, 128, 256
 * or 512 (1024 threads per SM in every case), which the autotuner times on
 * two batch rounds each once the strategy is decided -- or 0 if undecided.
 * Kind 3: the batch class's log capacity in permille of the static bound
 * (1..1000), or 0 if no call of the class has finished. */
int rc_autotune_lookup(int kind, uint64_t a, uint64_t b);

/* Kernel timing: when enabled, the library brackets its work with CUDA
 * events on the caller's stream and accumulates, per kind, the number of
 * intervals (or batch rounds), device milliseconds and algorithmic bytes
 * (12 per logged global access).  kind 0: the interpreter launch; kind 1:
 * everything after it until the interval's classification is done (owner-
 * table commit, compaction, sort and classification, and any wait for the
 * host in between); kind 2: batch calls (rc_check_batch), wall-clock
 * milliseconds of the host's own work in each call -- the set-up before the
 * first round (layout, descriptors, uploads queued) and the reports after
 * the last classification -- with launches counting the calls and bytes
 * zero.  Timing an interval
 * synchronises it, so the speculative launch of the next interval is off
 * while enabled.  Reset clears the sums. */
int rc_profile_enable(int on);
int rc_profile_reset(void);
int rc_profile_get(int kind, uint64_t *launches, double *ms, double *bytes);

/* Number of CUDA kernels the library has launched since it was loaded
 * (every launch counts, whatever the profiling state). */
uint64_t rc_kernel_launches(void);

/* ---- exhaustive interleavings of small instances
 *
 * The checker runs one canonical schedule per barrier interval and flags
 * conflicts conservatively.  Sec. 4 defines a race over ALL schedules: two
 * schedules reaching different shared states at a barrier.  rc_explore runs
 * the instance like rc_check and, before each of its first max_intervals
 * intervals, runs every schedule of that interval with one truly shared
 * memory from the checker's state at the interval's start: a flagged
 * interval is confirmed when several shared states are reachable at its
 * closing barrier or a read depends on the schedule. */
typedef struct {
  uint32_t interval;
  uint32_t n_end_states; /* distinct shared memories (global + local) at the closing barrier */
  uint32_t deviated;     /* 1: in some schedule some read differs from its work-item's solo run */
  uint32_t complete;     /* 1: every schedule explored within max_states */
  uint64_t n_states;     /* distinct states visited */
} rc_explore_interval;
/* Explore every schedule of the first max_intervals intervals of a small
 * instance (groups * group_size <= 16 work-items, <= 4096 cells, <= 64
 * registers).  out holds max_intervals entries; *n_out receives the number
 * filled (the run's intervals, at most max_intervals).  max_states bounds
 * the distinct states per interval (0: 1,000,000); beyond it an interval is
 * reported incomplete.  Errors: RC_E_INVALID, RC_E_CAPACITY, RC_E_CUDA. */
int rc_explore(const rc_bytecode *bc, uint32_t groups, uint32_t group_size, const rc_input *in, uint64_t max_states,
               rc_explore_interval *out, uint32_t max_intervals, uint32_t *n_out);

/* The interleaving product of two work-items (the fix proposed at the end of
 * Sec. 6 for a symbolic execution that misses branches on array values):
 * for every pair i < j of the instance's work-items, every schedule of the
 * two alone (all other work-items do not run) from the checker's state at
 * the start of each of the first max_intervals intervals.  It scales to
 * more work-items than rc_explore, at the price of missing races that need
 * three or more work-items to show. */
typedef struct {
  uint32_t interval;
  uint32_t n_pairs;          /* pairs (i < j): N (N - 1) / 2                          */
  uint32_t n_racy;           /* pairs reaching two or more shared memories            */
  uint32_t n_deviated;       /* pairs with a read that depends on the schedule        */
  uint32_t first_i, first_j; /* smallest racy pair in (i, j) order, 0xFFFFFFFF if none */
  uint32_t complete;         /* 1: every schedule explored within max_states          */
  uint32_t reserved;
  uint64_t n_states;         /* distinct (pair, state) items visited                  */
} rc_pair_interval;
/* groups * group_size <= 256 work-items, <= 4096 cells, <= 64 registers.
 * pair_detail (may be NULL) receives max_intervals x n_pairs values, pairs in
 * (i, j) order: distinct shared memories | (schedule-dependent read) << 31. */
int rc_explore_pairs(const rc_bytecode *bc, uint32_t groups, uint32_t group_size, const rc_input *in,
                     uint64_t max_states, rc_pair_interval *out, uint32_t max_intervals, uint32_t *n_out,
                     uint32_t *pair_detail);

/* ---- two-work-item NoRace pre-filter (no GPU work)
 *
 * A restricted, sound form of the paper's symbolic method (Sec. 5-6: two
 * renamed work-items i != j; Table 1's bounds premise).  Every register is
 * tracked as an affine form in tid, wg and the counters of constant-trip
 * loops (optionally reduced modulo a constant) by a fixpoint over the
 * bytecode's control flow; a compare-and-branch on an affine function of
 * tid (or wg) narrows the work-items that reach its then-region.  For the
 * launch shape groups x group_size and the input lengths (global_init is
 * not read), race_free = 1 means no two work-items
 * can make a conflicting pair of accesses in one barrier interval under any
 * schedule: every pair of accesses to one array (one a store) in a common
 * barrier region has disjoint index ranges, or the same index form that is
 * one-to-one on the work-items (one group's, for local arrays), or -- when
 * the work-items and loop counters of the pair can be enumerated (up to
 * 2^16 points per access, 2^20 per call) -- no cell reached by two work-items,
 * or both store one constant.  race_free = 0 decides nothing (the checker does);
 * first_pc_a/b name the first pair left open.  in_bounds = 1 means every
 * index is provably within its array. */
typedef struct {
  int32_t race_free;
  int32_t in_bounds;
  uint32_t first_pc_a, first_pc_b; /* bytecode positions, 0xFFFFFFFF if none */
  uint32_t n_pairs;                /* access pairs that may meet in one interval */
  uint32_t n_unresolved;           /* pairs the pre-filter could not clear      */
} rc_prove_result;
int rc_prove(const rc_bytecode *bc, uint32_t groups, uint32_t group_size, const rc_input *in, rc_prove_result *out);

/* Private accesses of the same analysis: flags[pc] = 1 (n_flags >= the
 * bytecode's instruction count) for a load or store whose cells never carry
 * a race or benign record.  Pairs with another work-item's access in a
 * common barrier interval (same array) are cleared only by disjoint index
 * ranges or a one-to-one index, never by equal values.  A store: every pair
 * with a load or store cleared, so no other work-item touches its cells in
 * its interval.  A load: every pair with a store cleared, and every pair
 * with another load L' cleared unless all of L''s pairs with stores are --
 * other work-items may read its cells, but none of them reads a cell that
 * a different work-item writes, so a work-item reading back its own store
 * never meets a reader of that cell.  The checker (owner-table and resident
 * runs) skips logging these accesses and claims only their stores.  This is
 * the analysis the checker runs for every launch shape, without rc_prove's
 * enumeration of small launches.  *n_private = the count. */
int rc_prove_private(const rc_bytecode *bc, uint32_t groups, uint32_t group_size, const rc_input *in,
                     uint8_t *flags, uint32_t n_flags, uint32_t *n_private);

/* The shared-access instructions of a compiled kernel (one per array read
 * or store of the kernel text, Sec. 3's v:=a[v] and a[v]:=e), in bytecode
 * order, which is text order: a statement's array reads left to right, an
 * index before the read that uses it, a store after the reads in its index
 * and value.  Entry k: pc[k] = the instruction's position (its index into
 * rc_prove_private's flags), is_store[k], mem[k] = the memory object
 * (declared order).  The caller owns the arrays; min(cap, count) entries
 * are written (cap 0: the arrays may be NULL) and *n_sites = count. */
int rc_access_sites(const rc_bytecode *bc, uint32_t *pc, uint8_t *is_store, uint32_t *mem, uint32_t cap,
                    uint32_t *n_sites);

/* The kernel translated into C++ source text (the thread-local rules of
 * Sec. 4 for one work-item, compiled instead of interpreted): one function
 *   RC_JIT_FN void fn_name(RC_JIT_CTX &cx, int32_t (&r)[n_regs],
 *                          uint32_t &pc, uint32_t &st)
 * that runs a work-item from pc (0, or the instruction after a barrier) to
 * its next barrier (st = 1, pc = where to resume), its exit (st = 2) or its
 * end (st = 3: a failed assume or assert, an out-of-bounds access); r[0..4]
 * hold tid, wg, gtid, group size and group count.  Shared memory is reached
 * through hooks the including code defines (RC_LD, RC_ST, RC_SIZE,
 * RC_ASSERT_FAIL, RC_AT_BARRIER; see translate.cpp), and the text calls
 * rc::sem_div, rc::sem_mod and rc::sem_index.  fn_name must be a C
 * identifier of at most 128 characters (else RC_E_INVALID).  Writes min(len, cap - 1) bytes and a NUL into buf (cap 0:
 * buf may be NULL); *len = the text's length.  The text compiles as CUDA
 * C++ and as plain C++. */
int rc_translate(const rc_bytecode *bc, const char *fn_name, char *buf, size_t cap, size_t *len);

/* ---- learned proposal: which candidate instances to check first
 *
 * The method needs, per kernel, a set of candidate instances (launch shape
 * and input); checking them in a good order finds a race sooner.  These
 * calls rank candidates with a small network trained on the checker's own
 * labels.  A ranking never decides a verdict: every race is found and
 * reported by rc_check; candidates never checked are not claimed race-free. */

#define RC_N_FEATURES 128
#define RC_MLP_IN 128
#define RC_MLP_HIDDEN 256
#define RC_MLP_PARAMS 164865 /* 256*128 + 256 + 2 * (256*256 + 256) + 256 + 1 */

/* Feature vector (RC_N_FEATURES floats) of the candidate instance (bc,
 * groups, group_size, in): opcode histogram and size counts of the kernel;
 * per access class (global/local x load/store) how indices depend on tid
 * and wg, how many work-items reach the accesses, branches on loaded
 * values, values that vary between work-items, and whether two work-items
 * of this shape must meet on a cell; collisions among a sample of the
 * instance's work-items evaluated on its input; the launch shape.  Host
 * inputs only (in->on_device must be 0).  Errors: RC_E_INVALID. */
int rc_features(const rc_bytecode *bc, uint32_t groups, uint32_t group_size, const rc_input *in, float *out);
/* rc_features for n candidates into out[n][RC_N_FEATURES], on n_threads host
 * threads (<= 0: one per 8 candidates, at most the host's cores; the
 * library keeps its worker threads between calls).  The result does not
 * depend on n_threads. */
int rc_features_batch(const rc_bytecode *const *bcs, const uint32_t *groups, const uint32_t *group_size,
                      const rc_input *inputs, size_t n, float *out, int n_threads);

/* Ranking network: MLP RC_MLP_IN -> 256 -> 256 -> 256 -> 1, ReLU hidden
 * layers, sigmoid output (probability that the candidate is racy).  FP32
 * master weights; products on BF16 tensor cores with FP32 accumulation.
 * Parameter vector layout (FP32, RC_MLP_PARAMS values): W1[256][128] b1[256]
 * W2[256][256] b2[256] W3[256][256] b3[256] w4[256] b4; layer l computes
 * h_l = relu(W_l h_{l-1} + b_l), the score is sigmoid(w4 . h3 + b4).
 * Feature, label and score arrays are device pointers (float, row-major
 * [n][RC_MLP_IN], [n], [n]); work runs on cuda_stream and is synchronised. */
typedef struct rc_mlp rc_mlp;
/* New network with He-uniform weights from `seed`, zero biases; capacity =
 * rows per device pass (training batch <= capacity). */
int rc_mlp_create(uint64_t seed, uint32_t capacity, rc_mlp **out);
void rc_mlp_free(rc_mlp *m);
int rc_mlp_get_params(const rc_mlp *m, float *host_out);
/* Every product (forward, data and weight gradients) on the tcgen05 kernels
 * with TMEM accumulators -- the three forward layers in one launch (backend
 * 1, the default) or one launch per layer (backend 2, the same values) -- or
 * on the mma.sync m16n8k16 kernels (backend 0).  rc_mlp_backend_error sets
 * *flag nonzero if a tcgen05 launch gave up waiting for its MMAs (its
 * outputs are then not valid). */
int rc_mlp_set_backend(rc_mlp *m, int backend);
int rc_mlp_backend_error(rc_mlp *m, uint32_t *flag);
int rc_mlp_set_params(rc_mlp *m, const float *host_in);
/* prob[i] = score of row i of x, for n rows. */
int rc_mlp_forward(rc_mlp *m, const float *x, uint64_t n, float *prob, void *cuda_stream);
/* Mean binary cross-entropy of the n <= capacity rows (labels y in {0,1})
 * and its gradient with respect to every parameter (host_grad: RC_MLP_PARAMS
 * floats, may be NULL); no update. */
int rc_mlp_grad(rc_mlp *m, const float *x, const float *y, uint32_t n, float *host_grad, float *host_loss,
                void *cuda_stream);
/* Train with Adam (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on the mean
 * binary cross-entropy, `epochs` passes over n rows in minibatches of
 * `batch`, rows shuffled per epoch from `seed`.  epoch_loss (host, epochs
 * floats, may be NULL) receives each epoch's mean minibatch loss. */
int rc_mlp_train(rc_mlp *m, const float *x, const float *y, uint64_t n, uint32_t epochs, uint32_t batch, float lr,
                 uint64_t seed, float *epoch_loss, void *cuda_stream);

/* Search for a racy candidate: check candidates (as rc_check) in descending
 * order of scores[i] (host array; ties keep their index order), or in index
 * order when scores is NULL (plain enumeration), until one report has status
 * RC_RACY or max_checks candidates (0 = all) were checked.  res->first is
 * that candidate's index or -1, res->checks the checks made, res->seconds
 * the host wall time of the checks.  found (may be NULL) receives the racy
 * candidate's report.  A check error stops the search and is returned. */
typedef struct {
  int64_t first;
  uint32_t checks;
  uint32_t reserved;
  double seconds;
} rc_search_result;
int rc_search(const rc_bytecode *const *bcs, const uint32_t *groups, const uint32_t *group_size,
              const rc_input *inputs, size_t n, const float *scores, uint32_t max_checks, rc_search_result *res,
              rc_report **found);

/* Ranked search in one call: the candidates' features (rc_features) are
 * computed on the host's worker threads, scored by `model` (rc_mlp_forward
 * on the stream of inputs[0]) or, when model is NULL, by the rule
 *   4 f[108] + 2 f[107] + (f[104] + f[105]) / 10   (float arithmetic)
 * (a race predicted by the index analysis, then sampled collisions), and
 * checked as rc_search does in descending score order (ties keep their
 * index order) until one is racy or max_checks checks (0 = all) were made.
 * With RC_RANK_OVERLAP the GPU does not wait for the ranking: candidates are
 * checked in index order while the features are computed, and the ranked
 * order takes over, skipping what was checked, once the scores exist (a
 * race found first ends the search and the feature work is abandoned).
 * Every reported race comes from an exact check.  res: the racy
 * candidate's index or -1, checks made (checks_unranked of them in index
 * order before the ranking), the call's host wall time and its parts.
 * found as for rc_search.  Host inputs only; errors as rc_search and
 * rc_features. */
#define RC_RANK_OVERLAP 1u
typedef struct {
  int64_t first;
  uint32_t checks;
  uint32_t checks_unranked;
  double seconds;          /* whole call */
  double features_seconds; /* from the call's start until every feature vector existed */
  double scoring_seconds;  /* network (or rule) scores and their order */
  double check_seconds;    /* in exact checks */
} rc_ranked_result;
int rc_search_ranked(rc_mlp *model, const rc_bytecode *const *bcs, const uint32_t *groups,
                     const uint32_t *group_size, const rc_input *inputs, size_t n, uint32_t max_checks,
                     uint32_t flags, rc_ranked_result *res, rc_report **found);

#ifdef __cplusplus
}
#endif
#endif /* RACECHECK_H */
