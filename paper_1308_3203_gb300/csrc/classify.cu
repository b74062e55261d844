// Race classification of one barrier interval from its access log sorted by
// (cell, work-item), and the commit of the interval's writes.
//
// Step 1 (run reduce): every run of records of one (cell, work-item) becomes
// a Summary: the range of values the work-item observed, the range it wrote,
// the value of its last write (highest sequence number) and its access count.
// The kernel of the last run also stores the number of summaries in device
// memory, so the later steps run over an upper bound (the record count)
// without the host reading the exact counts in between.
//
// Step 2 (per cell, over the summaries of that cell in work-item order):
//  * WW (Sec. 1 and the race rule of Sec. 4: differing values at a barrier
//    are a race, one common value is benign): each writer's LAST value
//    counts.  Two writers whose last values differ -> WW_RACE with witness
//    (smallest writer w1, smallest writer whose last value differs from
//    w1's); two or more writers, one value -> WW_BENIGN (w1, w2).
//  * RW: a read by r that observed o conflicts with a write by j != r of a
//    value v != o.  Witness: the lexicographically smallest (r, j).  A reader
//    r that observed one value c conflicts with the smallest writer j != r
//    that did not write c alone; one that observed several values conflicts
//    with the smallest writer j != r.  One forward pass over the writers
//    collects the few candidates this needs (w1, w2, the first two writers
//    differing from w1's value, the first writer after w2 differing from
//    w2's value); a second pass stops at the first reader with a conflict.
//  * commit: the cell takes the last write of its highest writer (the
//    schedule that runs work-items in id order).
#include "device.cuh"
#include "classify_cell.cuh"

namespace rc {
namespace {

constexpr int kThreads = 256;

__global__ void run_heads_kernel(const LogRec *r, uint64_t n, uint32_t *head) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t h = 1;
  if (i > 0) {
    const LogRec a = r[i - 1], b = r[i];
    h = (a.key != b.key || ((a.tw ^ b.tw) & 0x7FFFFFFFu) != 0) ? 1u : 0u;
  }
  head[i] = h;
}

__global__ void run_reduce_kernel(const LogRec *r, uint64_t n, const uint32_t *head,
                                  const uint32_t *runidx, Summary *sum, uint32_t *khead, uint32_t *nsum) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !head[i]) return;
  uint64_t j = 0;
  const Summary s = summarize_run(r, i, n, j);
  const uint32_t k = runidx[i];
  sum[k] = s;
  khead[k] = (i == 0 || r[i - 1].key != s.key) ? 1u : 0u;
  if (j == n) *nsum = k + 1;  // the last run
}

// The first summary of every cell, by cell index (keyidx: exclusive scan of
// the cell heads), and the number of cells in *a.ncell: the per-cell kernels
// then run one thread per cell, so that a warp's lanes all walk cells
// instead of one lane in a cell's worth of summaries.
__global__ void cell_starts_kernel(const uint32_t *khead, const uint32_t *keyidx, ClassifyArgs a) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nsum = *a.nsum;
  if (i >= nsum) return;
  const uint32_t h = khead[i], k = keyidx[i];
  if (h) a.cstart[k] = (uint32_t)i;
  if (i + 1 == nsum) *a.ncell = k + h;
}

// One thread per cell (launched over an upper bound).
__global__ void key_classify_kernel(const Summary *sum, uint32_t *nrec, ClassifyArgs a) {
  const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= *a.ncell) return;
  const uint64_t nsum = *a.nsum, i = a.cstart[q];
  if (i + kBigCell < nsum && sum[i + kBigCell].key == sum[i].key) {  // a large cell: one CTA's work
    a.big[atomicAdd(a.nbig, 1u)] = (uint32_t)i;
    return;
  }
  const CellResult c = classify_cell(sum, i, nsum);
  if (c.wrote && a.snap) a.snap[sum[i].key] = c.commit;  // no snapshot: commits were made already
  const uint32_t nr = (c.ww_cls ? 1u : 0u) + (c.rw_a != kNone ? 1u : 0u);
  nrec[q] = nr;
  if (nr) a.cellres[q] = c;
}

__global__ void key_emit_kernel(const Summary *sum, const uint32_t *nrec, const uint32_t *recoff, OutRec *out,
                                ClassifyArgs a) {
  const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= *a.ncell || nrec[q] == 0) return;
  const uint64_t nsum = *a.nsum, i = a.cstart[q];
  if (i + kBigCell < nsum && sum[i + kBigCell].key == sum[i].key) return;  // emitted by big_emit
  emit_cell(a, sum[i].key, a.cellres[q], recoff[q], out);
}

// ---- large cells: one CTA per cell, three sweeps over its summaries.
// Every candidate is "the first summary (in work-item order) with a
// property", so each thread keeps the first offsets it meets in its stride
// and the block takes the minimum: the same witnesses as classify_cell.
constexpr int kBigThreads = 256;

__device__ __forceinline__ void two_min(uint32_t &a1, uint32_t &a2, uint32_t b1, uint32_t b2) {
  const uint32_t m1 = min(a1, b1);
  a2 = min(max(a1, b1), min(a2, b2));  // a1 <= a2 and b1 <= b2
  a1 = m1;
}

// block-wide reductions; every thread gets the result (sh: 2 * 32 words)
__device__ __forceinline__ uint32_t block_sum(uint32_t x, uint32_t *sh) {
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
  __syncthreads();
  if ((threadIdx.x & 31u) == 0) sh[threadIdx.x >> 5] = x;
  __syncthreads();
  uint32_t t = 0;
  for (uint32_t w = 0; w < blockDim.x / 32u; w++) t += sh[w];
  return t;
}
__device__ __forceinline__ uint32_t block_min(uint32_t x, uint32_t *sh) {
  x = __reduce_min_sync(0xFFFFFFFFu, x);
  __syncthreads();
  if ((threadIdx.x & 31u) == 0) sh[threadIdx.x >> 5] = x;
  __syncthreads();
  uint32_t t = kNone;
  for (uint32_t w = 0; w < blockDim.x / 32u; w++) t = min(t, sh[w]);
  return t;
}
__device__ __forceinline__ uint32_t block_max(uint32_t x, uint32_t *sh) {
  x = __reduce_max_sync(0xFFFFFFFFu, x);
  __syncthreads();
  if ((threadIdx.x & 31u) == 0) sh[threadIdx.x >> 5] = x;
  __syncthreads();
  uint32_t t = 0;
  for (uint32_t w = 0; w < blockDim.x / 32u; w++) t = max(t, sh[w]);
  return t;
}
__device__ __forceinline__ void block_two_min(uint32_t &a1, uint32_t &a2, uint32_t *sh) {
  for (int o = 16; o; o >>= 1) {
    const uint32_t b1 = __shfl_xor_sync(0xFFFFFFFFu, a1, o), b2 = __shfl_xor_sync(0xFFFFFFFFu, a2, o);
    two_min(a1, a2, b1, b2);
  }
  __syncthreads();
  if ((threadIdx.x & 31u) == 0) {
    sh[threadIdx.x >> 5] = a1;
    sh[32 + (threadIdx.x >> 5)] = a2;
  }
  __syncthreads();
  a1 = kNone;
  a2 = kNone;
  for (uint32_t w = 0; w < blockDim.x / 32u; w++) two_min(a1, a2, sh[w], sh[32 + w]);
}

__global__ void __launch_bounds__(kBigThreads) big_classify_kernel(const Summary *sum, uint64_t nsum,
                                                                   const uint32_t *keyidx, uint32_t *nrec,
                                                                   ClassifyArgs a) {
  __shared__ uint32_t sh[64];
  __shared__ CellVals sv;
  __shared__ int32_t s_commit;
  const uint32_t t = threadIdx.x, nt = blockDim.x;
  const uint32_t nbig = *a.nbig;
  nsum = *a.nsum;
  for (uint32_t q = blockIdx.x; q < nbig; q += gridDim.x) {
    const uint64_t b = a.big[q];
    const uint32_t key = sum[b].key;
    // pass 1: extent, counts, first two writers, last writer
    uint32_t nacc = 0, nr = 0, nw = 0, f1 = kNone, f2 = kNone, lastw = 0, endo = kNone;
    for (uint64_t base = b;; base += nt) {
      const uint64_t i = base + t;
      const bool in = i < nsum && sum[i].key == key;
      if (in) {
        const Summary s = sum[i];
        const uint32_t o = (uint32_t)(i - b);
        nacc += s.meta & kMetaCount;
        if (s.meta & kMetaRead) nr++;
        if (s.meta & kMetaWrite) {
          nw++;
          if (f1 == kNone) f1 = o;
          else if (f2 == kNone) f2 = o;
          lastw = o + 1;
        }
      } else if (endo == kNone) {
        endo = (uint32_t)(i - b);
      }
      if (__syncthreads_or(!in)) break;  // sorted by cell: nothing of it lies further on
    }
    const uint32_t end = block_min(endo, sh);
    nacc = block_sum(nacc, sh);
    nr = block_sum(nr, sh);
    nw = block_sum(nw, sh);
    block_two_min(f1, f2, sh);
    lastw = block_max(lastw, sh);
    if (t == 0) {
      CellVals v{kNone, kNone, kNone, kNone, kNone, kNone, {true, 0}, {true, 0}, 0};
      if (f1 != kNone) {
        const Summary s = sum[b + f1];
        v.w1 = s.gtid;
        v.u1 = written(s);
        v.l1 = s.wlast;
      }
      if (f2 != kNone) {
        const Summary s = sum[b + f2];
        v.w2 = s.gtid;
        v.u2 = written(s);
      }
      sv = v;
      s_commit = lastw ? sum[b + lastw - 1].wlast : 0;
    }
    __syncthreads();
    const CellVals v0 = sv;
    // pass 2: writers after w1 (tb, d1, d2) and after w2 (e2)
    uint32_t tbo = kNone, e2o = kNone, d1o = kNone, d2o = kNone;
    if (nw >= 2) {
      for (uint32_t o = t; o < end; o += nt) {
        const Summary s = sum[b + o];
        if (!(s.meta & kMetaWrite) || o <= f1) continue;
        const Uni u = written(s);
        if (tbo == kNone && s.wlast != v0.l1) tbo = o;
        if (!v0.u1.mixed && !same(u, v0.u1)) {
          if (d1o == kNone) d1o = o;
          else if (d2o == kNone) d2o = o;
        }
        if (e2o == kNone && o > f2 && !same(u, v0.u2)) e2o = o;
      }
    }
    tbo = block_min(tbo, sh);
    e2o = block_min(e2o, sh);
    block_two_min(d1o, d2o, sh);
    if (t == 0) {
      if (tbo != kNone) sv.tb = sum[b + tbo].gtid;
      if (e2o != kNone) sv.e2 = sum[b + e2o].gtid;
      if (d1o != kNone) sv.d1 = sum[b + d1o].gtid;
      if (d2o != kNone) sv.d2 = sum[b + d2o].gtid;
    }
    __syncthreads();
    const CellVals v = sv;
    // pass 3: first reader with a conflict
    uint32_t ro = kNone;
    if (nw > 0 && nr > 0) {
      for (uint32_t o = t; o < end && ro == kNone; o += nt) {
        const Summary s = sum[b + o];
        if ((s.meta & kMetaRead) && reader_conflict(s, v) != kNone) ro = o;
      }
    }
    ro = block_min(ro, sh);
    if (t == 0) {
      CellResult c{};
      c.n_readers = nr;
      c.n_writers = nw;
      c.n_acc = nacc;
      set_ww(c, v);
      c.rw_a = kNone;
      if (ro != kNone) {
        const Summary s = sum[b + ro];
        c.rw_a = s.gtid;
        c.rw_b = reader_conflict(s, v);
      }
      c.wrote = nw > 0;
      c.commit = s_commit;
      if (c.wrote && a.snap) a.snap[key] = c.commit;
      nrec[keyidx[b]] = (c.ww_cls ? 1u : 0u) + (c.rw_a != kNone ? 1u : 0u);
      a.bigres[q] = c;
    }
    __syncthreads();
  }
}

__global__ void big_emit_kernel(const Summary *sum, const uint32_t *keyidx, const uint32_t *nrec,
                                const uint32_t *recoff, OutRec *out, ClassifyArgs a) {
  const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= *a.nbig) return;
  const uint32_t i = a.big[q], k = keyidx[i];
  if (nrec[k]) emit_cell(a, sum[i].key, a.bigres[q], recoff[k], out);
}

unsigned blocks_for(uint64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

void launch_run_heads(const LogRec *r, uint64_t n, uint32_t *head, cudaStream_t s) {
  if (n) count_launch();
  if (n) run_heads_kernel<<<blocks_for(n), kThreads, 0, s>>>(r, n, head);
}
void launch_run_reduce(const LogRec *r, uint64_t n, const uint32_t *head, const uint32_t *runidx,
                       Summary *sum, uint32_t *khead, uint32_t *nsum, cudaStream_t s) {
  if (n) count_launch();
  if (n) run_reduce_kernel<<<blocks_for(n), kThreads, 0, s>>>(r, n, head, runidx, sum, khead, nsum);
}
void launch_cell_starts(const uint32_t *khead, const uint32_t *keyidx, uint64_t n, const ClassifyArgs &a,
                        cudaStream_t s) {
  if (n) count_launch();
  if (n) cell_starts_kernel<<<blocks_for(n), kThreads, 0, s>>>(khead, keyidx, a);
}
void launch_key_classify(const Summary *sum, uint64_t n, uint32_t *nrec, const ClassifyArgs &a, cudaStream_t s) {
  if (n) count_launch();
  if (n) key_classify_kernel<<<blocks_for(n), kThreads, 0, s>>>(sum, nrec, a);
}
void launch_key_emit(const Summary *sum, uint64_t n, const uint32_t *nrec, const uint32_t *recoff, OutRec *out,
                     const ClassifyArgs &a, cudaStream_t s) {
  if (n) count_launch();
  if (n) key_emit_kernel<<<blocks_for(n), kThreads, 0, s>>>(sum, nrec, recoff, out, a);
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}
void launch_big_classify(const Summary *sum, uint64_t nsum, const uint32_t *keyidx, uint32_t *nrec,
                         const ClassifyArgs &a, cudaStream_t s) {
  if (nsum <= kBigCell) return;  // no cell can be large
  count_launch();
  const uint64_t grid = std::min<uint64_t>(big_cells_cap(nsum), (uint64_t)sm_count() * 8);
  big_classify_kernel<<<(unsigned)grid, kBigThreads, 0, s>>>(sum, nsum, keyidx, nrec, a);
}
void launch_big_emit(const Summary *sum, uint64_t nsum, const uint32_t *keyidx, const uint32_t *nrec,
                     const uint32_t *recoff, OutRec *out, const ClassifyArgs &a, cudaStream_t s) {
  if (nsum <= kBigCell) return;
  count_launch();
  big_emit_kernel<<<blocks_for(big_cells_cap(nsum)), kThreads, 0, s>>>(sum, keyidx, nrec, recoff, out, a);
}

}  // namespace rc
