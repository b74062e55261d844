// Device-wide exclusive scan and a stable LSD radix sort of access-log
// records by (cell, work-item).
//
// Scan: tiles of 2048 uint32 (256 threads x 8); per-tile sums are scanned
// recursively, then each tile is scanned and offset.
//
// Radix sort: 8-bit digits of the composite key (key << gbits | gtid), least
// significant first.  Per pass: (1) per-tile digit histograms, written digit-
// major so that (2) one exclusive scan gives every (digit, tile) its output
// offset, (3) each tile ranks its records stably - warps own contiguous
// 256-record segments, ranks within a warp come from __match_any_sync, and
// per-warp digit counters are prefixed across warps - and scatters them.
// Stability keeps the records of one (cell, work-item) in log order.
#include "device.cuh"

namespace rc {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;  // 2048
constexpr int kWarps = kThreads / 32;
static_assert(kThreads == 256, "thread d owns radix digit d");

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *warp_sums, uint32_t &total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t s = lane < kWarps ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kWarps) warp_sums[lane] = s;  // inclusive
  }
  __syncthreads();
  total = warp_sums[kWarps - 1];
  uint32_t before = w ? warp_sums[w - 1] : 0;
  uint32_t r = before + x - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kThreads) tile_sum_kernel(const uint32_t *in, uint64_t n, uint32_t *sums) {
  __shared__ uint32_t ws[kWarps];
  const uint64_t base = (uint64_t)blockIdx.x * kTile + (uint64_t)threadIdx.x * kItems;
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kItems; i++)
    if (base + i < n) s += in[base + i];
  uint32_t total;
  block_excl_scan(s, ws, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kThreads) tile_scan_kernel(const uint32_t *in, uint64_t n, uint32_t *out,
                                                             const uint32_t *offs) {
  __shared__ uint32_t ws[kWarps];
  const uint64_t base = (uint64_t)blockIdx.x * kTile + (uint64_t)threadIdx.x * kItems;
  uint32_t v[kItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kItems; i++) {
    v[i] = base + i < n ? in[base + i] : 0;
    s += v[i];
  }
  uint32_t total;
  uint32_t run = block_excl_scan(s, ws, total) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
  for (int i = 0; i < kItems; i++) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
}

// One CTA of 1024 threads scans up to kSmallScan values in one launch (the
// tiled scan takes three): warp w owns the contiguous chunk [w * 2048,
// (w + 1) * 2048), read coalesced 32 values at a time; a first sweep sums
// the chunk, the CTA scans the 32 warp sums, a second sweep writes the
// running prefix.
constexpr int kSmallThreads = 1024;
constexpr uint64_t kSmallChunk = 2048;
constexpr uint64_t kSmallScan = kSmallChunk * (kSmallThreads / 32);  // 65,536

__global__ void __launch_bounds__(kSmallThreads) small_scan_kernel(const uint32_t *in, uint64_t n, uint32_t *out) {
  __shared__ uint32_t wsum[32];
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  const uint64_t lo = (uint64_t)w * kSmallChunk, hi = lo + kSmallChunk < n ? lo + kSmallChunk : n;
  uint32_t part = 0;
  for (uint64_t i = lo + lane; i < hi; i += 32) part += in[i];
  part = __reduce_add_sync(0xFFFFFFFFu, part);
  if (lane == 0) wsum[w] = part;
  __syncthreads();
  if (w == 0) {  // exclusive scan of the 32 warp sums
    const uint32_t v = wsum[lane];
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    wsum[lane] = x - v;
  }
  __syncthreads();
  uint32_t carry = wsum[w];
  for (uint64_t base = lo; base < hi; base += 32) {
    const uint64_t i = base + lane;
    const uint32_t v = i < hi ? in[i] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    if (i < hi) out[i] = carry + x - v;
    carry += __shfl_sync(0xFFFFFFFFu, x, 31);
  }
}

__device__ __forceinline__ uint32_t digit_of(const LogRec &r, uint32_t gbits, uint32_t shift) {
  const uint64_t k = ((uint64_t)r.key << gbits) | (uint64_t)(r.tw & 0x7FFFFFFFu);
  return (uint32_t)(k >> shift) & 0xFFu;
}

__global__ void __launch_bounds__(kThreads) radix_hist_kernel(const LogRec *in, uint64_t n, uint32_t gbits,
                                                              uint32_t shift, uint32_t *hist,
                                                              uint32_t ntiles) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kTile;
#pragma unroll
  for (int i = 0; i < kItems; i++) {
    const uint64_t k = base + (uint64_t)i * kThreads + threadIdx.x;
    if (k < n) atomicAdd(&h[digit_of(in[k], gbits, shift)], 1u);
  }
  __syncthreads();
  hist[(uint64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads) radix_scatter_kernel(const LogRec *in, LogRec *out, uint64_t n,
                                                                 uint32_t gbits, uint32_t shift,
                                                                 const uint32_t *offs, uint32_t ntiles) {
  __shared__ uint32_t cnt[kWarps][256];
  __shared__ uint32_t dstart[256], gstart[256], ws[kWarps];
  __shared__ LogRec stage[kTile];  // 32 KB
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < kWarps * 256; k += kThreads) (&cnt[0][0])[k] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kTile + (uint64_t)w * (32 * kItems);
  const uint32_t lt_mask = (1u << lane) - 1u;
  LogRec rec[kItems];
  uint32_t dig[kItems], rank[kItems];
#pragma unroll
  for (int i = 0; i < kItems; i++) {
    const uint64_t k = base + (uint64_t)i * 32 + lane;
    const bool valid = k < n;
    if (valid) rec[i] = in[k];
    dig[i] = valid ? digit_of(rec[i], gbits, shift) : 256u;
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, dig[i]);
    const uint32_t before = __popc(peers & lt_mask);
    const uint32_t c = valid ? cnt[w][dig[i]] : 0u;
    rank[i] = c + before;
    __syncwarp();
    if (valid && lane == 31 - __clz(peers)) cnt[w][dig[i]] = c + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // prefix each digit's counts across warps (thread d owns digit d), then
  // over the digits: the tile's records in digit order in shared memory
  uint32_t run = 0;
  for (int q = 0; q < kWarps; q++) {
    const uint32_t t = cnt[q][threadIdx.x];
    cnt[q][threadIdx.x] = run;
    run += t;
  }
  uint32_t tile_n;
  const uint32_t first = block_excl_scan(run, ws, tile_n);
  dstart[threadIdx.x] = first;
  gstart[threadIdx.x] = offs[(uint64_t)threadIdx.x * ntiles + blockIdx.x];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kItems; i++)
    if (dig[i] < 256u) stage[dstart[dig[i]] + cnt[w][dig[i]] + rank[i]] = rec[i];
  __syncthreads();
  // consecutive threads write consecutive records of one digit's run:
  // coalesced stores instead of one scattered 16-byte store per record
  for (uint32_t i = threadIdx.x; i < tile_n; i += kThreads) {
    const LogRec r = stage[i];
    const uint32_t d = digit_of(r, gbits, shift);
    out[(uint64_t)gstart[d] + (i - dstart[d])] = r;
  }
}

uint64_t tiles_of(uint64_t n) { return (n + kTile - 1) / kTile; }

}  // namespace

size_t scan_tmp_words(uint64_t n) {
  size_t words = 0;
  for (uint64_t m = n; m > 1;) {
    m = tiles_of(m);
    words += 2 * m + 1;
  }
  return words + 1;
}

void scan_exclusive(const uint32_t *in, uint32_t *out, uint64_t n, uint32_t *tmp, cudaStream_t s) {
  if (n == 0) return;
  const uint64_t t = tiles_of(n);
  if (t > 1 && n <= kSmallScan) {  // one launch instead of three
    count_launch();
    small_scan_kernel<<<1, kSmallThreads, 0, s>>>(in, n, out);
    return;
  }
  if (t == 1) {
    count_launch();
    tile_scan_kernel<<<1, kThreads, 0, s>>>(in, n, out, nullptr);
    return;
  }
  uint32_t *sums = tmp, *soffs = tmp + t;
  count_launch();
  tile_sum_kernel<<<(unsigned)t, kThreads, 0, s>>>(in, n, sums);
  scan_exclusive(sums, soffs, t, tmp + 2 * t, s);
  count_launch();
  tile_scan_kernel<<<(unsigned)t, kThreads, 0, s>>>(in, n, out, soffs);
}

size_t sort_tmp_words(uint64_t n) {
  const uint64_t h = 256 * tiles_of(n);
  return 2 * h + scan_tmp_words(h);
}

void sort_log_into(const LogRec *in, LogRec *out, LogRec *scratch, uint64_t n, uint32_t gbits, uint32_t bits,
                   uint32_t *tmp, cudaStream_t s) {
  const uint32_t passes = n <= 1 ? 0 : (bits + 7) / 8;
  if (passes == 0) {
    if (n) cudaMemcpyAsync(out, in, n * sizeof(LogRec), cudaMemcpyDeviceToDevice, s);
    return;
  }
  // pass order chosen so that the last pass writes `out` and `in` is never written
  const uint32_t ntiles = (uint32_t)tiles_of(n);
  const uint64_t h = 256ull * ntiles;
  uint32_t *hist = tmp, *offs = tmp + h, *stmp = tmp + 2 * h;
  const LogRec *src = in;
  LogRec *dst = (passes % 2) ? out : scratch;
  for (uint32_t p = 0, shift = 0; p < passes; p++, shift += 8) {
    count_launch();
    radix_hist_kernel<<<ntiles, kThreads, 0, s>>>(src, n, gbits, shift, hist, ntiles);
    scan_exclusive(hist, offs, h, stmp, s);
    count_launch();
    radix_scatter_kernel<<<ntiles, kThreads, 0, s>>>(src, dst, n, gbits, shift, offs, ntiles);
    src = dst;
    dst = dst == out ? scratch : out;
  }
}

LogRec *sort_log(LogRec *a, LogRec *b, uint64_t n, uint32_t gbits, uint32_t bits, uint32_t *tmp,
                 cudaStream_t s) {
  if (n <= 1) return a;
  const uint32_t ntiles = (uint32_t)tiles_of(n);
  const uint64_t h = 256ull * ntiles;
  uint32_t *hist = tmp, *offs = tmp + h, *stmp = tmp + 2 * h;
  for (uint32_t shift = 0; shift < bits; shift += 8) {
    count_launch();
    radix_hist_kernel<<<ntiles, kThreads, 0, s>>>(a, n, gbits, shift, hist, ntiles);
    scan_exclusive(hist, offs, h, stmp, s);
    count_launch();
    radix_scatter_kernel<<<ntiles, kThreads, 0, s>>>(a, b, n, gbits, shift, offs, ntiles);
    LogRec *t = a;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace rc
