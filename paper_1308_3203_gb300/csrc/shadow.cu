// Shadow owner-table path of the classification.
//
// The interpreter claims, for every access, the cell's writer or reader word
// in the owner table (see shadow_claim).  After the interval:
//  * every written cell takes the last write of its highest writer (the
//    value the sort path's classifier commits: the schedule that runs
//    work-items in id order); that work-item's own-write table holds it, so
//    each work-item commits the cells whose highest writer it is;
//  * the log records of cells written by two or more work-items, or written
//    by one and read by another, are compacted (one warp-aggregated atomic
//    per 128 records) and classified exactly by the sort path, which then
//    commits nothing: the next interval needs only the commits.
#include <algorithm>

#include "device.cuh"

namespace rc {
namespace {

// one warp per log slice, 8 slices per block
__global__ void shadow_compact_kernel(const LogRec *log, uint32_t n_slices, uint64_t slice, const uint32_t *count,
                                      const uint32_t *owner, uint32_t tag, LogRec *out,
                                      unsigned long long *total) {
  const uint32_t w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= n_slices) return;
  compact_slice<8>(reinterpret_cast<const uint4 *>(log) + (uint64_t)w * slice, count[w], owner, tag,
                   reinterpret_cast<uint4 *>(out), total, threadIdx.x & 31u);
}

__global__ void shadow_commit_kernel(const uint2 *ow, const uint32_t *ow_count, uint64_t N, uint32_t ow_stride,
                                     const uint32_t *owner, uint32_t tag, int32_t *snap) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  const uint32_t nw = ow_count[t];
  const uint32_t hi = (tag << 26) | (uint32_t)t;
  for (uint32_t k = 0; k < nw; k++) {
    const uint2 e = ow[(uint64_t)k * ow_stride + t];
    if (owner[4ull * e.x] == hi) snap[e.x] = (int32_t)e.y;  // this work-item is the cell's highest writer
  }
}

__global__ void densify_kernel(const LogRec *log, uint32_t n_slices, uint64_t slice, const uint32_t *count,
                               const uint32_t *offs, LogRec *out) {
  const uint32_t w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= n_slices) return;
  const uint32_t n = count[w];
  const uint4 *src = reinterpret_cast<const uint4 *>(log) + (uint64_t)w * slice;
  uint4 *dst = reinterpret_cast<uint4 *>(out) + offs[w];
  for (uint32_t i = threadIdx.x & 31u; i < n; i += 32) dst[i] = src[i];
}

// n int32 values from src (pinned host memory the GPU reads over the
// CPU-GPU link, or device memory) to dst; 16-byte loads and stores when
// both are 16-byte aligned
__global__ void copy_words_kernel(const int32_t *__restrict__ src, int32_t *__restrict__ dst, uint64_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0) {
    const uint64_t n4 = n / 4;
    const int4 *s4 = reinterpret_cast<const int4 *>(src);
    int4 *d4 = reinterpret_cast<int4 *>(dst);
    for (uint64_t i = t; i < n4; i += stride) d4[i] = s4[i];
    for (uint64_t i = n4 * 4 + t; i < n; i += stride) dst[i] = src[i];
  } else {
    for (uint64_t i = t; i < n; i += stride) dst[i] = src[i];
  }
}

}  // namespace

void launch_copy_words(const int32_t *src, int32_t *dst, uint64_t n, cudaStream_t s) {
  if (!n) return;
  count_launch();
  const uint64_t blocks = std::min<uint64_t>((n / 4 + 255) / 256 + 1, (uint64_t)sm_count() * 16);
  copy_words_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, dst, n);
}

void launch_shadow_compact(const LogRec *log, uint32_t n_slices, uint64_t slice, const uint32_t *count,
                           const uint32_t *owner, uint32_t tag, LogRec *out, unsigned long long *total,
                           cudaStream_t s) {
  if (!n_slices) return;
  count_launch();
  shadow_compact_kernel<<<(n_slices + 7) / 8, 256, 0, s>>>(log, n_slices, slice, count, owner, tag, out, total);
}

void launch_shadow_commit(const uint2 *ow, const uint32_t *ow_count, uint64_t N, uint32_t ow_stride,
                          const uint32_t *owner, uint32_t tag, int32_t *snap, cudaStream_t s) {
  if (!N) return;
  count_launch();
  shadow_commit_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(ow, ow_count, N, ow_stride, owner, tag, snap);
}

void launch_densify(const LogRec *log, uint32_t n_slices, uint64_t slice, const uint32_t *count,
                    const uint32_t *offs, LogRec *out, cudaStream_t s) {
  if (!n_slices) return;
  count_launch();
  densify_kernel<<<(n_slices + 7) / 8, 256, 0, s>>>(log, n_slices, slice, count, offs, out);
}

}  // namespace rc
