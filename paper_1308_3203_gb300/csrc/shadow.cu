// Shadow owner-table path of the classification.
//
// The interpreter claims, for every access, the cell's writer or reader word
// in the owner table (see shadow_claim).  After the interval:
//  * cells with one writer and no other reader are race-free; their new
//    value is that work-item's last write, which its own-write table holds,
//    so each work-item commits its own cells;
//  * the log records of every other written cell are compacted (one warp-
//    aggregated atomic per warp and instruction) and classified exactly by
//    the sort path.
#include <cooperative_groups.h>

#include "device.cuh"

namespace cg = cooperative_groups;

namespace rc {
namespace {

__global__ void shadow_compact_kernel(const LogRec *log, uint64_t n, const unsigned long long *owner,
                                      uint32_t epoch, LogRec *out, unsigned long long *count) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 r = reinterpret_cast<const uint4 *>(log)[i];
  if (!shadow_needs_exact(owner, r.x, epoch)) return;
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned long long base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(count, (unsigned long long)g.size());
  base = g.shfl(base, 0);
  reinterpret_cast<uint4 *>(out)[base + g.thread_rank()] = r;
}

__global__ void shadow_commit_kernel(const uint2 *ow, const uint32_t *ow_count, uint64_t N, uint32_t ow_stride,
                                     const unsigned long long *owner, uint32_t epoch, int32_t *snap) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  const uint32_t nw = ow_count[t];
  const unsigned long long mine = ((unsigned long long)epoch << 32) | (uint32_t)t;
  for (uint32_t k = 0; k < nw; k++) {
    const uint2 e = ow[(uint64_t)k * ow_stride + t];
    if (owner[2ull * e.x] == mine) snap[e.x] = (int32_t)e.y;
  }
}

}  // namespace

void launch_shadow_compact(const LogRec *log, uint64_t n, const unsigned long long *owner, uint32_t epoch,
                           LogRec *out, unsigned long long *count, cudaStream_t s) {
  if (n) shadow_compact_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(log, n, owner, epoch, out, count);
}

void launch_shadow_commit(const uint2 *ow, const uint32_t *ow_count, uint64_t N, uint32_t ow_stride,
                          const unsigned long long *owner, uint32_t epoch, int32_t *snap, cudaStream_t s) {
  if (N)
    shadow_commit_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(ow, ow_count, N, ow_stride, owner, epoch,
                                                                     snap);
}

}  // namespace rc
