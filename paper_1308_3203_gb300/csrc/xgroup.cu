// Work-group-scoped barriers (OpenCL's barrier, against the kernel-wide one
// of Sec. 2 and Sec. 4's barrier-release rule): no barrier orders work-items
// of different groups, so every global cell is also classified over the
// whole run between groups.
//
// A table of one XgCell per global cell gathers, interval by interval from
// the access log, the smallest and largest writer and reader and the range
// of values written and observed (the observed range starts with the cell's
// value before the run).  At the end of the run, per cell:
//  * writers in two or more groups (the smallest and the largest writer lie
//    in different groups, as group = work-item / group size is monotone):
//    XG_WW_BENIGN when one value was written, else XG_WW_RACE; witness
//    (smallest writer, largest writer);
//  * a reader and a writer in different groups (the smallest and largest
//    reader and writer are not all in one group): XG_RW_RACE unless the
//    value before the run, every value written and every value observed are
//    one value (a read by another group may come before or after any write);
//    witness (r0, w0) if their groups differ, else (r0, w1) if those differ,
//    else (r1, w0) -- in the last case every writer is in r0's group, so r1
//    is not;
//  * n_readers / n_writers = reads / writes of the cell in the run.
// Records come out in cell order through an exclusive scan of per-cell
// record counts, XG_WW_* before XG_RW_RACE.
#include <algorithm>

#include "device.cuh"

namespace rc {
namespace {

constexpr int kThreads = 256;

unsigned grid_for(uint64_t items, uint64_t per_block) {
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((items + per_block - 1) / per_block, 1u << 20));
}

__global__ void xg_init_kernel(XgCell *xg, uint2 *cnt, const int32_t *snap, uint64_t GT) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < GT; k += stride) {
    const int32_t v = snap[k];
    xg[k] = XgCell{kNone, 0u, kNone, 0u, INT32_MAX, INT32_MIN, v, v};
    cnt[k] = make_uint2(0u, 0u);
  }
}

// one warp per log slice; records of local cells (key >= GT) are skipped
__global__ void xg_update_kernel(const LogRec *log, uint32_t n_slices, uint64_t slice, const uint32_t *count,
                                 uint64_t GT, XgCell *xg, uint2 *cnt) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32u);
  for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32u; w < n_slices; w += nwarps) {
    const LogRec *src = log + w * slice;
    const uint32_t n = count[w];
    for (uint32_t i = lane; i < n; i += 32u) {
      const LogRec r = src[i];
      if (r.key >= GT) continue;
      XgCell *c = xg + r.key;
      const uint32_t g = r.tw & 0x7FFFFFFFu;
      if (r.tw & 0x80000000u) {
        atomicMin(&c->wmin, g);
        atomicMax(&c->wmax, g);
        atomicMin(&c->vmin, r.val);
        atomicMax(&c->vmax, r.val);
        atomicAdd(&cnt[r.key].y, 1u);
      } else {
        atomicMin(&c->rmin, g);
        atomicMax(&c->rmax, g);
        atomicMin(&c->omin, r.val);
        atomicMax(&c->omax, r.val);
        atomicAdd(&cnt[r.key].x, 1u);
      }
    }
  }
}

struct XgOut {
  uint32_t n;
  uint32_t cls[2], ta[2], tb[2];
};

__device__ __forceinline__ XgOut xg_classify(const XgCell &c, uint32_t S) {
  XgOut o{};
  if (c.wmin == kNone) return o;  // nobody wrote the cell
  if (c.wmin / S != c.wmax / S) {
    o.cls[0] = c.vmin == c.vmax ? CLS_XG_WW_BENIGN : CLS_XG_WW_RACE;
    o.ta[0] = c.wmin;
    o.tb[0] = c.wmax;
    o.n = 1;
  }
  if (c.rmin == kNone) return o;
  const uint32_t r0 = c.rmin / S, r1 = c.rmax / S, w0 = c.wmin / S, w1 = c.wmax / S;
  const bool cross = !(r0 == r1 && w0 == w1 && r0 == w0);
  const bool one_value = c.omin == c.omax && c.vmin == c.vmax && c.omin == c.vmin;
  if (cross && !one_value) {
    o.cls[o.n] = CLS_XG_RW_RACE;
    if (r0 != w0) {
      o.ta[o.n] = c.rmin;
      o.tb[o.n] = c.wmin;
    } else if (r0 != w1) {
      o.ta[o.n] = c.rmin;
      o.tb[o.n] = c.wmax;
    } else {
      o.ta[o.n] = c.rmax;
      o.tb[o.n] = c.wmin;
    }
    o.n++;
  }
  return o;
}

__global__ void xg_count_kernel(const XgCell *xg, uint64_t GT, uint32_t S, uint32_t *nrec) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < GT; k += stride)
    nrec[k] = xg_classify(xg[k], S).n;
}

__global__ void xg_emit_kernel(const XgCell *xg, const uint2 *cnt, uint64_t GT, uint32_t S, const uint32_t *nrec,
                               const uint32_t *offs, OutRec *out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < GT; k += stride) {
    if (!nrec[k]) continue;
    const XgOut o = xg_classify(xg[k], S);
    const uint2 c = cnt[k];
    for (uint32_t i = 0; i < o.n; i++)
      out[offs[k] + i] = OutRec{kNone, 0u, 0u, (uint32_t)k, o.cls[i], o.ta[i], o.tb[i], c.x, c.y, c.x + c.y};
  }
}

}  // namespace

void launch_xg_init(XgCell *xg, uint2 *cnt, const int32_t *snap, uint64_t GT, cudaStream_t s) {
  if (!GT) return;
  count_launch();
  xg_init_kernel<<<grid_for(GT, kThreads), kThreads, 0, s>>>(xg, cnt, snap, GT);
}

void launch_xg_update(const LogRec *log, uint32_t n_slices, uint64_t slice, const uint32_t *count, uint64_t GT,
                      XgCell *xg, uint2 *cnt, cudaStream_t s) {
  if (!GT || !n_slices) return;
  count_launch();
  xg_update_kernel<<<grid_for(n_slices, kThreads / 32), kThreads, 0, s>>>(log, n_slices, slice, count, GT, xg, cnt);
}

void launch_xg_count(const XgCell *xg, uint64_t GT, uint32_t S, uint32_t *nrec, cudaStream_t s) {
  if (!GT) return;
  count_launch();
  xg_count_kernel<<<grid_for(GT, kThreads), kThreads, 0, s>>>(xg, GT, S, nrec);
}

void launch_xg_emit(const XgCell *xg, const uint2 *cnt, uint64_t GT, uint32_t S, const uint32_t *nrec,
                    const uint32_t *offs, OutRec *out, cudaStream_t s) {
  if (!GT) return;
  count_launch();
  xg_emit_kernel<<<grid_for(GT, kThreads), kThreads, 0, s>>>(xg, cnt, GT, S, nrec, offs, out);
}

}  // namespace rc
