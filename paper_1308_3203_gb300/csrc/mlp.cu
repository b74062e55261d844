// Learned proposal network: MLP 128 -> 256 -> 256 -> 256 -> 1 (ReLU, sigmoid
// score) over candidate features, trained on the exact checker's race / no
// race labels with binary cross-entropy and Adam.
//
// Numerics: FP32 master weights; the forward and backward products run on
// the tcgen05 tensor cores with FP32 accumulators in TMEM (mma.sync m16n8k16
// kernels selectable), with BF16 operands: the input features, the weight copies, the hidden activations
// h = relu(z) and the pre-activation gradients dz are rounded to BF16 where
// they are stored; biases, the output layer's dot product, the loss and all
// gradient sums stay in FP32.  Weight gradients reduce over the batch in a
// fixed order (split-K partials summed per element in split order), so a
// training run is deterministic.
//
// Parameter vector (FP32, also the layout of gradients and Adam moments):
//   W1[256][128] b1[256] W2[256][256] b2[256] W3[256][256] b3[256] w4[256] b4
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "racecheck.h"
#include "device.cuh"

namespace rc {
namespace {

constexpr int kIn = RC_MLP_IN, kHid = RC_MLP_HIDDEN;
constexpr size_t oW1 = 0, ob1 = oW1 + (size_t)kHid * kIn, oW2 = ob1 + kHid, ob2 = oW2 + (size_t)kHid * kHid,
                 oW3 = ob2 + kHid, ob3 = oW3 + (size_t)kHid * kHid, ow4 = ob3 + kHid, ob4 = ow4 + kHid,
                 kParams = ob4 + 1;
static_assert(kParams == RC_MLP_PARAMS, "parameter layout");

typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------------- GEMM
// C[M][N] = A[M][K] * B[K][N] on a 64 x 64 tile per CTA (4 warps, 32 x 32
// each), K in steps of 32.  Both operands are staged in shared memory with K
// contiguous ([row][k], rows padded to 40 elements so the fragment loads of
// a warp hit 32 distinct banks); modes differ in where the tiles come from:
//   FWD   A = act[M][K],           B[k][n] = W[n][k]      (W is [N][K])
//         out = relu(C + bias) as BF16 [M][N]
//   DGRAD A = dz[M][K],            B[k][n] = W[k][n]      (W is [K][N])
//         out = C where h[m][n] > 0, else 0, as BF16 [M][N]
//   WGRAD A[m][k] = dz[k][m],      B[k][n] = h[k][n]      (dz [rows][M], h [rows][N])
//         K = batch rows [z*kchunk, ...); out = FP32 partial z of C
constexpr int BM = 64, BN = 64, BK = 32, BKP = BK + 8, kGemmThreads = 128;
enum GemmMode { FWD = 0, DGRAD = 1, WGRAD = 2 };

struct GemmArgs {
  const bf16 *A;      // FWD/DGRAD: [M][K]; WGRAD: dz [rows][M]
  const bf16 *B;      // FWD: W [N][K]; DGRAD: W [K][N]; WGRAD: h [rows][N]
  const float *bias;  // FWD
  const bf16 *mask;   // DGRAD: h [M][N]
  bf16 *out;          // FWD/DGRAD: [M][N]
  float *part;        // WGRAD: [splits][M][N]
  int M, N, K;        // WGRAD: M = dz columns, N = h columns, K = rows
  int kchunk;         // WGRAD: rows per split
};

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// stage a 64 x 32 tile whose source rows are K-contiguous: tile[r][k] = src[(r0 + r) * ld + k0 + k]
__device__ __forceinline__ void stage_rows(bf16 (*tile)[BKP], const bf16 *src, int ld, int r0, int rmax, int k0) {
  const int t = threadIdx.x, r = t >> 1, h = (t & 1) * 16;
  uint4 v0 = make_uint4(0, 0, 0, 0), v1 = v0;
  if (r0 + r < rmax) {
    const uint4 *p = reinterpret_cast<const uint4 *>(src + (size_t)(r0 + r) * ld + k0 + h);
    v0 = p[0];
    v1 = p[1];
  }
  uint4 *q = reinterpret_cast<uint4 *>(&tile[r][h]);  // 80-byte rows: 16-byte aligned at h = 0, 16
  q[0] = v0;
  q[1] = v1;
}

// stage a 64 x 32 tile from a source whose rows run along the tile's rows:
// tile[r][k] = src[(k0 + k) * ld + r0 + r], source rows k0 + k < kmax
__device__ __forceinline__ void stage_cols(bf16 (*tile)[BKP], const bf16 *src, int ld, int r0, int k0, int kmax) {
  const int t = threadIdx.x, k = t >> 2, c = (t & 3) * 16;
  uint4 v[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
  if (k0 + k < kmax) {
    const uint4 *p = reinterpret_cast<const uint4 *>(src + (size_t)(k0 + k) * ld + r0 + c);
    v[0] = p[0];
    v[1] = p[1];
  }
  const bf16 *e = reinterpret_cast<const bf16 *>(v);
#pragma unroll
  for (int j = 0; j < 16; j++) tile[c + j][k] = e[j];
}

template <int MODE>
__global__ void __launch_bounds__(kGemmThreads) gemm_kernel(GemmArgs g) {
  __shared__ __align__(16) bf16 As[BM][BKP];
  __shared__ __align__(16) bf16 Bs[BN][BKP];
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane >> 2, tig = lane & 3;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  int kbeg = 0, kend = g.K;
  if (MODE == WGRAD) {
    kbeg = blockIdx.z * g.kchunk;
    kend = min(g.K, kbeg + g.kchunk);
  }
  float acc[2][4][4] = {};
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    if (MODE == FWD) {
      stage_rows(As, g.A, g.K, m0, g.M, k0);
      stage_rows(Bs, g.B, g.K, n0, g.N, k0);
    } else if (MODE == DGRAD) {
      stage_rows(As, g.A, g.K, m0, g.M, k0);
      stage_cols(Bs, g.B, g.N, n0, k0, g.K);
    } else {
      stage_cols(As, g.A, g.M, m0, k0, kend);
      stage_cols(Bs, g.B, g.N, n0, k0, kend);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; mi++) {
        const int r = wm + mi * 16 + grp;
        a[mi][0] = *reinterpret_cast<const uint32_t *>(&As[r][kk + tig * 2]);
        a[mi][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + tig * 2]);
        a[mi][2] = *reinterpret_cast<const uint32_t *>(&As[r][kk + tig * 2 + 8]);
        a[mi][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + tig * 2 + 8]);
      }
#pragma unroll
      for (int ni = 0; ni < 4; ni++) {
        const int c = wn + ni * 8 + grp;
        b[ni][0] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + tig * 2]);
        b[ni][1] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + tig * 2 + 8]);
      }
#pragma unroll
      for (int mi = 0; mi < 2; mi++)
#pragma unroll
        for (int ni = 0; ni < 4; ni++) mma_bf16(acc[mi][ni], a[mi], b[ni]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; mi++)
#pragma unroll
    for (int ni = 0; ni < 4; ni++)
#pragma unroll
      for (int h = 0; h < 2; h++) {  // h = 0: row grp, h = 1: row grp + 8
        const int r = m0 + wm + mi * 16 + grp + h * 8, c = n0 + wn + ni * 8 + tig * 2;
        if (r >= g.M) continue;
        const float v0 = acc[mi][ni][2 * h], v1 = acc[mi][ni][2 * h + 1];
        if (MODE == FWD) {
          const float z0 = v0 + g.bias[c], z1 = v1 + g.bias[c + 1];
          *reinterpret_cast<__nv_bfloat162 *>(g.out + (size_t)r * g.N + c) =
              __floats2bfloat162_rn(fmaxf(z0, 0.0f), fmaxf(z1, 0.0f));
        } else if (MODE == DGRAD) {
          const __nv_bfloat162 hm = *reinterpret_cast<const __nv_bfloat162 *>(g.mask + (size_t)r * g.N + c);
          const float d0 = __bfloat162float(hm.x) > 0.0f ? v0 : 0.0f;
          const float d1 = __bfloat162float(hm.y) > 0.0f ? v1 : 0.0f;
          *reinterpret_cast<__nv_bfloat162 *>(g.out + (size_t)r * g.N + c) = __floats2bfloat162_rn(d0, d1);
        } else {
          float *p = g.part + ((size_t)blockIdx.z * g.M + r) * g.N + c;
          p[0] = v0;
          p[1] = v1;
        }
      }
}

// ---------------------------------------------------------------- tcgen05 forward layer
// out[M][256] = relu(act[M][K] * W[256][K]^T + bias) on the 5th-generation
// tensor cores: one CTA (4 warps) per 128 rows x 64 output columns.  Both operands are staged in
// shared memory in the canonical K-major layout without swizzle: 8-row x
// 16-byte core matrices, 128 bytes each, core matrices along K adjacent
// (leading byte offset 128) and 8-row groups K/8 core matrices apart (stride
// byte offset K*16).  One thread issues K/16 MMAs of 128 x 64 x 16
// (kind::f16, BF16 operands, FP32 accumulator in 64 TMEM columns) and
// commits them to an mbarrier; after it fires, each warp reads its 32 rows
// of the accumulator (lanes 32w..32w+31), adds the bias, applies the ReLU
// and stores BF16.
constexpr int kTcRows = 128, kTcThreads = 128;
constexpr int kTcN = 64;  // output columns per CTA: the grid's second dimension covers the rest
constexpr uint32_t kTcWaitLimit = 1u << 26;  // mbarrier polls before the CTA gives up

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// 16-byte asynchronous copy global -> shared (zero fill when !valid; the
// source must still be a mapped address): the staging loops keep every copy
// of a thread in flight at once instead of waiting for each load
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(smem_dst)), "l"(gsrc),
               "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// shared-memory matrix descriptor: start, leading and stride byte offsets
// (all >> 4), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t tc_idesc(uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

template <int K>
__global__ void __launch_bounds__(kTcThreads) tc_fwd_kernel(const bf16 *__restrict__ act, const bf16 *__restrict__ W,
                                                            const float *__restrict__ bias, bf16 *__restrict__ out,
                                                            int M, uint32_t *err) {
  constexpr int KC = K / 8;                       // core matrices along K
  constexpr uint32_t A_BYTES = kTcRows * K * 2, B_BYTES = kTcN * K * 2;
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char *As = tsm, *Bs = tsm + A_BYTES;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(tsm + A_BYTES + B_BYTES);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int m0 = blockIdx.x * kTcRows, n0 = blockIdx.y * kTcN;
  // stage both operands, 16 bytes (8 elements along K) per copy; rows past
  // M are zero-filled
  for (int i = t; i < kTcRows * KC; i += kTcThreads) {
    const int r = i / KC, c = i % KC;
    const bool in = m0 + r < M;
    cp_async16(As + ((r >> 3) * KC + c) * 128 + (r & 7) * 16, act + (size_t)(in ? m0 + r : 0) * K + c * 8, in);
  }
  for (int i = t; i < kTcN * KC; i += kTcThreads) {
    const int n = i / KC, c = i % KC;
    cp_async16(Bs + ((n >> 3) * KC + c) * 128 + (n & 7) * 16, W + (size_t)(n0 + n) * K + c * 8, true);
  }
  cp_async_wait_all();
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // operands visible to the tensor cores
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "n"(kTcN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  if (t == 0) {
    const uint32_t a0 = smem_addr(As), b0 = smem_addr(Bs);
#pragma unroll 1
    for (int k = 0; k < K / 16; k++) {  // two core matrices along K per MMA
      const uint64_t ad = tc_desc(a0 + k * 256, 128, KC * 128), bd = tc_desc(b0 + k * 256, 128, KC * 128);
      const uint32_t acc = k > 0 ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
          "l"(ad), "l"(bd), "r"(tc_idesc(kTcN)), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_addr(mbar)));
  }
  // wait (bounded) for the MMAs to complete
  uint32_t done = 0;
  for (uint32_t it = 0; it < kTcWaitLimit && !done; it++)
    asm volatile(
        "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], 0;\n selp.b32 %0, 1, 0, P1;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(mbar)));
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!done) {
    if (t == 0) atomicOr(err, 1u);
  } else {
    const int r = warp * 32 + lane;  // accumulator row = TMEM lane
#pragma unroll 1
    for (int j = 0; j < kTcN / 32; j++) {
      uint32_t v[32];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
            "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
            "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
            "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * 32)));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m0 + r < M) {
        __align__(16) bf16 o[32];
#pragma unroll
        for (int q = 0; q < 32; q++)
          o[q] = __float2bfloat16_rn(fmaxf(__uint_as_float(v[q]) + bias[n0 + j * 32 + q], 0.0f));
        uint4 *dst = reinterpret_cast<uint4 *>(out + (size_t)(m0 + r) * kHid + n0 + j * 32);
#pragma unroll
        for (int q = 0; q < 4; q++) dst[q] = reinterpret_cast<const uint4 *>(o)[q];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTcN));
}

template <int K>
constexpr size_t tc_smem() {
  return (size_t)kTcRows * K * 2 + (size_t)kTcN * K * 2 + 16;
}

// ---- tcgen05 backward products.  The same tile layout and MMA sequence;
// operands whose source runs along M (or N) instead of K are transposed
// while staging, 8 x 8 blocks at a time.
constexpr int kTcK = 256;  // K per staged sub-tile

// tile[mn][k] (K-major core matrices, KC = kTcK / 8) = src[(k0 + k) * ld + mn0 + mn]
// for k < kn (else 0), mn < rows.  Each thread moves one 8 x 8 block: eight
// 16-byte source rows (8 M/N values at 8 consecutive K) are transposed in
// registers into eight 16-byte core-matrix rows (8 K values at one M/N).
__device__ __forceinline__ void tc_stage_mn(unsigned char *tile, const bf16 *src, int ld, int mn0, int rows, int k0,
                                            int kn) {
  constexpr int KC = kTcK / 8;
  const int G = rows / 8;
  for (int i = threadIdx.x; i < KC * G; i += kTcThreads) {
    const int c = i / G, g = i % G;  // K chunk, M/N group
    __align__(16) bf16 v[8][8];
#pragma unroll
    for (int e = 0; e < 8; e++) {
      const int k = c * 8 + e;
      uint4 x = make_uint4(0, 0, 0, 0);
      if (k < kn) x = *reinterpret_cast<const uint4 *>(src + (size_t)(k0 + k) * ld + mn0 + g * 8);
      *reinterpret_cast<uint4 *>(v[e]) = x;
    }
#pragma unroll
    for (int q = 0; q < 8; q++) {
      __align__(16) bf16 w[8];
#pragma unroll
      for (int e = 0; e < 8; e++) w[e] = v[e][q];
      *reinterpret_cast<uint4 *>(tile + (g * KC + c) * 128 + q * 16) = *reinterpret_cast<const uint4 *>(w);
    }
  }
}

// the MMAs of one staged sub-tile (K = kTcK) into TMEM, committed to mbar;
// returns false if the bounded wait ran out
__device__ __forceinline__ bool tc_mma_tile(const unsigned char *As, const unsigned char *Bs, uint32_t tmem,
                                            uint32_t idesc, bool accumulate, uint64_t *mbar, uint32_t phase) {
  constexpr int KC = kTcK / 8;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (threadIdx.x == 0) {
    const uint32_t a0 = smem_addr(As), b0 = smem_addr(Bs);
#pragma unroll 1
    for (int k = 0; k < kTcK / 16; k++) {
      const uint64_t ad = tc_desc(a0 + k * 256, 128, KC * 128), bd = tc_desc(b0 + k * 256, 128, KC * 128);
      const uint32_t acc = (accumulate || k > 0) ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
          "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_addr(mbar)));
  }
  uint32_t done = 0;
  for (uint32_t it = 0; it < kTcWaitLimit && !done; it++)
    asm volatile(
        "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n selp.b32 %0, 1, 0, P1;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(mbar)), "r"(phase));
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return __syncthreads_and(done) != 0;
}

__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t v[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
        "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
        "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t tc_begin(uint64_t *mbar, uint32_t *tslot) {
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "n"(kTcN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return *tslot;
}

__device__ __forceinline__ void tc_end(uint32_t tmem) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTcN));
}

// ---- the three hidden layers in one launch: one CTA per 128 rows keeps
// the rows' activations in shared memory from layer to layer.  Per layer the
// CTA stages the whole weight matrix (256 x K, K-major core matrices), one
// thread issues K/16 MMAs of 128 x 256 x 16 into 256 TMEM columns, and after
// the commit each warp reads its 32 rows back, adds the bias, applies the
// ReLU, rounds to BF16 and writes the result both to H_l in global memory
// (the backward pass reads it) and, in the operand layout, over the
// activation tile that the next layer's MMAs read.  Each element is the
// same FP32 sum of the same BF16 products as in tc_fwd_kernel, rounded at
// the same point.
constexpr int kTcFwd3N = 256;
constexpr size_t kTcFwd3Smem = (size_t)kTcRows * kHid * 2 + (size_t)kTcFwd3N * kHid * 2 + 16;

__global__ void __launch_bounds__(kTcThreads) tc_fwd3_kernel(const bf16 *__restrict__ X, const bf16 *__restrict__ Wb,
                                                             const float *__restrict__ P, bf16 *__restrict__ H1,
                                                             bf16 *__restrict__ H2, bf16 *__restrict__ H3, int M,
                                                             uint32_t *err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char *As = tsm, *Bs = tsm + (size_t)kTcRows * kHid * 2;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(tsm + kTcFwd3Smem - 16);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31, m0 = blockIdx.x * kTcRows;
  const int r = warp * 32 + lane;  // accumulator row = TMEM lane
  // layer 1's operand: the rows of X (K = 128), rows past M zero-filled
  {
    constexpr int KC = kIn / 8;
    for (int i = t; i < kTcRows * KC; i += kTcThreads) {
      const int rr = i / KC, c = i % KC;
      const bool in = m0 + rr < M;
      cp_async16(As + ((rr >> 3) * KC + c) * 128 + (rr & 7) * 16, X + (size_t)(in ? m0 + rr : 0) * kIn + c * 8, in);
    }
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "n"(kTcFwd3N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  bool ok = true;
  uint32_t tmem = 0;
#pragma unroll 1
  for (int l = 0; l < 3 && ok; l++) {
    const int K = l == 0 ? kIn : kHid, KC = K / 8;
    const bf16 *W = Wb + (l == 0 ? oW1 : l == 1 ? oW2 : oW3);
    const float *bias = P + (l == 0 ? ob1 : l == 1 ? ob2 : ob3);
    bf16 *H = l == 0 ? H1 : l == 1 ? H2 : H3;
    for (int i = t; i < kTcFwd3N * KC; i += kTcThreads) {
      const int n = i / KC, c = i % KC;
      cp_async16(Bs + ((n >> 3) * KC + c) * 128 + (n & 7) * 16, W + (size_t)n * K + c * 8, true);
    }
    cp_async_wait_all();
    // the staged operands (and the previous layer's activations written by
    // the epilogue) visible to the tensor cores; the previous layer's TMEM
    // reads finished before its accumulator is overwritten
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tmem = *tslot;
    if (t == 0) {
      const uint32_t a0 = smem_addr(As), b0 = smem_addr(Bs);
#pragma unroll 1
      for (int k = 0; k < K / 16; k++) {
        const uint64_t ad = tc_desc(a0 + k * 256, 128, KC * 128), bd = tc_desc(b0 + k * 256, 128, KC * 128);
        const uint32_t acc = k > 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(tc_idesc(kTcFwd3N)), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(mbar)));
    }
    uint32_t done = 0;
    for (uint32_t it = 0; it < kTcWaitLimit && !done; it++)
      asm volatile(
          "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n selp.b32 %0, 1, 0, P1;\n}\n"
          : "=r"(done)
          : "r"(smem_addr(mbar)), "r"((uint32_t)(l & 1)));
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ok = __syncthreads_and(done) != 0;
    if (!ok) break;
    // epilogue: H_l rows, and the next layer's operand over the activation tile
    constexpr int KCn = kHid / 8;
#pragma unroll 1
    for (int j = 0; j < kTcFwd3N / 32; j++) {
      uint32_t v[32];
      tc_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * 32), v);
      __align__(16) bf16 o[32];
#pragma unroll
      for (int q = 0; q < 32; q++)
        o[q] = __float2bfloat16_rn(fmaxf(__uint_as_float(v[q]) + bias[j * 32 + q], 0.0f));
      if (m0 + r < M) {
        uint4 *dst = reinterpret_cast<uint4 *>(H + (size_t)(m0 + r) * kHid + j * 32);
#pragma unroll
        for (int q = 0; q < 4; q++) dst[q] = reinterpret_cast<const uint4 *>(o)[q];
      }
      if (l < 2) {
#pragma unroll
        for (int q = 0; q < 4; q++)  // 8 values along K = one 16-byte core-matrix row
          *reinterpret_cast<uint4 *>(As + ((r >> 3) * KCn + j * 4 + q) * 128 + (r & 7) * 16) =
              reinterpret_cast<const uint4 *>(o)[q];
      }
    }
  }
  if (!ok && t == 0) atomicOr(err, 1u);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "n"(kTcFwd3N));
}

constexpr size_t kTcBwdSmem = (size_t)kTcRows * kTcK * 2 + (size_t)kTcN * kTcK * 2 + 16;

// dz_prev[M][256] = (dz[M][256] * W[256][256]) where h[M][256] > 0, as BF16
__global__ void __launch_bounds__(kTcThreads) tc_dgrad_kernel(const bf16 *__restrict__ dz, const bf16 *__restrict__ W,
                                                              const bf16 *__restrict__ h, bf16 *__restrict__ out,
                                                              int M, uint32_t *err) {
  constexpr int KC = kTcK / 8;
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char *As = tsm, *Bs = tsm + kTcRows * kTcK * 2;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(tsm + kTcBwdSmem - 16);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31, m0 = blockIdx.x * kTcRows, n0 = blockIdx.y * kTcN;
  for (int i = t; i < kTcRows * KC; i += kTcThreads) {  // A = dz rows, K contiguous
    const int r = i / KC, c = i % KC;
    const bool in = m0 + r < M;
    cp_async16(As + ((r >> 3) * KC + c) * 128 + (r & 7) * 16, dz + (size_t)(in ? m0 + r : 0) * kHid + c * 8, in);
  }
  tc_stage_mn(Bs, W, kHid, n0, kTcN, 0, kTcK);  // B[n][k] = W[k][n0 + n]
  cp_async_wait_all();
  const uint32_t tmem = tc_begin(mbar, tslot);
  if (!tc_mma_tile(As, Bs, tmem, tc_idesc(kTcN), false, mbar, 0)) {
    if (t == 0) atomicOr(err, 1u);
  } else {
    const int r = warp * 32 + lane;
#pragma unroll 1
    for (int j = 0; j < kTcN / 32; j++) {
      uint32_t v[32];
      tc_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * 32), v);
      if (m0 + r < M) {
        const bf16 *hm = h + (size_t)(m0 + r) * kHid + n0 + j * 32;
        __align__(16) bf16 o[32];
#pragma unroll
        for (int q = 0; q < 32; q++)
          o[q] = __float2bfloat16_rn(__bfloat162float(hm[q]) > 0.0f ? __uint_as_float(v[q]) : 0.0f);
        uint4 *dst = reinterpret_cast<uint4 *>(out + (size_t)(m0 + r) * kHid + n0 + j * 32);
#pragma unroll
        for (int q = 0; q < 4; q++) dst[q] = reinterpret_cast<const uint4 *>(o)[q];
      }
    }
  }
  tc_end(tmem);
}

// partial z of dW[256][N] = dz^T h over rows [z*kchunk, ...): the CTA at
// (blockIdx.x, blockIdx.y) takes output rows j = 128*x .. +127 and columns
// 64*y .. +63, K = batch rows in sub-tiles of kTcK accumulated in TMEM
__global__ void __launch_bounds__(kTcThreads) tc_wgrad_kernel(const bf16 *__restrict__ dz, const bf16 *__restrict__ h,
                                                              int N, int rows, int kchunk, float *__restrict__ part,
                                                              uint32_t *err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char *As = tsm, *Bs = tsm + kTcRows * kTcK * 2;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(tsm + kTcBwdSmem - 16);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int j0 = blockIdx.x * kTcRows, n0 = blockIdx.y * kTcN, z = blockIdx.z;
  const int kbeg = z * kchunk, kend = min(rows, kbeg + kchunk);
  const uint32_t tmem = tc_begin(mbar, tslot);
  bool ok = true;
  uint32_t phase = 0;
  for (int k0 = kbeg; k0 < kend && ok; k0 += kTcK, phase ^= 1u) {
    const int kn = min(kTcK, kend - k0);
    tc_stage_mn(As, dz, kHid, j0, kTcRows, k0, kn);  // A[j][r] = dz[r][j0 + j]
    tc_stage_mn(Bs, h, N, n0, kTcN, k0, kn);         // B[i][r] = h[r][n0 + i]
    ok = tc_mma_tile(As, Bs, tmem, tc_idesc(kTcN), k0 > kbeg, mbar, phase);
  }
  if (!ok) {
    if (t == 0) atomicOr(err, 1u);
  } else {
    const int r = warp * 32 + lane;  // output row j0 + r
    float *dst = part + ((size_t)z * kHid + j0 + r) * N + n0;
#pragma unroll 1
    for (int j = 0; j < kTcN / 32; j++) {
      uint32_t v[32];
      tc_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * 32), v);
#pragma unroll
      for (int q = 0; q < 32; q += 4)
        *reinterpret_cast<float4 *>(dst + j * 32 + q) =
            make_float4(__uint_as_float(v[q]), __uint_as_float(v[q + 1]), __uint_as_float(v[q + 2]),
                        __uint_as_float(v[q + 3]));
    }
  }
  tc_end(tmem);
}

// ---------------------------------------------------------------- small kernels
// rows of the (shuffled) batch: features to BF16, labels to FP32
__global__ void gather_kernel(const float *X, const float *Y, const uint32_t *idx, int n, bf16 *Xb, float *Yb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * kIn) return;
  const int r = i / kIn, c = i % kIn;
  const uint32_t s = idx ? idx[r] : (uint32_t)r;
  Xb[i] = __float2bfloat16_rn(X[(size_t)s * kIn + c]);
  if (c == 0 && Yb) Yb[r] = Y[s];
}

__device__ __forceinline__ float warp_sum(float x) {
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
  return x;
}

// output layer, one warp per row: logit = h3 . w4 + b4 (BF16 operands, FP32 sum)
__device__ __forceinline__ float head_logit(const bf16 *h3, const bf16 *w4b, float b4, int lane) {
  const uint4 hv = reinterpret_cast<const uint4 *>(h3)[lane];
  const uint4 wv = reinterpret_cast<const uint4 *>(w4b)[lane];
  const bf16 *he = reinterpret_cast<const bf16 *>(&hv), *we = reinterpret_cast<const bf16 *>(&wv);
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; j++) s += __bfloat162float(he[j]) * __bfloat162float(we[j]);
  return warp_sum(s) + b4;
}

__global__ void head_fwd_kernel(const bf16 *H3, const bf16 *w4b, const float *P, int n, float *prob) {
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (r >= n) return;
  const float z = head_logit(H3 + (size_t)r * kHid, w4b, P[ob4], lane);
  if (lane == 0) prob[r] = 1.0f / (1.0f + expf(-z));
}

// loss and the output layer's gradients: dl = (sigmoid(z) - y) / n,
// loss_r = log(1 + e^z) - y z, dz3 = dl * w4 where h3 > 0
__global__ void head_bwd_kernel(const bf16 *H3, const bf16 *w4b, const float *P, const float *Yb, int n,
                                float inv_n, float *dl, float *loss, bf16 *dZ3) {
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (r >= n) return;
  const bf16 *h = H3 + (size_t)r * kHid;
  const float z = head_logit(h, w4b, P[ob4], lane);
  const float y = Yb[r];
  const float p = 1.0f / (1.0f + expf(-z));
  const float d = (p - y) * inv_n;
  if (lane == 0) {
    dl[r] = d;
    loss[r] = fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z))) - y * z;
  }
  const uint4 hv = reinterpret_cast<const uint4 *>(h)[lane];
  const uint4 wv = reinterpret_cast<const uint4 *>(w4b)[lane];
  const bf16 *he = reinterpret_cast<const bf16 *>(&hv), *we = reinterpret_cast<const bf16 *>(&wv);
  __align__(16) bf16 o[8];
#pragma unroll
  for (int j = 0; j < 8; j++)
    o[j] = __float2bfloat16_rn(__bfloat162float(he[j]) > 0.0f ? d * __bfloat162float(we[j]) : 0.0f);
  reinterpret_cast<uint4 *>(dZ3 + (size_t)r * kHid)[lane] = *reinterpret_cast<const uint4 *>(o);
}

// column sums over a row chunk: part[chunk][c] = sum_r w[r] * A[r][c] (w = 1 if null)
constexpr int kColRows = 256;
__global__ void colsum_kernel(const bf16 *A, const float *w, int n, float *part) {
  const int c = threadIdx.x;  // blockDim = kHid
  const int r0 = blockIdx.x * kColRows, r1 = min(n, r0 + kColRows);
  float s = 0.0f;
  for (int r = r0; r < r1; r++) s += (w ? w[r] : 1.0f) * __bfloat162float(A[(size_t)r * kHid + c]);
  part[(size_t)blockIdx.x * kHid + c] = s;
}
// sum of dl over a row chunk (output bias)
__global__ void vecsum_kernel(const float *v, int n, float *part) {
  __shared__ float sh[32];
  const int r0 = blockIdx.x * kColRows;
  const int r = r0 + threadIdx.x;
  float s = (r < n && threadIdx.x < kColRows) ? v[r] : 0.0f;
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += sh[k];
    part[blockIdx.x] = t;
  }
}
// out[i] = scale * (sum over z of part[z][i]), summed in split order
__global__ void reduce_parts_kernel(const float *part, int splits, int count, float *out, float scale = 1.0f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  float s = 0.0f;
  for (int z = 0; z < splits; z++) s += part[(size_t)z * count + i];
  out[i] = s * scale;
}

__global__ void adam_kernel(float *P, const float *G, float *Mm, float *Vv, bf16 *Pb, size_t n, float lr, float b1,
                            float b2, float c1, float c2, float eps) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float m = b1 * Mm[i] + (1.0f - b1) * g;
  const float v = b2 * Vv[i] + (1.0f - b2) * g * g;
  Mm[i] = m;
  Vv[i] = v;
  const float p = P[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
  P[i] = p;
  Pb[i] = __float2bfloat16_rn(p);
}

__global__ void to_bf16_kernel(const float *P, bf16 *Pb, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) Pb[i] = __float2bfloat16_rn(P[i]);
}

unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace
}  // namespace rc

// ---------------------------------------------------------------- the network object
struct rc_mlp {
  uint32_t cap = 0;  // rows per pass
  int backend = 1;   // products: 0 mma.sync, 1 tcgen05 (forward layers fused), 2 tcgen05 (a launch per layer)
  uint32_t *tc_err = nullptr;  // device flag: a tcgen05 CTA gave up waiting for its MMAs
  float *P = nullptr, *G = nullptr, *Mm = nullptr, *Vv = nullptr;
  rc::bf16 *Pb = nullptr;
  rc::bf16 *Xb = nullptr, *H1 = nullptr, *H2 = nullptr, *H3 = nullptr, *D1 = nullptr, *D2 = nullptr;
  float *Yb = nullptr, *dl = nullptr, *loss = nullptr, *part = nullptr, *scal = nullptr;
  uint32_t *idx = nullptr;
  size_t part_floats = 0;
  uint64_t step = 0;
};

namespace rc {
namespace {

struct MlpFail {
  int code;
  const char *msg;
};
#define MK(x)                                                   \
  do {                                                          \
    cudaError_t e_ = (x);                                       \
    if (e_ != cudaSuccess) throw MlpFail{RC_E_CUDA, cudaGetErrorString(e_)}; \
  } while (0)

int wgrad_splits(int rows) { return std::max(1, std::min(64, (rows + 511) / 512)); }

// forward pass of rows [0, n) of the staged batch m->Xb (n <= cap)
void forward(rc_mlp *m, int n, cudaStream_t s) {
  const bf16 *Wb = m->Pb;
  if (m->backend == 1) {  // the three layers in one launch
    count_launch();
    tc_fwd3_kernel<<<(unsigned)((n + kTcRows - 1) / kTcRows), kTcThreads, kTcFwd3Smem, s>>>(
        m->Xb, Wb, m->P, m->H1, m->H2, m->H3, n, m->tc_err);
    return;
  }
  if (m->backend == 2) {  // one launch per layer
    const dim3 grid((unsigned)((n + kTcRows - 1) / kTcRows), kHid / kTcN);
    count_launch();
    tc_fwd_kernel<kIn><<<grid, kTcThreads, tc_smem<kIn>(), s>>>(m->Xb, Wb + oW1, m->P + ob1, m->H1, n, m->tc_err);
    count_launch();
    tc_fwd_kernel<kHid><<<grid, kTcThreads, tc_smem<kHid>(), s>>>(m->H1, Wb + oW2, m->P + ob2, m->H2, n, m->tc_err);
    count_launch();
    tc_fwd_kernel<kHid><<<grid, kTcThreads, tc_smem<kHid>(), s>>>(m->H2, Wb + oW3, m->P + ob3, m->H3, n, m->tc_err);
    return;
  }
  GemmArgs g{};
  g.M = n;
  g.N = kHid;
  dim3 grid(nblk(n, BM), kHid / BN);
  g.A = m->Xb, g.B = Wb + oW1, g.bias = m->P + ob1, g.out = m->H1, g.K = kIn;
  count_launch();
  gemm_kernel<FWD><<<grid, kGemmThreads, 0, s>>>(g);
  g.A = m->H1, g.B = Wb + oW2, g.bias = m->P + ob2, g.out = m->H2, g.K = kHid;
  count_launch();
  gemm_kernel<FWD><<<grid, kGemmThreads, 0, s>>>(g);
  g.A = m->H2, g.B = Wb + oW3, g.bias = m->P + ob3, g.out = m->H3, g.K = kHid;
  count_launch();
  gemm_kernel<FWD><<<grid, kGemmThreads, 0, s>>>(g);
}

// dW = dz^T h (+ split-K partials), db = column sums of dz
void weight_grads(rc_mlp *m, const bf16 *dz, const bf16 *h, int kin, int n, size_t oW, size_t ob, cudaStream_t s) {
  const int splits = wgrad_splits(n);
  if (m->backend != 0) {
    const int kchunk = (((n + splits - 1) / splits) + 15) / 16 * 16;
    const int zs = (n + kchunk - 1) / kchunk;
    count_launch();
    tc_wgrad_kernel<<<dim3(kHid / kTcRows, kin / kTcN, zs), kTcThreads, kTcBwdSmem, s>>>(dz, h, kin, n, kchunk,
                                                                                        m->part, m->tc_err);
    count_launch();
    reduce_parts_kernel<<<nblk((size_t)kHid * kin, 256), 256, 0, s>>>(m->part, zs, kHid * kin, m->G + oW);
    const int chunks = (n + kColRows - 1) / kColRows;
    count_launch();
    colsum_kernel<<<chunks, kHid, 0, s>>>(dz, nullptr, n, m->part);
    count_launch();
    reduce_parts_kernel<<<1, kHid, 0, s>>>(m->part, chunks, kHid, m->G + ob);
    return;
  }
  GemmArgs g{};
  g.A = dz;
  g.B = h;
  g.part = m->part;
  g.M = kHid;
  g.N = kin;
  g.K = n;
  g.kchunk = (((n + splits - 1) / splits) + BK - 1) / BK * BK;
  const int zs = (n + g.kchunk - 1) / g.kchunk;
  count_launch();
  gemm_kernel<WGRAD><<<dim3(kHid / BM, kin / BN, zs), kGemmThreads, 0, s>>>(g);
  count_launch();
  reduce_parts_kernel<<<nblk((size_t)kHid * kin, 256), 256, 0, s>>>(m->part, zs, kHid * kin, m->G + oW);
  const int chunks = (n + kColRows - 1) / kColRows;
  count_launch();
  colsum_kernel<<<chunks, kHid, 0, s>>>(dz, nullptr, n, m->part);
  count_launch();
  reduce_parts_kernel<<<1, kHid, 0, s>>>(m->part, chunks, kHid, m->G + ob);
}

// forward + backward of the staged batch; gradients into m->G, per-row losses into m->loss
void backward(rc_mlp *m, int n, cudaStream_t s) {
  forward(m, n, s);
  count_launch();
  head_bwd_kernel<<<nblk((size_t)n * 32, 256), 256, 0, s>>>(m->H3, m->Pb + ow4, m->P, m->Yb, n, 1.0f / n, m->dl,
                                                            m->loss, m->D2);
  // output layer: gw4 = sum_r dl_r h3_r, gb4 = sum_r dl_r
  const int chunks = (n + kColRows - 1) / kColRows;
  count_launch();
  colsum_kernel<<<chunks, kHid, 0, s>>>(m->H3, m->dl, n, m->part);
  count_launch();
  reduce_parts_kernel<<<1, kHid, 0, s>>>(m->part, chunks, kHid, m->G + ow4);
  count_launch();
  vecsum_kernel<<<chunks, kColRows, 0, s>>>(m->dl, n, m->part);
  count_launch();
  reduce_parts_kernel<<<1, 1, 0, s>>>(m->part, chunks, 1, m->G + ob4);
  // layer 3 (dz3 in D2), then dz2 = (dz3 W3) * [h2 > 0] into D1
  weight_grads(m, m->D2, m->H2, kHid, n, oW3, ob3, s);
  GemmArgs g{};
  g.M = n;
  g.N = kHid;
  g.K = kHid;
  g.A = m->D2, g.B = m->Pb + oW3, g.mask = m->H2, g.out = m->D1;
  const dim3 tgrid((unsigned)((n + kTcRows - 1) / kTcRows), kHid / kTcN);
  count_launch();
  if (m->backend != 0)
    tc_dgrad_kernel<<<tgrid, kTcThreads, kTcBwdSmem, s>>>(m->D2, m->Pb + oW3, m->H2, m->D1, n, m->tc_err);
  else
    gemm_kernel<DGRAD><<<dim3(nblk(n, BM), kHid / BN), kGemmThreads, 0, s>>>(g);
  weight_grads(m, m->D1, m->H1, kHid, n, oW2, ob2, s);
  g.A = m->D1, g.B = m->Pb + oW2, g.mask = m->H1, g.out = m->D2;  // dz1 into D2
  count_launch();
  if (m->backend != 0)
    tc_dgrad_kernel<<<tgrid, kTcThreads, kTcBwdSmem, s>>>(m->D1, m->Pb + oW2, m->H1, m->D2, n, m->tc_err);
  else
    gemm_kernel<DGRAD><<<dim3(nblk(n, BM), kHid / BN), kGemmThreads, 0, s>>>(g);
  weight_grads(m, m->D2, m->Xb, kIn, n, oW1, ob1, s);
}

void stage(rc_mlp *m, const float *X, const float *Y, const uint32_t *idx, int n, cudaStream_t s) {
  count_launch();
  gather_kernel<<<nblk((size_t)n * kIn, 256), 256, 0, s>>>(X, Y, idx, n, m->Xb, Y ? m->Yb : nullptr);
}

// mean of the per-row losses into m->scal[slot]
void mean_loss(rc_mlp *m, int n, int slot, cudaStream_t s) {
  const int chunks = (n + kColRows - 1) / kColRows;
  count_launch();
  vecsum_kernel<<<chunks, kColRows, 0, s>>>(m->loss, n, m->part);
  count_launch();
  reduce_parts_kernel<<<1, 1, 0, s>>>(m->part, chunks, 1, m->scal + slot, 1.0f / n);
}

void adam(rc_mlp *m, float lr, cudaStream_t s) {
  m->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - (float)std::pow(b1, (double)m->step), c2 = 1.0f - (float)std::pow(b2, (double)m->step);
  count_launch();
  adam_kernel<<<nblk(kParams, 256), 256, 0, s>>>(m->P, m->G, m->Mm, m->Vv, m->Pb, kParams, lr, b1, b2, c1, c2, 1e-8f);
}

uint64_t splitmix(uint64_t &x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <class F>
int guarded(F f) {
  try {
    f();
    return RC_OK;
  } catch (const MlpFail &e) {
    set_last_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc &) {
    set_last_error("out of host memory");
    return RC_E_NOMEM;
  }
}

}  // namespace
}  // namespace rc

using namespace rc;

extern "C" {

int rc_mlp_create(uint64_t seed, uint32_t capacity, rc_mlp **out) {
  if (!out || capacity == 0 || capacity > (1u << 24)) {
    set_last_error("bad arguments");
    return RC_E_INVALID;
  }
  rc_mlp *m = new (std::nothrow) rc_mlp();
  if (!m) return RC_E_NOMEM;
  const int rc = guarded([&] {
    m->cap = capacity;
    const size_t cap = capacity;
    const int max_splits = wgrad_splits((int)std::min<size_t>(cap, 1u << 30));
    m->part_floats = std::max<size_t>((size_t)max_splits * kHid * kHid, ((cap + kColRows - 1) / kColRows) * kHid);
    MK(cudaMalloc(&m->P, kParams * 4));
    MK(cudaMalloc(&m->G, kParams * 4));
    MK(cudaMalloc(&m->Mm, kParams * 4));
    MK(cudaMalloc(&m->Vv, kParams * 4));
    MK(cudaMalloc(&m->Pb, kParams * 2));
    MK(cudaMalloc(&m->Xb, cap * kIn * 2));
    MK(cudaMalloc(&m->H1, cap * kHid * 2));
    MK(cudaMalloc(&m->H2, cap * kHid * 2));
    MK(cudaMalloc(&m->H3, cap * kHid * 2));
    MK(cudaMalloc(&m->D1, cap * kHid * 2));
    MK(cudaMalloc(&m->D2, cap * kHid * 2));
    MK(cudaMalloc(&m->Yb, cap * 4));
    MK(cudaMalloc(&m->dl, cap * 4));
    MK(cudaMalloc(&m->loss, cap * 4));
    MK(cudaMalloc(&m->idx, cap * 4));
    MK(cudaMalloc(&m->part, m->part_floats * 4));
    MK(cudaMalloc(&m->scal, 4096 * 4));
    MK(cudaMalloc(&m->tc_err, 4));
    MK(cudaMemset(m->tc_err, 0, 4));
    MK(cudaFuncSetAttribute(tc_fwd_kernel<kIn>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem<kIn>()));
    MK(cudaFuncSetAttribute(tc_fwd_kernel<kHid>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem<kHid>()));
    MK(cudaFuncSetAttribute(tc_dgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcBwdSmem));
    MK(cudaFuncSetAttribute(tc_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcBwdSmem));
    MK(cudaFuncSetAttribute(tc_fwd3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcFwd3Smem));
    // He-uniform weights for the ReLU layers, zero biases
    std::vector<float> p(kParams, 0.0f);
    uint64_t st = seed;
    auto uni = [&](float a) { return (float)((splitmix(st) >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0) * a; };
    const float a1 = std::sqrt(6.0f / kIn), a2 = std::sqrt(6.0f / kHid), a4 = std::sqrt(3.0f / kHid);
    for (size_t i = 0; i < (size_t)kHid * kIn; i++) p[oW1 + i] = uni(a1);
    for (size_t i = 0; i < (size_t)kHid * kHid; i++) p[oW2 + i] = uni(a2);
    for (size_t i = 0; i < (size_t)kHid * kHid; i++) p[oW3 + i] = uni(a2);
    for (size_t i = 0; i < (size_t)kHid; i++) p[ow4 + i] = uni(a4);
    MK(cudaMemcpy(m->P, p.data(), kParams * 4, cudaMemcpyHostToDevice));
    MK(cudaMemset(m->Mm, 0, kParams * 4));
    MK(cudaMemset(m->Vv, 0, kParams * 4));
    MK(cudaMemset(m->G, 0, kParams * 4));
    count_launch();
    to_bf16_kernel<<<nblk(kParams, 256), 256>>>(m->P, m->Pb, kParams);
    MK(cudaGetLastError());
    MK(cudaDeviceSynchronize());
  });
  if (rc) {
    rc_mlp_free(m);
    return rc;
  }
  *out = m;
  return RC_OK;
}

void rc_mlp_free(rc_mlp *m) {
  if (!m) return;
  for (void *p : {(void *)m->P, (void *)m->G, (void *)m->Mm, (void *)m->Vv, (void *)m->Pb, (void *)m->Xb,
                  (void *)m->H1, (void *)m->H2, (void *)m->H3, (void *)m->D1, (void *)m->D2, (void *)m->Yb,
                  (void *)m->dl, (void *)m->loss, (void *)m->idx, (void *)m->part, (void *)m->scal,
                  (void *)m->tc_err})
    if (p) cudaFree(p);
  delete m;
}

int rc_mlp_set_backend(rc_mlp *m, int backend) {
  if (!m || backend < 0 || backend > 2) return RC_E_INVALID;
  m->backend = backend;
  return RC_OK;
}

int rc_mlp_backend_error(rc_mlp *m, uint32_t *flag) {
  if (!m || !flag) return RC_E_INVALID;
  return guarded([&] { MK(cudaMemcpy(flag, m->tc_err, 4, cudaMemcpyDeviceToHost)); });
}

int rc_mlp_get_params(const rc_mlp *m, float *out) {
  if (!m || !out) return RC_E_INVALID;
  return guarded([&] { MK(cudaMemcpy(out, m->P, kParams * 4, cudaMemcpyDeviceToHost)); });
}

int rc_mlp_set_params(rc_mlp *m, const float *in) {
  if (!m || !in) return RC_E_INVALID;
  return guarded([&] {
    MK(cudaMemcpy(m->P, in, kParams * 4, cudaMemcpyHostToDevice));
    count_launch();
    to_bf16_kernel<<<nblk(kParams, 256), 256>>>(m->P, m->Pb, kParams);
    MK(cudaGetLastError());
    MK(cudaDeviceSynchronize());
  });
}

int rc_mlp_forward(rc_mlp *m, const float *x, uint64_t n, float *prob, void *cuda_stream) {
  if (!m || (n && (!x || !prob))) return RC_E_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return guarded([&] {
    for (uint64_t r0 = 0; r0 < n; r0 += m->cap) {
      const int k = (int)std::min<uint64_t>(m->cap, n - r0);
      stage(m, x + r0 * kIn, nullptr, nullptr, k, s);
      forward(m, k, s);
      count_launch();
      head_fwd_kernel<<<nblk((size_t)k * 32, 256), 256, 0, s>>>(m->H3, m->Pb + ow4, m->P, k, prob + r0);
    }
    MK(cudaGetLastError());
    MK(cudaStreamSynchronize(s));
  });
}

int rc_mlp_grad(rc_mlp *m, const float *x, const float *y, uint32_t n, float *grad, float *loss, void *cuda_stream) {
  if (!m || n == 0 || n > m->cap || !x || !y) return RC_E_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return guarded([&] {
    stage(m, x, y, nullptr, (int)n, s);
    backward(m, (int)n, s);
    mean_loss(m, (int)n, 0, s);
    if (grad) MK(cudaMemcpyAsync(grad, m->G, kParams * 4, cudaMemcpyDeviceToHost, s));
    float l = 0;
    MK(cudaMemcpyAsync(&l, m->scal, 4, cudaMemcpyDeviceToHost, s));
    MK(cudaGetLastError());
    MK(cudaStreamSynchronize(s));
    if (loss) *loss = l;
  });
}

int rc_mlp_train(rc_mlp *m, const float *x, const float *y, uint64_t n, uint32_t epochs, uint32_t batch, float lr,
                 uint64_t seed, float *epoch_loss, void *cuda_stream) {
  if (!m || n == 0 || !x || !y || batch == 0 || batch > m->cap || n > 0xFFFFFFFFull || epochs > 4096)
    return RC_E_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return guarded([&] {
    std::vector<uint32_t> perm(n);
    uint32_t *didx = nullptr;
    MK(cudaMalloc(&didx, n * 4));
    struct Free {
      uint32_t *p;
      ~Free() { cudaFree(p); }
    } fr{didx};
    uint64_t st = seed;
    std::vector<float> sums(epochs, 0.0f);
    for (uint32_t e = 0; e < epochs; e++) {
      for (uint64_t i = 0; i < n; i++) perm[i] = (uint32_t)i;
      for (uint64_t i = n - 1; i > 0; i--) std::swap(perm[i], perm[splitmix(st) % (i + 1)]);
      MK(cudaMemcpyAsync(didx, perm.data(), n * 4, cudaMemcpyHostToDevice, s));
      uint32_t nb = 0;
      for (uint64_t r0 = 0; r0 < n; r0 += batch, nb++) {
        const int k = (int)std::min<uint64_t>(batch, n - r0);
        stage(m, x, y, didx + r0, k, s);
        backward(m, k, s);
        mean_loss(m, k, (int)std::min<uint32_t>(nb, 4095), s);
        adam(m, lr, s);
      }
      std::vector<float> ls(std::min<uint32_t>(nb, 4096));
      MK(cudaMemcpyAsync(ls.data(), m->scal, ls.size() * 4, cudaMemcpyDeviceToHost, s));
      MK(cudaStreamSynchronize(s));
      double t = 0;
      for (float v : ls) t += v;
      sums[e] = (float)(t / std::max<size_t>(ls.size(), 1));
    }
    MK(cudaGetLastError());
    if (epoch_loss) std::memcpy(epoch_loss, sums.data(), epochs * 4);
  });
}

}  // extern "C"
