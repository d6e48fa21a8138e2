// sepso_mlp.cu -- the learned prior of the planner on GB300 (sm_103a): an MLP
// (64x64 occupancy raster + start/target -> 1024 -> 512 -> 2T) with BF16 weights
// and FP32 accumulation, trained and run with the project's own kernels.
//
//   gemm_tc_kernel     C = A . B^T on the 5th-generation tensor cores: a TMA
//                      producer lane fills a ring of 128-byte-swizzled operand
//                      stages, an MMA lane issues tcgen05.mma (kind::f16, BF16
//                      inputs, FP32 accumulator in tensor memory) and frees each
//                      stage with tcgen05.commit, and eight warps read the
//                      accumulator back with tcgen05.ld for a fused epilogue
//                      (scale, bias, ReLU, the backward pass's ReLU mask, FP32
//                      and/or BF16 output, a transposed BF16 copy, column
//                      sums; K split into slices summed in order).  Tile N
//                      (64 / 128 / 256) per launch, and a persistent form.
//   raster_kernel      occupancy raster of the circles (cell centre inside a disk), each
//                      circle testing only the cells of its bounding box.
//   small kernels      row gather with a transposed copy, column sums (bias
//                      gradients), MSE loss gradient, split-K sums, Adam with the
//                      BF16 weight copies the products read.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <new>
#include <string>
#include <vector>

#include "sepso_device.cuh"
#include "sepso_internal.h"

namespace sepso {

// ---------------------------------------------------------------------------
// tcgen05 / cp.async helpers (inline PTX)
// ---------------------------------------------------------------------------
// 2D tiled TMA load (box of the tensor map at coordinates (x = k, y = row)) into
// shared memory, completing on an mbarrier with the transaction byte count.
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* smem_dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(smem_dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile written by TMA with the
// 128-byte swizzle: rows of 128 B (64 BF16 of K), 8-row atoms of 1024 B (the
// stride-dimension byte offset), leading-dimension offset unused for this layout
// (encoded as 1), fixed version bits 46..48 = 0b001, layout type 2 (128-byte
// swizzle) in bits 61..63.  The tile base is 1024-byte aligned; the k-th 16-wide
// K slice starts 32 k bytes further (the swizzle is a function of the address).
__device__ __forceinline__ uint64_t smem_desc_sw128(const void* p) {
  const uint64_t a = (uint64_t)((smem_addr(p) >> 4) & 0x3FFFu);
  return a | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t mma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------
// GEMM: C[M x N] = alpha * A[M x K] . B[N x K]^T (+ bias[n]) (then ReLU, or the
// ReLU mask mask[m][n] > 0), A and B row-major BF16 with K contiguous.
//
// One CTA computes a 128 x BN tile with eight warps.  Warp 0 (one lane) streams
// 128 x 64 and BN x 64 operand boxes into a ring of shared-memory stages with TMA
// (128-byte swizzle, zero fill past the matrix edges); warp 1 (one lane) issues
// four tcgen05.mma (M = 128, N = BN, K = 16) per stage into a BN-column FP32
// accumulator in tensor memory and frees the stage with tcgen05.commit; after the
// last stage all eight warps read the accumulator (warp w: rows 32 (w % 4) ..
// + 31, column half w / 4) with tcgen05.ld, stage it through shared memory and
// store it row-contiguously with the epilogue applied, then, when asked, a
// transposed BF16 copy and per-slab column sums.  A split product gives each CTA
// one K-slice (blockIdx.z) and stores its raw FP32 products.  Every wait is
// bounded; tensor memory is released on every path.
// ---------------------------------------------------------------------------
struct GemmArgs {
  const __nv_bfloat16* A;
  const __nv_bfloat16* B;
  int M, N, K, lda, ldb;
  float alpha;
  const float* bias;           // N, or null
  int relu;
  const __nv_bfloat16* mask;   // M x N (ldm), or null
  int ldm;
  float* Cf;                   // FP32 output, or null
  int ldcf;
  __nv_bfloat16* Cb;           // BF16 output, or null
  int ldcb;
  __nv_bfloat16* CbT;          // BF16 output transposed, CbT[n * ldct + m], or null
  int ldct;
  float* colpart;              // column sums of the output per 32-row slab: [ceil(M / 32)][N], or null
  float* part;                 // split K: raw FP32 products of K-slice z at part + z * M * N (row stride N)
  int kcb;                     // split K: K-blocks (of 64) per slice; 0 = the whole K in one slice
  int* status;
};

constexpr int kBM = 128, kBK = 64, kGemmThreads = 256;
constexpr int kRing = 192 * 1024;                         // operand stages
constexpr int kGemmSmem = kRing + 1024;                   // + alignment slack
template <int BN>
struct GemmTile {
  static constexpr int kABytes = kBM * kBK * 2;           // 16 KB
  static constexpr int kBBytes = BN * kBK * 2;
  static constexpr int kStage = kABytes + kBBytes;
  static constexpr int kStages = kRing / kStage;
  static_assert(kStages >= 2, "ring too small");
  static_assert(kBM * (BN + 4) * 4 <= kRing, "epilogue staging does not fit");
};

// BF16 element j (0..7) of eight packed in a uint4, as FP32 (exact).
__device__ __forceinline__ float bf16_of(const uint4& u, int j) {
  const uint32_t w = (j >> 1) == 0 ? u.x : (j >> 1) == 1 ? u.y : (j >> 1) == 2 ? u.z : u.w;
  return __uint_as_float((j & 1) ? (w & 0xffff0000u) : (w << 16));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // a in the low half
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Epilogue of a staged 128 x BN FP32 tile into the row-major outputs.  Work items
// are 8 columns of one row (consecutive threads: consecutive columns); the mask
// loads of a batch of items are all issued before the first of them is used, so
// that their latencies overlap.  A split-K slice stores its raw products to its
// slice of `part`.  With a transposed output or column sums the final values also
// go back into the tile.
template <int BN>
__device__ __forceinline__ void tile_epilogue_rows(const GemmArgs& g, float* tile, int m0, int n0, int tid) {
  constexpr int kLd = BN + 4, kUnits = BN / 8, kItems = kBM * kUnits, kBatch = 8;
  const bool raw = g.part != nullptr;
  float* Cf = raw ? g.part + (size_t)blockIdx.z * g.M * g.N : g.Cf;
  const int ldcf = raw ? g.N : g.ldcf;
  const __nv_bfloat16* mask = raw ? nullptr : g.mask;
  __nv_bfloat16* Cb = raw ? nullptr : g.Cb;
  const bool keep = !raw && (g.CbT || g.colpart);
  const int ncol = min(BN, g.N - n0), nrow = min(kBM, g.M - m0);
  const bool mvec = mask && (g.ldm & 7) == 0 && (reinterpret_cast<uintptr_t>(mask) & 15) == 0;
  const bool fvec = Cf && (ldcf & 3) == 0 && (reinterpret_cast<uintptr_t>(Cf) & 15) == 0;
  const bool bvec = Cb && (g.ldcb & 7) == 0 && (reinterpret_cast<uintptr_t>(Cb) & 15) == 0;
  const bool svec = g.bias && (reinterpret_cast<uintptr_t>(g.bias) & 15) == 0;
  for (int i0 = tid; i0 < kItems; i0 += kGemmThreads * kBatch) {
    uint4 mk[kBatch];
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      mk[b] = make_uint4(0u, 0u, 0u, 0u);
      const int it = i0 + b * kGemmThreads;
      const int rl = it / kUnits, c = (it % kUnits) * 8;
      if (mask && it < kItems && rl < nrow && c < ncol) {
        const __nv_bfloat16* mp = mask + (size_t)(m0 + rl) * g.ldm + (n0 + c);
        if (mvec && c + 8 <= ncol) {
          mk[b] = __ldg(reinterpret_cast<const uint4*>(mp));
        } else {
          uint32_t w0 = 0u, w1 = 0u, w2 = 0u, w3 = 0u;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            if (c + j < ncol) {
              const uint32_t h = (uint32_t)__bfloat16_as_ushort(mp[j]) << (16 * (j & 1));
              if ((j >> 1) == 0) w0 |= h;
              else if ((j >> 1) == 1) w1 |= h;
              else if ((j >> 1) == 2) w2 |= h;
              else w3 |= h;
            }
          }
          mk[b] = make_uint4(w0, w1, w2, w3);
        }
      }
    }
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      const int it = i0 + b * kGemmThreads;
      const int rl = it / kUnits, c = (it % kUnits) * 8;
      if (it >= kItems || rl >= nrow || c >= ncol) continue;
      float* tp = tile + rl * kLd + c;
      const float4 t0 = *reinterpret_cast<const float4*>(tp), t1 = *reinterpret_cast<const float4*>(tp + 4);
      float x[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
      const int nv = min(8, ncol - c);
      const int row = m0 + rl, col = n0 + c;
      if (!raw) {
        float bb[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (g.bias) {
          if (svec && nv == 8) {
            const float4 p = __ldg(reinterpret_cast<const float4*>(g.bias + col));
            const float4 q = __ldg(reinterpret_cast<const float4*>(g.bias + col + 4));
            bb[0] = p.x, bb[1] = p.y, bb[2] = p.z, bb[3] = p.w, bb[4] = q.x, bb[5] = q.y, bb[6] = q.z, bb[7] = q.w;
          } else {
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (j < nv) bb[j] = g.bias[col + j];
          }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (j < nv) {
            float y = x[j] * g.alpha;
            if (g.bias) y += bb[j];
            if (g.relu) y = fmaxf(y, 0.0f);
            if (mask && !(bf16_of(mk[b], j) > 0.0f)) y = 0.0f;
            x[j] = y;
          }
        }
        if (keep) {
          *reinterpret_cast<float4*>(tp) = make_float4(x[0], x[1], x[2], x[3]);
          *reinterpret_cast<float4*>(tp + 4) = make_float4(x[4], x[5], x[6], x[7]);
        }
      }
      if (Cf) {
        float* o = Cf + (size_t)row * ldcf + col;
        if (fvec && nv == 8) {
          *reinterpret_cast<float4*>(o) = make_float4(x[0], x[1], x[2], x[3]);
          *reinterpret_cast<float4*>(o + 4) = make_float4(x[4], x[5], x[6], x[7]);
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (j < nv) o[j] = x[j];
        }
      }
      if (Cb) {
        __nv_bfloat16* o = Cb + (size_t)row * g.ldcb + col;
        if (bvec && nv == 8) {
          *reinterpret_cast<uint4*>(o) = make_uint4(pack_bf16x2(x[0], x[1]), pack_bf16x2(x[2], x[3]),
                                                    pack_bf16x2(x[4], x[5]), pack_bf16x2(x[6], x[7]));
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (j < nv) o[j] = __float2bfloat16_rn(x[j]);
        }
      }
    }
  }
}

// Transposed BF16 output of the final tile values: lane = a pair of rows of a
// 64-row group, so that each store instruction writes 64 consecutive elements (128
// bytes) of one output row as BF16 pairs.
template <int BN>
__device__ __forceinline__ void tile_store_transposed(const GemmArgs& g, const float* tile, int m0, int n0, int warp,
                                                      int lane) {
  constexpr int kLd = BN + 4, kQuads = BN / 4;
  const int ncol = min(BN, g.N - n0), nrow = min(kBM, g.M - m0);
  const bool pair = (g.ldct & 1) == 0 && (reinterpret_cast<uintptr_t>(g.CbT) & 3) == 0;
  for (int it = warp; it < (kBM / 64) * kQuads; it += kGemmThreads / 32) {
    const int r0 = (it / kQuads) * 64 + 2 * lane, c = (it % kQuads) * 4;
    if (c >= ncol) continue;
    const float4 a = *reinterpret_cast<const float4*>(tile + r0 * kLd + c);
    const float4 b = *reinterpret_cast<const float4*>(tile + (r0 + 1) * kLd + c);
    if (r0 >= nrow) continue;
    const float xa[4] = {a.x, a.y, a.z, a.w}, xb[4] = {b.x, b.y, b.z, b.w};
    const bool two = r0 + 1 < nrow;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (c + j >= ncol) continue;
      __nv_bfloat16* o = g.CbT + (size_t)(n0 + c + j) * g.ldct + (m0 + r0);
      if (pair && two) {
        *reinterpret_cast<uint32_t*>(o) = pack_bf16x2(xa[j], xb[j]);
      } else {
        o[0] = __float2bfloat16_rn(xa[j]);
        if (two) o[1] = __float2bfloat16_rn(xb[j]);
      }
    }
  }
}

// Column sums of the final tile values over each 32-row slab (rows in order).
template <int BN>
__device__ __forceinline__ void tile_column_sums(const GemmArgs& g, const float* tile, int m0, int n0, int tid) {
  constexpr int kLd = BN + 4;
  const int ncol = min(BN, g.N - n0), nrow = min(kBM, g.M - m0);
  for (int it = tid; it < (kBM / 32) * BN; it += kGemmThreads) {
    const int slab = it / BN, c = it % BN;
    const int r0 = slab * 32;
    if (c >= ncol || r0 >= nrow) continue;
    const int r1 = min(r0 + 32, nrow);
    float s = 0.0f;
    for (int r = r0; r < r1; ++r) s += tile[r * kLd + c];
    g.colpart[(size_t)(m0 / 32 + slab) * g.N + (n0 + c)] = s;
  }
}

// The accumulator (128 x BN FP32 in tensor memory) through the staging tile in
// shared memory (row pitch BN + 4 floats: 16-byte aligned rows, and the eight
// threads of a quarter-warp land in distinct bank groups both when each writes its
// own row and when a warp reads one row) into the outputs.
template <int BN>
__device__ __forceinline__ void tile_epilogue_all(const GemmArgs& g, uint8_t* gsm, uint32_t tmem, int m0, int n0) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float* tile = reinterpret_cast<float*>(gsm);
  constexpr int kLd = BN + 4;
  // warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows), column half w / 4
  const int q = warp & 3, half = warp >> 2;
  const int r = q * 32 + lane;
  float v[32];
#pragma unroll 1
  for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2); c0 += 32) {
    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
    float4* dst = reinterpret_cast<float4*>(tile + r * kLd + c0);
#pragma unroll
    for (int i = 0; i < 8; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  }
  __syncthreads();
  tile_epilogue_rows<BN>(g, tile, m0, n0, tid);
  if (!g.part && (g.CbT || g.colpart)) {
    __syncthreads();  // the final values are back in the tile
    if (g.CbT) tile_store_transposed<BN>(g, tile, m0, n0, warp, lane);
    if (g.colpart) tile_column_sums<BN>(g, tile, m0, n0, tid);
  }
}

template <int BN>
__global__ void __launch_bounds__(kGemmThreads, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const GemmArgs g) {
  using TL = GemmTile<BN>;
  constexpr int S = TL::kStages;
  extern __shared__ uint8_t gsm_raw[];
  __shared__ uint64_t full[S], empty[S], done;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  uint8_t* gsm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  // this CTA's K-blocks: all of them, or K-slice blockIdx.z of a split product
  const int nkb_all = (g.K + kBK - 1) / kBK;
  const int kb0 = g.kcb > 0 ? (int)blockIdx.z * g.kcb : 0;
  const int nkb = g.kcb > 0 ? max(0, min(g.kcb, nkb_all - kb0)) : nkb_all;
  constexpr uint32_t kIdesc = mma_idesc_bf16(kBM, BN);

  if (warp == 0) tmem_alloc(&tmem_base, BN);
  if (tid == 32) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    s_fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    // producer: TMA boxes into the ring
    int issued = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % S;
      if (kb >= S && !mbar_wait_bounded(&empty[s], (uint32_t)((kb / S - 1) & 1), kWaitLimitNs)) {
        atomicExch(&s_fail, 1);
        break;
      }
      uint8_t* sa = gsm + s * TL::kStage;
      mbar_expect_tx(&full[s], (uint32_t)TL::kStage);
      tma_load_2d(sa, &tmA, (kb0 + kb) * kBK, m0, &full[s]);
      tma_load_2d(sa + TL::kABytes, &tmB, (kb0 + kb) * kBK, n0, &full[s]);
      issued = kb + 1;
    }
    // on a failure, let the boxes already in flight land before the CTA exits
    if (issued < nkb)
      for (int kb = max(0, issued - S); kb < issued; ++kb)
        mbar_wait_bounded(&full[kb % S], (uint32_t)((kb / S) & 1), kWaitLimitNs);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    int kb = 0;
    for (; kb < nkb; ++kb) {
      const int s = kb % S;
      if (!mbar_wait_bounded(&full[s], (uint32_t)((kb / S) & 1), kWaitLimitNs) || *(volatile int*)&s_fail) {
        atomicExch(&s_fail, 1);
        break;
      }
      tc_fence_after();
      const uint8_t* sa = gsm + s * TL::kStage;
      const uint8_t* sb = sa + TL::kABytes;
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk)
        mma_bf16(tmem, smem_desc_sw128(sa + kk * 32), smem_desc_sw128(sb + kk * 32), kIdesc,
                 (kb > 0 || kk > 0) ? 1u : 0u);
      // Free the stage only for a load that will reuse it: every commit is then
      // waited for by the producer or by `done`, and none can arrive on this CTA's
      // shared memory after it exits.
      if (kb + S < nkb) mma_commit(&empty[s]);
    }
    mma_commit(&done);  // tracks every MMA issued above
  }
  __syncwarp();
  // everyone: the accumulator is final once `done` completes
  if (!mbar_wait_bounded(&done, 0u, kWaitLimitNs)) atomicExch(&s_fail, 1);
  const bool fail = __syncthreads_or(*(volatile int*)&s_fail) != 0;
  if (fail) {
    if (tid == 0 && g.status) atomicExch(g.status, SEPSO_ETIMEOUT);
  } else if (nkb > 0) {
    tc_fence_after();
    tile_epilogue_all<BN>(g, gsm, tmem, m0, n0);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, BN);
}

// ---------------------------------------------------------------------------
// Persistent form: each CTA loops over tiles (t = blockIdx.x, + gridDim.x ...),
// with two BN-column accumulators in tensor memory so that the epilogue of one
// tile overlaps the main loop of the next.  Six warps: warp 0 lane 0 is the TMA
// producer (a ring of stages shared by all the CTA's tiles), warp 1 lane 0 issues
// the MMAs, warps 2..5 drain the accumulators (warp w reads TMEM lanes
// 32 (w % 4) .. + 31, as the hardware requires) through a per-warp 32 x 33 staging
// tile, storing rows of 32 consecutive columns (coalesced).
// ---------------------------------------------------------------------------
constexpr int kPThreads = 192;
constexpr int kStageWarpFloats = 32 * 33;
constexpr int kPRing = 192 * 1024 - 4 * kStageWarpFloats * 4 - 1024;  // ring + staging + alignment in 192 KB
constexpr int kPSmem = 192 * 1024;

template <int BN>
struct PTile {
  static constexpr int kABytes = kBM * kBK * 2;
  static constexpr int kStage = kABytes + BN * kBK * 2;
  static constexpr int kStages = (kPRing / kStage) < 8 ? (kPRing / kStage) : 8;
  static constexpr int kRingBytes = kStages * kStage;
  static_assert(kStages >= 2, "ring too small");
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

template <int BN>
__global__ void __launch_bounds__(kPThreads, 1)
    gemm_tc_persistent(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                       const GemmArgs g) {
  using TL = PTile<BN>;
  constexpr int S = TL::kStages;
  extern __shared__ uint8_t psm_raw[];
  __shared__ uint64_t full[S], empty[S], acc_full[2], acc_empty[2], done;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  uint8_t* ring = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(psm_raw) + 1023) & ~uintptr_t(1023));
  float* stage_all = reinterpret_cast<float*>(ring + TL::kRingBytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = (g.M + kBM - 1) / kBM, ntl = (g.N + BN - 1) / BN;
  const int tiles = mt * ntl;
  const int nkb = (g.K + kBK - 1) / kBK;
  constexpr uint32_t kIdesc = mma_idesc_bf16(kBM, BN);

  if (warp == 0) tmem_alloc(&tmem_base, 2 * BN);
  if (tid == 32) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 4);
    }
    mbar_init(&done, 1);
    s_fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // producer: one running k-block counter across the CTA's tiles
      long long it = 0;
      bool stop = false;
      for (int t = blockIdx.x; t < tiles && !stop; t += gridDim.x) {
        const int m0 = (t % mt) * kBM, n0 = (t / mt) * BN;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % S);
          const long long u = it / S;
          if (u >= 1 && !mbar_wait_bounded(&empty[s], (uint32_t)((u - 1) & 1), kWaitLimitNs)) {
            atomicExch(&s_fail, 1);
            stop = true;
            break;
          }
          if (*(volatile int*)&s_fail) {
            stop = true;
            break;
          }
          uint8_t* sa = ring + s * TL::kStage;
          mbar_expect_tx(&full[s], (uint32_t)TL::kStage);
          tma_load_2d(sa, &tmA, kb * kBK, m0, &full[s]);
          tma_load_2d(sa + TL::kABytes, &tmB, kb * kBK, n0, &full[s]);
        }
      }
      // boxes still in flight land before the CTA exits
      for (long long q = (it > S ? it - S : 0); q < it; ++q)
        mbar_wait_bounded(&full[q % S], (uint32_t)((q / S) & 1), kWaitLimitNs);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      long long it = 0;
      int lt = 0;
      bool stop = false;
      // k-blocks this CTA streams in all: a stage is freed only for a later load
      const long long total_it =
          (long long)((tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x) * nkb;
      for (int t = blockIdx.x; t < tiles && !stop; t += gridDim.x, ++lt) {
        const int a = lt & 1;
        const int v = lt >> 1;
        if (v >= 1 && !mbar_wait_bounded(&acc_empty[a], (uint32_t)((v - 1) & 1), kWaitLimitNs)) {
          atomicExch(&s_fail, 1);
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(a * BN);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % S);
          if (!mbar_wait_bounded(&full[s], (uint32_t)((it / S) & 1), kWaitLimitNs) || *(volatile int*)&s_fail) {
            atomicExch(&s_fail, 1);
            stop = true;
            break;
          }
          tc_fence_after();
          const uint8_t* sa = ring + s * TL::kStage;
          const uint8_t* sb = sa + TL::kABytes;
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk)
            mma_bf16(acc, smem_desc_sw128(sa + kk * 32), smem_desc_sw128(sb + kk * 32), kIdesc,
                     (kb > 0 || kk > 0) ? 1u : 0u);
          if (it + S < total_it) mma_commit(&empty[s]);
        }
        if (!stop) mma_commit(&acc_full[a]);
      }
      mma_commit(&done);  // tracks every MMA issued above
    }
  } else {
    // epilogue warps 2..5: TMEM lane quarter (warp % 4)
    const int q = warp & 3;
    float* st = stage_all + (warp - 2) * kStageWarpFloats;
    const bool vec_ok = true;
    (void)vec_ok;
    int lt = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++lt) {
      const int a = lt & 1;
      int ok = 1;
      if (lane == 0) ok = mbar_wait_bounded(&acc_full[a], (uint32_t)((lt >> 1) & 1), kWaitLimitNs) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok || *(volatile int*)&s_fail) {
        if (lane == 0) atomicExch(&s_fail, 1);
        break;
      }
      tc_fence_after();
      const int m0 = (t % mt) * kBM, n0 = (t / mt) * BN;
      const int rbase = m0 + q * 32;
      float v[32];
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        tmem_ld32(tmem + (uint32_t)(a * BN) + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
        // this lane holds row rbase + lane, columns c0 .. c0 + 31
#pragma unroll
        for (int c = 0; c < 32; ++c) st[lane * 33 + c] = v[c];
        __syncwarp();
        // lane = column: rows rbase .. rbase + 31, the 32 mask loads issued first
        const int col = n0 + c0 + lane;
        if (col < g.N && rbase < g.M) {
          float mk[32];
          if (g.mask) {
#pragma unroll
            for (int r = 0; r < 32; ++r) {
              const int row = rbase + r;
              mk[r] = row < g.M ? __bfloat162float(g.mask[(size_t)row * g.ldm + col]) : 0.0f;
            }
          }
          const float bcol = g.bias ? g.bias[col] : 0.0f;
          float csum = 0.0f;
#pragma unroll
          for (int r = 0; r < 32; ++r) {
            const int row = rbase + r;
            if (row < g.M) {
              float x = g.alpha * st[r * 33 + lane] + bcol;
              if (g.relu) x = fmaxf(x, 0.0f);
              if (g.mask && !(mk[r] > 0.0f)) x = 0.0f;
              if (g.Cf) g.Cf[(size_t)row * g.ldcf + col] = x;
              if (g.Cb) g.Cb[(size_t)row * g.ldcb + col] = __float2bfloat16_rn(x);
              st[r * 33 + lane] = x;
              csum += x;
            }
          }
          if (g.colpart) g.colpart[(size_t)(rbase / 32) * g.N + col] = csum;
        }
        if (g.CbT) {
          // lane = row: 32 consecutive rows of each transposed output row
          __syncwarp();
          const int row = rbase + lane;
          if (row < g.M) {
#pragma unroll 8
            for (int c = 0; c < 32; ++c) {
              const int cc = n0 + c0 + c;
              if (cc < g.N) g.CbT[(size_t)cc * g.ldct + row] = __float2bfloat16_rn(st[lane * 33 + c]);
            }
          }
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[a]);
    }
  }
  __syncwarp();
  // teardown: every MMA has completed before tensor memory is released
  if (!mbar_wait_bounded(&done, 0u, kWaitLimitNs)) atomicExch(&s_fail, 1);
  if (__syncthreads_or(*(volatile int*)&s_fail) && tid == 0 && g.status) atomicExch(g.status, SEPSO_ETIMEOUT);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 2 * BN);
}

}  // namespace sepso

namespace sepso {

// ---------------------------------------------------------------------------
// Features and labels of a chunk of scenes (one CTA per scene).
//   feature row: g*g occupancy cells (cell (i, j) occupied when its centre lies in
//   a closed disk; FP32 decision with explicit round-to-nearest operations), then
//   start / target over the map extent, then zeros up to K.
//   label row (when waypoints are given): offset of each waypoint from the point
//   of the straight start-target line at fraction (k + 1) / (T + 1), over the extent.
// ---------------------------------------------------------------------------
struct RasterArgs {
  int n, grid, K, ldx, T, O_max;
  float W, H;
  const float4* circ;      // staged circles (cx, cy, r, 0) of the chunk
  const int* coff;         // n + 1 prefix offsets into circ
  const float* pts;        // n x 4
  const float* wp;         // n x 2T, or null
  __nv_bfloat16* X;        // n rows of K features, row pitch ldx >= K (pad zero)
  float* Y;                // n rows of 2T, or null
};

__global__ void __launch_bounds__(256) raster_kernel(const RasterArgs a) {
  // Occupancy in shared memory, one byte per cell.  Each thread takes circles and
  // tests only the cells of the circle's bounding box (widened by one cell); the
  // test of a (cell, circle) pair is the same as over the whole grid, so a cell is
  // set exactly when its centre lies in some disk.
  extern __shared__ unsigned char occ[];
  const int s = blockIdx.x;
  const int c0 = a.coff[s], O = a.coff[s + 1] - c0;
  const int G = a.grid, g2 = G * G;
  for (int c = threadIdx.x; c < g2; c += blockDim.x) occ[c] = 0;
  __syncthreads();
  const float cw = a.W / (float)G, ch = a.H / (float)G;
  for (int o = threadIdx.x; o < O; o += blockDim.x) {
    const float4 q = a.circ[c0 + o];
    const float r2 = __fmul_rn(q.z, q.z);
    // cell index bounds, clamped in FP32 before the conversion (any finite circle)
    const float lim = (float)(G + 1);
    const int j0 = max(0, (int)fminf(fmaxf(floorf((q.x - q.z) / cw - 0.5f) - 1.0f, -1.0f), lim));
    const int j1 = min(G - 1, (int)fminf(fmaxf(ceilf((q.x + q.z) / cw - 0.5f) + 1.0f, -1.0f), lim));
    const int i0 = max(0, (int)fminf(fmaxf(floorf((q.y - q.z) / ch - 0.5f) - 1.0f, -1.0f), lim));
    const int i1 = min(G - 1, (int)fminf(fmaxf(ceilf((q.y + q.z) / ch - 0.5f) + 1.0f, -1.0f), lim));
    for (int i = i0; i <= i1; ++i) {
      const float y = __fmul_rn((float)i + 0.5f, ch);
      const float dy = __fsub_rn(y, q.y);
      const float dy2 = __fmul_rn(dy, dy);
      for (int j = j0; j <= j1; ++j) {
        const float x = __fmul_rn((float)j + 0.5f, cw);
        const float dx = __fsub_rn(x, q.x);
        if (__fadd_rn(__fmul_rn(dx, dx), dy2) <= r2) occ[i * G + j] = 1;
      }
    }
  }
  __syncthreads();
  __nv_bfloat16* row = a.X + (size_t)s * a.ldx;
  for (int c = threadIdx.x; c < g2; c += blockDim.x) row[c] = __float2bfloat16_rn(occ[c] ? 1.0f : 0.0f);
  const float* p = a.pts + 4 * s;
  for (int k = g2 + threadIdx.x; k < a.ldx; k += blockDim.x) {
    const int e = k - g2;
    const float v = (e < 4 && k < a.K) ? p[e] / ((e & 1) ? a.H : a.W) : 0.0f;
    row[k] = __float2bfloat16_rn(v);
  }
  if (a.wp != nullptr && a.Y != nullptr) {
    const int T = a.T;
    for (int d = threadIdx.x; d < 2 * T; d += blockDim.x) {
      const int k = d < T ? d : d - T;
      const float f = (float)(k + 1) / (float)(T + 1);
      const float s0 = d < T ? p[0] : p[1], t0 = d < T ? p[2] : p[3];
      const float ext = d < T ? a.W : a.H;
      a.Y[(size_t)s * 2 * T + d] = (a.wp[(size_t)s * 2 * T + d] - (s0 + f * (t0 - s0))) / ext;
    }
  }
}

// Labels of rows from device waypoints (row stride ld): the same encoding as above.
__global__ void label_kernel(const float* __restrict__ wp, int ld, int n, int T, const float* __restrict__ pts,
                             float W, float H, float* __restrict__ Y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * 2 * T) return;
  const int s = i / (2 * T), d = i - s * 2 * T;
  const int k = d < T ? d : d - T;
  const float f = (float)(k + 1) / (float)(T + 1);
  const float* p = pts + 4 * s;
  const float s0 = d < T ? p[0] : p[1], t0 = d < T ? p[2] : p[3];
  const float ext = d < T ? W : H;
  Y[i] = (wp[(size_t)s * ld + d] - (s0 + f * (t0 - s0))) / ext;
}

// Minibatch rows: idx[b] = Philox(seed; step, b) mod n_rows (with replacement).
__global__ void sample_kernel(int* idx, int B, int n_rows, uint32_t k0, uint32_t k1, uint32_t step) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) {
    const uint4 r = draw(k0, k1, step, (uint32_t)b, kStreamSample, 0u, 0u);
    idx[b] = (int)(r.x % (uint32_t)n_rows);
  }
}

// x[b] = X[r] (K bf16, 16-byte vectors), t[b] = Y[r], with r = idx[b] (or first + b
// without an index list).
// dY = (y - t) / B: FP32 (B x O), BF16 (B x ldb, columns O .. ldb-1 zero) and BF16
// transposed (O x B); loss += sum (y - t)^2 / 2B, one atomic per CTA.
__global__ void loss_grad_kernel(const float* __restrict__ y, const float* __restrict__ t, int B, int O,
                                 float* __restrict__ dyf, __nv_bfloat16* __restrict__ dyb, int ldb,
                                 __nv_bfloat16* __restrict__ dyT, float* loss) {
  __shared__ float wsum[32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float sq = 0.0f;
  if (i < B * ldb) {
    const int b = i / ldb, d = i - b * ldb;
    float g = 0.0f;
    if (d < O) {
      const float e = y[(size_t)b * O + d] - t[(size_t)b * O + d];
      sq = e * e;
      g = e / (float)B;
      dyf[(size_t)b * O + d] = g;
      dyT[(size_t)d * B + b] = __float2bfloat16_rn(g);
    }
    dyb[i] = __float2bfloat16_rn(g);
  }
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += wsum[w];
    if (s != 0.0f) atomicAdd(loss, 0.5f * s / (float)B);
  }
}

// Column sums, first stage: part[p][j] = sum of D[b][j] over rows b of 32-row block p
// (8 row lanes, then the lanes in order).
__global__ void colsum_part_kernel(const float* __restrict__ D, int B, int N, int ld, float* __restrict__ part) {
  __shared__ float s[8][33];
  const int j = blockIdx.x * 32 + threadIdx.x;
  const int b0 = blockIdx.y * 32;
  float acc = 0.0f;
  if (j < N)
    for (int b = b0 + threadIdx.y; b < min(B, b0 + 32); b += 8) acc += D[(size_t)b * ld + j];
  s[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && j < N) {
    float v = 0.0f;
    for (int r = 0; r < 8; ++r) v += s[r][threadIdx.x];
    part[(size_t)blockIdx.y * N + j] = v;
  }
}

// Split K: C = epilogue(alpha * (sum of the K-slices' FP32 products, in slice order)).
__global__ void splitk_reduce_kernel(const GemmArgs g, int slices) {
  const long long MN = (long long)g.M * g.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < MN; i += (long long)gridDim.x * blockDim.x) {
    float acc = 0.0f;
#pragma unroll 4
    for (int z = 0; z < slices; ++z) acc += __ldcs(g.part + z * MN + i);
    const int m = (int)(i / g.N), n = (int)(i - (long long)m * g.N);
    float x = acc * g.alpha;
    if (g.bias) x += g.bias[n];
    if (g.relu) x = fmaxf(x, 0.0f);
    if (g.mask && !(__bfloat162float(g.mask[(size_t)m * g.ldm + n]) > 0.0f)) x = 0.0f;
    if (g.Cf) g.Cf[(size_t)m * g.ldcf + n] = x;
    if (g.Cb) g.Cb[(size_t)m * g.ldcb + n] = __float2bfloat16_rn(x);
  }
}

// x[b] = X[row b] and xT[k][b] = X[row b][k] (row b = idx[b], or first + b; rows of
// K features at pitch ldx), t[b] = Y[row b]: 64 rows x 128 features per CTA, read
// and copied with 16-byte accesses, transposed through shared memory into 128-byte
// row segments of xT (K a multiple of 8, n even).
__global__ void __launch_bounds__(256) gather_t_kernel(const int* __restrict__ idx, int first, int n, int K, int ldx,
                                                       const __nv_bfloat16* __restrict__ X, const float* __restrict__ Y,
                                                       int O, __nv_bfloat16* __restrict__ x,
                                                       __nv_bfloat16* __restrict__ xT, float* __restrict__ t) {
  __shared__ uint32_t sm[64][65];  // 64 rows b x 64 feature pairs
  const int k0 = blockIdx.x * 128, b0 = blockIdx.y * 64;
  const int tid = threadIdx.x, lane = tid & 31;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int e = tid + i * 256;
    const int rb = e >> 4, qd = e & 15;  // row of the tile, 8-feature group
    const int b = b0 + rb, k = k0 + qd * 8;
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
    if (b < n && k < K) {
      const int r = idx ? idx[b] : first + b;
      w = *reinterpret_cast<const uint4*>(X + (size_t)r * ldx + k);
      *reinterpret_cast<uint4*>(x + (size_t)b * ldx + k) = w;
    }
    sm[rb][qd * 4 + 0] = w.x;
    sm[rb][qd * 4 + 1] = w.y;
    sm[rb][qd * 4 + 2] = w.z;
    sm[rb][qd * 4 + 3] = w.w;
  }
  if (blockIdx.x == 0) {
    for (int e = tid; e < 64 * O; e += 256) {
      const int rb = e / O, d = e - rb * O, b = b0 + rb;
      if (b < n) t[(size_t)b * O + d] = Y[(size_t)(idx ? idx[b] : first + b) * O + d];
    }
  }
  __syncthreads();
#pragma unroll 4
  for (int kk = tid >> 5; kk < 128; kk += 8) {
    const int k = k0 + kk, b = b0 + 2 * lane;
    if (k < K && b < n) {
      const int sh = (kk & 1) ? 16 : 0;
      const uint32_t lo = (sm[2 * lane][kk >> 1] >> sh) & 0xffffu, hi = (sm[2 * lane + 1][kk >> 1] >> sh) & 0xffffu;
      *reinterpret_cast<uint32_t*>(xT + (size_t)k * n + b) = lo | (hi << 16);
    }
  }
}

// db[j] = sum_b D[b][j]: 32 columns per CTA, 8 row lanes, fixed summation order.
__global__ void colsum_kernel(const float* __restrict__ D, int B, int N, int ld, float* __restrict__ db) {
  __shared__ float part[8][33];
  const int j = blockIdx.x * 32 + threadIdx.x;
  float s = 0.0f;
  if (j < N)
    for (int b = threadIdx.y; b < B; b += 8) s += D[(size_t)b * ld + j];
  part[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && j < N) {
    float v = 0.0f;
    for (int r = 0; r < 8; ++r) v += part[r][threadIdx.x];
    db[j] = v;
  }
}

// BF16 copies of the weights that the products read: W1 (h1 x k, at offset 0) in
// rows of pitch ldp (128-byte rows for the TMA boxes), W2 (h2 x h1, at off2) and
// W3 (o x h2, at off4) transposed (the backward pass's B operands).
struct BfMirrors {
  __nv_bfloat16* w1p;
  int h1, k, ldp;
  __nv_bfloat16* w2t;
  long long off2;
  int h2;
  __nv_bfloat16* w3t;
  long long off4;
  int o, o8;
};

__device__ __forceinline__ void mirror_store(const BfMirrors& mr, long long i, __nv_bfloat16 b) {
  if (i < (long long)mr.h1 * mr.k) {  // h1 * ldp < 2^31
    const int ii = (int)i, r = ii / mr.k;
    mr.w1p[r * mr.ldp + (ii - r * mr.k)] = b;
    return;
  }
  long long j = i - mr.off2;
  if (j >= 0 && j < (long long)mr.h2 * mr.h1) {
    const int jj = (int)j, r = jj / mr.h1;
    mr.w2t[(size_t)(jj - r * mr.h1) * mr.h2 + r] = b;
    return;
  }
  j = i - mr.off4;
  if (j >= 0 && j < (long long)mr.o * mr.h2) {
    const int jj = (int)j, r = jj / mr.h2;
    mr.w3t[(size_t)(jj - r * mr.h2) * mr.o8 + r] = b;
  }
}

__device__ __forceinline__ float adam_update(float& w, float& m, float& v, float g, float lr, float b1, float b2,
                                             float eps, float c1, float c2) {
  m = b1 * m + (1.0f - b1) * g;
  v = b2 * v + (1.0f - b2) * g * g;
  w = w - lr * (m / c1) / (sqrtf(v / c2) + eps);
  return w;
}

// Adam (Kingma and Ba, 2015) on FP32 masters, four parameters per thread step
// (16-byte accesses), then the BF16 copies: wb (all parameters) and the mirrors.
__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, __nv_bfloat16* __restrict__ wb, long long n, float lr,
                            float b1, float b2, float eps, float c1, float c2, const BfMirrors mr) {
  const long long n4 = n / 4;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4; q += stride) {
    float4 W = reinterpret_cast<float4*>(w)[q], M = reinterpret_cast<float4*>(m)[q];
    float4 V = reinterpret_cast<float4*>(v)[q];
    const float4 Gq = reinterpret_cast<const float4*>(g)[q];
    const float a = adam_update(W.x, M.x, V.x, Gq.x, lr, b1, b2, eps, c1, c2);
    const float b = adam_update(W.y, M.y, V.y, Gq.y, lr, b1, b2, eps, c1, c2);
    const float c = adam_update(W.z, M.z, V.z, Gq.z, lr, b1, b2, eps, c1, c2);
    const float d = adam_update(W.w, M.w, V.w, Gq.w, lr, b1, b2, eps, c1, c2);
    reinterpret_cast<float4*>(w)[q] = W;
    reinterpret_cast<float4*>(m)[q] = M;
    reinterpret_cast<float4*>(v)[q] = V;
    const __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
    uint2 u;
    u.x = *reinterpret_cast<const uint32_t*>(&lo);
    u.y = *reinterpret_cast<const uint32_t*>(&hi);
    reinterpret_cast<uint2*>(wb)[q] = u;
    mirror_store(mr, 4 * q, lo.x);
    mirror_store(mr, 4 * q + 1, lo.y);
    mirror_store(mr, 4 * q + 2, hi.x);
    mirror_store(mr, 4 * q + 3, hi.y);
  }
  for (long long i = 4 * n4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
    const float wi = adam_update(w[i], m[i], v[i], g[i], lr, b1, b2, eps, c1, c2);
    const __nv_bfloat16 bi = __float2bfloat16_rn(wi);
    wb[i] = bi;
    mirror_store(mr, i, bi);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, long long n,
                               const BfMirrors mr) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const __nv_bfloat16 b = __float2bfloat16_rn(w[i]);
    wb[i] = b;
    mirror_store(mr, i, b);
  }
}

// Waypoints of the network outputs: straight-line point + y * extent, clipped to the map.
__global__ void decode_kernel(const float* __restrict__ y, int n, int T, const float* __restrict__ pts, float W,
                              float H, float* __restrict__ out, int ldo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * 2 * T) return;
  const int s = i / (2 * T), d = i - s * 2 * T;
  const int k = d < T ? d : d - T;
  const float f = (float)(k + 1) / (float)(T + 1);
  const float* p = pts + 4 * s;
  const float s0 = d < T ? p[0] : p[1], t0 = d < T ? p[2] : p[3];
  const float ext = d < T ? W : H;
  out[(size_t)s * ldo + d] = fminf(fmaxf(s0 + f * (t0 - s0) + y[i] * ext, 0.0f), ext);
}

}  // namespace sepso

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
using sepso::GemmArgs;
using bf16 = __nv_bfloat16;

namespace {

thread_local std::string g_prior_error;

int pfail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int pfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_prior_error = buf;
  return code;
}

#define PCUDA(expr)                                                                          \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess) return pfail(SEPSO_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)
#define PTRY(expr)              \
  do {                          \
    const int r_ = (expr);      \
    if (r_ != SEPSO_OK) return r_; \
  } while (0)

size_t al256(size_t v) { return (v + 255) & ~size_t(255); }
int round8(int v) { return (v + 7) / 8 * 8; }
constexpr int kLossRing = 65536;

__device__ int g_gemm_status;

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Tensor map of a row-major BF16 matrix (rows x cols, row stride ld elements) read
// in boxes of 64 columns (128 B, the swizzle span) x box_rows rows; zero fill
// outside the matrix.  Encoded maps are kept in a small per-thread cache keyed by
// their arguments (the training loop reuses the same buffers every step).
struct MapKey {
  const void* base;
  int rows, cols, ld, box_rows;
  bool operator==(const MapKey& o) const {
    return base == o.base && rows == o.rows && cols == o.cols && ld == o.ld && box_rows == o.box_rows;
  }
};
constexpr int kMapCache = 64;
thread_local MapKey t_map_keys[kMapCache];
thread_local CUtensorMap t_maps[kMapCache];
thread_local int t_map_n = 0, t_map_next = 0;

int encode_map(CUtensorMap* map, const void* base, int rows, int cols, int ld, int box_rows);

int make_map(CUtensorMap* map, const void* base, int rows, int cols, int ld, int box_rows) {
  const MapKey k{base, rows, cols, ld, box_rows};
  for (int i = 0; i < t_map_n; ++i)
    if (t_map_keys[i] == k) {
      *map = t_maps[i];
      return SEPSO_OK;
    }
  PTRY(encode_map(map, base, rows, cols, ld, box_rows));
  const int slot = t_map_next;
  t_map_next = (t_map_next + 1) % kMapCache;
  t_map_n = std::min(t_map_n + 1, kMapCache);
  t_map_keys[slot] = k;
  t_maps[slot] = *map;
  return SEPSO_OK;
}

int encode_map(CUtensorMap* map, const void* base, int rows, int cols, int ld, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return pfail(SEPSO_ECUDA, "cuTensorMapEncodeTiled is not available");
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)sepso::kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return pfail(SEPSO_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return SEPSO_OK;
}

int g_num_sms = 0;

// Tile N for a product: the widest tile whose grid still covers the SMs, else the
// one with the fewest waves (ties to the wider tile).
int choose_tile_n(int M, int N) {
  if (g_num_sms <= 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      g_num_sms = 148;
  }
  const int mt = (M + sepso::kBM - 1) / sepso::kBM;
  int best = 64;
  double best_cost = 1e300;
  for (int bn : {256, 128, 64}) {
    const long long tiles = (long long)mt * ((N + bn - 1) / bn);
    const long long waves = (tiles + g_num_sms - 1) / g_num_sms;
    // per-tile time ~ bn, with narrower tiles paying more per output column
    const double per_tile = bn * (bn == 256 ? 1.0 : bn == 128 ? 1.15 : 1.6);
    const double cost = (double)waves * per_tile;
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = bn;
    }
  }
  return best;
}

template <int BN>
int gemm_launch_bn(const CUtensorMap& ta, const GemmArgs& g, cudaStream_t s, int slices = 1) {
  CUtensorMap tb;
  PTRY(make_map(&tb, g.B, g.N, g.K, g.ldb, BN));
  static thread_local int configured_device = -1;
  int dev = 0;
  PCUDA(cudaGetDevice(&dev));
  if (configured_device != dev) {
    PCUDA(cudaFuncSetAttribute(sepso::gemm_tc_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               sepso::kGemmSmem));
    configured_device = dev;
  }
  const dim3 grid((g.M + sepso::kBM - 1) / sepso::kBM, (g.N + BN - 1) / BN, slices);
  if (grid.y > 65535u || grid.z > 65535u) return pfail(SEPSO_EINVAL, "gemm: N or the K split too large");
  sepso::gemm_tc_kernel<BN><<<grid, sepso::kGemmThreads, sepso::kGemmSmem, s>>>(ta, tb, g);
  PCUDA(cudaGetLastError());
  return SEPSO_OK;
}

template <int BN>
int gemm_launch_persistent(const CUtensorMap& ta, const GemmArgs& g, cudaStream_t s) {
  CUtensorMap tb;
  PTRY(make_map(&tb, g.B, g.N, g.K, g.ldb, BN));
  static thread_local int configured_device = -1;
  int dev = 0;
  PCUDA(cudaGetDevice(&dev));
  if (configured_device != dev) {
    PCUDA(cudaFuncSetAttribute(sepso::gemm_tc_persistent<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               sepso::kPSmem));
    configured_device = dev;
  }
  const long long tiles = (long long)((g.M + sepso::kBM - 1) / sepso::kBM) * ((g.N + BN - 1) / BN);
  if (g_num_sms <= 0) choose_tile_n(g.M, g.N);  // fills the SM count
  const int grid = (int)std::min<long long>(tiles, (long long)g_num_sms);
  sepso::gemm_tc_persistent<BN><<<grid, sepso::kPThreads, sepso::kPSmem, s>>>(ta, tb, g);
  PCUDA(cudaGetLastError());
  return SEPSO_OK;
}

// Kernel and tile width for a product (positive: persistent; negative: one tile
// per CTA), from a sweep of both kernels on GB300 with the eight-warp epilogue
// (TFLOP/s, best persistent / best one per CTA):
//   8192^3 1230 / 1352, 4096^3 954 / 1051, 1024 x 4104 x 4096 639 / 849,
//   4096 x 1024 x 4104 610 / 817 (three quarters of a wave or more of 256-wide
//   tiles)                                                   -> one per CTA, 256
//   4096 x 512 x 1024 194 / 252, 4096 x 1024 x 512 170 / 225; with mask,
//   transposed copy and column sums 4096 x 512 x 40: 31.1 / 18.7 us -> one per CTA, 128
//   long K and few tiles (1024 x 1024 x 4104 at width 64: 237 / 262), or N <= 64
//   (4096 x 40 x 512: 11.0 / 8.7 us)                         -> one per CTA, 64
int choose_tile_n_auto(int M, int N, int K) {
  choose_tile_n(M, N);  // fills the SM count
  const long long mt = (M + sepso::kBM - 1) / sepso::kBM;
  const long long t256 = mt * ((N + 255) / 256);
  if (4 * t256 >= 3LL * g_num_sms) return -256;
  return (K >= 2048 || N <= 64) ? -64 : -128;
}

// tile_n: 0 automatic (persistent kernel); 64 / 128 / 256 the persistent kernel
// with that tile; -64 / -128 / -256 the one-tile-per-CTA kernel.
int gemm_check(const GemmArgs& g, int tile_n) {
  if (g.M < 1 || g.N < 1 || g.K < 8 || (g.K & 7) || (g.lda & 7) || (g.ldb & 7) || g.lda < g.K || g.ldb < g.K)
    return pfail(SEPSO_EINVAL, "gemm: bad sizes M %d N %d K %d lda %d ldb %d", g.M, g.N, g.K, g.lda, g.ldb);
  if (!g.A || !g.B || !aligned16(g.A) || !aligned16(g.B))
    return pfail(SEPSO_EINVAL, "gemm: A and B must be 16-byte aligned device arrays");
  if ((g.Cf && g.ldcf < g.N) || (g.Cb && g.ldcb < g.N) || (g.mask && g.ldm < g.N))
    return pfail(SEPSO_EINVAL, "gemm: output or mask row stride below N");
  if (tile_n != 0 && tile_n != 64 && tile_n != 128 && tile_n != 256 && tile_n != -64 && tile_n != -128 &&
      tile_n != -256)
    return pfail(SEPSO_EINVAL, "gemm: tile N %d (64, 128 or 256; negative for one tile per CTA)", tile_n);
  return SEPSO_OK;
}

int gemm_launch(const GemmArgs& g, cudaStream_t s, int tile_n = 0) {
  PTRY(gemm_check(g, tile_n));
  if (tile_n == 0) tile_n = choose_tile_n_auto(g.M, g.N, g.K);
  CUtensorMap ta;
  PTRY(make_map(&ta, g.A, g.M, g.K, g.lda, sepso::kBM));
  switch (tile_n) {
    case 64: return gemm_launch_persistent<64>(ta, g, s);
    case 128: return gemm_launch_persistent<128>(ta, g, s);
    case 256: return gemm_launch_persistent<256>(ta, g, s);
    case -64: return gemm_launch_bn<64>(ta, g, s);
    case -128: return gemm_launch_bn<128>(ta, g, s);
    case -256: return gemm_launch_bn<256>(ta, g, s);
    default: return pfail(SEPSO_EINVAL, "gemm: tile N %d", tile_n);
  }
}

// What a product needs beyond the plain epilogue: a transposed BF16 copy of the
// output, its column sums, or a split of K into slices whose FP32 products are
// summed in slice order (row-major outputs only).
struct GemmExtra {
  bf16* CbT = nullptr;
  int ldct = 0;
  float* colsum = nullptr;
  int ksplit = 1;
  float* ws = nullptr;  // device scratch of gemm_ws_bytes
  size_t ws_bytes = 0;
};

size_t gemm_ws_bytes(long long M, long long N, int ksplit, bool colsum) {
  if (ksplit > 1) return (size_t)ksplit * M * N * 4;
  return colsum ? (size_t)((M + 31) / 32) * N * 4 : 0;
}

// K slices for a product whose tiles fill few SMs: about one wave of CTAs, at
// least 4 K-blocks per slice, at most kMaxSlices.
constexpr int kMaxSlices = 16;
int auto_ksplit(int M, int N, int K, int bn) {
  choose_tile_n(M, N);  // fills the SM count
  const long long tiles = (long long)((M + sepso::kBM - 1) / sepso::kBM) * ((N + bn - 1) / bn);
  const long long nkb = (K + sepso::kBK - 1) / sepso::kBK;
  if (2 * tiles > g_num_sms) return 1;
  long long sl = std::min<long long>(g_num_sms / tiles, nkb / 4);
  sl = std::min<long long>(sl, kMaxSlices);
  return (int)std::max<long long>(sl, 1);
}

int gemm_run_check(const GemmArgs& g, const GemmExtra& e, int tile_n) {
  PTRY(gemm_check(g, tile_n));
  if (e.CbT && e.ldct < g.M) return pfail(SEPSO_EINVAL, "gemm: transposed output row stride %d below M", e.ldct);
  if (e.ksplit < 1 || e.ksplit > 4096) return pfail(SEPSO_EINVAL, "gemm: K split %d", e.ksplit);
  if (e.ksplit > 1 && (e.CbT || e.colsum))
    return pfail(SEPSO_EINVAL, "gemm: a K split supports the row-major outputs only");
  const size_t need = gemm_ws_bytes(g.M, g.N, e.ksplit, e.colsum != nullptr);
  if (need && (!e.ws || e.ws_bytes < need || !aligned16(e.ws)))
    return pfail(SEPSO_ENOSPC, "gemm: workspace of %zu bytes, need %zu (16-byte aligned)", e.ws_bytes, need);
  return SEPSO_OK;
}

// One product with its extras; *launches gets the kernels launched.
int gemm_run(GemmArgs g, const GemmExtra& e, cudaStream_t s, int tile_n, int* launches) {
  *launches = 0;
  PTRY(gemm_run_check(g, e, tile_n));
  g.CbT = nullptr;
  g.colpart = nullptr;
  g.part = nullptr;
  g.kcb = 0;
  if (e.ksplit > 1) {
    const int nkb = (g.K + sepso::kBK - 1) / sepso::kBK;
    const int kcb = (nkb + e.ksplit - 1) / e.ksplit;
    const int slices = (nkb + kcb - 1) / kcb;  // every slice non-empty
    GemmArgs r = g;
    r.alpha = 1.0f;
    r.bias = nullptr;
    r.relu = 0;
    r.mask = nullptr;
    r.Cf = nullptr;
    r.Cb = nullptr;
    r.part = e.ws;
    r.kcb = kcb;
    CUtensorMap ta;
    PTRY(make_map(&ta, g.A, g.M, g.K, g.lda, sepso::kBM));
    const int bn = tile_n ? std::abs(tile_n) : 128;
    if (bn == 64) PTRY(gemm_launch_bn<64>(ta, r, s, slices));
    else if (bn == 128) PTRY(gemm_launch_bn<128>(ta, r, s, slices));
    else PTRY(gemm_launch_bn<256>(ta, r, s, slices));
    GemmArgs f = g;
    f.part = e.ws;
    const long long MN = (long long)g.M * g.N;
    const int blocks = (int)std::min<long long>((MN + 255) / 256, 16LL * std::max(g_num_sms, 1));
    sepso::splitk_reduce_kernel<<<blocks, 256, 0, s>>>(f, slices);
    PCUDA(cudaGetLastError());
    *launches = 2;
    return SEPSO_OK;
  }
  g.CbT = e.CbT;
  g.ldct = e.ldct;
  g.colpart = e.colsum ? e.ws : nullptr;
  PTRY(gemm_launch(g, s, tile_n));
  *launches = 1;
  if (e.colsum) {
    sepso::colsum_kernel<<<(g.N + 31) / 32, dim3(32, 8), 0, s>>>(e.ws, (g.M + 31) / 32, g.N, g.N, e.colsum);
    PCUDA(cudaGetLastError());
    *launches = 2;
  }
  return SEPSO_OK;
}

struct PriorLayout {
  size_t prm, m, v, grad, wb, w1p, w2t, w3t, X, Y, P, scirc, scoff, spts, swp, idx, x, xT, h1, h1T, h2, h2T, y, t, dyf,
      dyb, dyT, dh2b, dh2T, dh1T, kpart, cpart, cpart2, loss, status, total;
};

struct Dims {
  int K, Kp, O, O8, H1, H2, B, g;  // Kp: feature row pitch, a multiple of 64 (128-byte rows)
  long long P;
  long long off[6];
};

bool make_dims(const sepso_prior_config* c, Dims* d) {
  if (!c || c->T < 1 || c->T > 64 || c->grid < 8 || c->grid > 256 || c->hidden1 < 8 || (c->hidden1 & 7) ||
      c->hidden2 < 8 || (c->hidden2 & 7) || c->max_batch < 8 || (c->max_batch & 7) || c->max_batch > 65536 ||
      c->capacity < 1 || c->max_circles < 0 || c->max_circles > 8192 || !(c->map_w > 0) || !(c->map_h > 0) ||
      !(c->lr > 0) || !(c->beta1 >= 0 && c->beta1 < 1) || !(c->beta2 >= 0 && c->beta2 < 1) || !(c->eps > 0))
    return false;
  d->g = c->grid;
  d->K = round8(c->grid * c->grid + 4);
  d->Kp = (d->K + 63) / 64 * 64;
  d->O = 2 * c->T;
  d->O8 = round8(d->O);
  d->H1 = c->hidden1;
  d->H2 = c->hidden2;
  d->B = c->max_batch;
  d->off[0] = 0;
  d->off[1] = d->off[0] + (long long)d->H1 * d->K;
  d->off[2] = d->off[1] + d->H1;
  d->off[3] = d->off[2] + (long long)d->H2 * d->H1;
  d->off[4] = d->off[3] + d->H2;
  d->off[5] = d->off[4] + (long long)d->O * d->H2;
  d->P = d->off[5] + d->O;
  return (long long)c->capacity * d->Kp < (1ll << 40) && (long long)d->H1 * d->Kp < (1ll << 31);
}

PriorLayout layout(const sepso_prior_config* c, const Dims& d) {
  PriorLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = al256(off);
    const size_t o = off;
    off += std::max<size_t>(bytes, 16);
    return o;
  };
  const size_t P = (size_t)d.P, B = (size_t)d.B, K = (size_t)d.K, O = (size_t)d.O;
  const size_t H1 = (size_t)d.H1, H2 = (size_t)d.H2, cap = (size_t)c->capacity;
  L.prm = take(P * 4);
  L.m = take(P * 4);
  L.v = take(P * 4);
  L.grad = take(P * 4);
  L.wb = take(P * 2);
  L.w1p = take(H1 * (size_t)d.Kp * 2);
  L.w2t = take(H1 * H2 * 2);
  L.w3t = take(H2 * d.O8 * 2);
  L.X = take(cap * (size_t)d.Kp * 2);
  L.Y = take(cap * O * 4);
  L.P = take(cap * 16);
  L.scirc = take(B * (size_t)std::max(c->max_circles, 1) * 16);
  L.scoff = take((B + 1) * 4);
  L.spts = take(B * 16);
  L.swp = take(B * O * 4);
  L.idx = take(B * 4);
  L.x = take(B * (size_t)d.Kp * 2);
  L.xT = take(K * B * 2);
  L.h1 = take(B * H1 * 2);
  L.h1T = take(H1 * B * 2);
  L.h2 = take(B * H2 * 2);
  L.h2T = take(H2 * B * 2);
  L.y = take(B * O * 4);
  L.t = take(B * O * 4);
  L.dyf = take(B * O * 4);
  L.dyb = take(B * d.O8 * 2);
  L.dyT = take(O * B * 2);
  L.dh2b = take(B * H2 * 2);
  L.dh2T = take(H2 * B * 2);
  L.dh1T = take(H1 * B * 2);
  L.kpart = take((size_t)kMaxSlices * std::max(O * H2, H2 * H1) * 4);  // K-split partial products
  L.cpart = take((B + 31) / 32 * std::max(std::max(H1, H2), O) * 4);    // column sums per 32-row slab
  L.cpart2 = take((B + 31) / 32 * O * 4);                                // the same for dY, on the side stream
  L.loss = take((size_t)kLossRing * 4);
  L.status = take(4);
  L.total = al256(off);
  return L;
}

}  // namespace

struct sepso_prior_ctx {
  sepso_prior_config c{};
  Dims d{};
  PriorLayout L{};
  cudaStream_t stream = nullptr;
  // The backward pass forks the weight gradients that do not feed the next
  // product onto a second stream and joins it before Adam.
  cudaStream_t side = nullptr;
  cudaEvent_t ev_dy = nullptr, ev_dh2 = nullptr, ev_join = nullptr;
  ~sepso_prior_ctx() {
    if (ev_dy) cudaEventDestroy(ev_dy);
    if (ev_dh2) cudaEventDestroy(ev_dh2);
    if (ev_join) cudaEventDestroy(ev_join);
    if (side) cudaStreamDestroy(side);
  }
  char* ws = nullptr;
  int64_t step = 0;      // Adam steps taken
  int64_t launches = 0;
  int loss_head = 0;     // next slot of the loss ring
  struct Pending {
    float* host;
    int n, slot;
  };
  std::vector<Pending> pending;
  template <class T>
  T* at(size_t o) const { return reinterpret_cast<T*>(ws + o); }
};

namespace {

int gemm(sepso_prior_ctx* h, const bf16* A, const bf16* B, int M, int N, int K, int lda, int ldb, const float* bias,
         int relu, const bf16* mask, int ldm, float* Cf, int ldcf, bf16* Cb, int ldcb,
         const GemmExtra& e = GemmExtra(), int tile_n = 0, cudaStream_t st = nullptr) {
  GemmArgs g{};
  g.A = A;
  g.B = B;
  g.M = M;
  g.N = N;
  g.K = K;
  g.lda = lda;
  g.ldb = ldb;
  g.alpha = 1.0f;
  g.bias = bias;
  g.relu = relu;
  g.mask = mask;
  g.ldm = ldm;
  g.Cf = Cf;
  g.ldcf = ldcf;
  g.Cb = Cb;
  g.ldcb = ldcb;
  g.status = h->at<int>(h->L.status);
  int n = 0;
  const int r = gemm_run(g, e, st ? st : h->stream, tile_n, &n);
  h->launches += n;
  return r;
}

// db[j] = sum over the B rows of D[.][j]: sums over 32-row blocks (into part), then
// over the blocks.
int colsum(sepso_prior_ctx* h, const float* D, int B, int N, int ld, float* db, float* part, cudaStream_t st) {
  const int nb = (B + 31) / 32;
  sepso::colsum_part_kernel<<<dim3((N + 31) / 32, nb), dim3(32, 8), 0, st>>>(D, B, N, ld, part);
  PCUDA(cudaGetLastError());
  sepso::colsum_kernel<<<(N + 31) / 32, dim3(32, 8), 0, st>>>(part, nb, N, N, db);
  h->launches += 2;
  PCUDA(cudaGetLastError());
  return SEPSO_OK;
}

// Forward pass of n <= B rows x (row pitch Kp): h1, h2 (BF16), y (FP32); for
// training also the transposed copies h1T, h2T (n columns) the weight gradients read.
int forward(sepso_prior_ctx* h, const bf16* x, int n, bool train) {
  const Dims& d = h->d;
  const float* prm = h->at<float>(h->L.prm);
  const bf16* wb = h->at<bf16>(h->L.wb);
  bf16* h1 = h->at<bf16>(h->L.h1);
  bf16* h2 = h->at<bf16>(h->L.h2);
  GemmExtra e1, e2;
  if (train) {
    e1.CbT = h->at<bf16>(h->L.h1T);
    e1.ldct = n;
    e2.CbT = h->at<bf16>(h->L.h2T);
    e2.ldct = n;
  }
  PTRY(gemm(h, x, h->at<bf16>(h->L.w1p), n, d.H1, d.K, d.Kp, d.Kp, prm + d.off[1], 1, nullptr, 0, nullptr, 0, h1,
            d.H1, e1));
  PTRY(gemm(h, h1, wb + d.off[2], n, d.H2, d.H1, d.H1, d.H1, prm + d.off[3], 1, nullptr, 0, nullptr, 0, h2, d.H2, e2));
  PTRY(gemm(h, h2, wb + d.off[4], n, d.O, d.H2, d.H2, d.H2, prm + d.off[5], 0, nullptr, 0, h->at<float>(h->L.y), d.O,
            nullptr, 0));
  return SEPSO_OK;
}

// Backward pass after forward(x, n, true) with targets in t: gradient into grad,
// the loss added to loss[slot].  n is a multiple of 8 (the K of the weight GEMMs).
// The ReLU-masked products write their BF16 output transposed (the next weight
// gradient's operand) and their column sums (the bias gradient) from the epilogue;
// the weight gradients with few output tiles split K.
int backward(sepso_prior_ctx* h, int n, int slot) {
  const Dims& d = h->d;
  float* grad = h->at<float>(h->L.grad);
  bf16 *h1 = h->at<bf16>(h->L.h1), *h2 = h->at<bf16>(h->L.h2);
  bf16 *dyb = h->at<bf16>(h->L.dyb), *dyT = h->at<bf16>(h->L.dyT);
  bf16 *h2T = h->at<bf16>(h->L.h2T), *h1T = h->at<bf16>(h->L.h1T), *xT = h->at<bf16>(h->L.xT);
  bf16 *dh2b = h->at<bf16>(h->L.dh2b), *dh2T = h->at<bf16>(h->L.dh2T), *dh1T = h->at<bf16>(h->L.dh1T);
  float* dyf = h->at<float>(h->L.dyf);
  const int tot = n * d.O8;
  sepso::loss_grad_kernel<<<(tot + 255) / 256, 256, 0, h->stream>>>(h->at<float>(h->L.y), h->at<float>(h->L.t), n, d.O,
                                                                    dyf, dyb, d.O8, dyT, h->at<float>(h->L.loss) + slot);
  ++h->launches;
  PCUDA(cudaGetLastError());
  GemmExtra kw;  // weight gradients: K split over the partial-product scratch
  kw.ws = h->at<float>(h->L.kpart);
  kw.ws_bytes = (size_t)kMaxSlices * std::max(d.O * d.H2, d.H2 * d.H1) * 4;
  GemmExtra mk;  // masked products: transposed output and column sums
  mk.ws = h->at<float>(h->L.cpart);
  mk.ws_bytes = (size_t)((d.B + 31) / 32) * std::max(std::max(d.H1, d.H2), d.O) * 4;
  mk.ldct = n;
  // The side stream takes gb3, gW3 (after dY) and gW2 (after dh2): products no
  // later product reads; the main stream carries dh2 -> dh1 -> gW1.  The side
  // stream has its own column-sum scratch; both split-K products are on it.
  cudaStream_t side = h->side;
  PCUDA(cudaEventRecord(h->ev_dy, h->stream));
  PCUDA(cudaStreamWaitEvent(side, h->ev_dy, 0));
  // layer 3: gb3 = colsum dY, gW3 = dY^T h2 (side); dh2 = (dY W3) * [h2 > 0] (+ dh2T,
  // gb2 = colsum dh2) (main)
  PTRY(colsum(h, dyf, n, d.O, d.O, grad + d.off[5], h->at<float>(h->L.cpart2), side));
  kw.ksplit = auto_ksplit(d.O, d.H2, n, 64);
  PTRY(gemm(h, dyT, h2T, d.O, d.H2, n, n, n, nullptr, 0, nullptr, 0, grad + d.off[4], d.H2, nullptr, 0, kw, -64,
            side));
  mk.CbT = dh2T;
  mk.colsum = grad + d.off[3];
  PTRY(gemm(h, dyb, h->at<bf16>(h->L.w3t), n, d.H2, d.O8, d.O8, d.O8, nullptr, 0, h2, d.H2, nullptr, 0, dh2b, d.H2,
            mk));
  PCUDA(cudaEventRecord(h->ev_dh2, h->stream));
  PCUDA(cudaStreamWaitEvent(side, h->ev_dh2, 0));
  // layer 2: gW2 = dh2^T h1 (side); dh1 = (dh2 W2) * [h1 > 0] (only dh1T, gb1 =
  // colsum dh1) (main)
  kw.ksplit = auto_ksplit(d.H2, d.H1, n, 128);
  PTRY(gemm(h, dh2T, h1T, d.H2, d.H1, n, n, n, nullptr, 0, nullptr, 0, grad + d.off[2], d.H1, nullptr, 0, kw, -128,
            side));
  mk.CbT = dh1T;
  mk.colsum = grad + d.off[1];
  PTRY(gemm(h, dh2b, h->at<bf16>(h->L.w2t), n, d.H1, d.H2, d.H2, d.H2, nullptr, 0, h1, d.H1, nullptr, 0, nullptr, 0,
            mk));
  // layer 1: gW1 = dh1^T x (main), then join the side stream
  PTRY(gemm(h, dh1T, xT, d.H1, d.K, n, n, n, nullptr, 0, nullptr, 0, grad + d.off[0], d.K, nullptr, 0));
  PCUDA(cudaEventRecord(h->ev_join, side));
  PCUDA(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
  return SEPSO_OK;
}

// The BF16 weight copies the products read: W1 at pitch Kp, W2 transposed (H1 x
// H2), W3 transposed (H2 x O8; columns O .. O8-1 stay zero from the workspace clear).
sepso::BfMirrors mirrors(sepso_prior_ctx* h) {
  const Dims& d = h->d;
  sepso::BfMirrors mr;
  mr.w1p = h->at<bf16>(h->L.w1p);
  mr.h1 = d.H1;
  mr.k = d.K;
  mr.ldp = d.Kp;
  mr.w2t = h->at<bf16>(h->L.w2t);
  mr.off2 = d.off[2];
  mr.h2 = d.H2;
  mr.w3t = h->at<bf16>(h->L.w3t);
  mr.off4 = d.off[4];
  mr.o = d.O;
  mr.o8 = d.O8;
  return mr;
}

// Training rows: x (n x K), its transpose xT (K x n) and the targets t.
int gather(sepso_prior_ctx* h, const int* idx, int first, int n, cudaStream_t st = nullptr) {
  const Dims& d = h->d;
  const dim3 grid((d.K + 127) / 128, (n + 63) / 64);
  sepso::gather_t_kernel<<<grid, 256, 0, st ? st : h->stream>>>(idx, first, n, d.K, d.Kp, h->at<bf16>(h->L.X), h->at<float>(h->L.Y),
                                                      d.O, h->at<bf16>(h->L.x), h->at<bf16>(h->L.xT),
                                                      h->at<float>(h->L.t));
  ++h->launches;
  PCUDA(cudaGetLastError());
  return SEPSO_OK;
}

int adam_step(sepso_prior_ctx* h) {
  const Dims& d = h->d;
  ++h->step;
  const double c1 = 1.0 - std::pow((double)h->c.beta1, (double)h->step);
  const double c2 = 1.0 - std::pow((double)h->c.beta2, (double)h->step);
  const long long blocks = std::min<long long>((d.P + 255) / 256, 152LL * 16);
  sepso::adam_kernel<<<(unsigned)blocks, 256, 0, h->stream>>>(
      h->at<float>(h->L.prm), h->at<float>(h->L.m), h->at<float>(h->L.v), h->at<float>(h->L.grad), h->at<bf16>(h->L.wb),
      d.P, h->c.lr, h->c.beta1, h->c.beta2, h->c.eps, (float)c1, (float)c2, mirrors(h));
  ++h->launches;
  PCUDA(cudaGetLastError());
  return SEPSO_OK;
}

int check_rows(const sepso_prior_ctx* h, int first, int n) {
  if (first < 0 || n < 0 || (long long)first + n > h->c.capacity)
    return pfail(SEPSO_EINVAL, "rows [%d, %d) outside the dataset's %d rows", first, first + n, h->c.capacity);
  return SEPSO_OK;
}

int read_status(sepso_prior_ctx* h) {
  int st = 0;
  PCUDA(cudaMemcpyAsync(&st, h->at<int>(h->L.status), 4, cudaMemcpyDeviceToHost, h->stream));
  PCUDA(cudaStreamSynchronize(h->stream));
  if (st != 0) {
    PCUDA(cudaMemsetAsync(h->at<int>(h->L.status), 0, 4, h->stream));
    PCUDA(cudaStreamSynchronize(h->stream));
    return pfail(st, "device-side error %d (tensor-core wait timed out)", st);
  }
  return SEPSO_OK;
}

int flush_pending(sepso_prior_ctx* h) {
  for (const auto& p : h->pending) {
    const int a = std::min(p.n, kLossRing - p.slot);
    PCUDA(cudaMemcpyAsync(p.host, h->at<float>(h->L.loss) + p.slot, (size_t)a * 4, cudaMemcpyDeviceToHost, h->stream));
    if (a < p.n)
      PCUDA(cudaMemcpyAsync(p.host + a, h->at<float>(h->L.loss), (size_t)(p.n - a) * 4, cudaMemcpyDeviceToHost,
                            h->stream));
  }
  h->pending.clear();
  PCUDA(cudaStreamSynchronize(h->stream));
  return SEPSO_OK;
}

}  // namespace

extern "C" {

int sepso_prior_workspace_size(const sepso_prior_config* cfg, size_t* bytes) {
  Dims d;
  if (!bytes || !make_dims(cfg, &d)) return pfail(SEPSO_EINVAL, "bad prior configuration");
  *bytes = layout(cfg, d).total;
  return SEPSO_OK;
}

int sepso_prior_create(const sepso_prior_config* cfg, void* d_workspace, size_t bytes, void* stream,
                       sepso_prior_handle* out) {
  if (!out) return pfail(SEPSO_EINVAL, "out is NULL");
  *out = nullptr;
  Dims d;
  if (!make_dims(cfg, &d)) return pfail(SEPSO_EINVAL, "bad prior configuration");
  const PriorLayout L = layout(cfg, d);
  if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255u))
    return pfail(SEPSO_ENOSPC, "workspace must be non-NULL and 256-byte aligned");
  if (bytes < L.total) return pfail(SEPSO_ENOSPC, "workspace of %zu bytes, need %zu", bytes, L.total);
  sepso_prior_ctx* h = new (std::nothrow) sepso_prior_ctx;
  if (!h) return pfail(SEPSO_ENOMEM, "host allocation failed");
  h->c = *cfg;
  h->d = d;
  h->L = L;
  h->ws = static_cast<char*>(d_workspace);
  h->stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_dy, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_dh2, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->ws, 0, L.total, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    delete h;
    return pfail(SEPSO_ECUDA, "workspace clear: %s", cudaGetErrorString(e));
  }
  *out = h;
  return SEPSO_OK;
}

void sepso_prior_destroy(sepso_prior_handle h) { delete h; }

int64_t sepso_prior_num_params(sepso_prior_handle h) { return h ? h->d.P : -1; }

int sepso_prior_set_params(sepso_prior_handle h, const float* params) {
  if (!h || !params) return pfail(SEPSO_EINVAL, "NULL argument");
  const size_t n = (size_t)h->d.P * 4;
  PCUDA(cudaMemcpyAsync(h->at<float>(h->L.prm), params, n, cudaMemcpyHostToDevice, h->stream));
  PCUDA(cudaMemsetAsync(h->at<float>(h->L.m), 0, n, h->stream));
  PCUDA(cudaMemsetAsync(h->at<float>(h->L.v), 0, n, h->stream));
  const long long blocks = std::min<long long>((h->d.P + 255) / 256, 152LL * 16);
  sepso::to_bf16_kernel<<<(unsigned)blocks, 256, 0, h->stream>>>(h->at<float>(h->L.prm), h->at<bf16>(h->L.wb), h->d.P,
                                                                  mirrors(h));
  ++h->launches;
  PCUDA(cudaGetLastError());
  h->step = 0;
  PCUDA(cudaStreamSynchronize(h->stream));
  return SEPSO_OK;
}

int sepso_prior_get_params(sepso_prior_handle h, float* params) {
  if (!h || !params) return pfail(SEPSO_EINVAL, "NULL argument");
  PCUDA(cudaMemcpyAsync(params, h->at<float>(h->L.prm), (size_t)h->d.P * 4, cudaMemcpyDeviceToHost, h->stream));
  PCUDA(cudaStreamSynchronize(h->stream));
  return SEPSO_OK;
}

int sepso_prior_add_scenes(sepso_prior_handle h, int32_t first, int32_t n, const float* points, const int32_t* counts,
                           const float* circles, const float* waypoints) {
  if (!h || (n > 0 && (!points || !counts))) return pfail(SEPSO_EINVAL, "NULL argument");
  PTRY(check_rows(h, first, n));
  const Dims& d = h->d;
  long long total = 0;
  for (int i = 0; i < n; ++i) {
    if (counts[i] < 0 || counts[i] > h->c.max_circles)
      return pfail(SEPSO_EINVAL, "scene %d: %d circles (max %d)", i, counts[i], h->c.max_circles);
    total += counts[i];
  }
  if (total > 0 && !circles) return pfail(SEPSO_EINVAL, "circles is NULL");
  std::vector<float4> hc;
  std::vector<int> off;
  long long c0 = 0;
  for (int s0 = 0; s0 < n; s0 += d.B) {
    const int m = std::min(d.B, n - s0);
    hc.clear();
    off.assign(1, 0);
    for (int i = 0; i < m; ++i) {
      for (int o = 0; o < counts[s0 + i]; ++o) {
        const float* q = circles + 3 * (c0 + o);
        hc.push_back(make_float4(q[0], q[1], q[2], 0.0f));
      }
      c0 += counts[s0 + i];
      off.push_back((int)hc.size());
    }
    if (!hc.empty())
      PCUDA(cudaMemcpyAsync(h->at<float4>(h->L.scirc), hc.data(), hc.size() * 16, cudaMemcpyHostToDevice, h->stream));
    PCUDA(cudaMemcpyAsync(h->at<int>(h->L.scoff), off.data(), off.size() * 4, cudaMemcpyHostToDevice, h->stream));
    PCUDA(cudaMemcpyAsync(h->at<float>(h->L.P) + 4LL * (first + s0), points + 4LL * s0, (size_t)m * 16,
                          cudaMemcpyHostToDevice, h->stream));
    if (waypoints)
      PCUDA(cudaMemcpyAsync(h->at<float>(h->L.swp), waypoints + (long long)s0 * d.O, (size_t)m * d.O * 4,
                            cudaMemcpyHostToDevice, h->stream));
    sepso::RasterArgs a;
    a.n = m;
    a.grid = d.g;
    a.K = d.K;
    a.ldx = d.Kp;
    a.T = h->c.T;
    a.O_max = h->c.max_circles;
    a.W = h->c.map_w;
    a.H = h->c.map_h;
    a.circ = h->at<float4>(h->L.scirc);
    a.coff = h->at<int>(h->L.scoff);
    a.pts = h->at<float>(h->L.P) + 4LL * (first + s0);
    a.wp = waypoints ? h->at<float>(h->L.swp) : nullptr;
    a.X = h->at<bf16>(h->L.X) + (long long)(first + s0) * d.Kp;
    a.Y = h->at<float>(h->L.Y) + (long long)(first + s0) * d.O;
    const size_t smem = (size_t)d.g * d.g;  // occupancy bytes
    if (smem > 48 * 1024)
      PCUDA(cudaFuncSetAttribute(sepso::raster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    sepso::raster_kernel<<<m, 256, smem, h->stream>>>(a);
    ++h->launches;
    PCUDA(cudaGetLastError());
    // the staging buffers are reused by the next chunk
    PCUDA(cudaStreamSynchronize(h->stream));
  }
  return SEPSO_OK;
}

int sepso_prior_set_labels(sepso_prior_handle h, int32_t first, int32_t n, const float* d_waypoints, int32_t ld) {
  if (!h || (n > 0 && !d_waypoints)) return pfail(SEPSO_EINVAL, "NULL argument");
  PTRY(check_rows(h, first, n));
  if (ld < h->d.O) return pfail(SEPSO_EINVAL, "ld %d below 2T = %d", ld, h->d.O);
  if (n == 0) return SEPSO_OK;
  const int tot = n * h->d.O;
  sepso::label_kernel<<<(tot + 255) / 256, 256, 0, h->stream>>>(d_waypoints, ld, n, h->c.T,
                                                                 h->at<float>(h->L.P) + 4LL * first, h->c.map_w,
                                                                 h->c.map_h, h->at<float>(h->L.Y) + (long long)first * h->d.O);
  ++h->launches;
  PCUDA(cudaGetLastError());
  return SEPSO_OK;
}

int sepso_prior_get_rows(sepso_prior_handle h, int32_t first, int32_t n, float* features, float* labels) {
  if (!h) return pfail(SEPSO_EINVAL, "NULL handle");
  PTRY(check_rows(h, first, n));
  const Dims& d = h->d;
  if (features && n > 0) {
    std::vector<uint16_t> raw((size_t)n * d.K);
    PCUDA(cudaMemcpy2DAsync(raw.data(), (size_t)d.K * 2, h->at<bf16>(h->L.X) + (long long)first * d.Kp,
                            (size_t)d.Kp * 2, (size_t)d.K * 2, (size_t)n, cudaMemcpyDeviceToHost, h->stream));
    PCUDA(cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i < raw.size(); ++i) {
      const uint32_t bits = (uint32_t)raw[i] << 16;
      std::memcpy(&features[i], &bits, 4);
    }
  }
  if (labels && n > 0) {
    PCUDA(cudaMemcpyAsync(labels, h->at<float>(h->L.Y) + (long long)first * d.O, (size_t)n * d.O * 4,
                          cudaMemcpyDeviceToHost, h->stream));
    PCUDA(cudaStreamSynchronize(h->stream));
  }
  return SEPSO_OK;
}

int sepso_prior_forward(sepso_prior_handle h, int32_t first, int32_t n, float* y) {
  if (!h || !y) return pfail(SEPSO_EINVAL, "NULL argument");
  PTRY(check_rows(h, first, n));
  const Dims& d = h->d;
  for (int s0 = 0; s0 < n; s0 += d.B) {
    const int m = std::min(d.B, n - s0);
    PTRY(forward(h, h->at<bf16>(h->L.X) + (long long)(first + s0) * d.Kp, m, false));
    PCUDA(cudaMemcpyAsync(y + (long long)s0 * d.O, h->at<float>(h->L.y), (size_t)m * d.O * 4, cudaMemcpyDeviceToHost,
                          h->stream));
    PTRY(read_status(h));
  }
  return SEPSO_OK;
}

int sepso_prior_grad(sepso_prior_handle h, int32_t first, int32_t n, float* grad, float* loss) {
  if (!h || !grad) return pfail(SEPSO_EINVAL, "NULL argument");
  PTRY(check_rows(h, first, n));
  if (n < 8 || (n & 7) || n > h->d.B) return pfail(SEPSO_EINVAL, "rows %d: need a multiple of 8 up to %d", n, h->d.B);
  const int slot = h->loss_head;
  h->loss_head = (h->loss_head + 1) % kLossRing;
  PCUDA(cudaMemsetAsync(h->at<float>(h->L.loss) + slot, 0, 4, h->stream));
  PTRY(gather(h, nullptr, first, n));
  PTRY(forward(h, h->at<bf16>(h->L.x), n, true));
  PTRY(backward(h, n, slot));
  PCUDA(cudaMemcpyAsync(grad, h->at<float>(h->L.grad), (size_t)h->d.P * 4, cudaMemcpyDeviceToHost, h->stream));
  if (loss) PCUDA(cudaMemcpyAsync(loss, h->at<float>(h->L.loss) + slot, 4, cudaMemcpyDeviceToHost, h->stream));
  return read_status(h);
}

int sepso_prior_train(sepso_prior_handle h, int32_t n_rows, int32_t first, int32_t steps, int32_t batch,
                      uint64_t seed, float* losses) {
  if (!h) return pfail(SEPSO_EINVAL, "NULL handle");
  if (batch < 8 || (batch & 7) || batch > h->d.B)
    return pfail(SEPSO_EINVAL, "batch %d: need a multiple of 8 up to %d", batch, h->d.B);
  if (steps < 0 || (losses && steps > kLossRing)) return pfail(SEPSO_EINVAL, "bad step count %d", steps);
  if (first >= 0) {
    PTRY(check_rows(h, first, batch));
  } else if (n_rows < 1 || n_rows > h->c.capacity) {
    return pfail(SEPSO_EINVAL, "n_rows %d outside [1, %d]", n_rows, h->c.capacity);
  }
  const int slot0 = h->loss_head;
  // A step's minibatch (row indices drawn with the Adam step count as the counter)
  // gathered on stream st.
  auto stage_rows = [&](cudaStream_t st, int64_t counter) -> int {
    if (first >= 0) return gather(h, nullptr, first, batch, st);
    sepso::sample_kernel<<<(batch + 255) / 256, 256, 0, st>>>(h->at<int>(h->L.idx), batch, n_rows, (uint32_t)seed,
                                                              (uint32_t)(seed >> 32), (uint32_t)counter);
    ++h->launches;
    PCUDA(cudaGetLastError());
    return gather(h, h->at<int>(h->L.idx), 0, batch, st);
  };
  if (steps > 0) PTRY(stage_rows(h->stream, h->step));
  for (int s = 0; s < steps; ++s) {
    const int slot = h->loss_head;
    h->loss_head = (h->loss_head + 1) % kLossRing;
    PCUDA(cudaMemsetAsync(h->at<float>(h->L.loss) + slot, 0, 4, h->stream));
    PTRY(forward(h, h->at<bf16>(h->L.x), batch, true));
    PTRY(backward(h, batch, slot));
    // The next minibatch is gathered on the side stream while Adam runs: both
    // stream through memory, and the rows are free once the backward pass is done.
    const bool more = s + 1 < steps;
    if (more) {
      PCUDA(cudaEventRecord(h->ev_dy, h->stream));
      PCUDA(cudaStreamWaitEvent(h->side, h->ev_dy, 0));
      PTRY(stage_rows(h->side, h->step + 1));
      PCUDA(cudaEventRecord(h->ev_join, h->side));
    }
    PTRY(adam_step(h));
    if (more) PCUDA(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
  }
  if (losses && steps > 0) {
    h->pending.push_back({losses, steps, slot0});
    PTRY(flush_pending(h));
  }
  return SEPSO_OK;
}

int sepso_prior_infer(sepso_prior_handle h, int32_t first, int32_t n, float* d_out, int32_t ld) {
  if (!h || (n > 0 && !d_out)) return pfail(SEPSO_EINVAL, "NULL argument");
  PTRY(check_rows(h, first, n));
  const Dims& d = h->d;
  if (ld < d.O) return pfail(SEPSO_EINVAL, "ld %d below 2T = %d", ld, d.O);
  for (int s0 = 0; s0 < n; s0 += d.B) {
    const int m = std::min(d.B, n - s0);
    PTRY(forward(h, h->at<bf16>(h->L.X) + (long long)(first + s0) * d.Kp, m, false));
    const int tot = m * d.O;
    sepso::decode_kernel<<<(tot + 255) / 256, 256, 0, h->stream>>>(h->at<float>(h->L.y), m, h->c.T,
                                                                    h->at<float>(h->L.P) + 4LL * (first + s0),
                                                                    h->c.map_w, h->c.map_h,
                                                                    d_out + (long long)s0 * ld, ld);
    ++h->launches;
    PCUDA(cudaGetLastError());
  }
  return SEPSO_OK;
}

int sepso_prior_sync(sepso_prior_handle h) {
  if (!h) return pfail(SEPSO_EINVAL, "NULL handle");
  PTRY(flush_pending(h));
  return read_status(h);
}

int64_t sepso_prior_launch_count(sepso_prior_handle h) { return h ? h->launches : -1; }

const char* sepso_prior_last_error(void) { return g_prior_error.c_str(); }

int sepso_gemm_bf16(const void* A, const void* B, int32_t M, int32_t N, int32_t K, int32_t lda, int32_t ldb,
                    float alpha, const float* bias, int32_t relu, const void* mask, int32_t ldm, float* Cf,
                    int32_t ldcf, void* Cb, int32_t ldcb, int32_t tile_n, void* stream) {
  GemmArgs g{};
  g.A = static_cast<const bf16*>(A);
  g.B = static_cast<const bf16*>(B);
  g.M = M;
  g.N = N;
  g.K = K;
  g.lda = lda;
  g.ldb = ldb;
  g.alpha = alpha;
  g.bias = bias;
  g.relu = relu;
  g.mask = static_cast<const bf16*>(mask);
  g.ldm = ldm;
  g.Cf = Cf;
  g.ldcf = ldcf;
  g.Cb = static_cast<bf16*>(Cb);
  g.ldcb = ldcb;
  PTRY(gemm_check(g, tile_n));  // before any CUDA call
  void* st = nullptr;
  PCUDA(cudaGetSymbolAddress(&st, g_gemm_status));
  g.status = static_cast<int*>(st);
  return gemm_launch(g, static_cast<cudaStream_t>(stream), tile_n);
}

int sepso_gemm_bf16_ex_workspace(int32_t M, int32_t N, int32_t ksplit, int32_t colsum, size_t* bytes) {
  if (!bytes || M < 1 || N < 1 || ksplit < 0) return pfail(SEPSO_EINVAL, "bad workspace query");
  *bytes = gemm_ws_bytes(M, N, std::max(ksplit, 1), colsum != 0);
  return SEPSO_OK;
}

int sepso_gemm_bf16_ex(const void* A, const void* B, int32_t M, int32_t N, int32_t K, int32_t lda, int32_t ldb,
                       float alpha, const float* bias, int32_t relu, const void* mask, int32_t ldm, float* Cf,
                       int32_t ldcf, void* Cb, int32_t ldcb, const sepso_gemm_extra* extra, int32_t tile_n,
                       void* stream) {
  GemmArgs g{};
  g.A = static_cast<const bf16*>(A);
  g.B = static_cast<const bf16*>(B);
  g.M = M;
  g.N = N;
  g.K = K;
  g.lda = lda;
  g.ldb = ldb;
  g.alpha = alpha;
  g.bias = bias;
  g.relu = relu;
  g.mask = static_cast<const bf16*>(mask);
  g.ldm = ldm;
  g.Cf = Cf;
  g.ldcf = ldcf;
  g.Cb = static_cast<bf16*>(Cb);
  g.ldcb = ldcb;
  GemmExtra e;
  if (extra) {
    e.CbT = static_cast<bf16*>(extra->Ct);
    e.ldct = extra->ldct;
    e.colsum = extra->colsum;
    e.ksplit = std::max(extra->ksplit, 1);
    e.ws = static_cast<float*>(extra->workspace);
    e.ws_bytes = extra->workspace_bytes;
  }
  if (extra && extra->ksplit < 0) return pfail(SEPSO_EINVAL, "gemm: K split %d", extra->ksplit);
  PTRY(gemm_run_check(g, e, tile_n));  // before any CUDA call
  void* st = nullptr;
  PCUDA(cudaGetSymbolAddress(&st, g_gemm_status));
  g.status = static_cast<int*>(st);
  int n = 0;
  return gemm_run(g, e, static_cast<cudaStream_t>(stream), tile_n, &n);
}

int sepso_gemm_bf16_sync(void* stream) {
  PCUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  int st = 0;
  PCUDA(cudaMemcpyFromSymbol(&st, g_gemm_status, 4));
  if (st != 0) {
    const int zero = 0;
    PCUDA(cudaMemcpyToSymbol(g_gemm_status, &zero, 4));
    return pfail(st, "device-side error %d (tensor-core wait timed out)", st);
  }
  return SEPSO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The prior as the request server uses it (declared in sepso_internal.h).
// ---------------------------------------------------------------------------
namespace sepso {

int prior_shape(const sepso_prior_ctx* h, int* T, int* max_circles, int* capacity, float* map_w, float* map_h,
                cudaStream_t* stream) {
  if (!h) return pfail(SEPSO_EINVAL, "NULL prior handle");
  if (T) *T = h->c.T;
  if (max_circles) *max_circles = h->c.max_circles;
  if (capacity) *capacity = h->c.capacity;
  if (map_w) *map_w = h->c.map_w;
  if (map_h) *map_h = h->c.map_h;
  if (stream) *stream = h->stream;
  return SEPSO_OK;
}

cudaStream_t prior_swap_stream(sepso_prior_ctx* h, cudaStream_t s) {
  const cudaStream_t old = h->stream;
  h->stream = s;
  return old;
}

int prior_propose_device(sepso_prior_ctx* h, int first, int n, const float4* circ, const int* coff, const float* pts,
                         float* out, int ld) {
  if (!h || (n > 0 && (!circ || !coff || !pts || !out))) return pfail(SEPSO_EINVAL, "NULL argument");
  if (n == 0) return SEPSO_OK;
  PTRY(check_rows(h, first, n));
  const Dims& d = h->d;
  PCUDA(cudaMemcpyAsync(h->at<float>(h->L.P) + 4LL * first, pts, (size_t)n * 16, cudaMemcpyDeviceToDevice,
                        h->stream));
  const size_t smem = (size_t)d.g * d.g;  // occupancy bytes
  if (smem > 48 * 1024)
    PCUDA(cudaFuncSetAttribute(sepso::raster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  for (int s0 = 0; s0 < n; s0 += d.B) {
    const int m = std::min(d.B, n - s0);
    sepso::RasterArgs a;
    a.n = m;
    a.grid = d.g;
    a.K = d.K;
    a.ldx = d.Kp;
    a.T = h->c.T;
    a.O_max = h->c.max_circles;
    a.W = h->c.map_w;
    a.H = h->c.map_h;
    a.circ = circ;        // the offsets are absolute into circ
    a.coff = coff + s0;
    a.pts = h->at<float>(h->L.P) + 4LL * (first + s0);
    a.wp = nullptr;
    a.X = h->at<bf16>(h->L.X) + (long long)(first + s0) * d.Kp;
    a.Y = nullptr;
    sepso::raster_kernel<<<m, 256, smem, h->stream>>>(a);
    ++h->launches;
    PCUDA(cudaGetLastError());
  }
  return sepso_prior_infer(h, first, n, out, ld);
}

}  // namespace sepso
