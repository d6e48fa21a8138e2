// sepso_device.cuh -- device-side building blocks of the SEPSO planner (sm_103a).
//
// Internal to libsepso: the workspace records, Philox4x32-10, the bulk-copy /
// mbarrier helpers, the bounded inter-CTA barrier and the segment-circle test.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sepso.h"

namespace sepso {

// ---------------------------------------------------------------------------
// Workspace records
// ---------------------------------------------------------------------------

// Per-run control block: iteration counter, bests' scalars, warm-start state.
struct RunCtl {
  int32_t k;          // iteration counter of Algorithm 1
  int32_t cycle;      // planning cycles completed (Philox counter word 2, low 24 bits)
  int32_t has_prev;   // a previous best path exists (enables PI)
  int32_t win_n;      // AT window fill
  int32_t win_head;   // AT window ring head
  int32_t stall;      // AT stall counter
  int32_t TQ;         // collision count of Tbest
  int32_t status;     // first device-side error of this run
  float Tfit;         // F(Tbest)
  float prev_lfv;     // LFV of the previous iteration (AT stall mode)
  uint32_t run_id;    // Philox counter word 3
  int32_t pad;
  long long plans_total;  // planning cycles finished by this run
  long long iters_total;  // iterations of Algorithm 1 run by this run
};

// Candidate published by one CTA each iteration: its best Pbest (lowest index on ties).
struct __align__(16) CandMeta {
  float fit;
  int32_t idx;  // particle index n within the group (INT32_MAX when the CTA is empty)
  int32_t q;    // collision count of that Pbest
  int32_t pad;
};

// Inter-CTA barrier of one run (own 128-byte line).
struct __align__(128) RunBarrier {
  unsigned int count;
  unsigned int gen;
  unsigned int pad[30];
};

enum : int { kModePlan = 0, kModeStep = 1 };

enum : uint32_t {
  kStreamVel = 0, kStreamInitX = 1, kStreamInitV = 2, kStreamPI = 3,
  kStreamHInitX = 5, kStreamHInitV = 6, kStreamHVel = 7
};

// Everything one launch of the swarm kernel needs (passed by value).
struct SwarmParams {
  int T, D, G, N, M;          // M = G * N
  int R;                      // runs in this launch
  int cpg, C, ppc;            // CTAs per group, CTAs per run, particles per CTA
  int split;                  // circle chunks per (particle, segment) item
  int O, Omax;                // obstacles now / capacity (shared-memory carve)
  float W, H, alpha;
  int beta, max_iters, at_mode, tw;
  float delta;
  int stall_iters;
  float stall_tol;
  int use_pi, n_pi;
  float pi_h;
  uint32_t key0, key1;
  int mode, step_iters;
  // device pointers
  const float4* circ;         // Omax x (cx, cy, r, r^2)
  const float* pts;           // start xy, target xy, start vel, target vel
  const float* hyper;         // R x G x 6
  float *X, *V, *P, *Pfit;    // R x M x D (X, V, P), R x M
  int32_t* PQ;                // R x M
  float *Gb, *Gfit;           // R x G x D, R x G
  int32_t* GQ;                // R x G
  float *Tb, *prevT, *res_wp; // R x D each
  RunCtl* ctl;                // R
  sepso_result* res;          // R
  double* win;                // R x tw
  CandMeta* cmeta;            // R x 2 x C
  float* crows;               // R x 2 x C x D
  RunBarrier* bar;            // R
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Counter layout: (c0, particle, stream << 24 | cycle, run).
__device__ __forceinline__ uint4 draw(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t particle,
                                      uint32_t stream, uint32_t cycle, uint32_t run) {
  return philox4x32_10(make_uint4(c0, particle, (stream << 24) | (cycle & 0x00ffffffu), run), k0, k1);
}

// Top 24 bits times 2^-24: exact in FP32, uniform on [0, 1).
__device__ __forceinline__ float u01(uint32_t x) { return (float)(x >> 8) * 5.9604644775390625e-08f; }

__device__ __forceinline__ float lane_of(uint4 v, int l) {
  const uint32_t w = (l == 0) ? v.x : (l == 1) ? v.y : (l == 2) ? v.z : v.w;
  return u01(w);
}

// ---------------------------------------------------------------------------
// Bulk copy (TMA engine, non-tensor) with mbarrier completion.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// dst (shared) and src (global) 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits with a time limit; false when the copy did not land in time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}

// ---------------------------------------------------------------------------
// Bounded barrier across the CTAs of one run (co-resident: cooperative launch).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

// Every CTA of the run calls this with the same n.  Returns false (in every
// thread of the CTA) when the wait gave up; the barrier is then unusable until
// the host re-zeroes it.
__device__ __forceinline__ bool run_barrier(RunBarrier* b, unsigned int n, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int g0 = ld_acquire(&b->gen);
    __threadfence();
    const unsigned int prev = atomicAdd(&b->count, 1u);
    if (prev == n - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      st_release(&b->gen, g0 + 1u);
    } else {
      unsigned int spins = 0;
      unsigned long long t0 = 0;
      while (ld_acquire(&b->gen) == g0) {
        if ((++spins & 255u) == 0u) {
          const unsigned long long t = global_ns();
          if (t0 == 0) t0 = t;
          else if (t - t0 > kWaitLimitNs) {
            ok = 0;
            break;
          }
        }
      }
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// ---------------------------------------------------------------------------
// Segment-circle test (Eq. penalty's Q for circular obstacles).
// The segment [a, b] is described by its midpoint m, unit direction u, normal
// n = (-u_y, u_x) and half-length h.  For a circle centre c, along = (c - m).u
// and perp = (c - m).n; the squared distance to the segment is
// max(|along| - h, 0)^2 + perp^2, compared with r^2 (strict: open disk).
// ---------------------------------------------------------------------------
struct SegFrame {
  float ux, uy, mu, mn, h;
};

__device__ __forceinline__ SegFrame seg_frame(float ax, float ay, float bx, float by, float* len_out) {
  const float dx = bx - ax, dy = by - ay;
  const float len = sqrtf(fmaf(dx, dx, dy * dy));
  float ux = 1.0f, uy = 0.0f;
  if (len > 0.0f) {
    const float inv = 1.0f / len;
    ux = dx * inv;
    uy = dy * inv;
  }
  const float mx = 0.5f * (ax + bx), my = 0.5f * (ay + by);
  SegFrame f;
  f.ux = ux;
  f.uy = uy;
  f.mu = fmaf(mx, ux, my * uy);
  f.mn = fmaf(my, ux, -(mx * uy));
  f.h = 0.5f * len;
  *len_out = len;
  return f;
}

__device__ __forceinline__ int seg_hits(const SegFrame& f, const float4* __restrict__ circ, int o0, int o1) {
  int hits = 0;
#pragma unroll 4
  for (int o = o0; o < o1; ++o) {
    const float4 c = circ[o];
    const float al = fmaf(c.x, f.ux, fmaf(c.y, f.uy, -f.mu));
    const float pe = fmaf(c.y, f.ux, fmaf(-c.x, f.uy, -f.mn));
    const float e = fmaxf(fabsf(al) - f.h, 0.0f);
    const float d2 = fmaf(e, e, pe * pe);
    hits += (d2 < c.w) ? 1 : 0;
  }
  return hits;
}

__device__ __forceinline__ float powi(float q, int beta) {
  float r = 1.0f;
  for (int i = 0; i < beta; ++i) r *= q;
  return r;
}

// Q and per-segment lengths of nl particles whose rows (D floats each) are in
// shared memory.  Items are (particle, segment, circle chunk); Q accumulates with
// shared-memory integer atomics (exact); lengths land in seg_len[i * (T+1) + s].
__device__ __forceinline__ void fitness_items(const float* sX, int nl, int T, int D, float sx, float sy,
                                              float tx, float ty, const float4* circ, int O, int split,
                                              int* sQ, float* seg_len) {
  const int nseg = T + 1;
  const int chunk = (O + split - 1) / split;
  const int items = nl * nseg * split;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int c = it % split;
    const int rest = it / split;
    const int s = rest % nseg;
    const int i = rest / nseg;
    const float* x = sX + i * D;
    const float ax = (s == 0) ? sx : x[s - 1];
    const float ay = (s == 0) ? sy : x[T + s - 1];
    const float bx = (s == T) ? tx : x[s];
    const float by = (s == T) ? ty : x[T + s];
    float len;
    const SegFrame f = seg_frame(ax, ay, bx, by, &len);
    const int o0 = c * chunk;
    const int o1 = min(O, o0 + chunk);
    const int hits = seg_hits(f, circ, o0, o1);
    if (hits) atomicAdd(&sQ[i], hits);
    if (c == 0) seg_len[i * nseg + s] = len;
  }
}

}  // namespace sepso
