// sepso_device.cuh -- device-side building blocks of the SEPSO planner (sm_103a).
//
// Internal to libsepso: the workspace records, Philox4x32-10, the bulk-copy /
// mbarrier helpers, the group-best exchange (atomic-min keys and a monotone
// barrier counter) and the segment-circle test.
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
  int32_t fin_launches;  // cluster-form launches finished by this run (end-of-launch barrier target)
  long long plans_total;  // planning cycles finished by this run
  long long iters_total;  // iterations of Algorithm 1 run by this run
};

// Group bests without moving rows through a reduction: every particle whose
// Pbest is below its group's best folds its key into the group's word with a
// 64-bit atomic min.  Fitness values are non-negative, so their IEEE bit
// patterns order like the values; the key is (fitness bits << 32) | (particle
// index n << 12) | min(Q, kQSat), and the minimum key is the lowest-index
// particle of minimum fitness (indices are unique, so Q never decides).  Words
// are triple-buffered by iteration (read during iteration k, reset by CTA 0
// during k + 1, reused at k + 3).  Such a particle also writes its row and Q to
// its slot, where readers fetch the winner's.
constexpr unsigned long long kKeyEmpty = ~0ull;

constexpr uint32_t kQSat = 0xfffu;  // Q field saturates here (exact Q then read from the slot)

__device__ __forceinline__ unsigned long long best_key(float fit, uint32_t idx, uint32_t q) {
  return ((unsigned long long)__float_as_uint(fit) << 32) | ((unsigned long long)(idx & 0xfffffu) << 12) |
         (unsigned long long)(q < kQSat ? q : kQSat);
}
__device__ __forceinline__ float key_fit(unsigned long long key) { return __uint_as_float((uint32_t)(key >> 32)); }
__device__ __forceinline__ int key_idx(unsigned long long key) { return (int)((uint32_t)key >> 12); }
__device__ __forceinline__ int key_q(unsigned long long key) { return (int)((uint32_t)key & kQSat); }

// Per-run barrier counter on its own 128-byte line.  It only grows: the CTAs of
// a run add 1 each per iteration, so the barrier of the run's gk-th iteration
// (counted across launches) is complete when the counter reaches C * gk.
struct __align__(128) RunCounter {
  unsigned int count;
  unsigned int fin;   // cluster form: one arrival per group at the end of each launch
  unsigned int pad[30];
};

enum : int { kModePlan = 0, kModeStep = 1 };

enum : uint32_t {
  kStreamVel = 0, kStreamInitX = 1, kStreamInitV = 2, kStreamPI = 3,
  kStreamPrior = 4, kStreamHInitX = 5, kStreamHInitV = 6, kStreamHVel = 7, kStreamSample = 8
};

// Everything one launch of the swarm kernel needs (passed by value).
struct SwarmParams {
  int T, D, G, N, M;          // M = G * N
  int R;                      // runs in this launch
  int cpg, C, ppc;            // CTAs per group, CTAs per run, particles per CTA
  int split;                  // circle chunks per (particle, segment) item
  int lp;                     // lanes per particle (power of two, <= 32)
  int items;                  // 1: fitness as (particle, segment, chunk) items over the CTA
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
  const float4* circ;         // Omax x (cx, cy, r, 4 r^2)
  const float4* pairs;        // the same circles as pair blocks (pair_block_f4(O) float4)
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
  unsigned long long* gword;  // R x 3 x G group best keys
  RunCounter* counter;        // R
  float* crows;               // R x 2 x M x (D + 4): candidate row, its Q, padding
  unsigned long long* grec;   // R x kRecDepth x G group records (cluster form)
  int cta_grid;               // CTAs per run of the grid-wide form (its barrier counts C * iterations)
  int poly;                   // obstacles are polygon edges (circ holds O edges as float4), not circles
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
// Acquire/release accesses for the candidate exchange between the CTAs of a run
// (co-resident: cooperative launch).  Waits on them are bounded by kWaitLimitNs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void red_min_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.min.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// After relaxed loads that observed a writer's stores: an acquire.  Before a
// writer's relaxed stores: a release of everything it wrote earlier.
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Polls a monotone counter until it reaches target (wrap-around safe) or the
// limit passes; false on a timeout.  The caller adds the acquire fence.
__device__ __forceinline__ bool counter_wait_bounded(const unsigned int* ctr, unsigned int target,
                                                     unsigned long long limit_ns) {
  unsigned int v = ld_relaxed_u32(ctr);
  if ((int)(v - target) >= 0) return true;
  const unsigned long long t0 = global_ns();
  do {
    if (global_ns() - t0 > limit_ns) return false;
    v = ld_relaxed_u32(ctr);
  } while ((int)(v - target) < 0);
  return true;
}



constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

// ---------------------------------------------------------------------------
// Cluster form of the exchange: the CTAs of one group form a thread-block
// cluster and trade their candidates through distributed shared memory; the
// groups of a run trade only (Gfit, Q) records through global memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Address of the same shared-memory location in CTA `rank` of this cluster.
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_peer_u64(uint32_t addr, unsigned long long v) {
  asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}
__device__ __forceinline__ void st_peer_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void st_peer_f32(uint32_t addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

__device__ __forceinline__ void st_peer_v4(uint32_t addr, float a, float b, float c, float d) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

// The cluster barrier for a warp that made no remote store this round: its arrival
// needs no release order (the wait still acquires the other CTAs' stores).
__device__ __forceinline__ void cluster_barrier_relaxed_arrive() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Every thread of every CTA of the cluster: the release orders this thread's
// earlier shared-memory stores (local and remote) before the arrival, the acquire
// makes the other CTAs' stores visible after the wait.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// A group's record of one iteration, one 64-bit word (single-copy atomic, so it
// needs no fence): Gfit bits << 32 | Q << 12 | tag.  Q < 2^20 always holds
// ((T + 1) * O <= 65 * 8192); the tag (iteration mod 4095) + 1 is never 0, so a
// zeroed ring holds no valid record.
constexpr int kRecDepth = 4;  // ring slots per group; groups of a run are at most one iteration apart
__device__ __forceinline__ uint32_t rec_tag(unsigned long long gk) { return (uint32_t)(gk % 4095ull) + 1u; }
__device__ __forceinline__ unsigned long long make_rec(float fit, int q, unsigned long long gk) {
  return ((unsigned long long)__float_as_uint(fit) << 32) | ((unsigned long long)((uint32_t)q & 0xfffffu) << 12) |
         rec_tag(gk);
}
__device__ __forceinline__ float rec_fit(unsigned long long v) { return __uint_as_float((uint32_t)(v >> 32)); }
__device__ __forceinline__ int rec_q(unsigned long long v) { return (int)(((uint32_t)v >> 12) & 0xfffffu); }
__device__ __forceinline__ uint32_t rec_tag_of(unsigned long long v) { return (uint32_t)v & 0xfffu; }

// ---------------------------------------------------------------------------
// Segment-circle test (Eq. penalty's Q for circular obstacles).
// The segment [a, b] is described by its midpoint m, unit direction u, normal
// n = (-u_y, u_x) and half-length h.  For a circle centre c, along = (c - m).u
// and perp = (c - m).n; the squared distance to the segment is
// max(|along| - h, 0)^2 + perp^2; the pair collides when it is below r^2 (open
// disk).  Everything is kept on the FP32 FMA pipe: with a = |along| - h,
// t = a + |a| = 2 max(a, 0) exactly, the normal is pre-scaled by 2 (exact) so
// that p2 = 2 perp, and s = 4r^2 - p2^2 - t^2 = 4 (r^2 - dist^2) is formed by two
// FMAs; hit = saturate(s * 2^100) is exactly 1 for s > 0 and 0 otherwise (a
// positive s is never below 2^-100 here), and hits accumulate in FP32 (exact
// below 2^24).  Circles are stored as (cx, cy, r, 4 r^2).
// ---------------------------------------------------------------------------
struct SegFrame {
  float ux, uy, mu, nx2, ny2, mn2, h;
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
  f.nx2 = -2.0f * uy;
  f.ny2 = 2.0f * ux;
  f.mn2 = fmaf(mx, f.nx2, my * f.ny2);
  f.h = 0.5f * len;
  *len_out = len;
  return f;
}

__device__ __forceinline__ float seg_hits(const SegFrame& f, const float4* __restrict__ circ, int o0, int o1) {
  float hits = 0.0f;
#pragma unroll 8
  for (int o = o0; o < o1; ++o) {
    const float4 c = circ[o];
    const float al = fmaf(c.x, f.ux, fmaf(c.y, f.uy, -f.mu));
    const float p2 = fmaf(c.x, f.nx2, fmaf(c.y, f.ny2, -f.mn2));
    const float a = fabsf(al) - f.h;
    const float t = a + fabsf(a);
    const float s = fmaf(-t, t, fmaf(-p2, p2, c.w));
    hits += __saturatef(s * 0x1p100f);
  }
  return hits;
}

// Length and Q of one particle by a lane group of lp lanes (a power of two <= 32,
// aligned within the warp): lanes take (segment, circle chunk) items of the row x
// (D = 2T floats in shared memory), then the group sums both with a fixed
// shuffle tree, so every lane of the group ends with the same deterministic
// values.  All 32 lanes of the warp must call this (live = false for lanes
// without a particle).
__device__ __forceinline__ void group_fitness(const float* x, bool live, int lp, int T, int split, int O,
                                              float sx, float sy, float tx, float ty, const float4* circ,
                                              float* len_out, int* q_out) {
  const int lsub = (threadIdx.x & 31) & (lp - 1);
  const int items = (T + 1) * split;
  const int chunk = (O + split - 1) / split;
  float len = 0.0f, hits = 0.0f;
  if (live) {
    // segment fastest: neighbouring lanes read the same circle (broadcast)
    for (int it = lsub; it < items; it += lp) {
      const int sg = it % (T + 1);
      const int c = it / (T + 1);
      const float ax = (sg == 0) ? sx : x[sg - 1];
      const float ay = (sg == 0) ? sy : x[T + sg - 1];
      const float bx = (sg == T) ? tx : x[sg];
      const float by = (sg == T) ? ty : x[T + sg];
      float l;
      const SegFrame f = seg_frame(ax, ay, bx, by, &l);
      if (c == 0) len += l;
      hits += seg_hits(f, circ, c * chunk, min(O, c * chunk + chunk));
    }
  }
  for (int off = lp >> 1; off > 0; off >>= 1) {
    len += __shfl_xor_sync(0xffffffffu, len, off);
    hits += __shfl_xor_sync(0xffffffffu, hits, off);
  }
  *len_out = len;
  *q_out = (int)hits;
}

// ---------------------------------------------------------------------------
// Packed form of the same test: two circles per FP32x2 instruction.
// Circles are stored in pairs: pair k holds circles 2k and 2k + 1 as
// cxy[k] = (cx_2k, cx_2k+1, cy_2k, cy_2k+1) and nr2[k] = (-r_2k^2, -r_2k+1^2), the
// K = ceil(O / 2) cxy records first, then the K nr2 records, the block padded to
// whole float4s (pair_block_f4 float4s); an odd O is completed by a circle of
// radius 0 at the origin (it never counts).  With m = max(|along| - h, 0) and the
// unscaled perpendicular p, a pair collides when m^2 + p^2 - r^2 < 0, formed as
// fma(m, m, fma(p, p, -r^2)): this is exactly -1/4 of the scaled form's s above
// (scaling by powers of two commutes with rounding), never -0, so the sign bit
// gives the same decision; hits accumulate as integers.
// ---------------------------------------------------------------------------
__host__ __device__ inline int circle_pairs(int O) { return (O + 1) >> 1; }
__host__ __device__ inline int pair_block_f4(int O) {
  const int K = circle_pairs(O);
  return K + ((K + 1) >> 1);
}

__device__ __forceinline__ unsigned long long pack2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack2(unsigned long long v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long fadd2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long fmul2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// The frame of segment [a, b] as scalars: unit direction, normal n = (-u_y, u_x),
// the negated projections of the midpoint on both, and the half-length.
struct FrameScalars {
  float ux, uy, nmu, nx, ny, nmn, h;
};

__device__ __forceinline__ FrameScalars frame_scalars(float ax, float ay, float bx, float by, float* len_out) {
  const float dx = bx - ax, dy = by - ay;
  const float len = sqrtf(fmaf(dx, dx, dy * dy));
  float ux = 1.0f, uy = 0.0f;
  if (len > 0.0f) {
    const float inv = 1.0f / len;
    ux = dx * inv;
    uy = dy * inv;
  }
  const float mx = 0.5f * (ax + bx), my = 0.5f * (ay + by);
  const float mu = fmaf(mx, ux, my * uy);
  const float nx = -uy, ny = ux;
  const float mn = fmaf(mx, nx, my * ny);
  FrameScalars f;
  f.ux = ux;
  f.uy = uy;
  f.nmu = -mu;
  f.nx = nx;
  f.ny = ny;
  f.nmn = -mn;
  f.h = 0.5f * len;
  *len_out = len;
  return f;
}

struct PairFrame {
  unsigned long long ux, uy, nmu, nx, ny, nmn;  // each value in both halves
  float h;
};

__device__ __forceinline__ PairFrame pair_frame(float ax, float ay, float bx, float by, float* len_out) {
  const FrameScalars s = frame_scalars(ax, ay, bx, by, len_out);
  PairFrame f;
  f.ux = pack2(s.ux, s.ux);
  f.uy = pack2(s.uy, s.uy);
  f.nmu = pack2(s.nmu, s.nmu);
  f.nx = pack2(s.nx, s.nx);
  f.ny = pack2(s.ny, s.ny);
  f.nmn = pack2(s.nmn, s.nmn);
  f.h = s.h;
  return f;
}

// Hits of one circle pair (cx, cy, -r^2 packed per circle) against a packed frame,
// the arithmetic of pair_hits.
__device__ __forceinline__ int pair_test(unsigned long long CX, unsigned long long CY, unsigned long long W,
                                         unsigned long long UX, unsigned long long UY, unsigned long long NMU,
                                         unsigned long long NX, unsigned long long NY, unsigned long long NMN,
                                         float h) {
  const unsigned long long AL = ffma2(CX, UX, ffma2(CY, UY, NMU));
  const unsigned long long P = ffma2(CX, NX, ffma2(CY, NY, NMN));
  float al0, al1;
  unpack2(AL, al0, al1);
  const float m0 = fmaxf(fabsf(al0) - h, 0.0f), m1 = fmaxf(fabsf(al1) - h, 0.0f);
  const unsigned long long S = ffma2(pack2(m0, m1), pack2(m0, m1), ffma2(P, P, W));
  float s0, s1;
  unpack2(S, s0, s1);
  return (int)(__float_as_uint(s0) >> 31) + (int)(__float_as_uint(s1) >> 31);
}

__device__ __forceinline__ int pair_hits(const PairFrame& f, const float4* __restrict__ cxy,
                                         const float2* __restrict__ nr2, int k0, int k1) {
  int hits = 0;
#pragma unroll 4
  for (int k = k0; k < k1; ++k) {
    const float4 c = cxy[k];
    const float2 w = nr2[k];
    hits += pair_test(pack2(c.x, c.y), pack2(c.z, c.w), pack2(w.x, w.y), f.ux, f.uy, f.nmu, f.nx, f.ny, f.nmn, f.h);
  }
  return hits;
}

// group_fitness on circle pairs (K of them; split chunks of pairs per segment).
__device__ __forceinline__ void group_fitness_pairs(const float* x, bool live, int lp, int T, int split, int K,
                                                    float sx, float sy, float tx, float ty,
                                                    const float4* cxy, const float2* nr2, float* len_out,
                                                    int* q_out) {
  const int lsub = (threadIdx.x & 31) & (lp - 1);
  const int items = (T + 1) * split;
  const int chunk = (K + split - 1) / split;
  float len = 0.0f;
  int hits = 0;
  if (live) {
    for (int it = lsub; it < items; it += lp) {
      const int sg = it % (T + 1);
      const int c = it / (T + 1);
      const float ax = (sg == 0) ? sx : x[sg - 1];
      const float ay = (sg == 0) ? sy : x[T + sg - 1];
      const float bx = (sg == T) ? tx : x[sg];
      const float by = (sg == T) ? ty : x[T + sg];
      float l;
      const PairFrame f = pair_frame(ax, ay, bx, by, &l);
      if (c == 0) len += l;
      hits += pair_hits(f, cxy, nr2, c * chunk, min(K, c * chunk + chunk));
    }
  }
  for (int off = lp >> 1; off > 0; off >>= 1) {
    len += __shfl_xor_sync(0xffffffffu, len, off);
    hits += __shfl_xor_sync(0xffffffffu, hits, off);
  }
  *len_out = len;
  *q_out = hits;
}

// ---------------------------------------------------------------------------
// Polygon obstacles (Sec. 3.3.1's map model: bounding boxes or outlines given by
// their edges).  Q counts the (path segment, edge) pairs that cross properly: the
// endpoints of each segment strictly on opposite sides of the other's line (four
// orientation products), so touching and collinear contacts do not count.  Edges
// are float4 (x0, y0, x1, y1).  The segment is a -> a + u, the edge d0 -> d0 + v.
// With w = d0 - a, the four orientations are o1 = u x w, o2 = u x (w + v) = o1 +
// u x v, o3 = v x (-w) and o4 = v x (u - w) = o3 - u x v: two products of w, one
// of u x v and two additions (12 operations where the four written out take 18).
// Each orientation is formed from differences of nearby points, so its rounding
// error stays of the order of the written-out form's.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int edge_crosses(float ax, float ay, float ux, float uy, const float4 d) {
  const float vx = d.z - d.x, vy = d.w - d.y;
  const float wx = d.x - ax, wy = d.y - ay;
  const float o1 = ux * wy - uy * wx;
  const float o3 = vy * wx - vx * wy;
  const float c = ux * vy - uy * vx;
  const float o2 = o1 + c, o4 = o3 - c;
  return (o1 * o2 < 0.0f) && (o3 * o4 < 0.0f);
}

// Edge pairs: the edges two by two as float4 (x0a, x0b, y0a, y0b) and float4 (vxa,
// vxb, -vya, -vyb), v = d1 - d0, an odd count padded with a zero edge (v = 0: o3 o4
// vanishes, no hit); edge_pair_f4(E) float4s.  Packed FP32x2 instructions then test
// a segment against two edges at once with edge_crosses' orientations: w = d0 - a,
// o1 = u x w, c = u x v, o2 = o1 + c, and the negated pair m3 = -o3 = v x w, m4 =
// -o4 = m3 + c, whose product is o3 o4.
__host__ __device__ inline int edge_pair_f4(int E) { return 2 * ((E + 1) / 2); }
__host__ __device__ inline void edge_pair(const float4 a, const float4 b, float4* out) {
  out[0] = make_float4(a.x, b.x, a.y, b.y);
  out[1] = make_float4(a.z - a.x, b.z - b.x, -(a.w - a.y), -(b.w - b.y));
}
// E edges (x0, y0, x1, y1 each) from host memory into edge_pair_f4(E) float4s.
inline void pack_edge_pairs(const float* e, int E, float4* out) {
  for (int k = 0; 2 * k < E; ++k) {
    const float* a = e + 8 * k;
    const float4 fa = make_float4(a[0], a[1], a[2], a[3]);
    const float4 fb = 2 * k + 1 < E ? make_float4(a[4], a[5], a[6], a[7]) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    edge_pair(fa, fb, out + 2 * k);
  }
}
// Crossings of segment a -> a + u with edge pairs k0 .. k1 - 1.
__device__ __forceinline__ int edge_pair_hits(float ax, float ay, float ux, float uy,
                                              const ulonglong2* __restrict__ ep, int k0, int k1) {
  const unsigned long long NAX = pack2(-ax, -ax), NAY = pack2(-ay, -ay), UX = pack2(ux, ux);
  const unsigned long long NUX = pack2(-ux, -ux), NUY = pack2(-uy, -uy);
  int hits = 0;
#pragma unroll 2
  for (int k = k0; k < k1; ++k) {
    const ulonglong2 d0 = ep[2 * k], v = ep[2 * k + 1];
    const unsigned long long WX = fadd2(d0.x, NAX), WY = fadd2(d0.y, NAY);
    const unsigned long long O1 = ffma2(UX, WY, fmul2(NUY, WX));
    const unsigned long long C = ffma2(NUX, v.y, fmul2(NUY, v.x));
    const unsigned long long M3 = ffma2(v.x, WY, fmul2(v.y, WX));
    const unsigned long long P12 = fmul2(O1, fadd2(O1, C)), P34 = fmul2(M3, fadd2(M3, C));
    float a12, b12, a34, b34;
    unpack2(P12, a12, b12);
    unpack2(P34, a34, b34);
    hits += (a12 < 0.0f && a34 < 0.0f) + (b12 < 0.0f && b34 < 0.0f);
  }
  return hits;
}

// The same for two segments (a -> a + u, a' -> a' + u') per edge pair read: two
// independent chains per loaded record.
__device__ __forceinline__ int edge_pair_hits2(float ax, float ay, float ux, float uy, float ax2, float ay2, float ux2,
                                               float uy2, const ulonglong2* __restrict__ ep, int K) {
  const unsigned long long NAX = pack2(-ax, -ax), NAY = pack2(-ay, -ay), UX = pack2(ux, ux);
  const unsigned long long NUX = pack2(-ux, -ux), NUY = pack2(-uy, -uy);
  const unsigned long long NAX2 = pack2(-ax2, -ax2), NAY2 = pack2(-ay2, -ay2), UX2 = pack2(ux2, ux2);
  const unsigned long long NUX2 = pack2(-ux2, -ux2), NUY2 = pack2(-uy2, -uy2);
  int hits = 0;
  for (int k = 0; k < K; ++k) {
    const ulonglong2 d0 = ep[2 * k], v = ep[2 * k + 1];
    const unsigned long long WX = fadd2(d0.x, NAX), WY = fadd2(d0.y, NAY);
    const unsigned long long WX2 = fadd2(d0.x, NAX2), WY2 = fadd2(d0.y, NAY2);
    const unsigned long long O1 = ffma2(UX, WY, fmul2(NUY, WX));
    const unsigned long long O1b = ffma2(UX2, WY2, fmul2(NUY2, WX2));
    const unsigned long long C = ffma2(NUX, v.y, fmul2(NUY, v.x));
    const unsigned long long Cb = ffma2(NUX2, v.y, fmul2(NUY2, v.x));
    const unsigned long long M3 = ffma2(v.x, WY, fmul2(v.y, WX));
    const unsigned long long M3b = ffma2(v.x, WY2, fmul2(v.y, WX2));
    const unsigned long long P12 = fmul2(O1, fadd2(O1, C)), P34 = fmul2(M3, fadd2(M3, C));
    const unsigned long long P12b = fmul2(O1b, fadd2(O1b, Cb)), P34b = fmul2(M3b, fadd2(M3b, Cb));
    float a12, b12, a34, b34, c12, d12, c34, d34;
    unpack2(P12, a12, b12);
    unpack2(P34, a34, b34);
    unpack2(P12b, c12, d12);
    unpack2(P34b, c34, d34);
    hits += (a12 < 0.0f && a34 < 0.0f) + (b12 < 0.0f && b34 < 0.0f) + (c12 < 0.0f && c34 < 0.0f) +
            (d12 < 0.0f && d34 < 0.0f);
  }
  return hits;
}

__device__ __forceinline__ int edge_hits(float ax, float ay, float bx, float by, const float4* __restrict__ edges,
                                         int e0, int e1) {
  const float ux = bx - ax, uy = by - ay;
  int hits = 0;
#pragma unroll 4
  for (int e = e0; e < e1; ++e) hits += edge_crosses(ax, ay, ux, uy, edges[e]);
  return hits;
}

// Length and Q of one particle among polygon edges by a lane group (as
// group_fitness_pairs): lanes take (segment, edge chunk) items, the group sums
// both with a fixed shuffle tree.
__device__ __forceinline__ void group_fitness_edges(const float* x, bool live, int lp, int T, int split, int E,
                                                    float sx, float sy, float tx, float ty, const float4* edges,
                                                    float* len_out, int* q_out) {
  const int lsub = (threadIdx.x & 31) & (lp - 1);
  const int items = (T + 1) * split;
  const int chunk = (E + split - 1) / split;
  float len = 0.0f;
  int hits = 0;
  if (live) {
    for (int it = lsub; it < items; it += lp) {
      const int sg = it % (T + 1);
      const int c = it / (T + 1);
      const float ax = (sg == 0) ? sx : x[sg - 1];
      const float ay = (sg == 0) ? sy : x[T + sg - 1];
      const float bx = (sg == T) ? tx : x[sg];
      const float by = (sg == T) ? ty : x[T + sg];
      if (c == 0) {
        const float dx = bx - ax, dy = by - ay;
        len += sqrtf(fmaf(dx, dx, dy * dy));
      }
      hits += edge_hits(ax, ay, bx, by, edges, c * chunk, min(E, c * chunk + chunk));
    }
  }
  for (int off = lp >> 1; off > 0; off >>= 1) {
    len += __shfl_xor_sync(0xffffffffu, len, off);
    hits += __shfl_xor_sync(0xffffffffu, hits, off);
  }
  *len_out = len;
  *q_out = hits;
}

// The same with the edges as edge pairs (edge_pair_f4(E) float4s): lanes take
// (segment, edge-pair chunk) items.
__device__ __forceinline__ void group_fitness_edge_pairs(const float* x, bool live, int lp, int T, int split, int E,
                                                         float sx, float sy, float tx, float ty, const float4* edges,
                                                         float* len_out, int* q_out) {
  const int lsub = (threadIdx.x & 31) & (lp - 1);
  const int items = (T + 1) * split;
  const int K = (E + 1) / 2;
  const int chunk = (K + split - 1) / split;
  const ulonglong2* ep = reinterpret_cast<const ulonglong2*>(edges);
  float len = 0.0f;
  int hits = 0;
  if (live) {
    for (int it = lsub; it < items; it += lp) {
      const int sg = it % (T + 1);
      const int c = it / (T + 1);
      const float ax = (sg == 0) ? sx : x[sg - 1];
      const float ay = (sg == 0) ? sy : x[T + sg - 1];
      const float bx = (sg == T) ? tx : x[sg];
      const float by = (sg == T) ? ty : x[T + sg];
      const float ux = bx - ax, uy = by - ay;
      if (c == 0) len += sqrtf(fmaf(ux, ux, uy * uy));
      hits += edge_pair_hits(ax, ay, ux, uy, ep, c * chunk, min(K, c * chunk + chunk));
    }
  }
  for (int off = lp >> 1; off > 0; off >>= 1) {
    len += __shfl_xor_sync(0xffffffffu, len, off);
    hits += __shfl_xor_sync(0xffffffffu, hits, off);
  }
  *len_out = len;
  *q_out = hits;
}

// Q and per-segment lengths of nl particles among polygon edges, as (particle,
// segment, edge chunk) items over the block (as fitness_items_pairs); sQ must be
// zero on entry.
__device__ __forceinline__ void fitness_items_edges(const float* sX, int nl, int T, int D, float sx, float sy,
                                                    float tx, float ty, const float4* edges, int E, int split,
                                                    int* sQ, float* seg_len) {
  const int nseg = T + 1;
  const int chunk = (E + split - 1) / split;
  const int per_c = nl * nseg;
  const int items = per_c * split;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int c = it / per_c;
    const int r = it - c * per_c;
    const int i = r / nseg;
    const int s = r - i * nseg;
    const float* x = sX + i * D;
    const float ax = (s == 0) ? sx : x[s - 1];
    const float ay = (s == 0) ? sy : x[T + s - 1];
    const float bx = (s == T) ? tx : x[s];
    const float by = (s == T) ? ty : x[T + s];
    const int hits = edge_hits(ax, ay, bx, by, edges, c * chunk, min(E, c * chunk + chunk));
    if (hits) atomicAdd(&sQ[i], hits);
    if (c == 0) {
      const float dx = bx - ax, dy = by - ay;
      seg_len[i * nseg + s] = sqrtf(fmaf(dx, dx, dy * dy));
    }
  }
}

// A particle's path length from its per-segment lengths seg[0 .. nseg), summed by a
// whole warp in a fixed order: lane l adds segments l, l + 32, l + 64 in turn, then
// a butterfly over the lanes.  Every lane returns the same value.
__device__ __forceinline__ float warp_len_sum(const float* seg, int nseg, int lane) {
  float v = 0.0f;
  for (int s = lane; s < nseg; s += 32) v += seg[s];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// float4s of a swarm kernel's obstacle area: the circle-pair blocks, or the edges.
__host__ __device__ inline int obstacle_f4(int Omax, int poly) {
  const int o = Omax > 0 ? Omax : 1;
  return poly ? o : pair_block_f4(o);
}

// Circle chunks per segment for a warp (32 lanes) evaluating one particle of T
// waypoints against O circles: the split (1..8) that minimises the per-lane work
// rounds * (chunk + setup), so that the warp's rounds are nearly full.
__host__ __device__ inline int warp_split(int T, int O) {
  int best = 1;
  long long best_cost = -1;
  for (int sp = 1; sp <= 8; ++sp) {
    const long long rounds = ((long long)(T + 1) * sp + 31) / 32;
    const long long chunk = (O + sp - 1) / sp;
    const long long cost = rounds * (chunk + 4);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = sp;
    }
  }
  return best;
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
    const int hits = (int)seg_hits(f, circ, o0, o1);
    if (hits) atomicAdd(&sQ[i], hits);
    if (c == 0) seg_len[i * nseg + s] = len;
  }
}

// Q and per-segment lengths of nl particles (rows in shared memory) against circle
// pairs, as (particle, segment, circle chunk) items spread over all threads of the
// block, chunk-major so that the lanes of a warp read the same circle pair (a
// broadcast).  Q accumulates with shared-memory integer atomics (exact); lengths
// land in seg_len[i * (T+1) + s].  sQ must be zero on entry.
__device__ __forceinline__ void fitness_items_pairs(const float* sX, int nl, int T, int D, float sx, float sy,
                                                    float tx, float ty, const float4* cxy, const float2* nr2,
                                                    int K, int split, int* sQ, float* seg_len) {
  const int nseg = T + 1;
  const int chunk = (K + split - 1) / split;
  const int per_c = nl * nseg;
  const int items = per_c * split;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int c = it / per_c;
    const int r = it - c * per_c;
    const int i = r / nseg;
    const int s = r - i * nseg;
    const float* x = sX + i * D;
    const float ax = (s == 0) ? sx : x[s - 1];
    const float ay = (s == 0) ? sy : x[T + s - 1];
    const float bx = (s == T) ? tx : x[s];
    const float by = (s == T) ? ty : x[T + s];
    float len;
    const PairFrame f = pair_frame(ax, ay, bx, by, &len);
    const int hits = pair_hits(f, cxy, nr2, c * chunk, min(K, c * chunk + chunk));
    if (hits) atomicAdd(&sQ[i], hits);
    if (c == 0) seg_len[i * nseg + s] = len;
  }
}

}  // namespace sepso
