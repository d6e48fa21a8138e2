// sepso_bf.cu -- DTPSO on the benchmark functions of Table BFs (BF1 Sphere, BF2
// Rosenbrock, BF3 Rastrigin, BF4 Griewank): the tensor-form iteration of Sec. 3.1 /
// Algorithm 1 with a closed-form objective over the box [lo, hi]^D.  Sized for the
// large-scale case of Sec. 4.1.2 (16K particles x 1K coordinates: 16M scalars per
// tensor, about 330 MB of HBM traffic per iteration) as well as the standard case of
// Sec. 4.1.1 (80 particles x 30 coordinates, many independent trials as runs).
//
// One launch per iteration; a CUDA graph holds a whole run.  Launch j (1-based):
//   1. (kUpdate) the velocity and position update of iteration j - 1 (Eqs.
//      TOF_omega, TOF_V with clipping to V_range, TOF_X with clipping to X_range),
//      from the bests of iteration j - 1;
//   2. (kEval) the fitness of the positions (iteration j) and the Pbest update,
//      and this launch's candidates for iteration j's Gbest.
// A run of K iterations is: init, launch 1 (kEval), launches 2..K (both), launch
// K + 1 (kUpdate only), so that the state after it is the state of Algorithm 1
// after K whole iterations (positions updated K times); a later step starts with
// a kEval-only launch.
// One warp owns one particle: its row of X, V and Pbest streams through once
// (float4), the new position row is kept in shared memory for the fitness, and an
// improved Pbest row is written from there.
//
// Bests cross the kernel boundary as 64-bit keys
//   ordered fitness (32) | priority (1) | particle (30) | Pbest parity (1),
// so that an atomicMin picks the lowest fitness, then the previous holder (priority
// 0: Eq. DPPSO's "strictly better" rule keeps the old best on a tie), then the
// lowest particle index -- the oracle's order.  A particle's Pbest row alternates
// between two buffers (its parity bit) each time it improves, so the row a key names
// is never overwritten in the launch that reads it: the holder of a best can only
// write the other parity, and it must improve again (and so replace itself as the
// holder) before it writes the first one again.  Keys of three consecutive
// iterations rotate (read j - 1, write j, clear j + 1); the Tbest holder is kept
// in two slots.  Rows of a loaded state live in an "external" table addressed by
// particle numbers >= M.
//
// Path objectives: 5 is a path among polygons (Sec. 3.3.1), 6 a path in three
// dimensions among spheres (the Conclusion's extension from 2D to 3D planning).
// Their rows are waypoint coordinates by axis ([x1..xT, y1..yT(, z1..zT)]), each
// axis with its own box, and a run may start with Priori Initialization (Sec.
// 3.3.3) around its previous best path; the planning cycle then enters every
// Philox counter, as in the planner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sepso.h"
#include "sepso_device.cuh"

namespace sepso {
namespace {

constexpr unsigned long long kEmpty = ~0ull;
constexpr int kUpdate = 1, kEval = 2;
constexpr int kUnroll = 4;
constexpr int kMaxD = 16384;
constexpr int kMaxRG = 4096;           // runs x groups: the CTA's key table
constexpr int kSmemTotal = 200 * 1024;  // shared-memory budget of the iteration kernel
constexpr int kMaxEdges = 4096;        // polygon edges held in shared memory
constexpr int kMaxSpheres = 4096;      // spheres held in shared memory

struct BfParams {
  int fn, D, Dp, G, N, M, R, K, hist_len;
  float lo, hi;
  // path objectives: coordinate j lies on axis (j >= half) + (j >= half2), x in
  // [lo, hi], y in [lo2, hi2], z in [lo3, hi3]; half = half2 = D for the benchmark
  // functions, half2 = D for objective 5
  int half, half2;
  float lo2, hi2, lo3, hi3, alpha;
  int beta, E;
  const float4* edges;        // objective 5: E polygon edges (x0, y0, x1, y1);
                              // objective 6: E spheres (cx, cy, cz, r)
  const float* pts;           // start, then target: 2 coordinates each (objective 5), 3 (objective 6)
  const int* warm;            // path objectives, device words: PI particles per group, PI
                              // half-width (float bits), planning cycle
  const float* prevT;         // R rows of Dp: each run's previous best path (the PI centre)
  // path objectives: Auto Truncation by stall counter (Sec. 3.3.4 with the stall
  // reading): a run stops after at_stall iterations without an improvement of its
  // Tbest fitness by more than stall_tol while its Tbest collides with nothing;
  // at_stall = 0: off
  int at_stall;
  float stall_tol;
  int* pq;                    // 2 x R*M: the collision count of each Pbest row, by parity
  int* at_state;              // 2 slots x R x {stall, previous Tbest fitness bits, stopped, stop iteration}
  uint32_t key0, key1, run_id;
  float* X;                   // R*M rows of Dp
  float* V;                   // R*M rows of Dp
  float* P;                   // 2 parities x R*M rows of Dp
  float* Pfit;                // R*M
  unsigned char* pcur;        // R*M: parity of the current Pbest row
  unsigned long long* keys;   // 3 x R*G
  unsigned long long* thold;  // 2 x R
  const float* hyper;         // R*G*6 (C1, C2, C3, w_init, w_end, V_limit)
  float* ext;                 // R x (G+1) rows of Dp: loaded Gbest rows, then Tbest
  float* hist;                // R x hist_len: Tbest fitness after each iteration
  float *Gb, *Gfit, *Tb, *Tfit;  // bests after the last launch (finish kernel)
};

// Order-preserving map of a float onto uint32 (any sign; NaN is never posted).
__device__ __forceinline__ uint32_t ord_of(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float float_of_ord(uint32_t o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}
__device__ __forceinline__ unsigned long long make_key(float fit, uint32_t prio, uint32_t idx, uint32_t par) {
  return ((unsigned long long)ord_of(fit) << 32) | ((unsigned long long)prio << 31) |
         ((unsigned long long)(idx & 0x3fffffffu) << 1) | (unsigned long long)(par & 1u);
}
__device__ __forceinline__ uint32_t key_idx(unsigned long long k) { return (uint32_t)(k >> 1) & 0x3fffffffu; }
__device__ __forceinline__ uint32_t key_par(unsigned long long k) { return (uint32_t)k & 1u; }

// The row a key names (null: no best yet, a zero row).
__device__ __forceinline__ const float* key_row(const BfParams& p, int r, unsigned long long k) {
  if (k == kEmpty) return nullptr;
  const uint32_t idx = key_idx(k);
  if ((int)idx < p.M)
    return p.P + ((size_t)key_par(k) * p.R * p.M + (size_t)r * p.M + idx) * p.Dp;
  return p.ext + ((size_t)r * (p.G + 1) + (idx - p.M)) * p.Dp;
}

// Tbest after an iteration: the best group key (lowest fitness, then lowest group)
// if strictly better than the previous holder, else the previous holder.
__device__ __forceinline__ unsigned long long resolve_T(const unsigned long long* gk, int G,
                                                        unsigned long long told) {
  unsigned long long best = kEmpty;
  for (int g = 0; g < G; ++g) {
    const unsigned long long k = gk[g];
    if (k != kEmpty && (best == kEmpty || (k >> 32) < (best >> 32))) best = k;
  }
  if (best != kEmpty && (told == kEmpty || (best >> 32) < (told >> 32))) return best;
  return told;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_prod(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Griewank's factor cos(x_i / sqrt(i)) for coordinate index i (0-based) as
// cos(pi y) with y = x / (pi sqrt(i + 1)): cospif reduces y exactly, and the scale
// takes one reciprocal square root and two products instead of a square root, a
// divide and cosf's argument reduction.
__device__ __forceinline__ float griewank_factor(float x, int i) {
  return cospif(x * (rsqrtf((float)(i + 1)) * 0.318309886183790672f));
}

// BF1..BF4 of one row (any address space), the whole warp; every lane gets the value.
//   Sphere      sum x_i^2
//   Rosenbrock  sum_{i<D} 100 (x_{i+1} - x_i^2)^2 + (x_i - 1)^2
//   Rastrigin   10 D + sum x_i^2 - 10 cos(2 pi x_i)
//   Griewank    1 + sum x_i^2 / 4000 - prod cos(x_i / sqrt(i)),  i = 1..D
template <int FN>
__device__ __forceinline__ float bf_row(const float* s, int D, int lane) {
  float acc = 0.0f;
  if (FN == 1) {
    for (int i = lane; i < D; i += 32) acc = fmaf(s[i], s[i], acc);
    return warp_sum(acc);
  } else if (FN == 2) {
    for (int i = lane; i + 1 < D; i += 32) {
      const float x = s[i];
      const float a = fmaf(-x, x, s[i + 1]), b = x - 1.0f;
      acc += fmaf(100.0f * a, a, b * b);
    }
    return warp_sum(acc);
  } else if (FN == 3) {
    for (int i = lane; i < D; i += 32) {
      const float x = s[i];
      acc += fmaf(x, x, -10.0f * cospif(2.0f * x));
    }
    return fmaf(10.0f, (float)D, warp_sum(acc));
  } else {
    float prod = 1.0f;
    for (int i = lane; i < D; i += 32) {
      const float x = s[i];
      acc = fmaf(x, x, acc);
      prod *= griewank_factor(x, i);
    }
    const float sum = warp_sum(acc);
    prod = warp_prod(prod);
    return 1.0f + sum / 4000.0f - prod;
  }
}

// Eq. penalty's Q^beta for an integer beta >= 1, by repeated multiplication.
__device__ __forceinline__ float pow_int(float q, int beta) {
  float r = q;
  for (int b = 1; b < beta; ++b) r *= q;
  return r;
}

// Box of coordinate j of a path objective: its axis (x, y or z) picks the bounds.
__device__ __forceinline__ int coord_axis(const BfParams& p, int j) { return (j >= p.half) + (j >= p.half2); }
__device__ __forceinline__ float axis_sel(int ax, float a, float b, float c) { return ax == 0 ? a : (ax == 1 ? b : c); }

// Shared memory of an iteration CTA before its obstacles and rows: this launch's
// candidate keys and the previous group keys (RG each), the Tbest keys (R) and the
// runs' stop flags (R).
__host__ __device__ inline size_t bf_keys_bytes(int RG, int R) {
  return ((size_t)(2 * RG + R) * 8 + (size_t)R * 4 + 15) / 16 * 16;
}

// Auto Truncation of the runs in launch j (path objectives).  With kUpdate, every
// CTA decides iteration j - 1 for each run from the run's Tbest key, the state the
// previous launch left in slot (j + 1) % 2 and the collision count of the Tbest row
// (its holder's Pbest count; unknown, so no stop, for a row of a loaded state); CTA 0
// writes the new state into slot j % 2.  Without kUpdate the flags come from slot
// j % 2 (written by the last whole launch).  sdone[r] != 0: run r has stopped --
// its particles neither move nor are evaluated again.
__device__ __forceinline__ void at_decide(const BfParams& p, int j, int mode, const unsigned long long* stk, int* sdone) {
  const int RM = p.R * p.M;
  for (int r = threadIdx.x; r < p.R; r += blockDim.x) {
    if (p.at_stall <= 0) {
      sdone[r] = 0;
      continue;
    }
    if (!(mode & kUpdate)) {
      sdone[r] = p.at_state[((size_t)(j % 2) * p.R + r) * 4 + 2];
      continue;
    }
    const int* in = p.at_state + ((size_t)((j + 1) % 2) * p.R + r) * 4;
    int stall = in[0], done = in[2], stop = in[3];
    float prev = __int_as_float(in[1]);
    if (!done) {
      const unsigned long long tk = stk[r];
      const float tf = tk == kEmpty ? INFINITY : float_of_ord((uint32_t)(tk >> 32));
      stall = tf < prev - p.stall_tol ? 0 : stall + 1;
      prev = tf;
      int tq = -1;
      if (tk != kEmpty && (int)key_idx(tk) < p.M)
        tq = p.pq[(size_t)key_par(tk) * RM + (size_t)r * p.M + key_idx(tk)];
      if (stall >= p.at_stall && tq == 0) {
        done = 1;
        stop = j - 1;
      }
    }
    sdone[r] = done;
    if (blockIdx.x == 0) {
      int* out = p.at_state + ((size_t)(j % 2) * p.R + r) * 4;
      out[0] = stall;
      out[1] = __float_as_int(prev);
      out[2] = done;
      out[3] = stop;
    }
  }
}

// Objective 6 (the Conclusion's extension to 3D planning of Eqs. path_fit, lenth,
// penalty): a segment as its midpoint m, unit direction u (zero for a zero-length
// segment), half-length h and length.  For a sphere centre c, with w = c - m and
// along = w.u, the squared distance from c to the segment is
// max(|along| - h, 0)^2 + |w - along u|^2 (the perpendicular part is formed as a
// vector, not as |w|^2 - along^2, so that it keeps its precision for long segments).
struct Seg3 {
  float mx, my, mz, ux, uy, uz, h, len;
};
__device__ __forceinline__ Seg3 seg3(float ax, float ay, float az, float bx, float by, float bz) {
  Seg3 g;
  const float dx = bx - ax, dy = by - ay, dz = bz - az;
  const float l2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  g.len = sqrtf(l2);
  const float inv = l2 > 0.0f ? 1.0f / g.len : 0.0f;
  g.ux = dx * inv;
  g.uy = dy * inv;
  g.uz = dz * inv;
  g.mx = 0.5f * (ax + bx);
  g.my = 0.5f * (ay + by);
  g.mz = 0.5f * (az + bz);
  g.h = 0.5f * g.len;
  return g;
}
// 1 when the segment passes closer than the radius to the sphere (cx, cy, cz, r^2).
__device__ __forceinline__ int sphere_hit(const Seg3& g, float4 c) {
  const float wx = c.x - g.mx, wy = c.y - g.my, wz = c.z - g.mz;
  const float al = fmaf(wx, g.ux, fmaf(wy, g.uy, wz * g.uz));
  const float px = fmaf(-al, g.ux, wx), py = fmaf(-al, g.uy, wy), pz = fmaf(-al, g.uz, wz);
  const float e = fmaxf(fabsf(al) - g.h, 0.0f);
  return fmaf(e, e, fmaf(px, px, fmaf(py, py, pz * pz))) < c.w;
}

// Objective 6 of one row, the whole warp (every lane gets the value): the T + 1
// segment lengths over the lanes, then per segment the spheres over the lanes.
// Waypoint i is (s[i], s[T + i], s[2T + i]); pts = start x, y, z, target x, y, z.
// kSquared: the spheres' fourth value already holds r^2 (shared-memory copies).
template <bool kSquared>
__device__ __forceinline__ float sphere_row(const float* s, int T, const float* pts, const float4* sph, int S,
                                            float alpha, int beta, int lane, int& qout) {
  float len = 0.0f;
  for (int k = lane; k <= T; k += 32) {
    const float ax = k == 0 ? pts[0] : s[k - 1], ay = k == 0 ? pts[1] : s[T + k - 1];
    const float az = k == 0 ? pts[2] : s[2 * T + k - 1];
    const float bx = k == T ? pts[3] : s[k], by = k == T ? pts[4] : s[T + k], bz = k == T ? pts[5] : s[2 * T + k];
    const float dx = bx - ax, dy = by - ay, dz = bz - az;
    len += sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
  }
  len = warp_sum(len);
  int q = 0;
  for (int k = 0; k <= T; ++k) {
    const float ax = k == 0 ? pts[0] : s[k - 1], ay = k == 0 ? pts[1] : s[T + k - 1];
    const float az = k == 0 ? pts[2] : s[2 * T + k - 1];
    const float bx = k == T ? pts[3] : s[k], by = k == T ? pts[4] : s[T + k], bz = k == T ? pts[5] : s[2 * T + k];
    const Seg3 g = seg3(ax, ay, az, bx, by, bz);
#pragma unroll 4
    for (int o = lane; o < S; o += 32) {
      float4 c = sph[o];
      if (!kSquared) c.w = c.w * c.w;
      q += sphere_hit(g, c);
    }
  }
  q = __reduce_add_sync(0xffffffffu, q);
  qout = q;
  return q > 0 ? len + alpha * pow_int((float)q, beta) : len;
}

// Objective 5 (Sec. 3.3.1 map model; Eqs. path_fit, lenth, penalty): length of the
// path start -> waypoints -> target plus alpha * Q^beta, Q = the number of proper
// crossings (strict orientation tests) between its T + 1 segments and the E obstacle
// edges.  Waypoint i is (s[i], s[T + i]).  The whole warp; every lane gets the value.
__device__ __forceinline__ float poly_row(const float* s, int T, const float* pts, const float4* edges, int E,
                                          float alpha, int beta, int lane, int& qout) {
  float len = 0.0f;
  for (int k = lane; k <= T; k += 32) {
    const float ax = k == 0 ? pts[0] : s[k - 1], ay = k == 0 ? pts[1] : s[T + k - 1];
    const float bx = k == T ? pts[2] : s[k], by = k == T ? pts[3] : s[T + k];
    const float dx = bx - ax, dy = by - ay;
    len += sqrtf(fmaf(dx, dx, dy * dy));
  }
  len = warp_sum(len);
  int q = 0;
  for (int k = 0; k <= T; ++k) {
    const float ax = k == 0 ? pts[0] : s[k - 1], ay = k == 0 ? pts[1] : s[T + k - 1];
    const float bx = k == T ? pts[2] : s[k], by = k == T ? pts[3] : s[T + k];
    const float ux = bx - ax, uy = by - ay;
    for (int e = lane; e < E; e += 32) {
      q += edge_crosses(ax, ay, ux, uy, edges[e]);
    }
  }
  q = __reduce_add_sync(0xffffffffu, q);
  qout = q;
  return q > 0 ? len + alpha * pow_int((float)q, beta) : len;
}

}  // namespace

// ---------------------------------------------------------------------------
// Initialisation (Algorithm 1): X uniform over [lo, hi]^D, V uniform in +-V_range
// with V_range = V_limit (hi - lo), Pbest row = X (parity 0), Pbest fitness +inf, no
// bests.  Four coordinates per Philox draw (counter: coordinate chunk, particle,
// stream, run), as in the path planner.  Path objectives: each axis its own box;
// with Priori Initialization (Sec. 3.3.3) the first n_pi particles of each group
// take X = clip(prevT + (2u - 1) h_PI) from the PI stream instead, and the planning
// cycle enters the counters.
// ---------------------------------------------------------------------------
__global__ void bf_init_kernel(const BfParams p) {
  const size_t nch = (size_t)p.Dp / 4;
  const size_t total = (size_t)p.R * p.M * nch;
  const bool path = p.fn >= 5;
  const int n_pi = path ? p.warm[0] : 0;
  const float pi_h = path ? __int_as_float(p.warm[1]) : 0.0f;
  const uint32_t cyc = path ? (uint32_t)p.warm[2] : 0u;
  for (size_t it = (size_t)blockIdx.x * blockDim.x + threadIdx.x; it < total;
       it += (size_t)gridDim.x * blockDim.x) {
    const size_t q = it / nch;
    const int c = (int)(it - q * nch);
    const int r = (int)(q / p.M), pi = (int)(q - (size_t)r * p.M);
    const int g = pi / p.N;
    const float vlim = p.hyper[((size_t)r * p.G + g) * 6 + 5];
    const bool by_pi = pi - g * p.N < n_pi;
    const uint4 ux = draw(p.key0, p.key1, (uint32_t)c, (uint32_t)pi, by_pi ? kStreamPI : kStreamInitX, cyc,
                          p.run_id + (uint32_t)r);
    const uint4 uv = draw(p.key0, p.key1, (uint32_t)c, (uint32_t)pi, kStreamInitV, cyc, p.run_id + (uint32_t)r);
    float xs[4], vs[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int jj = 4 * c + e;
      const bool in = jj < p.D;
      const int ax = coord_axis(p, jj);
      const float lo = axis_sel(ax, p.lo, p.lo2, p.lo3), hi = axis_sel(ax, p.hi, p.hi2, p.hi3);
      const float ex = hi - lo;
      float x = lo + lane_of(ux, e) * ex;
      if (by_pi && in)
        x = fminf(fmaxf(p.prevT[(size_t)r * p.Dp + jj] + (2.0f * lane_of(ux, e) - 1.0f) * pi_h, lo), hi);
      xs[e] = in ? x : 0.0f;
      vs[e] = in ? (2.0f * lane_of(uv, e) - 1.0f) * (vlim * ex) : 0.0f;
    }
    const float4 x4 = make_float4(xs[0], xs[1], xs[2], xs[3]);
    const float4 v4 = make_float4(vs[0], vs[1], vs[2], vs[3]);
    reinterpret_cast<float4*>(p.X + q * p.Dp)[c] = x4;
    reinterpret_cast<float4*>(p.V + q * p.Dp)[c] = v4;
    reinterpret_cast<float4*>(p.P + q * p.Dp)[c] = x4;
    reinterpret_cast<float4*>(p.P + ((size_t)p.R * p.M + q) * p.Dp)[c] = x4;
    if (c == 0) {
      p.Pfit[q] = INFINITY;
      p.pcur[q] = 0;
    }
  }
  const size_t nk = (size_t)3 * p.R * p.G;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nk; i += (size_t)gridDim.x * blockDim.x) {
    p.keys[i] = kEmpty;
    if (i < (size_t)2 * p.R) p.thold[i] = kEmpty;
  }
  // Auto Truncation: no stall, no previous Tbest, not stopped (both slots)
  if (path && p.at_stall > 0)
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)2 * p.R;
         i += (size_t)gridDim.x * blockDim.x) {
      int* st = p.at_state + i * 4;
      st[0] = 0;
      st[1] = __float_as_int(INFINITY);
      st[2] = 0;
      st[3] = 0;
    }
}

// ---------------------------------------------------------------------------
// One iteration launch (see the file comment).  j is the iteration whose fitness
// this launch evaluates; the update it applies first is iteration j - 1's.
// ---------------------------------------------------------------------------
template <int FN>
__global__ void __launch_bounds__(256, 2) bf_iter_kernel(const BfParams p, int j, int mode) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int RG = p.R * p.G;
  // shared memory: this launch's candidate keys, iteration j - 1's group keys and
  // Tbest keys (copied once per CTA), the polygon edges, one row per warp
  unsigned long long* ck = reinterpret_cast<unsigned long long*>(smem);
  unsigned long long* sgk = ck + RG;
  unsigned long long* stk = sgk + RG;
  int* sdone = reinterpret_cast<int*>(stk + p.R);
  const size_t keys_b = bf_keys_bytes(RG, p.R);
  float4* sedges = reinterpret_cast<float4*>(smem + keys_b);
  const int E = FN >= 5 ? p.E : 0;
  float* srow = reinterpret_cast<float*>(smem + keys_b + (size_t)E * 16) + (size_t)warp * p.Dp;
  const uint32_t cyc = FN >= 5 ? (uint32_t)p.warm[2] : 0u;
  const unsigned long long* kprev = p.keys + (size_t)((j + 2) % 3) * RG;  // iteration j - 1
  unsigned long long* kcur = p.keys + (size_t)(j % 3) * RG;
  for (int i = threadIdx.x; i < RG; i += blockDim.x) {
    ck[i] = kEmpty;
    if (mode & kUpdate) sgk[i] = kprev[i];
  }
  for (int i = threadIdx.x; i < E; i += blockDim.x) {
    float4 o = p.edges[i];
    if (FN == 6) o.w = o.w * o.w;   // spheres are tested against r^2
    sedges[i] = o;
  }
  if (blockIdx.x == 0) {
    unsigned long long* knext = p.keys + (size_t)((j + 1) % 3) * RG;   // read last in launch j - 1
    for (int i = threadIdx.x; i < RG; i += blockDim.x) knext[i] = kEmpty;
  }
  __syncthreads();
  if (mode & kUpdate) {
    // Tbest of iteration j - 1 per run: the group keys and the previous holder.
    for (int r = threadIdx.x; r < p.R; r += blockDim.x) {
      const unsigned long long tk = resolve_T(sgk + (size_t)r * p.G, p.G, p.thold[(size_t)(j % 2) * p.R + r]);
      stk[r] = tk;
      if (blockIdx.x == 0) {
        p.thold[(size_t)((j + 1) % 2) * p.R + r] = tk;
        if (j - 2 < p.hist_len)
          p.hist[(size_t)r * p.hist_len + (j - 2)] = tk == kEmpty ? INFINITY : float_of_ord((uint32_t)(tk >> 32));
      }
    }
    __syncthreads();
  }
  if (FN >= 5) {
    at_decide(p, j, mode, stk, sdone);
    __syncthreads();
  }

  const float ext = p.hi - p.lo;
  const int nch = p.Dp >> 2;
  const size_t total = (size_t)p.R * p.M;
  const size_t stride = (size_t)gridDim.x * nwarps;
  const size_t q0 = (size_t)blockIdx.x * nwarps + warp;
  // this particle's Pbest parity and fitness, loaded one particle ahead (only this
  // warp writes them)
  unsigned par_next = q0 < total ? p.pcur[q0] : 0u;
  float pf_next = q0 < total ? p.Pfit[q0] : 0.0f;
  for (size_t q = q0; q < total; q += stride) {
    const int r = (int)(q / p.M), pi = (int)(q - (size_t)r * p.M);
    const int g = pi / p.N;
    float4* xr = reinterpret_cast<float4*>(p.X + q * p.Dp);
    float4* s4 = reinterpret_cast<float4*>(srow);
    const unsigned par = par_next;
    float pf = pf_next;
    if (q + stride < total) {
      par_next = p.pcur[q + stride];
      pf_next = p.Pfit[q + stride];
    }
    const bool stopped = FN >= 5 && sdone[r] != 0;
    if (stopped) {
      // a stopped run: only its group keys carry over (previous holders, priority 0)
      if ((mode & kUpdate) && pi == 0 && lane < p.G) {
        const unsigned long long k0 = sgk[(size_t)r * p.G + lane];
        if (k0 != kEmpty) atomicMin(&ck[r * p.G + lane], k0 & ~(1ull << 31));
      }
      continue;
    }
    if (mode & kUpdate) {
      // Bests of iteration j - 1: this group's key and the run's Tbest key.
      const unsigned long long* gk = sgk + (size_t)r * p.G;
      const unsigned long long tk = stk[r];
      const float4* gr = reinterpret_cast<const float4*>(key_row(p, r, gk[g]));
      const float4* tr = reinterpret_cast<const float4*>(key_row(p, r, tk));
      const float* hy = p.hyper + ((size_t)r * p.G + g) * 6;
      const float c1 = hy[0], c2 = hy[1], c3 = hy[2], w_init = hy[3], w_end = hy[4];
      const float vmax = hy[5] * ext, vmax2 = hy[5] * (p.hi2 - p.lo2), vmax3 = hy[5] * (p.hi3 - p.lo3);
      const int k = j - 1;
      const float w = w_init - (w_init - w_end) / (float)p.K * (float)k;
      const uint4 rr = draw(p.key0, p.key1, (uint32_t)k, (uint32_t)pi, kStreamVel, cyc, p.run_id + (uint32_t)r);
      const float a1 = c1 * u01(rr.x), a2 = c2 * u01(rr.y), a3 = c3 * u01(rr.z);
      const bool need_T = c3 != 0.0f;
      float4* vr = reinterpret_cast<float4*>(p.V + q * p.Dp);
      const float4* pr = reinterpret_cast<const float4*>(p.P + ((size_t)par * total + q) * p.Dp);
      const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      // kUnroll chunks per lane in flight: all their loads are issued before any use.
      for (int c0 = lane; c0 < nch; c0 += 32 * kUnroll) {
        float4 x[kUnroll], v[kUnroll], pb[kUnroll], gb[kUnroll], tb[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int c = c0 + 32 * u;
          if (c < nch) {
            x[u] = xr[c];
            v[u] = vr[c];
            pb[u] = __ldg(pr + c);
            gb[u] = gr ? __ldg(gr + c) : zero;
            tb[u] = (need_T && tr) ? __ldg(tr + c) : zero;
          }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int c = c0 + 32 * u;
          if (c < nch) {
            float* xe = &x[u].x;
            float* ve = &v[u].x;
            const float* pe = &pb[u].x;
            const float* ge = &gb[u].x;
            const float* te = &tb[u].x;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              if (4 * c + e < p.D) {
                const int ax = FN >= 5 ? coord_axis(p, 4 * c + e) : 0;
                const float bv = axis_sel(ax, vmax, vmax2, vmax3);
                float vv = w * ve[e];
                vv = fmaf(a1, pe[e] - xe[e], vv);
                vv = fmaf(a2, ge[e] - xe[e], vv);
                if (need_T) vv = fmaf(a3, te[e] - xe[e], vv);
                vv = fminf(fmaxf(vv, -bv), bv);
                ve[e] = vv;
                xe[e] = fminf(fmaxf(xe[e] + vv, axis_sel(ax, p.lo, p.lo2, p.lo3)), axis_sel(ax, p.hi, p.hi2, p.hi3));
              }
            }
            xr[c] = x[u];
            vr[c] = v[u];
            s4[c] = x[u];
          }
        }
      }
      // The previous holder of this group's best keeps it on a tie (priority 0).
      if (pi == 0 && lane < p.G) {
        const unsigned long long k0 = gk[lane];
        if (k0 != kEmpty) atomicMin(&ck[r * p.G + lane], k0 & ~(1ull << 31));
      }
    } else {
      for (int c = lane; c < nch; c += 32) s4[c] = xr[c];
    }
    __syncwarp();
    if (!(mode & kEval)) continue;

    // Fitness of iteration j, Pbest update (strictly better only).
    int qcount = 0;
    const float F = FN == 5   ? poly_row(srow, p.half, p.pts, sedges, E, p.alpha, p.beta, lane, qcount)
                    : FN == 6 ? sphere_row<true>(srow, p.half, p.pts, sedges, E, p.alpha, p.beta, lane, qcount)
                              : bf_row<FN>(srow, p.D, lane);
    unsigned npar = par;
    if (F < pf) {
      npar = par ^ 1u;
      float4* dst = reinterpret_cast<float4*>(p.P + ((size_t)npar * total + q) * p.Dp);
      for (int c = lane; c < nch; c += 32) dst[c] = s4[c];
      pf = F;
      if (lane == 0) {
        p.Pfit[q] = F;
        p.pcur[q] = (unsigned char)npar;
        if (FN >= 5) p.pq[(size_t)npar * total + q] = qcount;
      }
    }
    if (lane == 0 && isfinite(pf)) atomicMin(&ck[r * p.G + g], make_key(pf, 1u, (uint32_t)pi, npar));
    __syncwarp();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < RG; i += blockDim.x)
    if (ck[i] != kEmpty) atomicMin(&kcur[i], ck[i]);
}

// ---------------------------------------------------------------------------
// A whole run of a small swarm in one launch: one CTA per run holds X, V, Pbest,
// the Gbest rows and the Tbest row in shared memory (rows at an odd stride, so
// that the threads' rows fall in different banks) and steps through all
// iterations with block barriers instead of kernel boundaries (the standard runs
// of Sec. 4.1.1: 80 particles x 30 coordinates per trial, one trial per CTA).
// Thread t owns particles t, t + blockDim, ...: it draws their random factors,
// updates their rows and sums their fitness coordinate by coordinate.  Group keys
// are merged with shared-memory atomics (previous holder first, at priority 0),
// then Tbest is decided; the update expressions, the Philox draws and the best
// rules are bf_iter_kernel's (the fitness is summed in coordinate order here, in
// lane-strided order there).  At the end the state is written back in the engine's
// layout (Pbest rows in parity 0, keys naming them, Tbest in both holder slots) so
// that sepso_bf_step, the bests kernel and the state calls continue from it.
// ---------------------------------------------------------------------------
template <int FN>
__device__ __forceinline__ float bf_row_serial(const float* x, int D) {
  float acc = 0.0f, prod = 1.0f;
  if constexpr (FN == 2) {
    for (int i = 0; i + 1 < D; ++i) {
      const float a = fmaf(-x[i], x[i], x[i + 1]), b = x[i] - 1.0f;
      acc += fmaf(100.0f * a, a, b * b);
    }
    return acc;
  } else {
  for (int i = 0; i < D; ++i) {
    const float xi = x[i];
    if (FN == 1) {
      acc = fmaf(xi, xi, acc);
    } else if (FN == 3) {
      acc += fmaf(xi, xi, -10.0f * cospif(2.0f * xi));
    } else {
      acc = fmaf(xi, xi, acc);
      prod *= griewank_factor(xi, i);
    }
  }
  if (FN == 1) return acc;
  if (FN == 3) return fmaf(10.0f, (float)D, acc);
  return 1.0f + acc / 4000.0f - prod;
  }
}

template <int FN>
__global__ void __launch_bounds__(256) bf_small_kernel(const BfParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int r = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int D = p.D, G = p.G, N = p.N, M = p.M, K = p.K;
  const int S = D + 1;  // shared-memory row stride
  float* sX = reinterpret_cast<float*>(smem);
  float* sV = sX + (size_t)M * S;
  float* sP = sV + (size_t)M * S;
  float* sG = sP + (size_t)M * S;
  float* sT = sG + (size_t)G * S;
  float* sPf = sT + S;
  unsigned long long* gkey = reinterpret_cast<unsigned long long*>(
      smem + ((size_t)(3 * M * S + G * S + S + M) * 4 + 7) / 8 * 8);
  unsigned long long* nkey = gkey + G;
  unsigned long long* s_tk = nkey + G;
  const float ext = p.hi - p.lo;
  const uint32_t run = p.run_id + (uint32_t)r;

  // Initialisation, as bf_init_kernel.
  for (int pi = tid; pi < M; pi += nt) {
    const float vlim = p.hyper[((size_t)r * G + pi / N) * 6 + 5];
    for (int c = 0; 4 * c < D; ++c) {
      const uint4 ux = draw(p.key0, p.key1, (uint32_t)c, (uint32_t)pi, kStreamInitX, 0u, run);
      const uint4 uv = draw(p.key0, p.key1, (uint32_t)c, (uint32_t)pi, kStreamInitV, 0u, run);
      for (int e = 0; e < 4 && 4 * c + e < D; ++e) {
        const float x = p.lo + lane_of(ux, e) * ext;
        sX[pi * S + 4 * c + e] = x;
        sP[pi * S + 4 * c + e] = x;
        sV[pi * S + 4 * c + e] = (2.0f * lane_of(uv, e) - 1.0f) * (vlim * ext);
      }
    }
    sPf[pi] = INFINITY;
  }
  for (int i = tid; i < G * S + S; i += nt) sG[i] = 0.0f;  // sG then sT
  for (int i = tid; i < G; i += nt) gkey[i] = kEmpty;
  if (tid == 0) *s_tk = kEmpty;
  __syncthreads();

  for (int j = 1; j <= K + 1; ++j) {
    // Update of iteration j - 1 (for j > 1); for j = K + 1 it is the last step.
    if (j > 1) {
      const int k = j - 1;
      const bool have_T = *s_tk != kEmpty;
      for (int pi = tid; pi < M; pi += nt) {
        const int g = pi / N;
        const float* hy = p.hyper + ((size_t)r * G + g) * 6;
        const float c1 = hy[0], c2 = hy[1], c3 = hy[2], w_init = hy[3], w_end = hy[4];
        const float vmax = hy[5] * ext;
        const float w = w_init - (w_init - w_end) / (float)K * (float)k;
        const bool need_T = c3 != 0.0f, have_G = gkey[g] != kEmpty;
        const uint4 rr = draw(p.key0, p.key1, (uint32_t)k, (uint32_t)pi, kStreamVel, 0u, run);
        const float a1 = c1 * u01(rr.x), a2 = c2 * u01(rr.y), a3 = c3 * u01(rr.z);
        float* x = sX + pi * S;
        float* v = sV + pi * S;
        const float* pb = sP + pi * S;
        const float* gb = sG + g * S;
        for (int i = 0; i < D; ++i) {
          const float xe = x[i];
          float vv = w * v[i];
          vv = fmaf(a1, pb[i] - xe, vv);
          vv = fmaf(a2, (have_G ? gb[i] : 0.0f) - xe, vv);
          if (need_T) vv = fmaf(a3, (have_T ? sT[i] : 0.0f) - xe, vv);
          vv = fminf(fmaxf(vv, -vmax), vmax);
          v[i] = vv;
          x[i] = fminf(fmaxf(xe + vv, p.lo), p.hi);
        }
      }
    }
    if (j > K) break;
    // Iteration j's group keys start from the previous holders (priority 0).
    for (int g = tid; g < G; g += nt) nkey[g] = gkey[g] == kEmpty ? kEmpty : (gkey[g] & ~(1ull << 31));
    __syncthreads();
    // Fitness of iteration j, Pbest (strictly better), candidates.
    for (int pi = tid; pi < M; pi += nt) {
      const float F = bf_row_serial<FN>(sX + pi * S, D);
      float pf = sPf[pi];
      if (F < pf) {
        for (int i = 0; i < D; ++i) sP[pi * S + i] = sX[pi * S + i];
        pf = F;
        sPf[pi] = F;
      }
      if (isfinite(pf)) atomicMin(&nkey[pi / N], make_key(pf, 1u, (uint32_t)pi, 0u));
    }
    __syncthreads();
    // New Gbest rows where the holder changed.
    for (int it = tid; it < G * D; it += nt) {
      const int g = it / D, i = it - g * D;
      const unsigned long long kk = nkey[g];
      if (kk != kEmpty && kk != gkey[g]) sG[g * S + i] = sP[(int)((kk >> 1) & 0x3fffffffu) * S + i];
    }
    __syncthreads();
    for (int g = tid; g < G; g += nt) gkey[g] = nkey[g];
    __syncthreads();
    // Tbest of iteration j.
    const unsigned long long told = *s_tk;
    const unsigned long long tk = resolve_T(gkey, G, told);
    if (tk != told) {
      int gw = 0;
      for (int g = 0; g < G; ++g)
        if (gkey[g] == tk) {
          gw = g;
          break;
        }
      for (int i = tid; i < D; i += nt) sT[i] = sG[gw * S + i];
    }
    __syncthreads();
    if (tid == 0) {
      *s_tk = tk;
      if (j - 1 < p.hist_len)
        p.hist[(size_t)r * p.hist_len + (j - 1)] = tk == kEmpty ? INFINITY : float_of_ord((uint32_t)(tk >> 32));
    }
    __syncthreads();
  }
  __syncthreads();

  // Write the state back in the engine's layout.
  const int Dp = p.Dp;
  const size_t q0 = (size_t)r * M;
  for (int it = tid; it < M * Dp; it += nt) {
    const int pi = it / Dp, i = it - pi * Dp;
    const bool in = i < D;
    p.X[(q0 + pi) * Dp + i] = in ? sX[pi * S + i] : 0.0f;
    p.V[(q0 + pi) * Dp + i] = in ? sV[pi * S + i] : 0.0f;
    p.P[(q0 + pi) * Dp + i] = in ? sP[pi * S + i] : 0.0f;
  }
  for (int i = tid; i < M; i += nt) {
    p.Pfit[q0 + i] = sPf[i];
    p.pcur[q0 + i] = 0;
  }
  const int RG = p.R * G;
  for (int g = tid; g < G; g += nt) {
    const unsigned long long kk = gkey[g];
    p.keys[(size_t)(K % 3) * RG + (size_t)r * G + g] = kk;
    p.keys[(size_t)((K + 1) % 3) * RG + (size_t)r * G + g] = kk == kEmpty ? kEmpty : (kk & ~(1ull << 31));
  }
  if (tid == 0) {
    p.thold[r] = *s_tk;
    p.thold[(size_t)p.R + r] = *s_tk;
  }
}

// ---------------------------------------------------------------------------
// Path objectives with a lane per particle: the iteration of bf_iter_kernel for
// short rows (paths of D <= kLaneMaxD coordinates), where a warp per particle would
// leave most lanes idle in the update and spread each path's few segments over the
// lanes.  Lane l of a warp owns one particle: it updates its row coordinate by
// coordinate, keeps the new row in shared memory (stride D + 1: the lanes' rows fall
// in different banks) and tests its T + 1 segments against every obstacle record
// (edge pairs of objective 5, sphere pairs of objective 6), each record read by all
// lanes at once (a broadcast).  Bests, keys and Pbest parities as in bf_iter_kernel.
// poly_lane_kernel runs objective 5, sphere_lane_kernel objective 6.
// ---------------------------------------------------------------------------
constexpr int kLaneMaxD = 64;
constexpr int kLaneBatch = 2;     // particles whose rows a lane-kernel warp moves at once
constexpr int kLaneThreads = 128;   // small CTAs: the single wave of lane CTAs spreads evenly over the SMs
constexpr int kLaneMinPerSm = 256;   // particles per SM from which objective 5 uses a lane each
constexpr long long kSmallMaxCoords = 8192;  // swarm size (G N D) up to which a run is one CTA

// Objective 5 in the lane kernel, on edge pairs (edge_pair_hits): shared memory
// holds the edges two by two (layout at edge_pair_f4).
__device__ __forceinline__ float poly_lane_pairs(const float* s, int T, const float* pts, const ulonglong2* ep, int K,
                                                 float alpha, int beta, int& qout) {
  // segment k: start (ax, ay), direction (ux, uy)
  auto seg = [&](int k, float& ax, float& ay, float& ux, float& uy) {
    ax = k == 0 ? pts[0] : s[k - 1];
    ay = k == 0 ? pts[1] : s[T + k - 1];
    ux = (k == T ? pts[2] : s[k]) - ax;
    uy = (k == T ? pts[3] : s[T + k]) - ay;
  };
  float len = 0.0f;
  for (int k = 0; k <= T; ++k) {
    float ax, ay, ux, uy;
    seg(k, ax, ay, ux, uy);
    len += sqrtf(fmaf(ux, ux, uy * uy));
  }
  // the crossings two segments per edge-pair read
  int q = 0, k = 0;
  for (; k + 1 <= T; k += 2) {
    float ax, ay, ux, uy, ax2, ay2, ux2, uy2;
    seg(k, ax, ay, ux, uy);
    seg(k + 1, ax2, ay2, ux2, uy2);
    q += edge_pair_hits2(ax, ay, ux, uy, ax2, ay2, ux2, uy2, ep, K);
  }
  if (k <= T) {
    float ax, ay, ux, uy;
    seg(k, ax, ay, ux, uy);
    q += edge_pair_hits(ax, ay, ux, uy, ep, 0, K);
  }
  qout = q;
  return q > 0 ? len + alpha * pow_int((float)q, beta) : len;
}

// Objective 6 in the lane kernel, on sphere pairs: shared memory holds the spheres
// two by two as float4 (cx0, cx1, cy0, cy1) and float4 (cz0, cz1, -r0^2, -r1^2) (an
// odd count padded with a sphere of radius 0, which nothing hits), so that packed
// FP32x2 instructions test a segment against two spheres at once: w = c - m,
// -along = w.(-u), p = w + (-along) u, and S = max(|along| - h, 0)^2 + |p|^2 - r^2
// per sphere, whose sign bit is the hit (S is never -0: the sum of -r^2 and
// squares is +0 at the least when it vanishes).
struct Seg3P {
  unsigned long long nmx, nmy, nmz, ux, uy, uz, nux, nuy, nuz;
  float h;
};
__device__ __forceinline__ Seg3P seg3p(const Seg3& g) {
  Seg3P f;
  f.nmx = pack2(-g.mx, -g.mx);
  f.nmy = pack2(-g.my, -g.my);
  f.nmz = pack2(-g.mz, -g.mz);
  f.ux = pack2(g.ux, g.ux);
  f.uy = pack2(g.uy, g.uy);
  f.uz = pack2(g.uz, g.uz);
  f.nux = pack2(-g.ux, -g.ux);
  f.nuy = pack2(-g.uy, -g.uy);
  f.nuz = pack2(-g.uz, -g.uz);
  f.h = g.h;
  return f;
}
__device__ __forceinline__ int sphere_pair_hits(const Seg3P& g, ulonglong2 a, ulonglong2 b) {
  const unsigned long long WX = fadd2(a.x, g.nmx), WY = fadd2(a.y, g.nmy), WZ = fadd2(b.x, g.nmz);
  const unsigned long long NAL = ffma2(WX, g.nux, ffma2(WY, g.nuy, fmul2(WZ, g.nuz)));
  const unsigned long long PX = ffma2(NAL, g.ux, WX), PY = ffma2(NAL, g.uy, WY), PZ = ffma2(NAL, g.uz, WZ);
  float n0, n1;
  unpack2(NAL, n0, n1);
  const float e0 = fmaxf(fabsf(n0) - g.h, 0.0f), e1 = fmaxf(fabsf(n1) - g.h, 0.0f);
  const unsigned long long E = pack2(e0, e1);
  const unsigned long long S = ffma2(E, E, ffma2(PX, PX, ffma2(PY, PY, ffma2(PZ, PZ, b.y))));
  float s0, s1;
  unpack2(S, s0, s1);
  return (int)(__float_as_uint(s0) >> 31) + (int)(__float_as_uint(s1) >> 31);
}

// Objective 6 of one lane's row (waypoint i = (s[i], s[T + i], s[2T + i])) against K
// sphere pairs: the segments two at a time, each pair read once for both.
__device__ __forceinline__ float sphere_lane(const float* s, int T, const float* pts, const ulonglong2* sp, int K,
                                             float alpha, int beta, int& qout) {
  float len = 0.0f;
  int q = 0;
  float ax = pts[0], ay = pts[1], az = pts[2];
  for (int k = 0; k <= T; k += 2) {
    const float bx = k == T ? pts[3] : s[k], by = k == T ? pts[4] : s[T + k], bz = k == T ? pts[5] : s[2 * T + k];
    const Seg3 g0 = seg3(ax, ay, az, bx, by, bz);
    len += g0.len;
    const Seg3P f0 = seg3p(g0);
    if (k + 1 <= T) {
      const int k1 = k + 1;
      const float cx = k1 == T ? pts[3] : s[k1], cy = k1 == T ? pts[4] : s[T + k1];
      const float cz = k1 == T ? pts[5] : s[2 * T + k1];
      const Seg3 g1 = seg3(bx, by, bz, cx, cy, cz);
      len += g1.len;
      const Seg3P f1 = seg3p(g1);
#pragma unroll 2
      for (int o = 0; o < K; ++o) {
        const ulonglong2 a = sp[2 * o], b = sp[2 * o + 1];
        q += sphere_pair_hits(f0, a, b) + sphere_pair_hits(f1, a, b);
      }
      ax = cx;
      ay = cy;
      az = cz;
    } else {
#pragma unroll 2
      for (int o = 0; o < K; ++o) q += sphere_pair_hits(f0, sp[2 * o], sp[2 * o + 1]);
    }
  }
  qout = q;
  return q > 0 ? len + alpha * pow_int((float)q, beta) : len;
}

// Bytes of the obstacle records the lane kernel stages for n records.
__host__ __device__ inline size_t lane_obstacle_bytes(int fn, int n) {
  return fn == 5 || fn == 6 ? (size_t)((n + 1) / 2) * 32 : (size_t)n * 16;
}

template <int FN>
__device__ __forceinline__ void path_lane_iter(const BfParams& p, int j, int mode, unsigned char* smem) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  const int RG = p.R * p.G;
  const int D = p.D, T = p.half;
  unsigned long long* ck = reinterpret_cast<unsigned long long*>(smem);
  unsigned long long* sgk = ck + RG;
  unsigned long long* stk = sgk + RG;
  int* sdone = reinterpret_cast<int*>(stk + p.R);
  const size_t keys_b = bf_keys_bytes(RG, p.R);
  float4* sedges = reinterpret_cast<float4*>(smem + keys_b);
  const int E = p.E;
  // the warp's 32 rows (stride D + 1), and this lane's own
  float* swarp = reinterpret_cast<float*>(smem + keys_b + lane_obstacle_bytes(FN, E)) + (size_t)warp * 32 * (D + 1);
  float* srow = swarp + (size_t)lane * (D + 1);
  const unsigned long long* kprev = p.keys + (size_t)((j + 2) % 3) * RG;
  unsigned long long* kcur = p.keys + (size_t)(j % 3) * RG;
  for (int i = threadIdx.x; i < RG; i += blockDim.x) {
    ck[i] = kEmpty;
    if (mode & kUpdate) sgk[i] = kprev[i];
  }
  if (FN == 6) {
    // sphere pairs (cx0, cx1, cy0, cy1), (cz0, cz1, -r0^2, -r1^2); the pad has r = 0
    for (int i = threadIdx.x; i < (E + 1) / 2; i += blockDim.x) {
      const float4 c0 = p.edges[2 * i];
      const float4 c1 = 2 * i + 1 < E ? p.edges[2 * i + 1] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      sedges[2 * i] = make_float4(c0.x, c1.x, c0.y, c1.y);
      sedges[2 * i + 1] = make_float4(c0.z, c1.z, -(c0.w * c0.w), -(c1.w * c1.w));
    }
  } else {
    // edge pairs (x0a, x0b, y0a, y0b), (vxa, vxb, -vya, -vyb); the pad is a zero edge
    for (int i = threadIdx.x; i < (E + 1) / 2; i += blockDim.x)
      edge_pair(p.edges[2 * i], 2 * i + 1 < E ? p.edges[2 * i + 1] : make_float4(0.0f, 0.0f, 0.0f, 0.0f),
                sedges + 2 * i);
  }
  const uint32_t cyc = (uint32_t)p.warm[2];
  if (blockIdx.x == 0) {
    unsigned long long* knext = p.keys + (size_t)((j + 1) % 3) * RG;
    for (int i = threadIdx.x; i < RG; i += blockDim.x) knext[i] = kEmpty;
  }
  __syncthreads();
  if (mode & kUpdate) {
    for (int r = threadIdx.x; r < p.R; r += blockDim.x) {
      const unsigned long long tk = resolve_T(sgk + (size_t)r * p.G, p.G, p.thold[(size_t)(j % 2) * p.R + r]);
      stk[r] = tk;
      if (blockIdx.x == 0) {
        p.thold[(size_t)((j + 1) % 2) * p.R + r] = tk;
        if (j - 2 < p.hist_len)
          p.hist[(size_t)r * p.hist_len + (j - 2)] = tk == kEmpty ? INFINITY : float_of_ord((uint32_t)(tk >> 32));
      }
    }
    __syncthreads();
  }
  if (FN >= 5) {
    at_decide(p, j, mode, stk, sdone);
    __syncthreads();
  }

  // A warp takes 32 consecutive particles; lane l evaluates particle qb + l.  Rows
  // move between global and shared memory one particle at a time over the lanes
  // (coalesced), the fitness runs a lane per particle from the shared-memory rows.
  const size_t total = (size_t)p.R * p.M;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t qb = (size_t)blockIdx.x * blockDim.x + (size_t)warp * 32; qb < total; qb += stride) {
    const size_t q = qb + lane;
    const bool valid = q < total;
    const int nv = (int)(total - qb < 32 ? total - qb : 32);
    int r = 0, pi = 0, g = 0;
    unsigned par = 0;
    float pf = INFINITY;
    bool live = false;   // a particle of a run that has not stopped
    if (valid) {
      r = (int)(q / p.M);
      pi = (int)(q - (size_t)r * p.M);
      g = pi / p.N;
      par = p.pcur[q];
      pf = p.Pfit[q];
      live = sdone[r] == 0;
    }
    if (mode & kUpdate) {
      // this lane's particle: inertia and random factors (one Philox draw)
      float w = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
      if (valid) {
        const float* hy = p.hyper + ((size_t)r * p.G + g) * 6;
        const float c1 = hy[0], c2 = hy[1], c3 = hy[2], w_init = hy[3], w_end = hy[4];
        const int k = j - 1;
        w = w_init - (w_init - w_end) / (float)p.K * (float)k;
        const uint4 rr = draw(p.key0, p.key1, (uint32_t)k, (uint32_t)pi, kStreamVel, cyc, p.run_id + (uint32_t)r);
        a1 = c1 * u01(rr.x);
        a2 = c2 * u01(rr.y);
        a3 = c3 * u01(rr.z);
      }
      // kLaneBatch particles at a time, all their loads issued before any is used
      for (int t0 = 0; t0 < nv; t0 += kLaneBatch) {
        float wt[kLaneBatch], a1t[kLaneBatch], a2t[kLaneBatch], a3t[kLaneBatch], vl[kLaneBatch];
        bool need_T[kLaneBatch], move[kLaneBatch];
        const float *gr[kLaneBatch], *tr[kLaneBatch], *pr[kLaneBatch];
        float *xr[kLaneBatch], *vr[kLaneBatch], *st[kLaneBatch];
#pragma unroll
        for (int u = 0; u < kLaneBatch; ++u) {
          const int t = min(t0 + u, nv - 1);
          wt[u] = __shfl_sync(full, w, t);
          a1t[u] = __shfl_sync(full, a1, t);
          a2t[u] = __shfl_sync(full, a2, t);
          a3t[u] = __shfl_sync(full, a3, t);
          const int rt = __shfl_sync(full, r, t), gt = __shfl_sync(full, g, t);
          const unsigned part = __shfl_sync(full, par, t);
          move[u] = t0 + u < nv && __shfl_sync(full, (int)live, t) != 0;
          const size_t qt = qb + t;
          const float* hy = p.hyper + ((size_t)rt * p.G + gt) * 6;
          need_T[u] = hy[2] != 0.0f;
          vl[u] = hy[5];
          gr[u] = key_row(p, rt, sgk[(size_t)rt * p.G + gt]);
          tr[u] = key_row(p, rt, stk[rt]);
          xr[u] = p.X + qt * p.Dp;
          vr[u] = p.V + qt * p.Dp;
          pr[u] = p.P + ((size_t)part * total + qt) * p.Dp;
          st[u] = swarp + (size_t)t * (D + 1);
        }
        for (int i = lane; i < D; i += 32) {
          const int ax = coord_axis(p, i);
          const float ext = axis_sel(ax, p.hi - p.lo, p.hi2 - p.lo2, p.hi3 - p.lo3);
          const float blo = axis_sel(ax, p.lo, p.lo2, p.lo3), bhi = axis_sel(ax, p.hi, p.hi2, p.hi3);
          float x[kLaneBatch], v[kLaneBatch], pb[kLaneBatch], gb[kLaneBatch], tb[kLaneBatch];
#pragma unroll
          for (int u = 0; u < kLaneBatch; ++u) {
            x[u] = xr[u][i];
            v[u] = vr[u][i];
            pb[u] = pr[u][i];
            gb[u] = gr[u] ? gr[u][i] : 0.0f;
            tb[u] = (need_T[u] && tr[u]) ? tr[u][i] : 0.0f;
          }
#pragma unroll
          for (int u = 0; u < kLaneBatch; ++u) {
            if (move[u]) {
              const float bv = vl[u] * ext;
              float vv = wt[u] * v[u];
              vv = fmaf(a1t[u], pb[u] - x[u], vv);
              vv = fmaf(a2t[u], gb[u] - x[u], vv);
              if (need_T[u]) vv = fmaf(a3t[u], tb[u] - x[u], vv);
              vv = fminf(fmaxf(vv, -bv), bv);
              vr[u][i] = vv;
              const float xn = fminf(fmaxf(x[u] + vv, blo), bhi);
              xr[u][i] = xn;
              st[u][i] = xn;
            }
          }
        }
      }
      if (valid && pi == 0) {
        const unsigned long long* gk = sgk + (size_t)r * p.G;
        for (int gg = 0; gg < p.G; ++gg) {
          const unsigned long long kk = gk[gg];
          if (kk != kEmpty) atomicMin(&ck[r * p.G + gg], kk & ~(1ull << 31));
        }
      }
    } else {
      for (int t = 0; t < nv; ++t) {
        const float* xr = p.X + (qb + t) * p.Dp;
        float* st = swarp + (size_t)t * (D + 1);
        for (int i = lane; i < D; i += 32) st[i] = xr[i];
      }
    }
    __syncwarp();
    if (mode & kEval) {
      float F = 0.0f;
      int qcount = 0;
      if (live)
        F = FN == 5 ? poly_lane_pairs(srow, T, p.pts, reinterpret_cast<const ulonglong2*>(sedges), (E + 1) / 2,
                                      p.alpha, p.beta, qcount)
                    : sphere_lane(srow, T, p.pts, reinterpret_cast<const ulonglong2*>(sedges), (E + 1) / 2, p.alpha,
                                  p.beta, qcount);
      const bool improved = live && F < pf;
      unsigned npar = par;
      if (improved) {
        npar = par ^ 1u;
        pf = F;
        p.Pfit[q] = F;
        p.pcur[q] = (unsigned char)npar;
        p.pq[(size_t)npar * total + q] = qcount;
      }
      // improved rows into their new Pbest buffer, one particle at a time over the lanes
      unsigned imask = __ballot_sync(full, improved);
      while (imask) {
        const int t = __ffs(imask) - 1;
        imask &= imask - 1;
        const unsigned nt = __shfl_sync(full, npar, t);
        float* dst = p.P + ((size_t)nt * total + qb + t) * p.Dp;
        const float* st = swarp + (size_t)t * (D + 1);
        for (int i = lane; i < D; i += 32) dst[i] = st[i];
      }
      if (live && isfinite(pf)) atomicMin(&ck[r * p.G + g], make_key(pf, 1u, (uint32_t)pi, npar));
    }
    __syncwarp();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < RG; i += blockDim.x)
    if (ck[i] != kEmpty) atomicMin(&kcur[i], ck[i]);
}

__global__ void __launch_bounds__(kLaneThreads, 5) poly_lane_kernel(const BfParams p, int j, int mode) {
  extern __shared__ __align__(16) unsigned char smem[];
  path_lane_iter<5>(p, j, mode, smem);
}

__global__ void __launch_bounds__(kLaneThreads, 5) sphere_lane_kernel(const BfParams p, int j, int mode) {
  extern __shared__ __align__(16) unsigned char smem[];
  path_lane_iter<6>(p, j, mode, smem);
}

// ---------------------------------------------------------------------------
// Bests after iteration k (the last launch): Gbest rows and fitness per group, the
// Tbest row and fitness, the last history entry.  One block per (run, slot), slot
// G = Tbest.  Reads only; a later launch continues from the same keys.
// ---------------------------------------------------------------------------
__global__ void bf_finish_kernel(const BfParams p, int k) {
  const int r = blockIdx.x / (p.G + 1), s = blockIdx.x - r * (p.G + 1);
  const int RG = p.R * p.G;
  const unsigned long long* gk = p.keys + (size_t)(k % 3) * RG + (size_t)r * p.G;
  unsigned long long key;
  float* out;
  if (s < p.G) {
    key = k > 0 ? gk[s] : kEmpty;
    out = p.Gb + ((size_t)r * p.G + s) * p.Dp;
    if (threadIdx.x == 0) p.Gfit[(size_t)r * p.G + s] = key == kEmpty ? INFINITY : float_of_ord((uint32_t)(key >> 32));
  } else {
    key = k > 0 ? resolve_T(gk, p.G, p.thold[(size_t)((k + 1) % 2) * p.R + r]) : kEmpty;
    out = p.Tb + (size_t)r * p.Dp;
    const float tf = key == kEmpty ? INFINITY : float_of_ord((uint32_t)(key >> 32));
    if (threadIdx.x == 0) {
      p.Tfit[r] = tf;
      if (k >= 1 && k - 1 < p.hist_len) p.hist[(size_t)r * p.hist_len + (k - 1)] = tf;
    }
  }
  const float* src = key_row(p, r, key);
  for (int i = threadIdx.x; i < p.Dp; i += blockDim.x) out[i] = src ? src[i] : 0.0f;
}

// Objective 5 of n paths (pitch ldx floats): fitness and Q, one warp per path.
__global__ void poly_eval_kernel(const float* X, int ldx, int T, int n, float4 st, const float4* edges, int E,
                                 float alpha, int beta, float* F, int* Q) {
  const int nwarps = blockDim.x >> 5, lane = threadIdx.x & 31;
  const float pts[4] = {st.x, st.y, st.z, st.w};
  for (int i = blockIdx.x * nwarps + (threadIdx.x >> 5); i < n; i += gridDim.x * nwarps) {
    int q;
    const float f = poly_row(X + (size_t)i * ldx, T, pts, edges, E, alpha, beta, lane, q);
    if (lane == 0) {
      F[i] = f;
      if (Q) Q[i] = q;
    }
  }
}

// Objective 6 of n paths (pitch ldx floats): fitness and Q, one warp per path;
// spheres (cx, cy, cz, r) read from global memory.
__global__ void sphere_eval_kernel(const float* X, int ldx, int T, int n, float4 st, float2 tg, const float4* sph,
                                   int S, float alpha, int beta, float* F, int* Q) {
  const int nwarps = blockDim.x >> 5, lane = threadIdx.x & 31;
  const float pts[6] = {st.x, st.y, st.z, st.w, tg.x, tg.y};
  for (int i = blockIdx.x * nwarps + (threadIdx.x >> 5); i < n; i += gridDim.x * nwarps) {
    int q;
    const float f = sphere_row<false>(X + (size_t)i * ldx, T, pts, sph, S, alpha, beta, lane, q);
    if (lane == 0) {
      F[i] = f;
      if (Q) Q[i] = q;
    }
  }
}

// Fitness of n rows (pitch ldx floats), one warp per row.
template <int FN>
__global__ void bf_eval_kernel(const float* X, int ldx, int D, int n, float* F) {
  const int nwarps = blockDim.x >> 5, lane = threadIdx.x & 31;
  for (int i = blockIdx.x * nwarps + (threadIdx.x >> 5); i < n; i += gridDim.x * nwarps) {
    const float f = bf_row<FN>(X + (size_t)i * ldx, D, lane);
    if (lane == 0) F[i] = f;
  }
}

}  // namespace sepso

// ===========================================================================
// Host side: the sepso_bf_* C ABI.
// ===========================================================================
namespace sepso {
namespace {

thread_local std::string g_bf_error;

int bffail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int bffail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_bf_error = buf;
  return code;
}

#define BFCUDA(expr)                                                                         \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess) return bffail(SEPSO_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

size_t a256(size_t v) { return (v + 255) & ~size_t(255); }

struct BfLayout {
  size_t X, V, P, Pfit, pcur, keys, thold, hyper, ext, hist, Gb, Gfit, Tb, Tfit, edges, pts, warm, prevT, pq, at, total;
};

// Obstacle records a handle holds: polygon edges (objective 5) or spheres (6).
int obstacle_capacity(const sepso_bf_config& c) {
  return c.fn == 5 ? c.max_edges : (c.fn == 6 ? c.max_spheres : 0);
}

int padded(int D) { return (D + 3) & ~3; }

BfLayout bf_layout(const sepso_bf_config& c) {
  const size_t Dp = (size_t)padded(c.D), R = (size_t)c.runs, G = (size_t)c.G;
  const size_t RM = R * G * (size_t)c.N;
  BfLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += a256(bytes);
    return at;
  };
  L.X = take(RM * Dp * 4);
  L.V = take(RM * Dp * 4);
  L.P = take(2 * RM * Dp * 4);
  L.Pfit = take(RM * 4);
  L.pcur = take(RM);
  L.keys = take(3 * R * G * 8);
  L.thold = take(2 * R * 8);
  L.hyper = take(R * G * 6 * 4);
  L.ext = take(R * (G + 1) * Dp * 4);
  L.hist = take(R * (size_t)c.max_iters * 4);
  L.Gb = take(R * G * Dp * 4);
  L.Gfit = take(R * G * 4);
  L.Tb = take(R * Dp * 4);
  L.Tfit = take(R * 4);
  L.edges = take((size_t)obstacle_capacity(c) * 16);
  L.pts = take(32);
  L.warm = take(16);
  L.prevT = take(c.fn >= 5 ? R * Dp * 4 : 0);
  L.pq = take(c.fn >= 5 ? 2 * RM * 4 : 0);
  L.at = take(2 * R * 16);
  L.total = off;
  return L;
}

int bf_validate(const sepso_bf_config* c) {
  if (!c) return bffail(SEPSO_EINVAL, "NULL config");
  if (c->fn < 1 || c->fn > 6) return bffail(SEPSO_EINVAL, "fn=%d is not one of 1..6", c->fn);
  if (c->fn == 6) {
    if (c->D < 3 || c->D % 3) return bffail(SEPSO_EINVAL, "a 3D path needs D = 3T >= 3 (D=%d)", c->D);
    if (!(c->map_w > 0.0f) || !(c->map_h > 0.0f) || !(c->map_d > 0.0f) || !std::isfinite(c->map_w) ||
        !std::isfinite(c->map_h) || !std::isfinite(c->map_d))
      return bffail(SEPSO_EINVAL, "box %g x %g x %g", (double)c->map_w, (double)c->map_h, (double)c->map_d);
    if (!std::isfinite(c->alpha) || c->alpha < 0.0f) return bffail(SEPSO_EINVAL, "alpha=%g", (double)c->alpha);
    if (c->beta < 1 || c->beta > 8) return bffail(SEPSO_EINVAL, "beta=%d outside [1, 8]", c->beta);
    if (c->max_spheres < 0 || c->max_spheres > kMaxSpheres)
      return bffail(SEPSO_EINVAL, "max_spheres=%d outside [0, %d]", c->max_spheres, kMaxSpheres);
  }
  if (c->at_stall < 0) return bffail(SEPSO_EINVAL, "at_stall=%d is negative", c->at_stall);
  if (c->at_stall > 0 && c->fn < 5)
    return bffail(SEPSO_EINVAL, "Auto Truncation belongs to the path objectives (fn=%d)", c->fn);
  if (c->at_stall > 0 && (!std::isfinite(c->stall_tol) || c->stall_tol < 0.0f))
    return bffail(SEPSO_EINVAL, "stall_tol=%g", (double)c->stall_tol);
  if (c->fn == 5) {
    if (c->D < 2 || c->D % 2) return bffail(SEPSO_EINVAL, "a path needs an even D >= 2 (D=%d)", c->D);
    if (!(c->map_w > 0.0f) || !(c->map_h > 0.0f) || !std::isfinite(c->map_w) || !std::isfinite(c->map_h))
      return bffail(SEPSO_EINVAL, "map %g x %g", (double)c->map_w, (double)c->map_h);
    if (!std::isfinite(c->alpha) || c->alpha < 0.0f) return bffail(SEPSO_EINVAL, "alpha=%g", (double)c->alpha);
    if (c->beta < 1 || c->beta > 8) return bffail(SEPSO_EINVAL, "beta=%d outside [1, 8]", c->beta);
    if (c->max_edges < 0 || c->max_edges > kMaxEdges)
      return bffail(SEPSO_EINVAL, "max_edges=%d outside [0, %d]", c->max_edges, kMaxEdges);
  }
  if (c->D < 1 || c->D > kMaxD) return bffail(SEPSO_EINVAL, "D=%d outside [1, %d]", c->D, kMaxD);
  if (c->G < 1 || c->G > 32) return bffail(SEPSO_EINVAL, "G=%d outside [1, 32]", c->G);
  if (c->N < 1) return bffail(SEPSO_EINVAL, "N=%d below 1", c->N);
  if (c->runs < 1) return bffail(SEPSO_EINVAL, "runs=%d below 1", c->runs);
  if (c->max_iters < 1) return bffail(SEPSO_EINVAL, "max_iters=%d below 1", c->max_iters);
  if (c->fn <= 4 && (!std::isfinite(c->lo) || !std::isfinite(c->hi) || !(c->lo < c->hi)))
    return bffail(SEPSO_EINVAL, "box [%g, %g] is empty or not finite", (double)c->lo, (double)c->hi);
  if ((long long)c->runs * c->G > kMaxRG)
    return bffail(SEPSO_EINVAL, "runs x G = %lld above %d", (long long)c->runs * c->G, kMaxRG);
  const long long M = (long long)c->G * c->N;
  if (M + c->G + 1 >= (1ll << 30)) return bffail(SEPSO_EINVAL, "G x N = %lld above 2^30", M);
  if ((long long)c->runs * M > (1ll << 31) - 1) return bffail(SEPSO_EINVAL, "runs x G x N above 2^31");
  return SEPSO_OK;
}

template <int FN>
cudaError_t iter_attr(size_t smem) {
  return cudaFuncSetAttribute(bf_iter_kernel<FN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
template <int FN>
cudaError_t iter_occ(int* bps, int threads, size_t smem) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, bf_iter_kernel<FN>, threads, smem);
}

}  // namespace
}  // namespace sepso

using namespace sepso;

struct sepso_bf_ctx {
  sepso_bf_config c;
  BfLayout L;
  BfParams p;
  char* ws = nullptr;
  cudaStream_t stream = nullptr;
  int threads = 0, grid = 0, init_grid = 0;
  size_t smem = 0;
  int grid_lane = 0;  // > 0: a path objective runs on poly_lane_kernel / sphere_lane_kernel
  size_t smem_lane = 0;
  size_t smem_small = 0;  // > 0: whole runs go to bf_small_kernel
  int64_t k = -1;  // iterations done; -1 before the first run or state
  int64_t launches = 0;
  bool hyper_set = false;
  bool scene_set = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

cudaError_t launch_iter(sepso_bf_ctx* h, int j, int mode) {
  if (h->grid_lane > 0) {
    if (h->c.fn == 6)
      sphere_lane_kernel<<<h->grid_lane, kLaneThreads, h->smem_lane, h->stream>>>(h->p, j, mode);
    else
      poly_lane_kernel<<<h->grid_lane, kLaneThreads, h->smem_lane, h->stream>>>(h->p, j, mode);
    return cudaGetLastError();
  }
  switch (h->c.fn) {
    case 1: bf_iter_kernel<1><<<h->grid, h->threads, h->smem, h->stream>>>(h->p, j, mode); break;
    case 2: bf_iter_kernel<2><<<h->grid, h->threads, h->smem, h->stream>>>(h->p, j, mode); break;
    case 3: bf_iter_kernel<3><<<h->grid, h->threads, h->smem, h->stream>>>(h->p, j, mode); break;
    case 4: bf_iter_kernel<4><<<h->grid, h->threads, h->smem, h->stream>>>(h->p, j, mode); break;
    case 5: bf_iter_kernel<5><<<h->grid, h->threads, h->smem, h->stream>>>(h->p, j, mode); break;
    default: bf_iter_kernel<6><<<h->grid, h->threads, h->smem, h->stream>>>(h->p, j, mode); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_finish(sepso_bf_ctx* h, int k) {
  bf_finish_kernel<<<h->c.runs * (h->c.G + 1), 128, 0, h->stream>>>(h->p, k);
  return cudaGetLastError();
}

// Iterations k0 + 1 .. k0 + n from a whole-iteration boundary, then the bests.
int enqueue_iterations(sepso_bf_ctx* h, int k0, int n) {
  for (int i = 1; i <= n; ++i) BFCUDA(launch_iter(h, k0 + i, i == 1 ? kEval : (kUpdate | kEval)));
  BFCUDA(launch_iter(h, k0 + n + 1, kUpdate));
  BFCUDA(launch_finish(h, k0 + n));
  return SEPSO_OK;
}

// init + iterations 1..K + the bests, on h->stream.
int enqueue_run(sepso_bf_ctx* h) {
  if (h->smem_small > 0) {
    const int R = h->c.runs;
    const size_t sm = h->smem_small;
    switch (h->c.fn) {
      case 1: bf_small_kernel<1><<<R, 256, sm, h->stream>>>(h->p); break;
      case 2: bf_small_kernel<2><<<R, 256, sm, h->stream>>>(h->p); break;
      case 3: bf_small_kernel<3><<<R, 256, sm, h->stream>>>(h->p); break;
      default: bf_small_kernel<4><<<R, 256, sm, h->stream>>>(h->p); break;
    }
    BFCUDA(cudaGetLastError());
    BFCUDA(launch_finish(h, h->c.max_iters));
    return SEPSO_OK;
  }
  bf_init_kernel<<<h->init_grid, 256, 0, h->stream>>>(h->p);
  BFCUDA(cudaGetLastError());
  return enqueue_iterations(h, 0, h->c.max_iters);
}

}  // namespace

extern "C" {

const char* sepso_bf_last_error(void) { return g_bf_error.c_str(); }

int sepso_bf_workspace_size(const sepso_bf_config* c, size_t* bytes) {
  const int rc = bf_validate(c);
  if (rc) return rc;
  if (!bytes) return bffail(SEPSO_EINVAL, "NULL bytes");
  *bytes = bf_layout(*c).total;
  return SEPSO_OK;
}

int sepso_bf_create(const sepso_bf_config* c, void* workspace, size_t bytes, void* stream, sepso_bf_handle* out) {
  int rc = bf_validate(c);
  if (rc) return rc;
  if (!out) return bffail(SEPSO_EINVAL, "NULL handle pointer");
  const BfLayout L = bf_layout(*c);
  if (!workspace || bytes < L.total)
    return bffail(SEPSO_ENOSPC, "workspace of %zu bytes below the %zu needed", bytes, L.total);
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return bffail(SEPSO_ENOSPC, "workspace not 256-byte aligned");
  const int Dp = padded(c->D);
  const int edge_b = obstacle_capacity(*c) * 16;
  const size_t RG = (size_t)c->runs * c->G;
  const size_t keys_b = bf_keys_bytes((int)RG, c->runs);
  const long long rows_budget = (long long)kSmemTotal - (long long)keys_b - edge_b;
  if (rows_budget < (long long)Dp * 4)
    return bffail(SEPSO_ERANGE, "D=%d with %d obstacle records and %zu group keys exceeds shared memory", c->D,
                  obstacle_capacity(*c), RG);
  const int nwarps = (int)std::min<long long>(8, rows_budget / ((long long)Dp * 4));
  const size_t smem = keys_b + (size_t)edge_b + (size_t)nwarps * Dp * 4;
  int dev = 0, sms = 0, bps = 0;
  BFCUDA(cudaGetDevice(&dev));
  BFCUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaError_t e = cudaSuccess;
  switch (c->fn) {
    case 1: e = iter_attr<1>(smem); if (e == cudaSuccess) e = iter_occ<1>(&bps, nwarps * 32, smem); break;
    case 2: e = iter_attr<2>(smem); if (e == cudaSuccess) e = iter_occ<2>(&bps, nwarps * 32, smem); break;
    case 3: e = iter_attr<3>(smem); if (e == cudaSuccess) e = iter_occ<3>(&bps, nwarps * 32, smem); break;
    case 4: e = iter_attr<4>(smem); if (e == cudaSuccess) e = iter_occ<4>(&bps, nwarps * 32, smem); break;
    case 5: e = iter_attr<5>(smem); if (e == cudaSuccess) e = iter_occ<5>(&bps, nwarps * 32, smem); break;
    default: e = iter_attr<6>(smem); if (e == cudaSuccess) e = iter_occ<6>(&bps, nwarps * 32, smem); break;
  }
  if (e != cudaSuccess) return bffail(SEPSO_ECUDA, "iteration kernel attributes: %s", cudaGetErrorString(e));
  if (bps < 1) return bffail(SEPSO_ERANGE, "iteration kernel does not fit an SM (%zu bytes of shared memory)", smem);
  sepso_bf_ctx* h = new (std::nothrow) sepso_bf_ctx();
  if (!h) return bffail(SEPSO_ENOMEM, "host allocation");
  h->c = *c;
  h->L = L;
  h->ws = static_cast<char*>(workspace);
  h->stream = static_cast<cudaStream_t>(stream);
  h->threads = nwarps * 32;
  h->smem = smem;
  const long long RM = (long long)c->runs * c->G * c->N;
  h->grid = (int)std::min<long long>((RM + nwarps - 1) / nwarps, (long long)bps * sms);
  // Small swarms (a trial of the standard runs) run whole in one CTA per run.
  if (c->fn <= 4 && (long long)c->G * c->N * c->D <= kSmallMaxCoords) {
    const size_t M = (size_t)c->G * c->N;
    const size_t S = (size_t)c->D + 1;
    const size_t ss = ((3 * M * S + (size_t)c->G * S + S + M) * 4 + 7) / 8 * 8 + 8 * (2 * (size_t)c->G + 1);
    if (ss <= (size_t)kSmemTotal) {
      switch (c->fn) {
        case 1: e = cudaFuncSetAttribute(bf_small_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss); break;
        case 2: e = cudaFuncSetAttribute(bf_small_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss); break;
        case 3: e = cudaFuncSetAttribute(bf_small_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss); break;
        default: e = cudaFuncSetAttribute(bf_small_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss); break;
      }
      if (e != cudaSuccess) {
        delete h;
        return bffail(SEPSO_ECUDA, "small-swarm kernel attributes: %s", cudaGetErrorString(e));
      }
      h->smem_small = ss;
    }
  }
  // A lane per particle pays once there are enough particles to give every SM's
  // lanes work (below that, one path's tests spread over a warp finish sooner).
  if (c->fn >= 5 && c->D <= kLaneMaxD && RM >= (long long)kLaneMinPerSm * sms) {
    const size_t sl = keys_b + lane_obstacle_bytes(c->fn, obstacle_capacity(*c)) + (size_t)kLaneThreads * (c->D + 1) * 4;
    int bl = 0;
    const void* lk = c->fn == 6 ? (const void*)sphere_lane_kernel : (const void*)poly_lane_kernel;
    e = cudaFuncSetAttribute(lk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sl);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl, lk, kLaneThreads, sl);
    if (e != cudaSuccess) {
      delete h;
      return bffail(SEPSO_ECUDA, "lane kernel attributes: %s", cudaGetErrorString(e));
    }
    if (bl > 0) {
      h->smem_lane = sl;
      h->grid_lane = (int)std::min<long long>((RM + kLaneThreads - 1) / kLaneThreads, (long long)bl * sms);
    }
  }
  const long long init_items = RM * (Dp / 4);
  h->init_grid = (int)std::max<long long>(1, std::min<long long>((init_items + 255) / 256, 8ll * sms));
  BfParams& p = h->p;
  p.fn = c->fn;
  p.D = c->D;
  p.Dp = Dp;
  p.G = c->G;
  p.N = c->N;
  p.M = c->G * c->N;
  p.R = c->runs;
  p.K = c->max_iters;
  p.hist_len = c->max_iters;
  const bool path = c->fn >= 5;
  const int T = c->fn == 6 ? c->D / 3 : c->D / 2;
  p.lo = path ? 0.0f : c->lo;
  p.hi = path ? c->map_w : c->hi;
  p.half = path ? T : c->D;
  p.half2 = c->fn == 6 ? 2 * T : c->D;
  p.lo2 = path ? 0.0f : c->lo;
  p.hi2 = path ? c->map_h : c->hi;
  p.lo3 = path ? 0.0f : c->lo;
  p.hi3 = c->fn == 6 ? c->map_d : p.hi2;
  p.alpha = c->alpha;
  p.beta = c->beta;
  p.E = 0;
  p.key0 = (uint32_t)(c->seed & 0xffffffffu);
  p.key1 = (uint32_t)(c->seed >> 32);
  p.run_id = c->run_id;
  char* w = h->ws;
  p.X = reinterpret_cast<float*>(w + L.X);
  p.V = reinterpret_cast<float*>(w + L.V);
  p.P = reinterpret_cast<float*>(w + L.P);
  p.Pfit = reinterpret_cast<float*>(w + L.Pfit);
  p.pcur = reinterpret_cast<unsigned char*>(w + L.pcur);
  p.keys = reinterpret_cast<unsigned long long*>(w + L.keys);
  p.thold = reinterpret_cast<unsigned long long*>(w + L.thold);
  p.hyper = reinterpret_cast<const float*>(w + L.hyper);
  p.ext = reinterpret_cast<float*>(w + L.ext);
  p.hist = reinterpret_cast<float*>(w + L.hist);
  p.Gb = reinterpret_cast<float*>(w + L.Gb);
  p.Gfit = reinterpret_cast<float*>(w + L.Gfit);
  p.Tb = reinterpret_cast<float*>(w + L.Tb);
  p.Tfit = reinterpret_cast<float*>(w + L.Tfit);
  p.edges = reinterpret_cast<const float4*>(w + L.edges);
  p.pts = reinterpret_cast<const float*>(w + L.pts);
  p.warm = reinterpret_cast<const int*>(w + L.warm);
  p.prevT = reinterpret_cast<const float*>(w + L.prevT);
  p.at_stall = c->at_stall;
  p.stall_tol = c->stall_tol;
  p.pq = reinterpret_cast<int*>(w + L.pq);
  p.at_state = reinterpret_cast<int*>(w + L.at);
  e = cudaMemsetAsync(workspace, 0, L.total, h->stream);
  if (e != cudaSuccess) {
    delete h;
    return bffail(SEPSO_ECUDA, "workspace clear: %s", cudaGetErrorString(e));
  }
  *out = h;
  return SEPSO_OK;
}

int sepso_bf_destroy(sepso_bf_handle h) {
  if (!h) return SEPSO_OK;
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  delete h;
  return SEPSO_OK;
}

int sepso_bf_set_hyper(sepso_bf_handle h, const float* hyper, int32_t run) {
  if (!h || !hyper) return bffail(SEPSO_EINVAL, "NULL argument");
  if (run < -1 || run >= h->c.runs) return bffail(SEPSO_EINVAL, "run=%d outside [-1, %d)", run, h->c.runs);
  const int G = h->c.G;
  for (int i = 0; i < G * 6; ++i)
    if (!std::isfinite(hyper[i])) return bffail(SEPSO_EINVAL, "hyper-parameter %d is not finite", i);
  for (int g = 0; g < G; ++g)
    if (hyper[g * 6 + 5] < 0.0f) return bffail(SEPSO_EINVAL, "V_limit of group %d is negative", g);
  float* dst = reinterpret_cast<float*>(h->ws + h->L.hyper);
  const int r0 = run < 0 ? 0 : run, r1 = run < 0 ? h->c.runs : run + 1;
  for (int r = r0; r < r1; ++r)
    BFCUDA(cudaMemcpyAsync(dst + (size_t)r * G * 6, hyper, (size_t)G * 6 * 4, cudaMemcpyHostToDevice, h->stream));
  BFCUDA(cudaStreamSynchronize(h->stream));
  if (run < 0) h->hyper_set = true;
  return SEPSO_OK;
}

int sepso_bf_set_polygons(sepso_bf_handle h, const float* start, const float* target, const float* edges,
                          int32_t E) {
  if (!h || !start || !target || (E > 0 && !edges)) return bffail(SEPSO_EINVAL, "NULL argument");
  if (h->c.fn != 5) return bffail(SEPSO_EINVAL, "polygons belong to objective 5 (fn=%d)", h->c.fn);
  if (E < 0 || E > h->c.max_edges) return bffail(SEPSO_EINVAL, "E=%d outside [0, max_edges=%d]", E, h->c.max_edges);
  for (int i = 0; i < 2; ++i)
    if (!std::isfinite(start[i]) || !std::isfinite(target[i])) return bffail(SEPSO_EINVAL, "start/target not finite");
  for (int i = 0; i < 4 * E; ++i)
    if (!std::isfinite(edges[i])) return bffail(SEPSO_EINVAL, "edge coordinate %d is not finite", i);
  const float pts[4] = {start[0], start[1], target[0], target[1]};
  if (E > 0)
    BFCUDA(cudaMemcpyAsync(h->ws + h->L.edges, edges, (size_t)E * 16, cudaMemcpyHostToDevice, h->stream));
  BFCUDA(cudaMemcpyAsync(h->ws + h->L.pts, pts, 16, cudaMemcpyHostToDevice, h->stream));
  BFCUDA(cudaStreamSynchronize(h->stream));
  if (h->p.E != E && h->exec) {   // the captured launches carry the old edge count
    cudaGraphExecDestroy(h->exec);
    cudaGraphDestroy(h->graph);
    h->exec = nullptr;
    h->graph = nullptr;
  }
  h->p.E = E;
  h->scene_set = true;
  return SEPSO_OK;
}

int sepso_poly_evaluate(int32_t T, int32_t n, const float* X, int32_t ldx, const float* start, const float* target,
                        const float* edges, int32_t E, float alpha, int32_t beta, float* F, int32_t* Q,
                        void* stream) {
  if (T < 1 || n < 0 || ldx < 2 * T || E < 0 || beta < 1 || beta > 8 || !std::isfinite(alpha))
    return bffail(SEPSO_EINVAL, "T=%d, n=%d, ldx=%d, E=%d, beta=%d", T, n, ldx, E, beta);
  if (!start || !target) return bffail(SEPSO_EINVAL, "NULL start/target");
  if (n == 0) return SEPSO_OK;
  if (!X || !F || (E > 0 && !edges)) return bffail(SEPSO_EINVAL, "NULL argument");
  if (E > 0 && reinterpret_cast<uintptr_t>(edges) % 16) return bffail(SEPSO_EINVAL, "edges not 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = std::min((n + 7) / 8, 4096);
  poly_eval_kernel<<<grid, 256, 0, s>>>(X, ldx, T, n, make_float4(start[0], start[1], target[0], target[1]),
                                        reinterpret_cast<const float4*>(edges), E, alpha, beta, F, Q);
  BFCUDA(cudaGetLastError());
  return SEPSO_OK;
}

int sepso_bf_set_spheres(sepso_bf_handle h, const float* start, const float* target, const float* spheres,
                         int32_t S) {
  if (!h || !start || !target || (S > 0 && !spheres)) return bffail(SEPSO_EINVAL, "NULL argument");
  if (h->c.fn != 6) return bffail(SEPSO_EINVAL, "spheres belong to objective 6 (fn=%d)", h->c.fn);
  if (S < 0 || S > h->c.max_spheres)
    return bffail(SEPSO_EINVAL, "S=%d outside [0, max_spheres=%d]", S, h->c.max_spheres);
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(start[i]) || !std::isfinite(target[i])) return bffail(SEPSO_EINVAL, "start/target not finite");
  for (int i = 0; i < 4 * S; ++i)
    if (!std::isfinite(spheres[i])) return bffail(SEPSO_EINVAL, "sphere value %d is not finite", i);
  for (int o = 0; o < S; ++o)
    if (spheres[4 * o + 3] < 0.0f) return bffail(SEPSO_EINVAL, "sphere %d has a negative radius", o);
  const float pts[8] = {start[0], start[1], start[2], target[0], target[1], target[2], 0.0f, 0.0f};
  if (S > 0)
    BFCUDA(cudaMemcpyAsync(h->ws + h->L.edges, spheres, (size_t)S * 16, cudaMemcpyHostToDevice, h->stream));
  BFCUDA(cudaMemcpyAsync(h->ws + h->L.pts, pts, 32, cudaMemcpyHostToDevice, h->stream));
  BFCUDA(cudaStreamSynchronize(h->stream));
  if (h->p.E != S && h->exec) {   // the captured launches carry the old sphere count
    cudaGraphExecDestroy(h->exec);
    cudaGraphDestroy(h->graph);
    h->exec = nullptr;
    h->graph = nullptr;
  }
  h->p.E = S;
  h->scene_set = true;
  return SEPSO_OK;
}

int sepso_bf_set_warm_start(sepso_bf_handle h, const float* prevT, float pi_gamma, float pi_h, uint32_t cycle) {
  if (!h) return bffail(SEPSO_EINVAL, "NULL handle");
  if (h->c.fn < 5) return bffail(SEPSO_EINVAL, "warm starts belong to the path objectives (fn=%d)", h->c.fn);
  if (!std::isfinite(pi_gamma) || pi_gamma < 0.0f || pi_gamma > 1.0f)
    return bffail(SEPSO_EINVAL, "pi_gamma=%g outside [0, 1]", (double)pi_gamma);
  if (!std::isfinite(pi_h) || pi_h < 0.0f) return bffail(SEPSO_EINVAL, "pi_h=%g", (double)pi_h);
  if (cycle >= (1u << 24)) return bffail(SEPSO_EINVAL, "cycle=%u above 2^24 - 1", cycle);
  if (pi_gamma > 0.0f && !prevT) return bffail(SEPSO_EINVAL, "PI without a previous path");
  const int R = h->c.runs, D = h->c.D, Dp = h->p.Dp;
  if (prevT)
    for (long long i = 0; i < (long long)R * D; ++i)
      if (!std::isfinite(prevT[i])) return bffail(SEPSO_EINVAL, "prevT[%lld] is not finite", i);
  // Particles per group placed by PI: ceil(gamma N), in double precision.
  const int n_pi = prevT ? (int)std::min<double>(h->c.N, std::ceil((double)pi_gamma * (double)h->c.N)) : 0;
  int32_t words[4];
  words[0] = n_pi;
  std::memcpy(&words[1], &pi_h, 4);
  words[2] = (int32_t)cycle;
  words[3] = 0;
  if (prevT)
    BFCUDA(cudaMemcpy2DAsync(h->ws + h->L.prevT, (size_t)Dp * 4, prevT, (size_t)D * 4, (size_t)D * 4, R,
                             cudaMemcpyHostToDevice, h->stream));
  BFCUDA(cudaMemcpyAsync(h->ws + h->L.warm, words, 16, cudaMemcpyHostToDevice, h->stream));
  BFCUDA(cudaStreamSynchronize(h->stream));
  return SEPSO_OK;
}

int sepso_sphere_evaluate(int32_t T, int32_t n, const float* X, int32_t ldx, const float* start, const float* target,
                          const float* spheres, int32_t S, float alpha, int32_t beta, float* F, int32_t* Q,
                          void* stream) {
  if (T < 1 || n < 0 || ldx < 3 * T || S < 0 || beta < 1 || beta > 8 || !std::isfinite(alpha))
    return bffail(SEPSO_EINVAL, "T=%d, n=%d, ldx=%d, S=%d, beta=%d", T, n, ldx, S, beta);
  if (!start || !target) return bffail(SEPSO_EINVAL, "NULL start/target");
  if (n == 0) return SEPSO_OK;
  if (!X || !F || (S > 0 && !spheres)) return bffail(SEPSO_EINVAL, "NULL argument");
  if (S > 0 && reinterpret_cast<uintptr_t>(spheres) % 16) return bffail(SEPSO_EINVAL, "spheres not 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = std::min((n + 7) / 8, 4096);
  sphere_eval_kernel<<<grid, 256, 0, s>>>(X, ldx, T, n, make_float4(start[0], start[1], start[2], target[0]),
                                          make_float2(target[1], target[2]),
                                          reinterpret_cast<const float4*>(spheres), S, alpha, beta, F, Q);
  BFCUDA(cudaGetLastError());
  return SEPSO_OK;
}

int sepso_bf_run_async(sepso_bf_handle h, int32_t use_graph) {
  if (!h) return bffail(SEPSO_EINVAL, "NULL handle");
  if (!h->hyper_set) return bffail(SEPSO_ESTATE, "run before set_hyper for every run");
  if (h->c.fn == 5 && !h->scene_set) return bffail(SEPSO_ESTATE, "run before set_polygons");
  if (h->c.fn == 6 && !h->scene_set) return bffail(SEPSO_ESTATE, "run before set_spheres");
  if (!use_graph) {
    const int rc = enqueue_run(h);
    if (rc) return rc;
  } else {
    if (!h->exec) {
      cudaStream_t cap = nullptr;
      BFCUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      cudaStream_t keep = h->stream;
      h->stream = cap;
      cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      int rc = SEPSO_OK;
      if (e == cudaSuccess) rc = enqueue_run(h);
      cudaGraph_t g = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(cap, &g);
      h->stream = keep;
      cudaStreamDestroy(cap);
      if (e != cudaSuccess || e2 != cudaSuccess || rc) {
        if (g) cudaGraphDestroy(g);
        return rc ? rc : bffail(SEPSO_ECUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
      }
      h->graph = g;
      BFCUDA(cudaGraphInstantiate(&h->exec, g, 0));
    }
    BFCUDA(cudaGraphLaunch(h->exec, h->stream));
  }
  h->launches += h->c.max_iters + 3;
  h->k = h->c.max_iters;
  return SEPSO_OK;
}

int sepso_bf_step(sepso_bf_handle h, int32_t iters) {
  if (!h) return bffail(SEPSO_EINVAL, "NULL handle");
  if (iters < 0) return bffail(SEPSO_EINVAL, "iters=%d is negative", iters);
  if (h->k < 0) return bffail(SEPSO_ESTATE, "step before a run or a loaded state");
  if (h->k + iters > (1ll << 30)) return bffail(SEPSO_EINVAL, "iteration count above 2^30");
  if (iters == 0) return SEPSO_OK;
  const int rc = enqueue_iterations(h, (int)h->k, iters);
  if (rc) return rc;
  h->k += iters;
  h->launches += iters + 2;
  return SEPSO_OK;
}

int sepso_bf_sync(sepso_bf_handle h) {
  if (!h) return bffail(SEPSO_EINVAL, "NULL handle");
  BFCUDA(cudaStreamSynchronize(h->stream));
  return SEPSO_OK;
}

int sepso_bf_read(sepso_bf_handle h, int32_t run, float* best_x, float* best_fit, int32_t* iters) {
  if (!h) return bffail(SEPSO_EINVAL, "NULL handle");
  if (run < 0 || run >= h->c.runs) return bffail(SEPSO_EINVAL, "run=%d outside [0, %d)", run, h->c.runs);
  if (h->k < 0) return bffail(SEPSO_ESTATE, "read before a run");
  if (best_x)
    BFCUDA(cudaMemcpyAsync(best_x, h->p.Tb + (size_t)run * h->p.Dp, (size_t)h->c.D * 4, cudaMemcpyDeviceToHost,
                           h->stream));
  if (best_fit) BFCUDA(cudaMemcpyAsync(best_fit, h->p.Tfit + run, 4, cudaMemcpyDeviceToHost, h->stream));
  int32_t st[4] = {0, 0, 0, 0};
  if (h->c.at_stall > 0)   // the state the last whole launch (k + 1) left
    BFCUDA(cudaMemcpyAsync(st, h->p.at_state + ((size_t)((h->k + 1) % 2) * h->c.runs + run) * 4, 16,
                           cudaMemcpyDeviceToHost, h->stream));
  BFCUDA(cudaStreamSynchronize(h->stream));
  if (iters) *iters = st[2] ? st[3] : (int32_t)h->k;
  return SEPSO_OK;
}

int sepso_bf_history(sepso_bf_handle h, int32_t run, float* hist) {
  if (!h || !hist) return bffail(SEPSO_EINVAL, "NULL argument");
  if (run < 0 || run >= h->c.runs) return bffail(SEPSO_EINVAL, "run=%d outside [0, %d)", run, h->c.runs);
  BFCUDA(cudaMemcpyAsync(hist, h->p.hist + (size_t)run * h->p.hist_len, (size_t)h->p.hist_len * 4,
                         cudaMemcpyDeviceToHost, h->stream));
  BFCUDA(cudaStreamSynchronize(h->stream));
  return SEPSO_OK;
}

int64_t sepso_bf_launch_count(sepso_bf_handle h) { return h ? h->launches : -1; }

const char* sepso_bf_kernel_name(sepso_bf_handle h) {
  if (!h) return "";
  if (h->smem_small > 0) return "bf_small_kernel (runs), bf_iter_kernel (steps)";
  if (h->grid_lane > 0) return h->c.fn == 6 ? "sphere_lane_kernel" : "poly_lane_kernel";
  static const char* names[] = {"", "bf_iter_kernel<1>", "bf_iter_kernel<2>", "bf_iter_kernel<3>",
                                "bf_iter_kernel<4>", "bf_iter_kernel<5>", "bf_iter_kernel<6>"};
  return names[h->c.fn];
}

int sepso_bf_get_state(sepso_bf_handle h, int32_t run, float* X, float* V, float* P, float* Pfit, float* Gb,
                       float* Gfit, float* Tb, float* Tfit, int32_t* k) {
  if (!h) return bffail(SEPSO_EINVAL, "NULL handle");
  if (run < 0 || run >= h->c.runs) return bffail(SEPSO_EINVAL, "run=%d outside [0, %d)", run, h->c.runs);
  if (h->k < 0) return bffail(SEPSO_ESTATE, "no state before a run");
  const BfParams& p = h->p;
  const size_t D4 = (size_t)p.D * 4, Dp4 = (size_t)p.Dp * 4, M = (size_t)p.M, RM = (size_t)p.R * M;
  const size_t q0 = (size_t)run * M;
  cudaStream_t s = h->stream;
  if (X) BFCUDA(cudaMemcpy2DAsync(X, D4, p.X + q0 * p.Dp, Dp4, D4, M, cudaMemcpyDeviceToHost, s));
  if (V) BFCUDA(cudaMemcpy2DAsync(V, D4, p.V + q0 * p.Dp, Dp4, D4, M, cudaMemcpyDeviceToHost, s));
  std::vector<float> P0, P1;
  std::vector<unsigned char> par;
  if (P) {
    P0.resize(M * p.D);
    P1.resize(M * p.D);
    par.resize(M);
    BFCUDA(cudaMemcpy2DAsync(P0.data(), D4, p.P + q0 * p.Dp, Dp4, D4, M, cudaMemcpyDeviceToHost, s));
    BFCUDA(cudaMemcpy2DAsync(P1.data(), D4, p.P + (RM + q0) * p.Dp, Dp4, D4, M, cudaMemcpyDeviceToHost, s));
    BFCUDA(cudaMemcpyAsync(par.data(), p.pcur + q0, M, cudaMemcpyDeviceToHost, s));
  }
  if (Pfit) BFCUDA(cudaMemcpyAsync(Pfit, p.Pfit + q0, M * 4, cudaMemcpyDeviceToHost, s));
  if (Gb)
    BFCUDA(cudaMemcpy2DAsync(Gb, D4, p.Gb + (size_t)run * p.G * p.Dp, Dp4, D4, p.G, cudaMemcpyDeviceToHost, s));
  if (Gfit) BFCUDA(cudaMemcpyAsync(Gfit, p.Gfit + (size_t)run * p.G, (size_t)p.G * 4, cudaMemcpyDeviceToHost, s));
  if (Tb) BFCUDA(cudaMemcpyAsync(Tb, p.Tb + (size_t)run * p.Dp, D4, cudaMemcpyDeviceToHost, s));
  if (Tfit) BFCUDA(cudaMemcpyAsync(Tfit, p.Tfit + run, 4, cudaMemcpyDeviceToHost, s));
  BFCUDA(cudaStreamSynchronize(s));
  if (P)
    for (size_t i = 0; i < M; ++i)
      std::memcpy(P + i * p.D, (par[i] ? P1 : P0).data() + i * p.D, D4);
  if (k) *k = (int32_t)h->k;
  return SEPSO_OK;
}

int sepso_bf_set_state(sepso_bf_handle h, int32_t run, const float* X, const float* V, const float* P,
                       const float* Pfit, const float* Gb, const float* Gfit, const float* Tb, const float* Tfit,
                       int32_t k) {
  if (!h || !X || !V || !P || !Pfit || !Gb || !Gfit || !Tb || !Tfit) return bffail(SEPSO_EINVAL, "NULL argument");
  if (run < 0 || run >= h->c.runs) return bffail(SEPSO_EINVAL, "run=%d outside [0, %d)", run, h->c.runs);
  if (k < 0) return bffail(SEPSO_EINVAL, "k=%d is negative", k);
  if (h->k >= 0 && h->c.runs > 1 && k != h->k)
    return bffail(SEPSO_EINVAL, "k=%d differs from the other runs' %lld", k, (long long)h->k);
  const BfParams& p = h->p;
  const size_t M = (size_t)p.M;
  for (size_t i = 0; i < M * p.D; ++i)
    if (!std::isfinite(X[i]) || !std::isfinite(V[i]) || !std::isfinite(P[i]))
      return bffail(SEPSO_EINVAL, "X, V or P holds a non-finite value at %zu", i);
  for (size_t i = 0; i < M; ++i)
    if (std::isnan(Pfit[i])) return bffail(SEPSO_EINVAL, "Pfit[%zu] is NaN", i);
  for (int g = 0; g < p.G; ++g)
    if (std::isnan(Gfit[g])) return bffail(SEPSO_EINVAL, "Gfit[%d] is NaN", g);
  if (std::isnan(Tfit[0])) return bffail(SEPSO_EINVAL, "Tfit is NaN");
  const size_t D4 = (size_t)p.D * 4, Dp4 = (size_t)p.Dp * 4, RM = (size_t)p.R * M;
  const size_t q0 = (size_t)run * M;
  const int RG = p.R * p.G;
  cudaStream_t s = h->stream;
  BFCUDA(cudaMemcpy2DAsync(p.X + q0 * p.Dp, Dp4, X, D4, D4, M, cudaMemcpyHostToDevice, s));
  BFCUDA(cudaMemcpy2DAsync(p.V + q0 * p.Dp, Dp4, V, D4, D4, M, cudaMemcpyHostToDevice, s));
  BFCUDA(cudaMemcpy2DAsync(p.P + q0 * p.Dp, Dp4, P, D4, D4, M, cudaMemcpyHostToDevice, s));
  BFCUDA(cudaMemcpy2DAsync(p.P + (RM + q0) * p.Dp, Dp4, P, D4, D4, M, cudaMemcpyHostToDevice, s));
  BFCUDA(cudaMemsetAsync(p.pcur + q0, 0, M, s));
  BFCUDA(cudaMemcpyAsync(p.Pfit + q0, Pfit, M * 4, cudaMemcpyHostToDevice, s));
  float* ext = p.ext + (size_t)run * (p.G + 1) * p.Dp;
  BFCUDA(cudaMemcpy2DAsync(ext, Dp4, Gb, D4, D4, p.G, cudaMemcpyHostToDevice, s));
  BFCUDA(cudaMemcpyAsync(ext + (size_t)p.G * p.Dp, Tb, D4, cudaMemcpyHostToDevice, s));
  // Keys naming the external rows: iteration k's group keys, the same keys already
  // posted (as previous holders) into iteration k + 1's table, and Tbest in both
  // holder slots (the next launches read it as iteration k's).
  auto host_key = [](float fit, uint32_t idx) -> unsigned long long {
    if (!(fit < INFINITY)) return kEmpty;
    uint32_t u;
    std::memcpy(&u, &fit, 4);
    const uint32_t o = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)o << 32) | ((unsigned long long)(idx & 0x3fffffffu) << 1);
  };
  std::vector<unsigned long long> gk((size_t)p.G);
  for (int g = 0; g < p.G; ++g) gk[g] = host_key(Gfit[g], (uint32_t)(p.M + g));
  const unsigned long long tk = host_key(Tfit[0], (uint32_t)(p.M + p.G));
  unsigned long long* keys = p.keys;
  BFCUDA(cudaMemcpyAsync(keys + (size_t)(k % 3) * RG + (size_t)run * p.G, gk.data(), (size_t)p.G * 8,
                         cudaMemcpyHostToDevice, s));
  BFCUDA(cudaMemcpyAsync(keys + (size_t)((k + 1) % 3) * RG + (size_t)run * p.G, gk.data(), (size_t)p.G * 8,
                         cudaMemcpyHostToDevice, s));
  BFCUDA(cudaMemcpyAsync(p.thold + run, &tk, 8, cudaMemcpyHostToDevice, s));
  BFCUDA(cudaMemcpyAsync(p.thold + (size_t)p.R + run, &tk, 8, cudaMemcpyHostToDevice, s));
  if (h->c.at_stall > 0) {   // a loaded state starts with no stall and no stop
    float inf = INFINITY;
    int32_t fresh[4] = {0, 0, 0, 0};
    std::memcpy(&fresh[1], &inf, 4);
    for (int slot = 0; slot < 2; ++slot)
      BFCUDA(cudaMemcpyAsync(p.at_state + ((size_t)slot * p.R + run) * 4, fresh, 16, cudaMemcpyHostToDevice, s));
  }
  h->k = k;
  BFCUDA(launch_finish(h, k));
  BFCUDA(cudaStreamSynchronize(s));
  h->launches += 1;
  return SEPSO_OK;
}

int sepso_bf_evaluate(int32_t fn, int32_t D, int32_t n, const float* X, int32_t ldx, float* F, void* stream) {
  if (fn < 1 || fn > 4)
    return bffail(SEPSO_EINVAL, "fn=%d is not one of BF1..BF4 (paths: sepso_poly_evaluate, sepso_sphere_evaluate)", fn);
  if (D < 1 || n < 0 || ldx < D) return bffail(SEPSO_EINVAL, "D=%d, n=%d, ldx=%d", D, n, ldx);
  if (n == 0) return SEPSO_OK;
  if (!X || !F) return bffail(SEPSO_EINVAL, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = std::min((n + 7) / 8, 4096);
  switch (fn) {
    case 1: bf_eval_kernel<1><<<grid, 256, 0, s>>>(X, ldx, D, n, F); break;
    case 2: bf_eval_kernel<2><<<grid, 256, 0, s>>>(X, ldx, D, n, F); break;
    case 3: bf_eval_kernel<3><<<grid, 256, 0, s>>>(X, ldx, D, n, F); break;
    default: bf_eval_kernel<4><<<grid, 256, 0, s>>>(X, ldx, D, n, F); break;
  }
  BFCUDA(cudaGetLastError());
  return SEPSO_OK;
}

}  // extern "C"
