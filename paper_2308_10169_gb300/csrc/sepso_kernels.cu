// sepso_kernels.cu -- CUDA kernels of the SEPSO planner for GB300 (sm_103a).
//
//   swarm_kernel     one cooperative persistent launch runs whole planning cycles
//                    (or plain continuation steps) of R independent swarms:
//                    Algorithm 1 of the paper (fitness, P/G/T update,
//                    Eq. TOF_omega, Eq. TOF_V with clip, Eq. TOF_X with clip),
//                    Priori Initialization (Sec. 3.3.3) and Auto Truncation
//                    (Sec. 3.3.4), all on the device.
//   evaluate_kernel  fitness (Eqs. path_fit / lenth / penalty) of a batch of paths.
//   advance_kernel   the dynamic scene step (Fig. PP caption).
//   hsef_*_kernel    the outer H-swarm of HSEF (Sec. 3.2.1, Eq. fit_h).
//
// Work split of swarm_kernel: run r owns C = G * cpg CTAs; CTA (g, q) owns
// particles [q * ppc, q * ppc + ppc) of group g and keeps their X, V, P rows in
// shared memory for the whole launch.  Each iteration every particle whose Pbest
// is below its group's best leaves its row in a parity-double-buffered slot and
// folds its key (fitness bits, index, Q) into the group's word with a 64-bit
// atomic min; each CTA then arrives at the run's monotone barrier counter; after
// the barrier every CTA reads the same G words, so all CTAs hold identical Gbest
// / Tbest values and take identical truncation decisions, and each fetches the
// winning rows it needs.  A slot of parity k & 1 is rewritten only at k + 2,
// after the barrier of k + 1, i.e. after every CTA has finished reading the
// slots of k.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cstdint>

#include "sepso_device.cuh"
#include "sepso_internal.h"

namespace sepso {

__host__ __device__ inline int align_up(int v, int a) { return (v + a - 1) / a * a; }

__host__ __device__ SmemLayout SmemLayout::make(int obst_f4, int ppc, int D, int T, int G, int tw) {
  SmemLayout s;
  // A 1 KB gap before the pair blocks: with the blocks at offset 0 the dynamic
  // workload's iterations measured 1% slower (same results); the cause is not known.
  int off = 1024;
  s.pairs = off;
  off = align_up(off + obst_f4 * 16, 16);  // circle-pair blocks or polygon edges
  s.win = off;
  off = align_up(off + tw * 8, 16);
  s.X = off;
  off = align_up(off + ppc * D * 4, 16);
  s.V = off;
  off = align_up(off + ppc * D * 4, 16);
  s.P = off;
  off = align_up(off + ppc * D * 4, 16);
  s.R = off;
  off = align_up(off + ppc * 16, 16);
  s.Gown = off;
  off = align_up(off + D * 4, 16);
  s.Tb = off;
  off = align_up(off + D * 4, 16);
  s.Pfit = off;
  off += ppc * 4;
  s.PQ = off;
  off += ppc * 4;
  s.Q = off;
  off += ppc * 4;
  s.Imp = off;
  off += ppc * 4;
  s.Len = off;
  off += ppc * (T + 1) * 4;
  s.Gfit = off;
  off += G * 4;
  s.GQ = off;
  off += G * 4;
  s.Gsrc = off;
  off += G * 4;
  s.total = align_up(off, 16);
  return s;
}

// ---------------------------------------------------------------------------
// The Auto Truncation window test (Sec. 3.3.4, first criterion), run by one warp.
//
// The decision is the one a two-pass FP64 population standard deviation of the n
// newest ring entries (oldest first) takes against delta.  Each lane holds at most
// two entries (tw <= 64), FP32 values held as doubles; an FP32 pass over the warp
// gives the sum of squared deviations ss together with a bound on its rounding
// error, and settles every window whose deviation is not within that bound (plus
// a 1e-6 relative margin, far above the FP64 computation's own error) of the
// threshold n * delta^2; the rest, and windows with non-finite values, take the
// FP64 two-pass sums in ring order on lane 0.
//
// Error bound.  With u = 2^-24, L = adds on a summation path (<= 1 + 5 here) and
// g = (L + 4) u: |s - sum x| <= g A, A = sum |x|;  m = rn(s / n) is within
// e = (g + 2u) A / n of the true mean mu;  sum (x - m)^2 = SS + n (mu - m)^2 for
// the true SS; each rounded square carries at most 3u and the sum g, so
// ss (1 - 2g) - n e^2 <= SS <= ss (1 + 2g).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ bool window_std_below(const double* win, int tw, int n, int head, float delta,
                                 int lane) {
  if (!(delta > 0.0f)) return false;  // a standard deviation is never below 0 (or NaN)
  const int i0 = lane, i1 = lane + 32;
  const double w0 = i0 < n ? win[(head - n + i0 + 2 * tw) % tw] : 0.0;
  const double w1 = i1 < n ? win[(head - n + i1 + 2 * tw) % tw] : 0.0;
  const float x0 = (float)w0, x1 = (float)w1;
  // entries the kernel records are FP32 values; a window loaded with other doubles
  // goes to the FP64 sums
  const bool exact = __all_sync(0xffffffffu, (double)x0 == w0 && (double)x1 == w1);
  const float s = warp_sum_f32(x0 + x1);
  const float a = warp_sum_f32(fabsf(x0) + fabsf(x1));
  const float nf = (float)n;
  const float m = __fdiv_rn(s, nf);
  const float d0 = i0 < n ? __fsub_rn(x0, m) : 0.0f;
  const float d1 = i1 < n ? __fsub_rn(x1, m) : 0.0f;
  const float ss = warp_sum_f32(__fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1)));
  const float u = 5.9604645e-8f, g = 10.0f * u;
  const float A = a * (1.0f + g);
  const float e = (g + 2.0f * u) * A / nf;
  const float e64 = (nf + 2.0f) * 1.2e-16f * A / nf;
  const float thr = nf * delta * delta;
  const float hi = ss * (1.0f + 2.0f * g) + nf * e64 * e64;
  const float lo = ss * (1.0f - 2.0f * g) - nf * e * e;
  if (exact && isfinite(ss) && isfinite(A) && isfinite(thr) && isfinite(hi)) {
    if (hi < thr * (1.0f - 1e-6f)) return true;
    if (lo > thr * (1.0f + 1e-6f)) return false;
  }
  bool below = false;
  if (lane == 0) {
    double sum = 0.0;
    for (int i = 0; i < n; ++i) sum += win[(head - n + i + 2 * tw) % tw];
    const double mean = sum / (double)n;
    double sq = 0.0;
    for (int i = 0; i < n; ++i) {
      const double d = win[(head - n + i + 2 * tw) % tw] - mean;
      sq += d * d;
    }
    below = sqrt(sq / (double)n) < (double)delta;
  }
  return __shfl_sync(0xffffffffu, below ? 1 : 0, 0) != 0;
}

// ---------------------------------------------------------------------------
// The fused persistent iteration.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) swarm_kernel(const SwarmParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t s_mbar;
  __shared__ int s_stop;

  const SmemLayout L = SmemLayout::make(obstacle_f4(p.Omax, p.poly), p.ppc, p.D, p.T, p.G, p.tw);
  float4* sPairs = reinterpret_cast<float4*>(smem + L.pairs);
  double* sWin = reinterpret_cast<double*>(smem + L.win);
  float* sX = reinterpret_cast<float*>(smem + L.X);
  float* sV = reinterpret_cast<float*>(smem + L.V);
  float* sP = reinterpret_cast<float*>(smem + L.P);
  float* sR = reinterpret_cast<float*>(smem + L.R);
  int* sQi = reinterpret_cast<int*>(smem + L.Q);        // item mode: Q per particle
  float* sLen = reinterpret_cast<float*>(smem + L.Len);  // item mode: length per (particle, segment)
  float* sG = reinterpret_cast<float*>(smem + L.Gown);
  float* sT = reinterpret_cast<float*>(smem + L.Tb);
  float* sPfit = reinterpret_cast<float*>(smem + L.Pfit);
  int* sPQ = reinterpret_cast<int*>(smem + L.PQ);
  float* sGfit = reinterpret_cast<float*>(smem + L.Gfit);
  int* sGQ = reinterpret_cast<int*>(smem + L.GQ);
  int* sGsrc = reinterpret_cast<int*>(smem + L.Gsrc);

  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  const int T = p.T, D = p.D, G = p.G, N = p.N;
  const int b = blockIdx.x;
  const int r = b / p.C;
  const int cr = b - r * p.C;
  const int g = cr / p.cpg;
  const int q = cr - g * p.cpg;
  const int n0 = q * p.ppc;
  const int nl = max(0, min(p.ppc, N - n0));
  RunCtl* ctl = p.ctl + r;

  const float* hy = p.hyper + ((size_t)r * G + g) * 6;
  const float c1 = hy[0], c2 = hy[1], c3 = hy[2], w_init = hy[3], w_end = hy[4], vlim = hy[5];
  const float sx = p.pts[0], sy = p.pts[1], tx = p.pts[2], ty = p.pts[3];
  const uint32_t cycle = (uint32_t)ctl->cycle;
  const uint32_t run = ctl->run_id;

  // Obstacles -> shared memory through the bulk-copy engine: the scene's
  // circle-pair blocks, kept current by set_scene and the scene advance.
  if (tid == 0) mbar_init(&s_mbar, 1);
  __syncthreads();
  if (tid == 0 && p.O > 0) {
    const uint32_t bytes = (uint32_t)(p.poly ? p.O : pair_block_f4(p.O)) * 16u;
    mbar_expect_tx(&s_mbar, bytes);
    bulk_g2s(sPairs, p.poly ? p.circ : p.pairs, bytes, &s_mbar);
  }

  float* gX = p.X + ((size_t)r * p.M + (size_t)g * N + n0) * D;
  float* gV = p.V + ((size_t)r * p.M + (size_t)g * N + n0) * D;
  float* gP = p.P + ((size_t)r * p.M + (size_t)g * N + n0) * D;
  float* gPfit = p.Pfit + (size_t)r * p.M + (size_t)g * N + n0;
  int32_t* gPQ = p.PQ + (size_t)r * p.M + (size_t)g * N + n0;
  float* gGb = p.Gb + (size_t)r * G * D;  // G rows, kept current by the CTAs that win them
  float* gTb = p.Tb + (size_t)r * D;      // kept current likewise

  float Tfit;
  int TQ, k;
  // AT state, tracked by the lanes of warp 0
  int win_n = 0, win_head = 0, stall = 0;
  float prev_lfv = INFINITY;

  if (p.mode == kModePlan) {
    // Initialisation (Algorithm 1) with Priori Initialization (Sec. 3.3.3).
    const int n_pi = (p.use_pi && ctl->has_prev) ? p.n_pi : 0;
    const float* prevT = p.prevT + (size_t)r * D;
    const int nch = (D + 3) >> 2;
    for (int it = tid; it < nl * nch; it += nt) {
      const int i = it / nch, ch = it - i * nch;
      const int n = n0 + i;
      const uint32_t pid = (uint32_t)(g * N + n);
      const bool pi = n < n_pi;
      const uint4 ux = draw(p.key0, p.key1, (uint32_t)ch, pid, pi ? kStreamPI : kStreamInitX, cycle, run);
      const uint4 uv = draw(p.key0, p.key1, (uint32_t)ch, pid, kStreamInitV, cycle, run);
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int j = ch * 4 + l;
        if (j < D) {
          const float ext = (j < T) ? p.W : p.H;
          float x;
          if (pi) x = fminf(fmaxf(prevT[j] + (2.0f * lane_of(ux, l) - 1.0f) * p.pi_h, 0.0f), ext);
          else x = lane_of(ux, l) * ext;
          sX[i * D + j] = x;
          sP[i * D + j] = x;
          sV[i * D + j] = (2.0f * lane_of(uv, l) - 1.0f) * (vlim * ext);
        }
      }
    }
    for (int i = tid; i < nl; i += nt) {
      sPfit[i] = INFINITY;
      sPQ[i] = 0;
    }
    for (int j = tid; j < D; j += nt) {
      sG[j] = 0.0f;
      sT[j] = 0.0f;
      if (q == 0) gGb[g * D + j] = 0.0f;  // before this CTA's first publication
      if (cr == 0) gTb[j] = 0.0f;
    }
    for (int j = tid; j < G; j += nt) {
      sGfit[j] = INFINITY;
      sGQ[j] = 0;
    }
    Tfit = INFINITY;
    TQ = 0;
    k = 0;
    if (tid < 32 && p.at_mode == SEPSO_AT_STD_WINDOW) {
      if (cycle != 0) {
        win_n = ctl->win_n;
        win_head = ctl->win_head;
        for (int i = lane; i < p.tw; i += 32) sWin[i] = p.win[(size_t)r * p.tw + i];
      }
    }
  } else {
    for (int it = tid; it < nl * D; it += nt) {
      sX[it] = gX[it];
      sV[it] = gV[it];
      sP[it] = gP[it];
    }
    for (int i = tid; i < nl; i += nt) {
      sPfit[i] = gPfit[i];
      sPQ[i] = gPQ[i];
    }
    for (int j = tid; j < D; j += nt) {
      sG[j] = gGb[g * D + j];
      sT[j] = gTb[j];
    }
    for (int j = tid; j < G; j += nt) {
      sGfit[j] = p.Gfit[(size_t)r * G + j];
      sGQ[j] = p.GQ[(size_t)r * G + j];
    }
    Tfit = ctl->Tfit;
    TQ = ctl->TQ;
    k = ctl->k;
  }

  bool failed = false;
  const int K = circle_pairs(p.O);
  if (p.O > 0) {
    const bool landed = mbar_wait_bounded(&s_mbar, 0, kWaitLimitNs);
    if (__syncthreads_or(landed ? 0 : 1)) {
      failed = true;
      if (tid == 0) {
        ctl->status = SEPSO_ETIMEOUT;
        mbar_wait_bounded(&s_mbar, 0, kWaitLimitNs);  // once more: no copy in flight at exit
      }
    }
  } else {
    __syncthreads();
  }
  const float2* sNr2 = reinterpret_cast<const float2*>(sPairs + K);

  for (int i = tid; i < nl; i += nt) sQi[i] = 0;
  __syncthreads();
  const int nseg = T + 1;
  // Iterations already run by this run (across launches): they index the
  // barrier count and the rotation of the group words.
  const unsigned long long kbase = (unsigned long long)ctl->iters_total;
  const int rstride = D + 4;
  const bool need_T = c3 != 0.0f;  // the Tbest row enters this group's update
  int last_t_src = -2, last_tg = -1;
  size_t last_rbase = 0;
  int done = 0;
  while (!failed) {
    if (p.mode == kModeStep && done >= p.step_iters) break;
    ++k;
    ++done;
    // This iteration's R1..R3 (independent of the exchange), drawn by the last threads.
    for (int i = nt - 1 - tid; i < nl; i += nt) {
      const uint4 o = draw(p.key0, p.key1, (uint32_t)k, (uint32_t)(g * N + n0 + i), kStreamVel, cycle, run);
      sR[i * 4 + 0] = c1 * u01(o.x);
      sR[i * 4 + 1] = c2 * u01(o.y);
      sR[i * 4 + 2] = c3 * u01(o.z);
    }
    const unsigned long long gk = kbase + (unsigned long long)done;  // the run's iteration count
    const size_t rbase = ((size_t)r * 2 + (size_t)(gk & 1ull)) * p.M;    // candidate rows
    const size_t wbase = ((size_t)r * 3 + (size_t)(gk % 3ull)) * G;      // group words of gk
    const size_t wprev = ((size_t)r * 3 + (size_t)((gk + 2ull) % 3ull)) * G;  // of gk - 1

    // Fitness = F(X^k), Pbest test and publication, one lane group (lp lanes) per
    // particle: lanes take (segment, circle chunk) items, the group sums length
    // and Q with a fixed shuffle tree.  A particle whose Pbest is below its
    // group's current best writes its row and Q to its slot and folds its key
    // into the group word.
    if (p.items) {
      // (particle, segment, chunk) items over the whole CTA, then one warp per
      // particle sums its segment lengths in segment order and takes Q.
      if (p.poly) fitness_items_edges(sX, nl, T, D, sx, sy, tx, ty, sPairs, p.O, p.split, sQi, sLen);
      else fitness_items_pairs(sX, nl, T, D, sx, sy, tx, ty, sPairs, sNr2, K, p.split, sQi, sLen);
      __syncthreads();
    }
    {
      const int lp = p.items ? 32 : p.lp;
      const int ppw = 32 / lp;
      const int lsub = lane & (lp - 1);
      for (int i0 = warp * ppw; i0 < nl; i0 += nwarps * ppw) {
        const int i = i0 + lane / lp;
        const bool live = i < nl;
        float len = 0.0f;
        int qq = 0;
        if (p.items) {
          len = warp_len_sum(sLen + i * nseg, nseg, lane);  // lp = 32: the warp's one particle
          if (lsub == 0) {
            qq = sQi[i];
            sQi[i] = 0;  // ready for the next iteration (read again only after two barriers)
          }
        } else {
          if (p.poly)
            group_fitness_edges(sX + (live ? i : 0) * D, live, lp, T, p.split, p.O, sx, sy, tx, ty, sPairs, &len,
                                &qq);
          else
            group_fitness_pairs(sX + (live ? i : 0) * D, live, lp, T, p.split, K, sx, sy, tx, ty, sPairs, sNr2,
                                &len, &qq);
        }
        int imp = 0, pub = 0;
        float pf = INFINITY;
        int pq = 0;
        if (live && lsub == 0) {
          const float F = len + p.alpha * powi((float)qq, p.beta);
          pf = sPfit[i];
          pq = sPQ[i];
          if (F < pf) {
            imp = 1;
            pf = F;
            pq = qq;
            sPfit[i] = F;
            sPQ[i] = qq;
          }
          pub = pf < sGfit[g];
        }
        const int leader = lane & ~(lp - 1);
        imp = __shfl_sync(0xffffffffu, imp, leader);
        pub = __shfl_sync(0xffffffffu, pub, leader);
        if (live && (imp || pub)) {
          const size_t m = (size_t)g * N + n0 + i;
          float* slot = p.crows + (rbase + m) * rstride;
          for (int j = lsub; j < D; j += lp) {
            const float v = imp ? sX[i * D + j] : sP[i * D + j];
            if (imp) sP[i * D + j] = v;
            if (pub) slot[j] = v;
          }
          if (pub && lsub == 0) {
            slot[D] = __int_as_float(pq);
            red_min_u64(p.gword + wbase + g, best_key(pf, (uint32_t)(n0 + i), (uint32_t)pq));
          }
        }
      }
    }
    __syncthreads();
    // Arrive: the release orders this CTA's rows and keys before the arrival.
    if (tid == 0) red_release_add(&p.counter[r].count, 1u);

    // Barrier: every CTA of the run has arrived once per iteration, gk times in all.
    int timed_out = 0;
    if (tid == 0) {
      const unsigned int target = (unsigned int)p.C * (unsigned int)gk;
      timed_out = counter_wait_bounded(&p.counter[r].count, target, kWaitLimitNs) ? 0 : 1;
      fence_acq_rel_gpu();  // with the relaxed load that saw the count: an acquire
    }
    if (__syncthreads_or(timed_out)) {
      if (tid == 0) ctl->status = SEPSO_ETIMEOUT;
      failed = true;
      break;
    }

    // Group bests: a group improved when its word holds a key below its Gfit; the
    // winner is particle key_idx of that group (slot g * N + n).  The key carries
    // Q saturated at kQSat; the exact value is then read from the slot.
    for (int gg = tid; gg < G; gg += nt) {
      const unsigned long long key = __ldcg(p.gword + wbase + gg);
      int src = -1;
      if (key != kKeyEmpty && key_fit(key) < sGfit[gg]) {
        sGfit[gg] = key_fit(key);
        src = gg * N + key_idx(key);
        const int qs = key_q(key);
        sGQ[gg] = (qs < (int)kQSat) ? qs : __float_as_int(__ldcg(p.crows + (rbase + src) * rstride + D));
      }
      sGsrc[gg] = src;
    }
    if (cr == 0) {
      for (int gg = tid; gg < G; gg += nt) p.gword[wprev + gg] = kKeyEmpty;  // read by all during gk - 1
    }
    __syncthreads();

    // Tbest (every thread, identical registers).
    float tb = INFINITY;
    int tg = -1;
    for (int gg = 0; gg < G; ++gg) {
      const float v = sGfit[gg];
      if (v < tb) {
        tb = v;
        tg = gg;
      }
    }
    int t_src = -2;  // -2 unchanged; -1 the (unchanged) row of group tg; >= 0 a candidate slot
    if (tg >= 0 && tb < Tfit) {
      Tfit = tb;
      TQ = sGQ[tg];
      t_src = sGsrc[tg];
    }
    // This group's new Gbest row, and the persistent copies kept by the winners.
    const int gsrc = sGsrc[g];
    if (gsrc >= 0) {
      for (int j = tid; j < D; j += nt) sG[j] = __ldcg(p.crows + (rbase + gsrc) * rstride + j);
    }
    // (a winning particle's P row is final for this iteration: the update below
    // does not touch P)
    const int own_lo = g * N + n0, own_hi = g * N + n0 + nl;
    if (gsrc >= own_lo && gsrc < own_hi)
      for (int j = tid; j < D; j += nt) gGb[g * D + j] = sP[(gsrc - own_lo) * D + j];
    if (t_src >= own_lo && t_src < own_hi)
      for (int j = tid; j < D; j += nt) gTb[j] = sP[(t_src - own_lo) * D + j];
    if (t_src == -1 && tg == g && q == 0) {
      for (int j = tid; j < D; j += nt) gTb[j] = sG[j];  // group g did not improve: sG is stable
    }
    if (need_T) {
      if (t_src >= 0) {
        for (int j = tid; j < D; j += nt) sT[j] = __ldcg(p.crows + (rbase + t_src) * rstride + j);
      } else if (t_src == -1) {
        for (int j = tid; j < D; j += nt) sT[j] = __ldcg(gGb + tg * D + j);
      }
    }
    last_t_src = t_src;
    last_tg = tg;
    last_rbase = rbase;

    // Auto Truncation (Sec. 3.3.4) and the iteration cap, decided by warp 0 (its
    // lanes track the same window fill, head and stall counter).
    if (tid < 32) {
      int stop = 0;
      if (p.mode == kModePlan) {
        if (p.at_mode == SEPSO_AT_STD_WINDOW) {
          if (lane == 0) sWin[win_head] = (double)Tfit;
          __syncwarp();
          win_head = (win_head + 1) % p.tw;
          if (win_n < p.tw) ++win_n;
          if (win_n >= 2 && TQ == 0 && window_std_below(sWin, p.tw, win_n, win_head, p.delta, lane))
            stop = 1;
        } else if (p.at_mode == SEPSO_AT_STALL) {
          if (Tfit < prev_lfv - p.stall_tol) stall = 0;
          else ++stall;
          prev_lfv = Tfit;
          if (stall >= p.stall_iters && TQ == 0) stop = 1;
        }
        if (k >= p.max_iters) stop = 1;
      }
      if (tid == 0) s_stop = stop;
    }
    __syncthreads();
    if (s_stop) break;

    // Eq. TOF_omega, Eq. TOF_V (+ clip to V_range), Eq. TOF_X (+ clip to X_range).
    const float w = w_init - (w_init - w_end) / (float)p.max_iters * (float)k;
    for (int it = tid; it < nl * D; it += nt) {
      const int i = it / D;
      const int j = it - i * D;
      const float x = sX[it];
      float v = w * sV[it];
      v = fmaf(sR[i * 4 + 0], sP[it] - x, v);
      v = fmaf(sR[i * 4 + 1], sG[j] - x, v);
      if (need_T) v = fmaf(sR[i * 4 + 2], sT[j] - x, v);
      const float ext = (j < T) ? p.W : p.H;
      const float vmax = vlim * ext;
      v = fminf(fmaxf(v, -vmax), vmax);
      sV[it] = v;
      sX[it] = fminf(fmaxf(x + v, 0.0f), ext);
    }
    __syncthreads();
  }

  // Write back the swarm (state for sepso_step / sepso_get_state).
  for (int it = tid; it < nl * D; it += nt) {
    gX[it] = sX[it];
    gV[it] = sV[it];
    gP[it] = sP[it];
  }
  for (int i = tid; i < nl; i += nt) {
    gPfit[i] = sPfit[i];
    gPQ[i] = sPQ[i];
  }
  if (q == 0 && tid == 0) {
    p.Gfit[(size_t)r * G + g] = sGfit[g];
    p.GQ[(size_t)r * G + g] = sGQ[g];
  }
  if (cr == 0) {
    // The Tbest row: from this iteration's candidate slot if it changed in the
    // last iteration, else from the persistent copies written in earlier ones.
    const float* src = gTb;
    if (last_t_src >= 0) src = p.crows + (last_rbase + last_t_src) * (D + 4);
    else if (last_t_src == -1) src = gGb + last_tg * D;
    for (int j = tid; j < D; j += nt) sT[j] = __ldcg(src + j);
    __syncthreads();
    for (int j = tid; j < D; j += nt) {
      gTb[j] = sT[j];
      if (p.mode == kModePlan) {
        p.res_wp[(size_t)r * D + j] = sT[j];
        p.prevT[(size_t)r * D + j] = sT[j];
      }
    }
    if (tid == 0) {
      ctl->Tfit = Tfit;
      ctl->TQ = TQ;
      ctl->k = k;
      ctl->iters_total += done;
      if (p.mode == kModePlan) {
        ctl->plans_total += 1;
        float len = 0.0f;
        for (int s = 0; s < nseg; ++s) {
          const float ax = (s == 0) ? sx : sT[s - 1];
          const float ay = (s == 0) ? sy : sT[T + s - 1];
          const float bx = (s == T) ? tx : sT[s];
          const float by = (s == T) ? ty : sT[T + s];
          const float dx = bx - ax, dy = by - ay;
          len += sqrtf(fmaf(dx, dx, dy * dy));
        }
        sepso_result* res = p.res + r;
        res->cost = Tfit;
        res->length = len;
        res->Q = TQ;
        res->iters = k;
        res->status = failed ? SEPSO_ETIMEOUT : ctl->status;
        ctl->has_prev = 1;
        ctl->cycle = (int32_t)cycle + 1;
        ctl->stall = stall;
        ctl->prev_lfv = prev_lfv;
        if (p.at_mode == SEPSO_AT_STD_WINDOW) {
          ctl->win_n = win_n;
          ctl->win_head = win_head;
          for (int i = 0; i < p.tw; ++i) p.win[(size_t)r * p.tw + i] = sWin[i];
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Cluster form of the fused iteration, for swarms in which no group's update uses
// Tbest (C3 = 0 in every group, as in the sampled and HSEF-evolved settings): Eq.
// TOF_V then needs only the group's own Gbest, so the exchange that gates each
// update can stay inside the group.  Run r, group g owns one thread-block cluster
// of S = p.cpg CTAs (cluster rank q owns particles [q ppc, q ppc + ppc)).  Per
// iteration k:
//   1. fitness of X^k; the Pbest test is kept aside (F, Q, improved?), P is not
//      written yet;
//   2. warp 0 reads the G group records of iteration k - 1 (each group's Gfit and
//      Q after its best update, published one iteration earlier), updates Tbest
//      with them and takes the Auto Truncation decision of k - 1, as Algorithm 1
//      takes it right after that best update;
//   3. each CTA writes its best candidate key (the lowest-index particle of lowest
//      post-update Pbest fitness below the group's Gfit), its decision word and
//      the candidate's row into its slot in every CTA of the cluster (distributed
//      shared memory), then the cluster barrier;
//   4. the decision is the largest word of the cluster (0 go on, 1 stop at k - 1,
//      2 failed), so every CTA takes it alike; on a stop at k - 1 iteration k is
//      discarded: X and V of k - 1 are still in the other buffer, P and Gbest are
//      untouched, and Tbest of k - 1 is the result (Algorithm 1 returns Tbest
//      after the stopping iteration's best update and never applies its update);
//   5. otherwise the Pbest updates are applied, the new Gbest is the lowest key of
//      the cluster's slots (its row from the winner's slot), rank 0 publishes the
//      group's record of k, and the update of Eqs. TOF_omega, TOF_V and TOF_X runs.
// The iteration cap (or the step count) ends the loop after step 5; the groups
// then meet once at the run's end counter, and CTA 0 of the run applies the last
// records to Tbest and takes its row from the holder group's Gbest row.  The
// decisions, bests and arithmetic are those of swarm_kernel, so both forms give
// identical results.  Slots of parity k & 1 are rewritten at k + 2, after the
// cluster barrier of k + 1, which every CTA reaches only after reading them.
// ---------------------------------------------------------------------------
// Floats of one exchange slot: D row values, Q, the decision word and the 64-bit key,
// rounded up to whole 16-byte vectors.
__host__ __device__ inline int cluster_slot_stride(int D) { return (D + 4 + 3) & ~3; }

__host__ __device__ ClusterLayout ClusterLayout::make(int obst_f4, int ppc, int D, int T, int G, int tw, int S,
                                                      int spec) {
  ClusterLayout s;
  int off = 1024;
  s.pairs = off;
  off = align_up(off + obst_f4 * 16, 16);  // circle-pair blocks or polygon edges
  s.win = off;
  off = align_up(off + tw * 8, 16);
  s.rec = off;
  off = align_up(off + G * 8, 16);
  s.X0 = off;
  off = align_up(off + ppc * D * 4, 16);
  s.X1 = s.X0;
  if (spec) {
    s.X1 = off;
    off = align_up(off + ppc * D * 4, 16);
  }
  s.V0 = off;
  off = align_up(off + ppc * D * 4, 16);
  s.V1 = s.V0;
  if (spec) {
    s.V1 = off;
    off = align_up(off + ppc * D * 4, 16);
  }
  s.P = off;
  off = align_up(off + ppc * D * 4, 16);
  s.R = off;
  off = align_up(off + ppc * 16, 16);
  s.Gown = off;
  off = align_up(off + D * 4, 16);
  s.xrow = off;  // slots: the candidate row, its Q, the decision word, the key (cluster_slot_stride floats)
  off = align_up(off + 2 * S * cluster_slot_stride(D) * 4, 16);
  s.Pfit = off;
  off += ppc * 4;
  s.PQ = off;
  off += ppc * 4;
  s.Q = off;
  off += ppc * 4;
  s.F = off;
  off += ppc * 4;
  s.FQ = off;
  off += ppc * 4;
  s.Imp = off;
  off += ppc * 4;
  s.xdec = off;
  off += 2 * S * 4;
  s.Len = off;
  off += ppc * (T + 1) * 4;
  s.total = align_up(off, 16);
  return s;
}

// Tbest from the G group records held by lanes 0..G-1 of warp 0 (strictly better,
// lowest group first), then Auto Truncation of that iteration; returns the stop
// decision.  Every lane ends with the same values.
__device__ __forceinline__ bool cluster_tbest_at(const SwarmParams& p, unsigned long long rec, int lane, float& Tfit,
                                                 int& TQ, int& tholder, double* sWin, int& win_n, int& win_head,
                                                 int& stall, float& prev_lfv) {
  const bool has = lane < p.G;
  const float f = has ? rec_fit(rec) : INFINITY;
  // lowest (fitness, group): fitness values are non-negative, their bits order like them
  unsigned long long key = has ? (((unsigned long long)__float_as_uint(f) << 32) | (unsigned)lane) : ~0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
    key = other < key ? other : key;
  }
  const int tg = (int)(key & 0xffffffffu);
  const float tb = __uint_as_float((uint32_t)(key >> 32));
  const int tq = __shfl_sync(0xffffffffu, has ? rec_q(rec) : 0, tg & 31);
  if (tb < Tfit) {
    Tfit = tb;
    TQ = tq;
    tholder = tg;
  }
  bool stop = false;
  if (p.mode == kModePlan) {
    if (p.at_mode == SEPSO_AT_STD_WINDOW) {
      if (lane == 0) sWin[win_head] = (double)Tfit;
      __syncwarp();
      win_head = (win_head + 1) % p.tw;
      if (win_n < p.tw) ++win_n;
      if (win_n >= 2 && TQ == 0 && window_std_below(sWin, p.tw, win_n, win_head, p.delta, lane)) stop = true;
    } else if (p.at_mode == SEPSO_AT_STALL) {
      if (Tfit < prev_lfv - p.stall_tol) stall = 0;
      else ++stall;
      prev_lfv = Tfit;
      if (stall >= p.stall_iters && TQ == 0) stop = true;
    }
  }
  return stop;
}

// Lanes 0..G-1 of warp 0: the records of iteration gk (prefetched in rec), waited
// for with the time limit; true when one did not come.
__device__ __forceinline__ bool cluster_wait_records(const unsigned long long* slot, int lane, int G,
                                                     unsigned long long gk, unsigned long long& rec) {
  int late = 0;
  if (lane < G) {
    const uint32_t want = rec_tag(gk);
    if (rec_tag_of(rec) != want) {
      const unsigned long long t0 = global_ns();
      do {
        rec = ld_relaxed_u64(slot + lane);
      } while (rec_tag_of(rec) != want && global_ns() - t0 <= kWaitLimitNs);
      late = rec_tag_of(rec) != want;
    }
  }
  return __any_sync(0xffffffffu, late) != 0;
}

__global__ void __launch_bounds__(512) swarm_cluster_kernel(const SwarmParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t s_mbar;
  __shared__ unsigned long long s_key;
  __shared__ uint32_t s_dec;

  const int S = p.cpg;
  const ClusterLayout L = ClusterLayout::make(obstacle_f4(p.Omax, p.poly), p.ppc, p.D, p.T, p.G, p.tw, S, p.spec);
  float4* sPairs = reinterpret_cast<float4*>(smem + L.pairs);
  double* sWin = reinterpret_cast<double*>(smem + L.win);
  uint32_t* sXdec = reinterpret_cast<uint32_t*>(smem + L.xdec);
  float* sXrow = reinterpret_cast<float*>(smem + L.xrow);
  float* sX0 = reinterpret_cast<float*>(smem + L.X0);
  float* sX1 = reinterpret_cast<float*>(smem + L.X1);
  float* sV0 = reinterpret_cast<float*>(smem + L.V0);
  float* sV1 = reinterpret_cast<float*>(smem + L.V1);
  float* sP = reinterpret_cast<float*>(smem + L.P);
  float* sR = reinterpret_cast<float*>(smem + L.R);
  float* sG = reinterpret_cast<float*>(smem + L.Gown);
  float* sPfit = reinterpret_cast<float*>(smem + L.Pfit);
  int* sPQ = reinterpret_cast<int*>(smem + L.PQ);
  int* sQi = reinterpret_cast<int*>(smem + L.Q);
  float* sF = reinterpret_cast<float*>(smem + L.F);
  int* sFQ = reinterpret_cast<int*>(smem + L.FQ);
  int* sImp = reinterpret_cast<int*>(smem + L.Imp);
  float* sLen = reinterpret_cast<float*>(smem + L.Len);

  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  const int T = p.T, D = p.D, G = p.G, N = p.N;
  const int b = blockIdx.x;
  const int r = b / p.C;
  const int cr = b - r * p.C;
  const int g = cr / S;
  const uint32_t q = cluster_rank();  // = cr - g * S: a cluster is S consecutive blocks
  const int n0 = (int)q * p.ppc;
  const int nl = max(0, min(p.ppc, N - n0));
  RunCtl* ctl = p.ctl + r;

  const float* hy = p.hyper + ((size_t)r * G + g) * 6;
  const float c1 = hy[0], c2 = hy[1], w_init = hy[3], w_end = hy[4], vlim = hy[5];
  const float sx = p.pts[0], sy = p.pts[1], tx = p.pts[2], ty = p.pts[3];
  const uint32_t cycle = (uint32_t)ctl->cycle;
  const uint32_t run = ctl->run_id;
  // read before any group arrives at the end counter (the last arrival's reader
  // advances it only after all arrivals)
  const int nfin = ctl->fin_launches;

  if (tid == 0) {
    mbar_init(&s_mbar, 1);
    s_key = kKeyEmpty;
  }
  __syncthreads();
  if (tid == 0 && p.O > 0) {
    const uint32_t bytes = (uint32_t)(p.poly ? p.O : pair_block_f4(p.O)) * 16u;
    mbar_expect_tx(&s_mbar, bytes);
    bulk_g2s(sPairs, p.poly ? p.circ : p.pairs, bytes, &s_mbar);
  }

  float* gX = p.X + ((size_t)r * p.M + (size_t)g * N + n0) * D;
  float* gV = p.V + ((size_t)r * p.M + (size_t)g * N + n0) * D;
  float* gP = p.P + ((size_t)r * p.M + (size_t)g * N + n0) * D;
  float* gPfit = p.Pfit + (size_t)r * p.M + (size_t)g * N + n0;
  int32_t* gPQ = p.PQ + (size_t)r * p.M + (size_t)g * N + n0;
  float* gGb = p.Gb + (size_t)r * G * D;
  float* gTb = p.Tb + (size_t)r * D;
  unsigned long long* grec = p.grec + (size_t)r * kRecDepth * G;

  float Tfit, gfit;
  int TQ, k, gq;
  int tholder = -1;  // group whose Gbest row is Tbest's; -1: the row already in gTb
  int win_n = 0, win_head = 0, stall = 0;
  float prev_lfv = INFINITY;

  if (p.mode == kModePlan) {
    // Initialisation (Algorithm 1) with Priori Initialization (Sec. 3.3.3).
    const int n_pi = (p.use_pi && ctl->has_prev) ? p.n_pi : 0;
    const float* prevT = p.prevT + (size_t)r * D;
    const int nch = (D + 3) >> 2;
    for (int it = tid; it < nl * nch; it += nt) {
      const int i = it / nch, ch = it - i * nch;
      const int n = n0 + i;
      const uint32_t pid = (uint32_t)(g * N + n);
      const bool pi = n < n_pi;
      const uint4 ux = draw(p.key0, p.key1, (uint32_t)ch, pid, pi ? kStreamPI : kStreamInitX, cycle, run);
      const uint4 uv = draw(p.key0, p.key1, (uint32_t)ch, pid, kStreamInitV, cycle, run);
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int j = ch * 4 + l;
        if (j < D) {
          const float ext = (j < T) ? p.W : p.H;
          float x;
          if (pi) x = fminf(fmaxf(prevT[j] + (2.0f * lane_of(ux, l) - 1.0f) * p.pi_h, 0.0f), ext);
          else x = lane_of(ux, l) * ext;
          sX0[i * D + j] = x;
          sP[i * D + j] = x;
          sV0[i * D + j] = (2.0f * lane_of(uv, l) - 1.0f) * (vlim * ext);
        }
      }
    }
    for (int i = tid; i < nl; i += nt) {
      sPfit[i] = INFINITY;
      sPQ[i] = 0;
    }
    for (int j = tid; j < D; j += nt) {
      sG[j] = 0.0f;
      if (q == 0) gGb[g * D + j] = 0.0f;
      if (cr == 0) gTb[j] = 0.0f;
    }
    Tfit = INFINITY;
    TQ = 0;
    k = 0;
    gfit = INFINITY;
    gq = 0;
    if (tid < 32 && p.at_mode == SEPSO_AT_STD_WINDOW && cycle != 0) {
      win_n = ctl->win_n;
      win_head = ctl->win_head;
      for (int i = lane; i < p.tw; i += 32) sWin[i] = p.win[(size_t)r * p.tw + i];
    }
  } else {
    for (int it = tid; it < nl * D; it += nt) {
      sX0[it] = gX[it];
      sV0[it] = gV[it];
      sP[it] = gP[it];
    }
    for (int i = tid; i < nl; i += nt) {
      sPfit[i] = gPfit[i];
      sPQ[i] = gPQ[i];
    }
    for (int j = tid; j < D; j += nt) sG[j] = gGb[g * D + j];
    gfit = p.Gfit[(size_t)r * G + g];
    gq = p.GQ[(size_t)r * G + g];
    Tfit = ctl->Tfit;
    TQ = ctl->TQ;
    k = ctl->k;
  }

  bool failed = false;
  const int K = circle_pairs(p.O);
  if (p.O > 0) {
    const bool landed = mbar_wait_bounded(&s_mbar, 0, kWaitLimitNs);
    if (__syncthreads_or(landed ? 0 : 1)) {
      failed = true;
      if (tid == 0) {
        ctl->status = SEPSO_ETIMEOUT;
        mbar_wait_bounded(&s_mbar, 0, kWaitLimitNs);  // once more: no copy in flight at exit
      }
    }
  } else {
    __syncthreads();
  }
  const float2* sNr2 = reinterpret_cast<const float2*>(sPairs + K);
  for (int i = tid; i < nl; i += nt) sQi[i] = 0;

  const unsigned long long kbase = (unsigned long long)ctl->iters_total;
  // Every CTA of the cluster has started before any remote store; a failed copy
  // in any of them stops the whole cluster (the slots of parity kbase & 1 are
  // free until iteration kbase + 2).
  cluster_barrier();
  const int p0 = (int)(kbase & 1ull);
  if (tid < S) st_peer_u32(peer_addr(sXdec + p0 * S + q, (uint32_t)tid), failed ? 2u : 0u);
  cluster_barrier();
  {
    uint32_t any = 0;
    for (int s2 = 0; s2 < S; ++s2) any |= sXdec[p0 * S + s2];
    failed = any != 0;
  }

  const int nseg = T + 1;
  int done = 0, xb = 0;
  bool capstop = false;
  unsigned long long gk_last = kbase;
  while (!failed) {
    if (p.mode == kModeStep && done >= p.step_iters) break;
    ++k;
    ++done;
    const unsigned long long gk = kbase + (unsigned long long)done;
    const int par = (int)(gk & 1ull);
    float* cX = xb ? sX1 : sX0;
    float* cV = xb ? sV1 : sV0;
    const bool have_prev = done > 1;
    const unsigned long long* prev_slot = grec + (size_t)((gk - 1ull) % (unsigned long long)kRecDepth) * G;
    unsigned long long rec = 0;
    if (have_prev && tid < G) rec = ld_relaxed_u64(prev_slot + tid);  // in flight during the fitness
    for (int i = nt - 1 - tid; i < nl; i += nt) {
      const uint4 o = draw(p.key0, p.key1, (uint32_t)k, (uint32_t)(g * N + n0 + i), kStreamVel, cycle, run);
      sR[i * 4 + 0] = c1 * u01(o.x);
      sR[i * 4 + 1] = c2 * u01(o.y);
    }

    // 1. Fitness F(X^k) and the Pbest test, kept aside.
    if (p.items) {
      if (p.poly) fitness_items_edges(cX, nl, T, D, sx, sy, tx, ty, sPairs, p.O, p.split, sQi, sLen);
      else fitness_items_pairs(cX, nl, T, D, sx, sy, tx, ty, sPairs, sNr2, K, p.split, sQi, sLen);
      __syncthreads();
    }
    {
      // In item mode warp 0 leaves the particles to the other warps and reads the
      // groups' records meanwhile (step 2).
      const bool skip0 = p.items && nwarps > 1;
      const int lp = p.items ? 32 : p.lp;
      const int ppw = 32 / lp;
      const int lsub = lane & (lp - 1);
      const int w0 = skip0 ? warp - 1 : warp, nw = skip0 ? nwarps - 1 : nwarps;
      if (w0 >= 0) {
        for (int i0 = w0 * ppw; i0 < nl; i0 += nw * ppw) {
          const int i = i0 + lane / lp;
          const bool live = i < nl;
          float len = 0.0f;
          int qq = 0;
          if (p.items) {
            len = warp_len_sum(sLen + i * nseg, nseg, lane);
            if (lsub == 0) {
              qq = sQi[i];
              sQi[i] = 0;
            }
          } else if (p.poly) {
            group_fitness_edges(cX + (live ? i : 0) * D, live, lp, T, p.split, p.O, sx, sy, tx, ty, sPairs, &len,
                                &qq);
          } else {
            group_fitness_pairs(cX + (live ? i : 0) * D, live, lp, T, p.split, K, sx, sy, tx, ty, sPairs, sNr2,
                                &len, &qq);
          }
          if (live && lsub == 0) {
            const float F = len + p.alpha * powi((float)qq, p.beta);
            const float pf = sPfit[i];
            const int imp = F < pf;
            const float cf = imp ? F : pf;
            const int cq = imp ? qq : sPQ[i];
            sF[i] = F;
            sFQ[i] = qq;
            sImp[i] = imp;
            if (cf < gfit) atomicMin(&s_key, best_key(cf, (uint32_t)(n0 + i), (uint32_t)cq));
          }
        }
      }
    }
    // 2. Tbest and Auto Truncation of iteration k - 1 from the groups' records.
    if (warp == 0) {
      uint32_t dec = 0;
      if (have_prev) {
        const bool late = cluster_wait_records(prev_slot, lane, G, gk - 1ull, rec);
        if (late) {
          dec = 2;
        } else if (cluster_tbest_at(p, rec, lane, Tfit, TQ, tholder, sWin, win_n, win_head, stall, prev_lfv)) {
          dec = 1;
        }
      }
      if (lane == 0) s_dec = dec;
    }
    __syncthreads();

    // 3. Candidate row, its Q, the decision word and the key into this CTA's slot in
    // every CTA of the cluster, as 16-byte vectors (the row only when there is a
    // candidate); only the warps that store remotely arrive with release order.
    const unsigned long long lkey = s_key;
    const uint32_t mydec = s_dec;
    const int XS = cluster_slot_stride(D);
    const int nv = XS / 4;           // vectors per slot
    const int v_tail = (D + 3) / 4;  // first vector past the row: Q, decision, key live in the slot tail
    bool pushed = false;
    {
      const bool have = lkey != kKeyEmpty;
      const int iw = have ? key_idx(lkey) - n0 : 0;
      const bool wimp = have && sImp[iw] != 0;
      const float* src = wimp ? cX + iw * D : sP + iw * D;
      const int qx = have ? (wimp ? sFQ[iw] : sPQ[iw]) : 0;
      const int v0 = have ? 0 : (D / 4);  // without a candidate only the vectors holding the tail
      const int per = nv - v0;
      float* slot = sXrow + (par * S + q) * XS;
      for (int t = tid; t < S * per; t += nt) {
        const int peer = t / per, v = v0 + (t - peer * per);
        float e[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int j = 4 * v + c;
          float x = 0.0f;
          if (j < D) x = src[j];
          else if (j == D) x = __int_as_float(qx);
          else if (j == D + 1) x = __uint_as_float(mydec);
          else if (j == D + 2) x = __uint_as_float((uint32_t)lkey);
          else if (j == D + 3) x = __uint_as_float((uint32_t)(lkey >> 32));
          e[c] = x;
        }
        st_peer_v4(peer_addr(slot + 4 * v, (uint32_t)peer), e[0], e[1], e[2], e[3]);
        pushed = true;
      }
      (void)v_tail;
    }
    if (__any_sync(0xffffffffu, pushed)) cluster_barrier();
    else cluster_barrier_relaxed_arrive();
    if (tid == 0) s_key = kKeyEmpty;

    // 4. The cluster's decision and best key, reduced by every warp over the S slots.
    uint32_t cdec = 0;
    unsigned long long gkey = kKeyEmpty;
    int gw = 0;
    {
      const float* sl = sXrow + (par * S + (lane < S ? lane : 0)) * XS;
      if (lane < S) {
        cdec = __float_as_uint(sl[D + 1]);
        gkey = ((unsigned long long)__float_as_uint(sl[D + 3]) << 32) | __float_as_uint(sl[D + 2]);
        gw = lane;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        cdec = max(cdec, __shfl_xor_sync(0xffffffffu, cdec, o));
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, gkey, o);
        const int ow = __shfl_xor_sync(0xffffffffu, gw, o);
        if (ok < gkey || (ok == gkey && ow < gw)) {
          gkey = ok;
          gw = ow;
        }
      }
    }
    if (cdec >= 2) {
      failed = true;
      if (tid == 0) ctl->status = SEPSO_ETIMEOUT;
      break;
    }
    if (cdec == 1) {  // stop at k - 1: discard iteration k
      if (p.spec) xb ^= 1;
      --k;
      --done;
      break;
    }

    // 5. The group's Gbest and its record; Pbest and the update (one pass).
    const float* grow = sG;  // this iteration's Gbest row
    const bool gimp = gkey != kKeyEmpty && key_fit(gkey) < gfit;
    if (gimp) {
      grow = sXrow + (par * S + gw) * XS;
      gfit = key_fit(gkey);
      gq = __float_as_int(grow[D]);
    }
    if (q == 0) {
      if (gimp)
        for (int j = tid; j < D; j += nt) gGb[g * D + j] = grow[j];
      if (tid == 0) st_relaxed_u64(grec + (size_t)(gk % (unsigned long long)kRecDepth) * G + g, make_rec(gfit, gq, gk));
    }
    gk_last = gk;
    for (int i = tid; i < nl; i += nt) {
      if (sImp[i]) {
        sPfit[i] = sF[i];
        sPQ[i] = sFQ[i];
      }
    }
    if (p.mode == kModePlan && k >= p.max_iters) {  // the cap: Algorithm 1 stops before the update
      for (int it = tid; it < nl * D; it += nt)
        if (sImp[it / D]) sP[it] = cX[it];
      capstop = true;
      break;
    }

    // Eq. TOF_omega, Eq. TOF_V (+ clip to V_range), Eq. TOF_X (+ clip to X_range),
    // with the Pbest rows of this iteration (each element by the thread that updates it).
    float* nX = p.spec ? (xb ? sX0 : sX1) : cX;
    float* nV = p.spec ? (xb ? sV0 : sV1) : cV;
    const float w = w_init - (w_init - w_end) / (float)p.max_iters * (float)k;
    for (int it = tid; it < nl * D; it += nt) {
      const int i = it / D;
      const int j = it - i * D;
      const float x = cX[it];
      if (sImp[i]) sP[it] = x;
      float v = w * cV[it];
      v = fmaf(sR[i * 4 + 0], sP[it] - x, v);
      v = fmaf(sR[i * 4 + 1], grow[j] - x, v);
      const float ext = (j < T) ? p.W : p.H;
      const float vmax = vlim * ext;
      v = fminf(fmaxf(v, -vmax), vmax);
      nV[it] = v;
      nX[it] = fminf(fmaxf(x + v, 0.0f), ext);
    }
    if (p.spec) xb ^= 1;
    // the next iterations read this Gbest row from sG; nobody reads sG in this one
    // when it changed (the update above read the slot), and the slot stays valid
    // until the next cluster barrier
    if (gimp)
      for (int j = tid; j < D; j += nt) sG[j] = grow[j];
    __syncthreads();
    if (p.mode == kModeStep && done >= p.step_iters) {  // a plain continuation ends after the update
      capstop = true;
      break;
    }
  }

  // Write back the swarm (state for sepso_step / sepso_get_state).
  {
    const float* fX = xb ? sX1 : sX0;
    const float* fV = xb ? sV1 : sV0;
    for (int it = tid; it < nl * D; it += nt) {
      gX[it] = fX[it];
      gV[it] = fV[it];
      gP[it] = sP[it];
    }
  }
  for (int i = tid; i < nl; i += nt) {
    gPfit[i] = sPfit[i];
    gPQ[i] = sPQ[i];
  }
  if (q == 0 && tid == 0) {
    p.Gfit[(size_t)r * G + g] = gfit;
    p.GQ[(size_t)r * G + g] = gq;
  }
  __syncthreads();
  cluster_barrier();  // no shared-memory access between the CTAs after this point
  if (q == 0 && tid == 0) red_release_add(&p.counter[r].fin, 1u);
  if (cr != 0) return;

  // CTA 0 of the run: every group has written its rows and last record.
  int timed_out = 0;
  if (tid == 0) {
    timed_out = counter_wait_bounded(&p.counter[r].fin, (unsigned int)G * (unsigned int)(nfin + 1), kWaitLimitNs)
                    ? 0
                    : 1;
    fence_acq_rel_gpu();
  }
  if (__syncthreads_or(timed_out)) {
    failed = true;
    if (tid == 0) ctl->status = SEPSO_ETIMEOUT;
  }
  if (!failed && capstop && warp == 0) {
    // the records of the last iteration (the loop ended after publishing them)
    unsigned long long rec = lane < G ? ld_relaxed_u64(grec + (size_t)(gk_last % (unsigned long long)kRecDepth) * G + lane) : 0ull;
    if (cluster_wait_records(grec + (size_t)(gk_last % (unsigned long long)kRecDepth) * G, lane, G, gk_last, rec)) {
      if (lane == 0) ctl->status = SEPSO_ETIMEOUT;
    } else {
      cluster_tbest_at(p, rec, lane, Tfit, TQ, tholder, sWin, win_n, win_head, stall, prev_lfv);
    }
  }
  if (tid == 0) s_dec = (uint32_t)(tholder + 1);  // Tbest is tracked by warp 0 alone
  __syncthreads();
  // Tbest's row: the holder group's Gbest row (which changes only together with
  // Tbest), staged in the exchange slots (free after the last cluster barrier).
  float* sTrow = sXrow;
  const int holder = (int)s_dec - 1;
  const float* src = (holder >= 0) ? gGb + (size_t)holder * D : gTb;
  for (int j = tid; j < D; j += nt) sTrow[j] = __ldcg(src + j);
  __syncthreads();
  for (int j = tid; j < D; j += nt) {
    gTb[j] = sTrow[j];
    if (p.mode == kModePlan) {
      p.res_wp[(size_t)r * D + j] = sTrow[j];
      p.prevT[(size_t)r * D + j] = sTrow[j];
    }
  }
  for (int j = tid; j < 3 * G; j += nt) p.gword[(size_t)r * 3 * G + j] = kKeyEmpty;
  if (tid == 0) {
    // the grid-wide form's barrier counts C per iteration of the run, and expects
    // its group words empty: keep both as if it had run these iterations
    atomicAdd(&p.counter[r].count, (unsigned int)p.cta_grid * (unsigned int)done);
    ctl->Tfit = Tfit;
    ctl->TQ = TQ;
    ctl->k = k;
    ctl->iters_total += done;
    ctl->fin_launches = nfin + 1;
    if (p.mode == kModePlan) {
      ctl->plans_total += 1;
      float len = 0.0f;
      for (int s = 0; s < nseg; ++s) {
        const float ax = (s == 0) ? sx : sTrow[s - 1];
        const float ay = (s == 0) ? sy : sTrow[T + s - 1];
        const float bx = (s == T) ? tx : sTrow[s];
        const float by = (s == T) ? ty : sTrow[T + s];
        const float dx = bx - ax, dy = by - ay;
        len += sqrtf(fmaf(dx, dx, dy * dy));
      }
      sepso_result* res = p.res + r;
      res->cost = Tfit;
      res->length = len;
      res->Q = TQ;
      res->iters = k;
      res->status = failed ? SEPSO_ETIMEOUT : ctl->status;
      ctl->has_prev = 1;
      ctl->cycle = (int32_t)cycle + 1;
      ctl->stall = stall;
      ctl->prev_lfv = prev_lfv;
      if (p.at_mode == SEPSO_AT_STD_WINDOW) {
        ctl->win_n = win_n;
        ctl->win_head = win_head;
        for (int i = 0; i < p.tw; ++i) p.win[(size_t)r * p.tw + i] = sWin[i];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Fitness of a batch of paths.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) evaluate_kernel(const EvalParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t s_mbar;
  const int D = p.D, T = p.T, nseg = T + 1;
  float4* sC = reinterpret_cast<float4*>(smem);
  float* sX = reinterpret_cast<float*>(smem + align_up((p.Omax > 0 ? p.Omax : 1) * 16, 16));
  int* sQ = reinterpret_cast<int*>(sX + p.per_cta * D);
  float* sLen = reinterpret_cast<float*>(sQ + p.per_cta);
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * p.per_cta;
  const int nl = max(0, min(p.per_cta, p.n - i0));

  if (tid == 0) mbar_init(&s_mbar, 1);
  __syncthreads();
  if (tid == 0 && p.O > 0) {
    mbar_expect_tx(&s_mbar, (uint32_t)p.O * 16u);
    bulk_g2s(sC, p.circ, (uint32_t)p.O * 16u, &s_mbar);
  }
  for (int it = tid; it < nl * D; it += blockDim.x) sX[it] = p.X[(size_t)i0 * D + it];
  for (int i = tid; i < nl; i += blockDim.x) sQ[i] = 0;
  if (p.O > 0) {
    const bool landed = mbar_wait_bounded(&s_mbar, 0, kWaitLimitNs);
    if (__syncthreads_or(landed ? 0 : 1)) {
      if (tid == 0) {
        atomicExch(p.status, SEPSO_ETIMEOUT);
        mbar_wait_bounded(&s_mbar, 0, kWaitLimitNs);  // once more: no copy in flight at exit
      }
      return;
    }
  } else {
    __syncthreads();
  }
  if (p.poly)
    fitness_items_edges(sX, nl, T, D, p.pts[0], p.pts[1], p.pts[2], p.pts[3], sC, p.O, p.split, sQ, sLen);
  else
    fitness_items(sX, nl, T, D, p.pts[0], p.pts[1], p.pts[2], p.pts[3], sC, p.O, p.split, sQ, sLen);
  __syncthreads();
  for (int i = tid; i < nl; i += blockDim.x) {
    float len = 0.0f;
    for (int s = 0; s < nseg; ++s) len += sLen[i * nseg + s];
    const int qq = sQ[i];
    if (p.F) p.F[i0 + i] = len + p.alpha * powi((float)qq, p.beta);
    if (p.Q) p.Q[i0 + i] = qq;
    if (p.len) p.len[i0 + i] = len;
  }
}

// ---------------------------------------------------------------------------
// Dynamic scene: c += v; a velocity component flips when the disk crosses the
// border it is moving towards (Fig. PP caption).  Start/target: radius 0.
// ---------------------------------------------------------------------------
// (circle records keep 4 r^2 in .w; the radius itself does not change)
__device__ __forceinline__ void move1(float& c, float& v, float r, float hi) {
  c += v;
  if (c - r < 0.0f && v < 0.0f) v = -v;
  if (c + r > hi && v > 0.0f) v = -v;
}

// Circle-pair blocks of a circle list (the layout the fitness reads), from scratch.
__global__ void pairs_kernel(const float4* __restrict__ circ, int O, float4* __restrict__ pairs) {
  const int K = circle_pairs(O);
  float2* nr2 = reinterpret_cast<float2*>(pairs + K);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    const float4 a = circ[2 * k];
    const float4 b = (2 * k + 1 < O) ? circ[2 * k + 1] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    pairs[k] = make_float4(a.x, b.x, a.y, b.y);
    nr2[k] = make_float2(-(a.z * a.z), (2 * k + 1 < O) ? -(b.z * b.z) : 0.0f);
  }
}

// The scene step; the moved centres also go into the circle-pair blocks (radii,
// and so the blocks' -r^2 entries, do not change).
__global__ void advance_kernel(float4* circ, float2* cvel, float* pts, float4* pairs, int O, float W, float H,
                               int steps) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < O; o += gridDim.x * blockDim.x) {
    float4 c = circ[o];
    float2 v = cvel[o];
    for (int s = 0; s < steps; ++s) {
      move1(c.x, v.x, c.z, W);
      move1(c.y, v.y, c.z, H);
    }
    circ[o] = c;
    cvel[o] = v;
    float* pb = reinterpret_cast<float*>(pairs + (o >> 1));
    pb[o & 1] = c.x;
    pb[2 + (o & 1)] = c.y;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    float sx = pts[0], sy = pts[1], tx = pts[2], ty = pts[3];
    float svx = pts[4], svy = pts[5], tvx = pts[6], tvy = pts[7];
    for (int s = 0; s < steps; ++s) {
      move1(sx, svx, 0.0f, W);
      move1(sy, svy, 0.0f, H);
      move1(tx, tvx, 0.0f, W);
      move1(ty, tvy, 0.0f, H);
    }
    pts[0] = sx; pts[1] = sy; pts[2] = tx; pts[3] = ty;
    pts[4] = svx; pts[5] = svy; pts[6] = tvx; pts[7] = tvy;
  }
}

// Polygon obstacles (the box obstacles of Sec. 4.3, moved as the Fig. PP caption
// moves the obstacles): one thread per polygon translates its edges by its
// velocity, then flips a velocity component when the polygon's bounding box lies
// past the border it is moving towards.  Start and target move as with circles.
__global__ void advance_poly_kernel(float4* edges, float2* pvel, const int* poff, int P, float* pts, float W,
                                    float H, int steps) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < P; q += gridDim.x * blockDim.x) {
    float2 v = pvel[q];
    const int e0 = poff[q], e1 = poff[q + 1];
    for (int st = 0; st < steps; ++st) {
      float xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
      for (int e = e0; e < e1; ++e) {
        float4 d = edges[e];
        d.x += v.x;
        d.y += v.y;
        d.z += v.x;
        d.w += v.y;
        edges[e] = d;
        xmin = fminf(xmin, fminf(d.x, d.z));
        xmax = fmaxf(xmax, fmaxf(d.x, d.z));
        ymin = fminf(ymin, fminf(d.y, d.w));
        ymax = fmaxf(ymax, fmaxf(d.y, d.w));
      }
      if (e1 > e0) {
        if ((xmin < 0.0f && v.x < 0.0f) || (xmax > W && v.x > 0.0f)) v.x = -v.x;
        if ((ymin < 0.0f && v.y < 0.0f) || (ymax > H && v.y > 0.0f)) v.y = -v.y;
      }
    }
    pvel[q] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    float sx = pts[0], sy = pts[1], tx = pts[2], ty = pts[3];
    float svx = pts[4], svy = pts[5], tvx = pts[6], tvy = pts[7];
    for (int st = 0; st < steps; ++st) {
      move1(sx, svx, 0.0f, W);
      move1(sy, svy, 0.0f, H);
      move1(tx, tvx, 0.0f, W);
      move1(ty, tvy, 0.0f, H);
    }
    pts[0] = sx; pts[1] = sy; pts[2] = tx; pts[3] = ty;
    pts[4] = svx; pts[5] = svy; pts[6] = tvx; pts[7] = tvy;
  }
}

// ---------------------------------------------------------------------------
// HSEF outer swarm (single CTA; the L-runs are the runs of swarm_kernel).
// ---------------------------------------------------------------------------
__device__ void hsef_write_hyper(const HsefParams& p) {
  const int G = p.G, DH = 3 * G;
  for (int it = threadIdx.x; it < p.HM * G; it += blockDim.x) {
    const int h = it / G, g = it - h * G;
    const float* x = p.HX + (size_t)h * DH;
    float* dst = p.hyper + ((size_t)h * G + g) * 6;
    dst[0] = x[G + g];
    dst[1] = x[2 * G + g];
    dst[2] = 0.0f;
    dst[3] = x[g];
    dst[4] = x[g];
    dst[5] = p.l_vlimit;
  }
}

__global__ void hsef_init_kernel(const HsefParams p) {
  const int G = p.G, DH = 3 * G;
  for (int it = threadIdx.x; it < p.HM * DH; it += blockDim.x) {
    const int h = it / DH, j = it - h * DH;
    const int hg = h / p.HN;
    const int kind = j / G;
    const float lo = p.lo[kind], hi = p.hi[kind];
    const uint4 ux = draw(p.key0, p.key1, (uint32_t)(j / 4), (uint32_t)h, kStreamHInitX, 0u, 0u);
    const uint4 uv = draw(p.key0, p.key1, (uint32_t)(j / 4), (uint32_t)h, kStreamHInitV, 0u, 0u);
    const float x = lo + lane_of(ux, j & 3) * (hi - lo);
    const float vmax = p.hhyper[hg * 6 + 5] * (hi - lo);
    p.HX[it] = x;
    p.HV[it] = (2.0f * lane_of(uv, j & 3) - 1.0f) * vmax;
    p.HP[it] = x;
  }
  for (int h = threadIdx.x; h < p.HM; h += blockDim.x) {
    p.HPfit[h] = INFINITY;
    p.ctl[h].cycle = 0;
    p.ctl[h].has_prev = 0;
    p.ctl[h].run_id = p.run_id;
  }
  for (int g = threadIdx.x; g < p.HG; g += blockDim.x) p.HGfit[g] = INFINITY;
  for (int j = threadIdx.x; j < p.HG * DH; j += blockDim.x) p.HGb[j] = 0.0f;
  for (int j = threadIdx.x; j < DH; j += blockDim.x) p.HTb[j] = 0.0f;
  if (threadIdx.x == 0) *p.HTfit = INFINITY;
  __syncthreads();
  hsef_write_hyper(p);
}

// Evolution e (1-based): H-fitness = LFV of each L-run (Eq. fit_h), H bests,
// then Eqs. TOF_omega / TOF_V / TOF_X on the H-swarm inside the (w, C1, C2) box.
__global__ void hsef_update_kernel(const HsefParams p, int e) {
  const int G = p.G, DH = 3 * G, HN = p.HN;
  for (int h = threadIdx.x; h < p.HM; h += blockDim.x) {
    const float f = p.res[h].cost;
    if (f < p.HPfit[h]) {
      p.HPfit[h] = f;
      for (int j = 0; j < DH; ++j) p.HP[(size_t)h * DH + j] = p.HX[(size_t)h * DH + j];
    }
  }
  __syncthreads();
  for (int g = threadIdx.x; g < p.HG; g += blockDim.x) {
    float best = INFINITY;
    int bi = -1;
    for (int n = 0; n < HN; ++n) {
      const float v = p.HPfit[g * HN + n];
      if (v < best) {
        best = v;
        bi = n;
      }
    }
    if (bi >= 0 && best < p.HGfit[g]) {
      p.HGfit[g] = best;
      for (int j = 0; j < DH; ++j) p.HGb[(size_t)g * DH + j] = p.HP[(size_t)(g * HN + bi) * DH + j];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float best = INFINITY;
    int bg = -1;
    for (int g = 0; g < p.HG; ++g) {
      if (p.HGfit[g] < best) {
        best = p.HGfit[g];
        bg = g;
      }
    }
    if (bg >= 0 && best < *p.HTfit) {
      *p.HTfit = best;
      for (int j = 0; j < DH; ++j) p.HTb[j] = p.HGb[(size_t)bg * DH + j];
    }
    if (p.history) p.history[e - 1] = *p.HTfit;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < p.HM * DH; it += blockDim.x) {
    const int h = it / DH, j = it - h * DH;
    const int hg = h / HN;
    const float* hh = p.hhyper + hg * 6;
    const int kind = j / G;
    const float lo = p.lo[kind], hi = p.hi[kind];
    const float w = hh[3] - (hh[3] - hh[4]) / (float)p.E * (float)e;
    const uint4 o = draw(p.key0, p.key1, (uint32_t)e, (uint32_t)h, kStreamHVel, 0u, 0u);
    const float x = p.HX[it];
    float v = w * p.HV[it];
    v = fmaf(hh[0] * u01(o.x), p.HP[it] - x, v);
    v = fmaf(hh[1] * u01(o.y), p.HGb[(size_t)hg * DH + j] - x, v);
    v = fmaf(hh[2] * u01(o.z), p.HTb[j] - x, v);
    const float vmax = hh[5] * (hi - lo);
    v = fminf(fmaxf(v, -vmax), vmax);
    p.HV[it] = v;
    p.HX[it] = fminf(fmaxf(x + v, lo), hi);
  }
  for (int h = threadIdx.x; h < p.HM; h += blockDim.x) {
    p.ctl[h].cycle = e;
    p.ctl[h].has_prev = 0;
  }
  __syncthreads();
  hsef_write_hyper(p);
}

// ---------------------------------------------------------------------------
// Launch wrappers (host).
// ---------------------------------------------------------------------------
// Allow up to `smem_bytes` of dynamic shared memory, less the kernel's static part.
cudaError_t configure_swarm_kernel(size_t smem_bytes) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, swarm_kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(swarm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(smem_bytes - a.sharedSizeBytes));
}

cudaError_t swarm_occupancy(int threads, size_t smem_bytes, int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, swarm_kernel, threads, smem_bytes);
}

cudaError_t launch_swarm(const SwarmParams& p, int grid, int threads, size_t smem, cudaStream_t s) {
  void* args[] = {const_cast<SwarmParams*>(&p)};
  return cudaLaunchCooperativeKernel((const void*)swarm_kernel, dim3(grid), dim3(threads), args, smem, s);
}

cudaError_t configure_cluster_kernel(size_t smem_bytes) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, swarm_cluster_kernel);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(swarm_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(smem_bytes - a.sharedSizeBytes));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(swarm_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

static cudaLaunchConfig_t cluster_config(int S, int grid, int threads, size_t smem, cudaStream_t s,
                                         cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)S;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

cudaError_t cluster_max_active(int S, int threads, size_t smem_bytes, int* clusters) {
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = cluster_config(S, S, threads, smem_bytes, nullptr, attr);
  return cudaOccupancyMaxActiveClusters(clusters, (void*)swarm_cluster_kernel, &cfg);
}

cudaError_t launch_swarm_cluster(const SwarmParams& p, int grid, int threads, size_t smem, cudaStream_t s) {
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = cluster_config(p.cpg, grid, threads, smem, s, attr);
  return cudaLaunchKernelEx(&cfg, swarm_cluster_kernel, p);
}

cudaError_t launch_advance_poly(float4* edges, float2* pvel, const int* poff, int P, float* pts, float W, float H,
                                int steps, cudaStream_t s) {
  advance_poly_kernel<<<std::max(1, (P + 127) / 128), 128, 0, s>>>(edges, pvel, poff, P, pts, W, H, steps);
  return cudaGetLastError();
}

cudaError_t launch_evaluate(const EvalParams& p, cudaStream_t s) {
  const size_t smem = (size_t)align_up((p.Omax > 0 ? p.Omax : 1) * 16, 16) +
                      (size_t)p.per_cta * p.D * 4 + (size_t)p.per_cta * 4 +
                      (size_t)p.per_cta * (p.T + 1) * 4;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes a;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, evaluate_kernel);
  if (e == cudaSuccess && smem + a.sharedSizeBytes > (size_t)optin) return cudaErrorInvalidValue;
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(evaluate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)a.sharedSizeBytes);
  if (e != cudaSuccess) return e;
  const int grid = (p.n + p.per_cta - 1) / p.per_cta;
  evaluate_kernel<<<grid, 256, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_advance(float4* circ, float2* cvel, float* pts, float4* pairs, int O, float W, float H,
                           int steps, cudaStream_t s) {
  const int threads = 128;
  const int grid = O > 0 ? (O + threads - 1) / threads : 1;
  advance_kernel<<<grid, threads, 0, s>>>(circ, cvel, pts, pairs, O, W, H, steps);
  return cudaGetLastError();
}

cudaError_t launch_pairs(const float4* circ, int O, float4* pairs, cudaStream_t s) {
  const int K = circle_pairs(O);
  if (K == 0) return cudaSuccess;
  pairs_kernel<<<(K + 255) / 256, 256, 0, s>>>(circ, O, pairs);
  return cudaGetLastError();
}

cudaError_t launch_hsef_init(const HsefParams& p, cudaStream_t s) {
  hsef_init_kernel<<<1, 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_hsef_update(const HsefParams& p, int e, cudaStream_t s) {
  hsef_update_kernel<<<1, 256, 0, s>>>(p, e);
  return cudaGetLastError();
}

// Watchdog self-test: the two kinds of bounded wait the kernels use (an mbarrier
// that no copy completes, a counter that no CTA increments) are left to run out;
// bit 0 / bit 1 of *fired report that each gave up.
__global__ void watchdog_selftest_kernel(const unsigned int* never, unsigned long long limit_ns, int* fired) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int f = 0;
    if (!mbar_wait_bounded(&bar, 0u, limit_ns)) f |= 1;
    if (!counter_wait_bounded(never, 1u, limit_ns)) f |= 2;
    *fired = f;
  }
}

// The Auto Truncation window test on its own: one warp per window.
__global__ void at_window_kernel(const double* win, const int32_t* ns, const int32_t* heads, int tw,
                                 float delta, int32_t* out) {
  const int i = blockIdx.x;
  const bool below = window_std_below(win + (size_t)i * tw, tw, ns[i], heads[i], delta, threadIdx.x);
  if (threadIdx.x == 0) out[i] = below ? 1 : 0;
}

cudaError_t launch_at_window(const double* win, const int32_t* ns, const int32_t* heads, int count, int tw,
                             float delta, int32_t* out, cudaStream_t s) {
  at_window_kernel<<<count, 32, 0, s>>>(win, ns, heads, tw, delta, out);
  return cudaGetLastError();
}

// Philox4x32-10 on given counters: the planner's own generator (the function every
// kernel draws R1..R3 and the initial positions with), one counter per thread.
__global__ void philox_kernel(const uint4* ctr, long long n, uint32_t k0, uint32_t k1, uint4* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = philox4x32_10(ctr[i], k0, k1);
}

cudaError_t launch_philox(const uint4* ctr, long long n, uint64_t seed, uint4* out, int num_sms, cudaStream_t s) {
  const long long blocks = std::min<long long>((n + 255) / 256, 8LL * (num_sms > 0 ? num_sms : 1));
  philox_kernel<<<(int)std::max<long long>(blocks, 1), 256, 0, s>>>(ctr, n, (uint32_t)(seed & 0xffffffffu),
                                                                   (uint32_t)(seed >> 32), out);
  return cudaGetLastError();
}

cudaError_t launch_watchdog_selftest(const unsigned int* never, unsigned long long limit_ns, int* fired,
                                     cudaStream_t s) {
  watchdog_selftest_kernel<<<1, 32, 0, s>>>(never, limit_ns, fired);
  return cudaGetLastError();
}

}  // namespace sepso
