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
// of S = p.cpg CTAs; CTA q (its rank in the cluster) owns particles
// [q ppc, q ppc + ppc) of the group, one warp each, plus a control warp (the last
// warp).  A particle's state lives in its warp's registers: lane l < T holds
// waypoint l (x = X[l], y = X[T + l]) with its velocity and Pbest coordinates and
// the group's Gbest coordinates; the Pbest and Gbest fitness and Q are the same in
// every lane.  Round j of a launch runs iteration k = k0 + j:
//   1. each particle warp evaluates F(X^k) (lane s builds segment s's frame, lane
//      l tests obstacles l, l + 32, ... against every segment), applies its Pbest
//      test and, when its Pbest is below the group's Gfit, stages its Pbest row
//      and Q in its CTA's shared memory; it writes its key (or the empty key) into
//      its own key slot of the round in every CTA of the cluster (plain remote
//      stores: 64-bit atomic min on distributed shared memory was measured to lose
//      updates on GB300, so every warp owns a slot and readers reduce);
//   2. the control warp of rank 0 reads every group's record of iteration
//      k - kLag (Gfit and Q after that iteration's best update), updates Tbest,
//      takes that iteration's Auto Truncation decision and writes the decision
//      word of the round into every CTA of the cluster;
//   3. one cluster barrier;
//   4. every warp reads the round's decision and reduces the round's key slots in
//      its own shared memory.  A stop at k - kLag restores that iteration's state from two
//      register snapshots (Algorithm 1 returns Tbest after the stopping
//      iteration's best update and moves no particle after it); otherwise the
//      group's Gbest follows the key (the winner's row and Q are read from its
//      CTA's stage), rank 0's control warp publishes the group's record of k and
//      each particle warp applies Eqs. TOF_omega, TOF_V and TOF_X to its row.
// At the iteration cap the position update is skipped and, with Auto Truncation
// on, kLag - 1 more rounds collect the decisions of the last iterations.  The
// groups then meet once at the run's end counter, and CTA 0 of the run applies the
// records it has not seen yet and takes Tbest's row from the holder group's Gbest
// row (the holder's row changes only together with Tbest).  The decisions, bests
// and arithmetic are those of swarm_kernel, so both forms give identical results
// and states.
//
// Reuse of the exchange buffers: key slots and stage rows of parity gk & 1 (and
// the decision word of round j, slot j % 3) are rewritten two rounds later, after
// the barrier of the round in between, which every reader reaches only after
// reading them.  A record ring slot of iteration gk is rewritten at
// gk + kRecDepth; every group reads the records of gk - kLag before its barrier of
// gk, so no reader still needs a slot when it is rewritten.
// ---------------------------------------------------------------------------
constexpr int kLag = 2;  // Auto Truncation decided kLag iterations late (slack for the records)

// Floats of one stage row: (x_l, y_l) pairs for l < T, then Q, padded.
__host__ __device__ inline int cluster_stage_stride(int T) { return 2 * T + 4; }
constexpr int kFrameFloats = 8;  // one segment frame in a warp's frame area

__host__ __device__ ClusterLayout ClusterLayout::make(int obst_f4, int ppc, int T, int tw, int S) {
  ClusterLayout s;
  int off = 1024;
  s.pairs = off;
  off = align_up(off + obst_f4 * 16, 16);  // circle-pair blocks or polygon edges
  s.win = off;
  off = align_up(off + tw * 8, 16);
  s.keys = off;  // two parities x S ranks x ppc warps
  off = align_up(off + 2 * S * ppc * 8, 16);
  s.stage = off;
  off = align_up(off + 2 * ppc * cluster_stage_stride(T) * 4, 16);
  s.frames = off;
  off += ppc * 32 * kFrameFloats * 4;  // per particle warp: frames of up to 32 segments
  s.total = align_up(off, 16);
  return s;
}

__device__ __forceinline__ float2 ld_peer_f2(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ int ld_peer_s32(uint32_t addr) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
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

// Lanes 0..G-1 of a warp: the records of iteration gk (prefetched in rec), waited
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

// The circle pairs a lane keeps in registers for a whole launch: with PG =
// ceil(K / kLanePairs) lanes per segment group and SG = 32 / PG groups, lane l holds
// pairs kLanePairs (l % PG) + i and takes segments l / PG, l / PG + SG, ...; pairs
// past K hold a value that never hits (-r^2 = +1).  A lane then reads one compact
// frame per segment for kLanePairs pairs, which keeps the frames' shared-memory
// reads below the arithmetic.
constexpr int kLanePairs = 4;
struct LanePairs {
  unsigned long long cx[kLanePairs], cy[kLanePairs], w[kLanePairs];
  int s0, ds;  // first segment of the lane and the stride
};

__device__ __forceinline__ LanePairs lane_pairs(const float4* cxy, const float2* nr2, int K, int lane) {
  LanePairs lp;
  const int PG = max(1, (K + kLanePairs - 1) / kLanePairs);
  const int SG = max(1, 32 / PG);
  const int pg = lane % PG;
  lp.s0 = (lane / PG < SG) ? lane / PG : 32;  // lanes past the last group take no segment
  lp.ds = SG;
#pragma unroll
  for (int i = 0; i < kLanePairs; ++i) {
    const int k = pg * kLanePairs + i;
    float4 c = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float2 w = make_float2(1.0f, 1.0f);
    if (k < K) {
      c = cxy[k];
      w = nr2[k];
    }
    lp.cx[i] = pack2(c.x, c.y);
    lp.cy[i] = pack2(c.z, c.w);
    lp.w[i] = pack2(w.x, w.y);
  }
  return lp;
}

// Length and Q of the warp's particle among circle pairs, its row in registers
// (lane l < T holds waypoint l): lane s <= T builds segment s's frame (two float4:
// ux, uy, -mu, nx and ny, -mn, h) in the warp's frame area fr, then every lane
// tests its register pairs against its segments (K <= 32 kLanePairs), or pairs l,
// l + 32, ... against every segment (larger K), with the arithmetic of pair_hits.
// The length is summed in warp_len_sum's order (lane s holds segment s), Q
// exactly; every lane returns both.
__device__ __forceinline__ void warp_fitness_pairs(float x, float y, int T, int lane, float sx, float sy, float tx,
                                                   float ty, const LanePairs& lp, const float4* __restrict__ cxy,
                                                   const float2* __restrict__ nr2, int K, float* fr, float* len_out,
                                                   int* q_out) {
  const float xp = __shfl_up_sync(0xffffffffu, x, 1), yp = __shfl_up_sync(0xffffffffu, y, 1);
  float4* f4 = reinterpret_cast<float4*>(fr);
  float len = 0.0f;
  if (lane <= T) {
    const float ax = lane == 0 ? sx : xp, ay = lane == 0 ? sy : yp;
    const float bx = lane == T ? tx : x, by = lane == T ? ty : y;
    const FrameScalars f = frame_scalars(ax, ay, bx, by, &len);
    f4[2 * lane] = make_float4(f.ux, f.uy, f.nmu, f.nx);
    f4[2 * lane + 1] = make_float4(f.ny, f.nmn, f.h, 0.0f);
  }
  __syncwarp();
  int hits = 0;
  if (K <= 32 * kLanePairs) {
    for (int s = lp.s0; s <= T; s += lp.ds) {
      const float4 a = f4[2 * s], b = f4[2 * s + 1];
      const unsigned long long UX = pack2(a.x, a.x), UY = pack2(a.y, a.y), NMU = pack2(a.z, a.z),
                               NX = pack2(a.w, a.w), NY = pack2(b.x, b.x), NMN = pack2(b.y, b.y);
#pragma unroll
      for (int i = 0; i < kLanePairs; ++i) hits += pair_test(lp.cx[i], lp.cy[i], lp.w[i], UX, UY, NMU, NX, NY, NMN, b.z);
    }
  } else {
    for (int k = lane; k < K; k += 32) {
      const float4 c = cxy[k];
      const float2 w = nr2[k];
      const unsigned long long CX = pack2(c.x, c.y), CY = pack2(c.z, c.w), W = pack2(w.x, w.y);
#pragma unroll 2
      for (int s = 0; s <= T; ++s) {
        const float4 a = f4[2 * s], b = f4[2 * s + 1];
        hits += pair_test(CX, CY, W, pack2(a.x, a.x), pack2(a.y, a.y), pack2(a.z, a.z), pack2(a.w, a.w),
                          pack2(b.x, b.x), pack2(b.y, b.y), b.z);
      }
    }
  }
  __syncwarp();  // every lane has read the frames before the next round rewrites them
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    len += __shfl_xor_sync(0xffffffffu, len, o);
    hits += __shfl_xor_sync(0xffffffffu, hits, o);
  }
  *len_out = len;
  *q_out = hits;
}

// The same among polygon edges: lane s <= T stores segment s's start and direction, lane l
// tests edges l, l + 32, ... against every segment (edge_crosses).
__device__ __forceinline__ void warp_fitness_edges(float x, float y, int T, int lane, float sx, float sy, float tx,
                                                   float ty, const float4* __restrict__ edges, int E, float* fr,
                                                   float* len_out, int* q_out) {
  const float xp = __shfl_up_sync(0xffffffffu, x, 1), yp = __shfl_up_sync(0xffffffffu, y, 1);
  float4* f4 = reinterpret_cast<float4*>(fr);
  float len = 0.0f;
  if (lane <= T) {
    const float ax = lane == 0 ? sx : xp, ay = lane == 0 ? sy : yp;
    const float bx = lane == T ? tx : x, by = lane == T ? ty : y;
    const float dx = bx - ax, dy = by - ay;
    len = sqrtf(fmaf(dx, dx, dy * dy));
    f4[2 * lane] = make_float4(ax, ay, dx, dy);
  }
  __syncwarp();
  int hits = 0;
  for (int e = lane; e < E; e += 32) {
    const float4 d = edges[e];
#pragma unroll 4
    for (int s = 0; s <= T; ++s) {
      const float4 sg = f4[2 * s];
      hits += edge_crosses(sg.x, sg.y, sg.z, sg.w, d);
    }
  }
  __syncwarp();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    len += __shfl_xor_sync(0xffffffffu, len, o);
    hits += __shfl_xor_sync(0xffffffffu, hits, o);
  }
  *len_out = len;
  *q_out = hits;
}

// A particle lane's state at the end of one iteration (after its best updates).
struct LaneSnap {
  float x, y, vx, vy, px, py, gx, gy, pfit, gfit;
  int pq, gq;
};

__global__ void __launch_bounds__(kClusterMaxThreads, 1) swarm_cluster_kernel(const SwarmParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t s_mbar;
  __shared__ uint32_t s_dec[3];
  __shared__ uint32_t s_any[3];
  __shared__ uint32_t s_init[16];

  const int S = p.cpg;
  const ClusterLayout L = ClusterLayout::make(obstacle_f4(p.Omax, p.poly), p.ppc, p.T, p.tw, S);
  const float4* sObst = reinterpret_cast<const float4*>(smem + L.pairs);
  double* sWin = reinterpret_cast<double*>(smem + L.win);
  unsigned long long* sKeys = reinterpret_cast<unsigned long long*>(smem + L.keys);
  float* sStage = reinterpret_cast<float*>(smem + L.stage);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool ctrl = warp == (int)(blockDim.x >> 5) - 1;  // the control warp
  const int T = p.T, D = p.D, G = p.G, N = p.N, ppc = p.ppc;
  const int SR = cluster_stage_stride(T);
  const int r = blockIdx.x / p.C;
  const int cr = blockIdx.x - r * p.C;
  const int g = cr / S;
  const uint32_t q = cluster_rank();  // = cr - g * S: a cluster is S consecutive blocks
  const int n = (int)q * ppc + warp;  // the warp's particle (index within the group)
  const bool live = !ctrl && warp < ppc && n < N;
  const bool wl = live && lane < T;  // the lane holds a waypoint
  float* fr = reinterpret_cast<float*>(smem + L.frames) + (size_t)(live ? warp : 0) * 32 * kFrameFloats;
  RunCtl* ctl = p.ctl + r;

  const float* hy = p.hyper + ((size_t)r * G + g) * 6;
  const float c1 = hy[0], c2 = hy[1], w_init = hy[3], w_end = hy[4], vlim = hy[5];
  const float sx = p.pts[0], sy = p.pts[1], tx = p.pts[2], ty = p.pts[3];
  const uint32_t cycle = (uint32_t)ctl->cycle;
  const uint32_t run = ctl->run_id;
  const bool plan = p.mode == kModePlan;
  // read before any group arrives at the end counter (the last arrival's reader
  // advances it only after all arrivals)
  const int nfin = ctl->fin_launches;
  const int k0 = plan ? 0 : ctl->k;
  const unsigned long long kbase = (unsigned long long)ctl->iters_total;

  if (tid == 0) {
    mbar_init(&s_mbar, 1);
    for (int i = 0; i < 3; ++i) {
      s_dec[i] = 0u;
      s_any[i] = 0u;
    }
  }
  for (int i = tid; i < 2 * S * ppc; i += blockDim.x) sKeys[i] = kKeyEmpty;  // slots of absent particles stay empty
  __syncthreads();
  if (tid == 0 && p.O > 0) {
    const uint32_t bytes = (uint32_t)(p.poly ? p.O : pair_block_f4(p.O)) * 16u;
    mbar_expect_tx(&s_mbar, bytes);
    bulk_g2s(const_cast<float4*>(sObst), p.poly ? p.circ : p.pairs, bytes, &s_mbar);
  }

  const size_t prow = ((size_t)r * p.M + (size_t)g * N + (size_t)(live ? n : 0)) * D;
  float* gGb = p.Gb + (size_t)r * G * D;
  float* gTb = p.Tb + (size_t)r * D;
  unsigned long long* grec = p.grec + (size_t)r * kRecDepth * G;

  LaneSnap c = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, INFINITY, INFINITY, 0, 0};
  // Tbest and Auto Truncation state (meaningful in the control warp of rank 0)
  float Tfit = INFINITY;
  int TQ = 0, tholder = -1;  // tholder: group whose Gbest row is Tbest's; -1: the row already in gTb
  int win_n = 0, win_head = 0, stall = 0;
  float prev_lfv = INFINITY;

  if (plan) {
    // Initialisation (Algorithm 1) with Priori Initialization (Sec. 3.3.3):
    // coordinate j takes word j % 4 of the draw whose counter word 0 is j / 4.
    const int n_pi = (p.use_pi && ctl->has_prev) ? p.n_pi : 0;
    if (wl) {
      const uint32_t pid = (uint32_t)(g * N + n);
      const bool pi = n < n_pi;
      const uint32_t stream = pi ? kStreamPI : kStreamInitX;
      const int jx = lane, jy = T + lane;
      const uint4 uxa = draw(p.key0, p.key1, (uint32_t)(jx >> 2), pid, stream, cycle, run);
      const uint4 uxb = draw(p.key0, p.key1, (uint32_t)(jy >> 2), pid, stream, cycle, run);
      const uint4 uva = draw(p.key0, p.key1, (uint32_t)(jx >> 2), pid, kStreamInitV, cycle, run);
      const uint4 uvb = draw(p.key0, p.key1, (uint32_t)(jy >> 2), pid, kStreamInitV, cycle, run);
      if (pi) {
        const float* prevT = p.prevT + (size_t)r * D;
        c.x = fminf(fmaxf(prevT[jx] + (2.0f * lane_of(uxa, jx & 3) - 1.0f) * p.pi_h, 0.0f), p.W);
        c.y = fminf(fmaxf(prevT[jy] + (2.0f * lane_of(uxb, jy & 3) - 1.0f) * p.pi_h, 0.0f), p.H);
      } else {
        c.x = lane_of(uxa, jx & 3) * p.W;
        c.y = lane_of(uxb, jy & 3) * p.H;
      }
      c.vx = (2.0f * lane_of(uva, jx & 3) - 1.0f) * (vlim * p.W);
      c.vy = (2.0f * lane_of(uvb, jy & 3) - 1.0f) * (vlim * p.H);
      c.px = c.x;
      c.py = c.y;
    }
    if (cr == 0 && ctrl)
      for (int j = lane; j < D; j += 32) gTb[j] = 0.0f;
    if (ctrl && q == 0 && p.at_mode == SEPSO_AT_STD_WINDOW && cycle != 0) {
      win_n = ctl->win_n;
      win_head = ctl->win_head;
      for (int i = lane; i < p.tw; i += 32) sWin[i] = p.win[(size_t)r * p.tw + i];
    }
  } else {
    if (wl) {
      c.x = p.X[prow + lane];
      c.y = p.X[prow + T + lane];
      c.vx = p.V[prow + lane];
      c.vy = p.V[prow + T + lane];
      c.px = p.P[prow + lane];
      c.py = p.P[prow + T + lane];
      c.gx = gGb[(size_t)g * D + lane];
      c.gy = gGb[(size_t)g * D + T + lane];
    }
    if (live) {
      c.pfit = p.Pfit[prow / D];
      c.pq = p.PQ[prow / D];
    }
    c.gfit = p.Gfit[(size_t)r * G + g];
    c.gq = p.GQ[(size_t)r * G + g];
    Tfit = ctl->Tfit;
    TQ = ctl->TQ;
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
  const float2* sNr2 = reinterpret_cast<const float2*>(sObst + K);
  const LanePairs lpairs = lane_pairs(sObst, sNr2, p.poly ? 0 : K, lane);
  // Every CTA of the cluster has started (and set its words) before any remote
  // access; a failed copy in any of them stops the whole cluster.
  cluster_barrier();
  if (tid < S) st_peer_u32(peer_addr(&s_init[q], (uint32_t)tid), failed ? 1u : 0u);
  cluster_barrier();
  {
    uint32_t any = 0;
    for (int s2 = 0; s2 < S; ++s2) any |= s_init[s2];
    failed = any != 0;
  }

  const bool at_on = plan && p.at_mode != SEPSO_AT_OFF;
  const int n_compute = plan ? p.max_iters : p.step_iters;
  const int n_rounds = n_compute + (at_on ? kLag - 1 : 0);
  LaneSnap A = c, B = c;  // the state at the end of the last iteration, and of the one before
  int done = 0;           // iterations completed by this launch
  int stop_round = 0;     // the round that learned of an Auto Truncation stop
  unsigned long long proc = kbase;  // records applied to Tbest through this iteration count
  unsigned long long rec = 0ull;    // control warp of rank 0, lanes < G: the next records to apply
  for (int j = 1; !failed && j <= n_rounds; ++j) {
    const bool compute = j <= n_compute;
    const unsigned long long gk = kbase + (unsigned long long)j;
    const int slot = j % 3;
    const int par = (int)(gk & 1ull);
    float a1 = 0.0f, a2 = 0.0f;
    if (compute && live) {
      // R1, R2 of this iteration (one scalar per particle), F(X^k), the Pbest test
      const uint4 o = draw(p.key0, p.key1, (uint32_t)(k0 + j), (uint32_t)(g * N + n), kStreamVel, cycle, run);
      a1 = c1 * u01(o.x);
      a2 = c2 * u01(o.y);
      float len;
      int qq;
      if (p.poly) warp_fitness_edges(c.x, c.y, T, lane, sx, sy, tx, ty, sObst, p.O, fr, &len, &qq);
      else warp_fitness_pairs(c.x, c.y, T, lane, sx, sy, tx, ty, lpairs, sObst, sNr2, K, fr, &len, &qq);
      const float F = len + p.alpha * powi((float)qq, p.beta);
      if (F < c.pfit) {
        c.pfit = F;
        c.pq = qq;
        c.px = c.x;
        c.py = c.y;
      }
      unsigned long long key = kKeyEmpty;
      if (c.pfit < c.gfit) {  // a candidate for the group's best: stage the row
        float* st = sStage + (size_t)(par * ppc + warp) * SR;
        if (lane < T) reinterpret_cast<float2*>(st)[lane] = make_float2(c.px, c.py);
        if (lane == 0) reinterpret_cast<int*>(st)[2 * T] = c.pq;
        key = best_key(c.pfit, (uint32_t)n, (uint32_t)c.pq);
        if (lane < S) st_peer_u32(peer_addr(&s_any[slot], (uint32_t)lane), 1u);  // the round has a candidate
      }
      if (lane < S) st_peer_u64(peer_addr(sKeys + ((size_t)par * S + q) * ppc + warp, (uint32_t)lane), key);
    }
    if (ctrl && q == 0) {
      // Tbest and Auto Truncation of iteration gk - kLag from every group's record
      uint32_t dec = 0;
      if (j > kLag) {
        const unsigned long long gr = gk - (unsigned long long)kLag;
        const unsigned long long* rs = grec + (size_t)(gr % (unsigned long long)kRecDepth) * G;
        if (cluster_wait_records(rs, lane, G, gr, rec)) {  // rec: prefetched in the previous round
          dec = 2;
        } else {
          proc = gr;
          if (cluster_tbest_at(p, rec, lane, Tfit, TQ, tholder, sWin, win_n, win_head, stall, prev_lfv) && at_on)
            dec = 1;
        }
      }
      if (lane < S) st_peer_u32(peer_addr(&s_dec[slot], (uint32_t)lane), dec);
    }
    cluster_barrier();
    const uint32_t dec = s_dec[slot];
    const uint32_t any = s_any[slot];
    if (ctrl && lane == 0) s_any[(j + 2) % 3] = 0u;  // the flag of round j - 1, read by every warp before this barrier
    if (ctrl && q == 0 && lane < G && j + 1 > kLag)  // the records the next round applies, in flight meanwhile
      rec = ld_relaxed_u64(grec + (size_t)((gk + 1ull - (unsigned long long)kLag) % (unsigned long long)kRecDepth) * G + lane);
    if (dec >= 2) {
      failed = true;
      if (tid == 0) ctl->status = SEPSO_ETIMEOUT;
      break;
    }
    if (dec == 1) {  // Auto Truncation stopped at iteration k0 + j - kLag: its state is B
      c = B;
      done = j - kLag;
      stop_round = j;
      break;
    }
    if (!compute) continue;  // a round that only collects a decision
    // the group's lowest key of the round (the lowest-index particle of lowest
    // Pbest): each lane's lowest slot, then the lowest fitness bits over the warp,
    // then the lowest index bits among the lanes that hold them
    unsigned long long gkey = kKeyEmpty;
    if (any) {
      const unsigned long long* kk = sKeys + (size_t)par * S * ppc;
      for (int i = lane; i < S * ppc; i += 32) gkey = min(gkey, kk[i]);
      const uint32_t hi = __reduce_min_sync(0xffffffffu, (uint32_t)(gkey >> 32));
      const uint32_t lo = __reduce_min_sync(0xffffffffu, (uint32_t)(gkey >> 32) == hi ? (uint32_t)gkey : 0xffffffffu);
      gkey = ((unsigned long long)hi << 32) | lo;
    }
    if (gkey != kKeyEmpty && key_fit(gkey) < c.gfit) {
      const int nw = key_idx(gkey);
      const int qw = nw / ppc;
      const float* st = sStage + (size_t)(par * ppc + (nw - qw * ppc)) * SR;
      c.gfit = key_fit(gkey);
      c.gq = key_q(gkey);
      if (c.gq >= (int)kQSat) c.gq = ld_peer_s32(peer_addr(st + 2 * T, (uint32_t)qw));
      if (wl) {
        const float2 v = ld_peer_f2(peer_addr(st + 2 * lane, (uint32_t)qw));
        c.gx = v.x;
        c.gy = v.y;
      }
    }
    if (ctrl && q == 0 && lane == 0)
      st_relaxed_u64(grec + (size_t)(gk % (unsigned long long)kRecDepth) * G + g, make_rec(c.gfit, c.gq, gk));
    B = A;
    A = c;
    done = j;
    if (plan && j == n_compute) continue;  // the cap: Algorithm 1 stops after the best update
    if (wl) {
      // Eq. TOF_omega, Eq. TOF_V (+ clip to V_range), Eq. TOF_X (+ clip to X_range)
      const float w = w_init - (w_init - w_end) / (float)p.max_iters * (float)(k0 + j);
      float v = w * c.vx;
      v = fmaf(a1, c.px - c.x, v);
      v = fmaf(a2, c.gx - c.x, v);
      const float vmx = vlim * p.W;
      v = fminf(fmaxf(v, -vmx), vmx);
      c.vx = v;
      c.x = fminf(fmaxf(c.x + v, 0.0f), p.W);
      v = w * c.vy;
      v = fmaf(a1, c.py - c.y, v);
      v = fmaf(a2, c.gy - c.y, v);
      const float vmy = vlim * p.H;
      v = fminf(fmaxf(v, -vmy), vmy);
      c.vy = v;
      c.y = fminf(fmaxf(c.y + v, 0.0f), p.H);
    }
  }

  // Write back the swarm (state for sepso_step / sepso_get_state).
  if (wl) {
    p.X[prow + lane] = c.x;
    p.X[prow + T + lane] = c.y;
    p.V[prow + lane] = c.vx;
    p.V[prow + T + lane] = c.vy;
    p.P[prow + lane] = c.px;
    p.P[prow + T + lane] = c.py;
  }
  if (live && lane == 0) {
    p.Pfit[prow / D] = c.pfit;
    p.PQ[prow / D] = c.pq;
  }
  if (q == 0 && warp == 0) {  // particle 0's warp holds the group's Gbest
    if (lane < T) {
      gGb[(size_t)g * D + lane] = c.gx;
      gGb[(size_t)g * D + T + lane] = c.gy;
    }
    if (lane == 0) {
      p.Gfit[(size_t)r * G + g] = c.gfit;
      p.GQ[(size_t)r * G + g] = c.gq;
    }
  }
  __syncthreads();
  cluster_barrier();  // no shared-memory access between the CTAs after this point
  if (q == 0 && ctrl && lane == 0) {
    // records of iterations a stop discarded: the next launch counts iterations from
    // the stop, so their tags would match its first rounds
    if (stop_round > 0)
      for (int jj = stop_round - kLag + 1; jj < stop_round; ++jj)
        if (jj >= 1 && jj <= n_compute)
          grec[(size_t)((kbase + (unsigned long long)jj) % (unsigned long long)kRecDepth) * G + g] = 0ull;
    red_release_add(&p.counter[r].fin, 1u);
  }
  if (cr != 0 || !ctrl) return;

  // The control warp of CTA 0 of the run: every group has written its rows and
  // records; apply the records not yet applied, then the results.
  int timed_out = 0;
  if (lane == 0) {
    timed_out = counter_wait_bounded(&p.counter[r].fin, (unsigned int)G * (unsigned int)(nfin + 1), kWaitLimitNs)
                    ? 0
                    : 1;
    fence_acq_rel_gpu();
  }
  __syncwarp();
  if (__shfl_sync(0xffffffffu, timed_out, 0)) {
    failed = true;
    if (lane == 0) ctl->status = SEPSO_ETIMEOUT;
  }
  const unsigned long long gk_final = kbase + (unsigned long long)done;
  for (unsigned long long gr = proc + 1; !failed && gr <= gk_final; ++gr) {
    const unsigned long long* rs = grec + (size_t)(gr % (unsigned long long)kRecDepth) * G;
    unsigned long long rec = lane < G ? ld_relaxed_u64(rs + lane) : 0ull;
    if (cluster_wait_records(rs, lane, G, gr, rec)) {
      failed = true;
      if (lane == 0) ctl->status = SEPSO_ETIMEOUT;
    } else {
      cluster_tbest_at(p, rec, lane, Tfit, TQ, tholder, sWin, win_n, win_head, stall, prev_lfv);
    }
  }
  // Tbest's row: the holder group's Gbest row, staged in this CTA's (now unused)
  // stage area
  float* sTrow = sStage;
  const float* src = (tholder >= 0) ? gGb + (size_t)tholder * D : gTb;
  for (int j = lane; j < D; j += 32) sTrow[j] = __ldcg(src + j);
  __syncwarp();
  const int k = k0 + done;
  for (int j = lane; j < D; j += 32) {
    gTb[j] = sTrow[j];
    if (plan) {
      p.res_wp[(size_t)r * D + j] = sTrow[j];
      p.prevT[(size_t)r * D + j] = sTrow[j];
    }
  }
  for (int j = lane; j < 3 * G; j += 32) p.gword[(size_t)r * 3 * G + j] = kKeyEmpty;
  if (lane == 0) {
    // the grid-wide form's barrier counts C per iteration of the run, and expects
    // its group words empty: keep both as if it had run these iterations
    atomicAdd(&p.counter[r].count, (unsigned int)p.cta_grid * (unsigned int)done);
    ctl->Tfit = Tfit;
    ctl->TQ = TQ;
    ctl->k = k;
    ctl->iters_total += done;
    ctl->fin_launches = nfin + 1;
    if (plan) {
      ctl->plans_total += 1;
      const int nseg = T + 1;
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
