// sepso_batch.cu -- many independent scenes of uneven size (T, O, N, G) planned
// together on GB300 (sm_103a).
//
// One launch of batch_kernel advances every unfinished scene by one iteration of
// Algorithm 1.  The launch covers a host-built list of work items (scene, group,
// tile of particles), sorted by their cost (particles x segments x circles) so
// the largest items start first.  Each item:
//   1. (from the second launch on) reads its scene's group words of the previous
//      iteration and applies the group/global best updates (every item of a scene
//      computes the same values; the scene's first item stores them and the
//      winning rows for the next launch), then Eq. TOF_omega / TOF_V / TOF_X with
//      clipping for its particles;
//   2. evaluates the fitness of its particles (Eqs. path_fit / lenth / penalty)
//      with the circles bulk-copied into shared memory, applies the Pbest test
//      and publishes particles below the group best (row + Q into a slot, a
//      (fitness, index, Q) key into the group word with a 64-bit atomic min).
// The kernel boundary is the barrier of every scene at once.  A run is one reset
// launch plus max_iters + 1 iteration launches, captured once into a CUDA graph
// and replayed.  An autotuner times (tile, threads) candidates on the loaded
// batch; a particle is always evaluated by one warp, so the shape never changes
// results.  The random streams are keyed by the scene's
// run id, so a scene's result does not depend on what else is in the batch.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sepso_batch.cuh"
#include "sepso_device.cuh"
#include "sepso_internal.h"

namespace sepso {

// Bests of every scene empty, group words empty.
__global__ void batch_reset_kernel(const BatchParams p) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < p.nscenes; s += stride) {
    const BatchScene S = p.sc[s];
    for (int g = 0; g < 2 * S.G; ++g) {
      p.Gfit2[S.gso + g] = INFINITY;
      p.GQ2[S.gso + g] = 0;
    }
    for (int g = 0; g < 3 * S.G; ++g) p.words[S.wo + g] = kKeyEmpty;
    p.Tfit2[2 * s] = INFINITY;
    p.Tfit2[2 * s + 1] = INFINITY;
    p.TQ2[2 * s] = 0;
    p.TQ2[2 * s + 1] = 0;
    if (p.stall2 != nullptr) {
      p.stall2[2 * s] = p.stall2[2 * s + 1] = 0;
      p.plv2[2 * s] = p.plv2[2 * s + 1] = INFINITY;
      p.done[s] = 0;
    }
  }
}

// A failed device-side index check: the first one is recorded (status[1..3]: the
// check, the scene or work item, the index) and the access it guards is skipped.
__device__ __forceinline__ void batch_check_failed(int* status, int site, int a, int b) {
  if (atomicCAS(status + 1, 0, site) == 0) {
    status[2] = a;
    status[3] = b;
  }
  atomicCAS(status, 0, SEPSO_EBOUNDS);
}

__global__ void __launch_bounds__(512, 2) batch_kernel(const BatchParams p, int j) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t s_mbar;
  const int4 tl = p.tiles[blockIdx.x];
  const int s = tl.x, g = tl.y, n0 = tl.z, nl = tl.w;
  if (s < 0 || s >= p.nscenes) {
    if (threadIdx.x == 0) batch_check_failed(p.status, 1, (int)blockIdx.x, s);
    return;
  }
  const BatchScene S = p.sc[s];
  if (g < 0 || g >= S.G || n0 < 0 || nl < 1 || nl > p.tile || n0 + nl > S.N || S.D > p.Dmax || S.G > p.Gmax ||
      S.O > p.Omax) {
    if (threadIdx.x == 0) batch_check_failed(p.status, 2, s, (int)blockIdx.x);
    return;
  }
  const int jl = j - S.j0;  // this launch is the scene's jl-th
  if (jl < 1 || jl > S.max_iters + 1) return;  // not started, or finished
  if (p.done != nullptr && p.done[s]) return;   // truncated earlier

  const BatchSmem L = BatchSmem::make(p.Omax, p.tile, p.Dmax, p.Gmax);
  float4* sC = reinterpret_cast<float4*>(smem + L.circ);
  float* sX = reinterpret_cast<float*>(smem + L.X);
  float* sV = reinterpret_cast<float*>(smem + L.V);
  float* sP = reinterpret_cast<float*>(smem + L.P);
  float* sR = reinterpret_cast<float*>(smem + L.R);
  float* sG = reinterpret_cast<float*>(smem + L.G);
  float* sT = reinterpret_cast<float*>(smem + L.T);
  float* sPfit = reinterpret_cast<float*>(smem + L.Pfit);
  int* sPQ = reinterpret_cast<int*>(smem + L.PQ);
  float* sGfit = reinterpret_cast<float*>(smem + L.Gfit);
  int* sGQ = reinterpret_cast<int*>(smem + L.GQ);
  int* sGsrc = reinterpret_cast<int*>(smem + L.Gsrc);

  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  const int T = S.T, D = S.D, G = S.G, N = S.N, M = S.M;
  const bool fit_phase = jl <= S.max_iters;
  const bool first = (g == 0 && n0 == 0);

  if (tid == 0) mbar_init(&s_mbar, 1);
  __syncthreads();
  if (tid == 0 && fit_phase && S.O > 0) {
    const uint32_t bytes = (uint32_t)(S.poly ? edge_pair_f4(S.O) : pair_block_f4(S.O)) * 16u;
    mbar_expect_tx(&s_mbar, bytes);
    bulk_g2s(sC, p.circ + S.co, bytes, &s_mbar);
  }

  const float* hy = p.hyper + S.ho + g * 6;
  const float c1 = hy[0], c2 = hy[1], c3 = hy[2], w_init = hy[3], w_end = hy[4], vlim = hy[5];
  const float sx = p.pts[4 * s], sy = p.pts[4 * s + 1], tx = p.pts[4 * s + 2], ty = p.pts[4 * s + 3];
  float* gX = p.X + S.xo + (long long)(g * N + n0) * D;
  float* gV = p.V + S.xo + (long long)(g * N + n0) * D;
  float* gP = p.P + S.xo + (long long)(g * N + n0) * D;
  float* gPfit = p.Pfit + S.mo + g * N + n0;
  int32_t* gPQ = p.PQ + S.mo + g * N + n0;
  float* gGb = p.Gb + S.go;
  float* gTb = p.Tb + S.to;
  const uint32_t run = S.run_id;

  const uint32_t cyc = S.cycle;
  if (jl == 1) {
    // Initialisation (Algorithm 1), with Priori Initialization (Sec. 3.3.3) around
    // the agent's previous best path when it has one, after the first n_pr
    // particles placed the same way around the learned prior's proposal when the
    // scene uses it.
    const int n_pi = (S.has_prev && p.agent_prevT != nullptr && S.agent >= 0) ? S.n_pi : 0;
    const float* prevT = (n_pi > 0) ? p.agent_prevT + (long long)S.agent * p.Dmax : nullptr;
    const int n_pr = (p.prior_path != nullptr && p.prior_use[s] != 0) ? S.n_pr : 0;
    const float* priT = (n_pr > 0) ? p.prior_path + (long long)s * p.Dmax : nullptr;
    const int nch = (D + 3) >> 2;
    for (int it = tid; it < nl * nch; it += nt) {
      const int i = it / nch, ch = it - i * nch;
      const uint32_t pid = (uint32_t)(g * N + n0 + i);
      const int n = n0 + i;
      const float* ctr = (n < n_pr) ? priT : (n < n_pr + n_pi) ? prevT : nullptr;
      const uint32_t stream = (n < n_pr) ? kStreamPrior : (n < n_pr + n_pi) ? kStreamPI : kStreamInitX;
      const uint4 ux = draw(S.key0, S.key1, (uint32_t)ch, pid, stream, cyc, run);
      const uint4 uv = draw(S.key0, S.key1, (uint32_t)ch, pid, kStreamInitV, cyc, run);
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int jj = ch * 4 + l;
        if (jj < D) {
          const float ext = (jj < T) ? p.W : p.H;
          const float x = ctr ? fminf(fmaxf(ctr[jj] + (2.0f * lane_of(ux, l) - 1.0f) * S.pi_h, 0.0f), ext)
                              : lane_of(ux, l) * ext;
          sX[i * D + jj] = x;
          sP[i * D + jj] = x;
          sV[i * D + jj] = (2.0f * lane_of(uv, l) - 1.0f) * (vlim * ext);
        }
      }
    }
    for (int i = tid; i < nl; i += nt) {
      sPfit[i] = INFINITY;
      sPQ[i] = 0;
    }
    for (int gg = tid; gg < G; gg += nt) sGfit[gg] = INFINITY;
    __syncthreads();
  } else {
    // Bests of iteration k = j - 1 (every item of the scene computes the same).
    const int k = jl - 1;
    const float* oGfit = p.Gfit2 + S.gso + ((k - 1) & 1) * G;
    const int32_t* oGQ = p.GQ2 + S.gso + ((k - 1) & 1) * G;
    const unsigned long long* wk = p.words + S.wo + (k % 3) * G;
    const long long sk = S.so + (long long)(k & 1) * M * (D + 4);  // slots written at iteration k
    for (int gg = tid; gg < G; gg += nt) {
      float gf = oGfit[gg];
      int gq = oGQ[gg];
      int src = -1;
      unsigned long long key = wk[gg];
      if (key != kKeyEmpty && key_idx(key) >= N) {  // every item of the scene sees the same word
        if (g == 0 && n0 == 0) batch_check_failed(p.status, 3, s, key_idx(key));
        key = kKeyEmpty;
      }
      if (key != kKeyEmpty && key_fit(key) < gf) {
        gf = key_fit(key);
        src = gg * N + key_idx(key);
        const int qs = key_q(key);
        gq = (qs < (int)kQSat) ? qs : __float_as_int(p.slots[sk + (long long)src * (D + 4) + D]);
      }
      sGfit[gg] = gf;
      sGQ[gg] = gq;
      sGsrc[gg] = src;
    }
    __syncthreads();
    float Tfit = p.Tfit2[2 * s + ((k - 1) & 1)];
    int TQ = p.TQ2[2 * s + ((k - 1) & 1)];
    float tb = INFINITY;
    int tg = -1;
    for (int gg = 0; gg < G; ++gg) {
      if (sGfit[gg] < tb) {
        tb = sGfit[gg];
        tg = gg;
      }
    }
    int t_src = -2;  // -2 unchanged; -1 the unchanged row of group tg; >= 0 a slot
    if (tg >= 0 && tb < Tfit) {
      Tfit = tb;
      TQ = sGQ[tg];
      t_src = sGsrc[tg];
    }
    const float* trow = (t_src >= 0) ? p.slots + sk + (long long)t_src * (D + 4)
                                     : (t_src == -1 ? gGb + tg * D : gTb);
    // Truncation: the cap, or Auto Truncation by stall counter (Sec. 3.3.4).
    bool stop = (k == S.max_iters);
    int stall = 0;
    if (S.at_stall > 0) {
      const float plv = p.plv2[2 * s + ((k - 1) & 1)];
      stall = (Tfit < plv - S.stall_tol) ? 0 : p.stall2[2 * s + ((k - 1) & 1)] + 1;
      if (stall >= S.at_stall && TQ == 0) stop = true;
    }
    if (first) {
      if (S.at_stall > 0 && tid == 0) {
        p.stall2[2 * s + (k & 1)] = stall;
        p.plv2[2 * s + (k & 1)] = Tfit;
      }
      // Store the new scalars (other parity) and rows for the next launch; clear
      // the words the launch after next will fill.
      for (int gg = tid; gg < G; gg += nt) {
        p.Gfit2[S.gso + (k & 1) * G + gg] = sGfit[gg];
        p.GQ2[S.gso + (k & 1) * G + gg] = sGQ[gg];
        p.words[S.wo + ((k + 2) % 3) * G + gg] = kKeyEmpty;
      }
      if (tid == 0) {
        p.Tfit2[2 * s + (k & 1)] = Tfit;
        p.TQ2[2 * s + (k & 1)] = TQ;
      }
      for (int it = tid; it < G * D; it += nt) {
        const int gg = it / D, jj = it - gg * D;
        if (sGsrc[gg] >= 0) gGb[it] = p.slots[sk + (long long)sGsrc[gg] * (D + 4) + jj];
      }
      if (t_src != -2)
        for (int jj = tid; jj < D; jj += nt) gTb[jj] = trow[jj];
    }
    if (stop) {
      // Algorithm 1 returns F(Tbest): write the scene's result (and, for a
      // request, the agent's warm-start path).
      if (first) {
        float* warm = (S.agent >= 0 && p.agent_prevT != nullptr) ? p.agent_prevT + (long long)S.agent * p.Dmax
                                                                 : nullptr;
        for (int jj = tid; jj < D; jj += nt) {
          const float v = trow[jj];
          p.res_wp[S.to + jj] = v;
          sT[jj] = v;
          if (warm) warm[jj] = v;
        }
        __syncthreads();
        if (tid == 0) {
          float len = 0.0f;
          for (int sg = 0; sg <= T; ++sg) {
            const float ax = (sg == 0) ? sx : sT[sg - 1];
            const float ay = (sg == 0) ? sy : sT[T + sg - 1];
            const float bx = (sg == T) ? tx : sT[sg];
            const float by = (sg == T) ? ty : sT[T + sg];
            const float dx = bx - ax, dy = by - ay;
            len += sqrtf(fmaf(dx, dx, dy * dy));
          }
          sepso_result* r = p.res + s;
          r->cost = Tfit;
          r->length = len;
          r->Q = TQ;
          r->iters = k;
          r->status = SEPSO_OK;
          if (p.done != nullptr) p.done[s] = 1;
        }
      }
      // The obstacle bulk copy issued at the start must land before the CTA exits
      // (its shared memory is handed to the next CTA).
      if (tid == 0 && fit_phase && S.O > 0) mbar_wait_bounded(&s_mbar, 0, kWaitLimitNs);
      return;
    }
    // Rows for this group's update.
    const int gsrc = sGsrc[g];
    const float* grow = (gsrc >= 0) ? p.slots + sk + (long long)gsrc * (D + 4) : gGb + g * D;
    const bool need_T = c3 != 0.0f;
    for (int jj = tid; jj < D; jj += nt) {
      sG[jj] = grow[jj];
      if (need_T) sT[jj] = trow[jj];
    }
    for (int it = tid; it < nl * D; it += nt) {
      sX[it] = gX[it];
      sV[it] = gV[it];
      sP[it] = gP[it];
    }
    for (int i = tid; i < nl; i += nt) {
      sPfit[i] = gPfit[i];
      sPQ[i] = gPQ[i];
      const uint4 o = draw(S.key0, S.key1, (uint32_t)k, (uint32_t)(g * N + n0 + i), kStreamVel, cyc, run);
      sR[i * 4 + 0] = c1 * u01(o.x);
      sR[i * 4 + 1] = c2 * u01(o.y);
      sR[i * 4 + 2] = c3 * u01(o.z);
    }
    __syncthreads();
    // Eq. TOF_omega, Eq. TOF_V (+ clip to V_range), Eq. TOF_X (+ clip to X_range).
    const float w = w_init - (w_init - w_end) / (float)S.max_iters * (float)k;
    for (int it = tid; it < nl * D; it += nt) {
      const int i = it / D;
      const int jj = it - i * D;
      const float x = sX[it];
      float v = w * sV[it];
      v = fmaf(sR[i * 4 + 0], sP[it] - x, v);
      v = fmaf(sR[i * 4 + 1], sG[jj] - x, v);
      if (need_T) v = fmaf(sR[i * 4 + 2], sT[jj] - x, v);
      const float ext = (jj < T) ? p.W : p.H;
      const float vmax = vlim * ext;
      v = fminf(fmaxf(v, -vmax), vmax);
      sV[it] = v;
      sX[it] = fminf(fmaxf(x + v, 0.0f), ext);
    }
    __syncthreads();
  }

  // Fitness of iteration j, Pbest test and publication.
  if (S.O > 0 && !mbar_wait_bounded(&s_mbar, 0, kWaitLimitNs)) {
    if (threadIdx.x == 0) atomicExch(p.status, SEPSO_ETIMEOUT);
  }
  __syncthreads();
  {
    // A warp per particle; the lanes also split the circles so that the warp's
    // rounds are nearly full.  Both depend only on the scene, so results do not
    // depend on the launch shape.
    const int lp = 32;
    const int ppw = 1;
    const int lsub = lane;
    const int K = circle_pairs(S.O);
    const int split = warp_split(T, S.poly ? (S.O + 1) / 2 : K);
    const float2* sNr2 = reinterpret_cast<const float2*>(sC + K);
    const long long sj = S.so + (long long)(jl & 1) * M * (D + 4);
    for (int i0 = warp * ppw; i0 < nl; i0 += nwarps * ppw) {
      const int i = i0 + lane / lp;
      const bool live = i < nl;
      float len;
      int qq;
      if (S.poly)
        group_fitness_edge_pairs(sX + (live ? i : 0) * D, live, lp, T, split, S.O, sx, sy, tx, ty, sC, &len, &qq);
      else
        group_fitness_pairs(sX + (live ? i : 0) * D, live, lp, T, split, K, sx, sy, tx, ty, sC, sNr2, &len, &qq);
      if (S.nteam > 1)  // the team mates' paths as moving obstacles
        qq += agent_conflicts(sX + (live ? i : 0) * D, T, sx, sy, tx, ty, p.agent_rows + (long long)S.team0 * (p.Dmax + 4),
                              p.Dmax + 4, S.nteam, s - S.team0, S.sep2, lane);
      int imp = 0, pub = 0;
      float pf = INFINITY;
      int pq = 0;
      if (live && lsub == 0) {
        const float F = len + S.alpha * powi((float)qq, S.beta);
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
        float* slot = p.slots + sj + (long long)(g * N + n0 + i) * (D + 4);
        for (int jj = lsub; jj < D; jj += lp) {
          const float v = imp ? sX[i * D + jj] : sP[i * D + jj];
          if (imp) sP[i * D + jj] = v;
          if (pub) slot[jj] = v;
        }
        if (pub && lsub == 0) {
          slot[D] = __int_as_float(pq);
          red_min_u64(p.words + S.wo + (jl % 3) * G + g, best_key(pf, (uint32_t)(n0 + i), (uint32_t)pq));
        }
      }
    }
  }
  __syncthreads();
  for (int it = tid; it < nl * D; it += nt) {
    gX[it] = sX[it];
    gV[it] = sV[it];
    gP[it] = sP[it];
  }
  for (int i = tid; i < nl; i += nt) {
    gPfit[i] = sPfit[i];
    gPQ[i] = sPQ[i];
  }
}

cudaError_t batch_configure(int* smem_optin_out) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, batch_kernel);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess && smem_optin_out) *smem_optin_out = optin - (int)fa.sharedSizeBytes;
  return e;
}

cudaError_t launch_batch_reset(const BatchParams& p, cudaStream_t s) {
  batch_reset_kernel<<<std::max(1, std::min(1024, (p.nscenes + 255) / 256)), 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_batch_iter(const BatchParams& p, int j, int ntiles, int threads, size_t smem, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  batch_kernel<<<ntiles, threads, smem, s>>>(p, j);
  return cudaGetLastError();
}

// Learned-prior gate, one warp per scene: the proposal seeds the scene only when
// its fitness (Sec. 3.3.2, FP32, the swarm's own evaluation) is below that of the
// scene's previous path, or the scene has none.
__global__ void batch_gate_kernel(const BatchParams p) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= p.nscenes) return;  // warp-uniform
  const int s = warp;
  const BatchScene S = p.sc[s];
  int32_t* use = const_cast<int32_t*>(p.prior_use);
  if (S.n_pr == 0) {
    if (lane == 0) use[s] = 0;
    return;
  }
  const float sx = p.pts[4 * s], sy = p.pts[4 * s + 1], tx = p.pts[4 * s + 2], ty = p.pts[4 * s + 3];
  const int K = circle_pairs(S.O);
  const int split = warp_split(S.T, S.poly ? (S.O + 1) / 2 : K);
  const float4* cxy = p.circ + S.co;
  const float2* nr2 = reinterpret_cast<const float2*>(cxy + K);
  float len;
  int q;
  if (S.poly)
    group_fitness_edge_pairs(p.prior_path + (long long)s * p.Dmax, true, 32, S.T, split, S.O, sx, sy, tx, ty, cxy, &len,
                        &q);
  else
    group_fitness_pairs(p.prior_path + (long long)s * p.Dmax, true, 32, S.T, split, K, sx, sy, tx, ty, cxy, nr2,
                        &len, &q);
  const float f_prior = len + S.alpha * powi((float)q, S.beta);
  int ok = 1;
  if (S.has_prev && S.n_pi > 0) {
    if (S.poly)
      group_fitness_edge_pairs(p.agent_prevT + (long long)s * p.Dmax, true, 32, S.T, split, S.O, sx, sy, tx, ty, cxy,
                          &len, &q);
    else
      group_fitness_pairs(p.agent_prevT + (long long)s * p.Dmax, true, 32, S.T, split, K, sx, sy, tx, ty, cxy, nr2,
                          &len, &q);
    const float f_prev = len + S.alpha * powi((float)q, S.beta);
    ok = f_prior < f_prev;
  }
  if (lane == 0) use[s] = ok;
}

// Timed paths of the agents from the scenes' results: start, the result's
// waypoints, target (one scene per warp lane group).
__global__ void agent_rows_kernel(const BatchParams p) {
  const int ld = p.Dmax + 4;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < (long long)p.nscenes * ld;
       it += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(it / ld), j = (int)(it - (long long)s * ld);
    const BatchScene S = p.sc[s];
    const int T = S.T, P = T + 2;
    if (j >= 2 * P) continue;
    const int xy = j / P, k = j - xy * P;  // coordinate, point
    float v;
    if (k == 0) v = p.pts[4 * s + xy];
    else if (k == P - 1) v = p.pts[4 * s + 2 + xy];
    else v = p.res_wp[S.to + xy * T + (k - 1)];
    p.agent_rows[(long long)s * ld + j] = v;
  }
}

cudaError_t launch_agent_rows(const BatchParams& p, cudaStream_t s) {
  const long long total = (long long)p.nscenes * (p.Dmax + 4);
  agent_rows_kernel<<<(int)std::min<long long>((total + 255) / 256, 4096), 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_batch_gate(const BatchParams& p, cudaStream_t s) {
  const int threads = 128;
  const int blocks = (p.nscenes * 32 + threads - 1) / threads;
  batch_gate_kernel<<<blocks, threads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace sepso

using namespace sepso;

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

thread_local std::string g_batch_error;

int bfail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int bfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_batch_error = buf;
  return code;
}

#define BCUDA(expr)                                                                        \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess) return bfail(SEPSO_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

size_t al256(size_t v) { return (v + 255) & ~size_t(255); }

constexpr int kMinTile = 8;

struct BatchLayout {
  size_t sc, tiles, X, V, P, Pfit, PQ, slots, Gb, Tb, circ, hyper, pts, words, Gfit2, GQ2, Tfit2, TQ2, res_wp, res,
      stall2, plv2, done, prevT, priorT, prior_use, status, arows, total;
  long long nX, nM, nS, nG, nT, nC, nH, nW, nGS, ntiles_max, Dmax;
};

int check_scenes(const sepso_batch_scene* sc, int32_t n) {
  if (!sc || n < 1) return bfail(SEPSO_EINVAL, "need at least one scene");
  for (int s = 0; s < n; ++s) {
    const sepso_batch_scene& c = sc[s];
    if (c.T < 1 || c.T > 64 || c.G < 1 || c.G > 32 || c.N < 1 || c.N >= (1 << 20) || c.O < 0 || c.O > 8192 ||
        c.max_iters < 1 || c.beta < 1 || c.beta > 8 || !std::isfinite(c.alpha) || c.alpha < 0)
      return bfail(SEPSO_EINVAL, "scene %d: bad shape or parameters", s);
    if (c.obstacle_kind != 0 && c.obstacle_kind != 1)
      return bfail(SEPSO_EINVAL, "scene %d: obstacle_kind %d is neither 0 (circles) nor 1 (polygons)", s,
                   c.obstacle_kind);
    if (c.stall_iters < 0 || !std::isfinite(c.stall_tol) || c.stall_tol < 0 || c.n_pi < 0 || c.n_prior < 0 ||
        c.n_pi > c.N || c.n_prior > c.N || !std::isfinite(c.pi_halfwidth) || c.pi_halfwidth < 0)
      return bfail(SEPSO_EINVAL, "scene %d: bad truncation or warm-start parameters", s);
  }
  return SEPSO_OK;
}

BatchLayout batch_layout(const sepso_batch_scene* sc, int32_t n) {
  BatchLayout L{};
  for (int s = 0; s < n; ++s) {
    const long long D = 2 * sc[s].T, M = (long long)sc[s].G * sc[s].N;
    L.nX += M * D;
    L.nM += M;
    L.nS += 2 * M * (D + 4);
    L.nG += (long long)sc[s].G * D;
    L.nT += D;
    L.nC += sc[s].O > 0 ? (sc[s].obstacle_kind ? edge_pair_f4(sc[s].O) : pair_block_f4(sc[s].O)) : 0;
    L.nH += 6LL * sc[s].G;
    L.nW += 3LL * sc[s].G;
    L.nGS += 2LL * sc[s].G;
    L.ntiles_max += (long long)sc[s].G * ((sc[s].N + kMinTile - 1) / kMinTile);
    L.Dmax = std::max(L.Dmax, D);
  }
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = al256(off);
    const size_t o = off;
    off += bytes;
    return o;
  };
  L.sc = take((size_t)n * sizeof(BatchScene));
  L.tiles = take((size_t)L.ntiles_max * sizeof(int4));
  L.X = take((size_t)L.nX * 4);
  L.V = take((size_t)L.nX * 4);
  L.P = take((size_t)L.nX * 4);
  L.Pfit = take((size_t)L.nM * 4);
  L.PQ = take((size_t)L.nM * 4);
  L.slots = take((size_t)L.nS * 4);
  L.Gb = take((size_t)L.nG * 4);
  L.Tb = take((size_t)L.nT * 4);
  L.circ = take((size_t)std::max(L.nC, 1LL) * 16);
  L.hyper = take((size_t)L.nH * 4);
  L.pts = take((size_t)n * 16);
  L.words = take((size_t)L.nW * 8);
  L.Gfit2 = take((size_t)L.nGS * 4);
  L.GQ2 = take((size_t)L.nGS * 4);
  L.Tfit2 = take((size_t)n * 8);
  L.TQ2 = take((size_t)n * 8);
  L.res_wp = take((size_t)L.nT * 4);
  L.res = take((size_t)n * sizeof(sepso_result));
  L.stall2 = take((size_t)n * 8);
  L.plv2 = take((size_t)n * 8);
  L.done = take((size_t)n * 4);
  L.prevT = take((size_t)n * L.Dmax * 4);
  L.priorT = take((size_t)n * L.Dmax * 4);
  L.prior_use = take((size_t)n * 4);
  L.status = take(16);  // status, then the first failed index check: site, scene, index
  L.arows = take((size_t)n * (L.Dmax + 4) * 4);  // multi-agent timed paths
  L.total = al256(off);
  return L;
}

}  // namespace

struct sepso_batch_ctx {
  std::vector<sepso_batch_scene> scenes;
  std::vector<BatchScene> desc;
  int n = 0;
  float W = 0, H = 0;
  int device = 0, num_sms = 0, smem_optin = 0;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  BatchLayout L{};
  int Omax = 0, Dmax = 0, Gmax = 0, Kmax = 0;
  sepso_batch_shape shape{32, 256, 32, 0};
  int ntiles = 0;
  size_t smem = 0;
  bool inputs = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;
  std::vector<int> team_size;  // per scene, when teams are set
  float sep2 = 0.0f;

  ~sepso_batch_ctx() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
  template <class T>
  T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
};

namespace {

BatchParams batch_params(const sepso_batch_ctx* h) {
  BatchParams p;
  p.sc = h->at<BatchScene>(h->L.sc);
  p.tiles = h->at<int4>(h->L.tiles);
  p.ntiles = h->ntiles;
  p.nscenes = h->n;
  p.W = h->W;
  p.H = h->H;
  p.Omax = h->Omax;
  p.Dmax = h->Dmax;
  p.Gmax = h->Gmax;
  p.tile = h->shape.tile;
  p.X = h->at<float>(h->L.X);
  p.V = h->at<float>(h->L.V);
  p.P = h->at<float>(h->L.P);
  p.Pfit = h->at<float>(h->L.Pfit);
  p.PQ = h->at<int32_t>(h->L.PQ);
  p.slots = h->at<float>(h->L.slots);
  p.Gb = h->at<float>(h->L.Gb);
  p.Tb = h->at<float>(h->L.Tb);
  p.circ = h->at<float4>(h->L.circ);
  p.hyper = h->at<float>(h->L.hyper);
  p.pts = h->at<float>(h->L.pts);
  p.words = h->at<unsigned long long>(h->L.words);
  p.Gfit2 = h->at<float>(h->L.Gfit2);
  p.GQ2 = h->at<int32_t>(h->L.GQ2);
  p.Tfit2 = h->at<float>(h->L.Tfit2);
  p.TQ2 = h->at<int32_t>(h->L.TQ2);
  p.res_wp = h->at<float>(h->L.res_wp);
  p.res = h->at<sepso_result>(h->L.res);
  p.status = h->at<int>(h->L.status);
  p.stall2 = h->at<int32_t>(h->L.stall2);
  p.plv2 = h->at<float>(h->L.plv2);
  p.done = h->at<int32_t>(h->L.done);
  p.agent_prevT = h->at<float>(h->L.prevT);
  p.prior_path = h->at<float>(h->L.priorT);
  p.prior_use = h->at<int32_t>(h->L.prior_use);
  p.agent_rows = h->at<float>(h->L.arows);
  return p;
}

// Work items for a tile size, largest first.
int build_tiles(sepso_batch_ctx* h, int tile) {
  std::vector<int4> t;
  std::vector<double> cost;
  for (int s = 0; s < h->n; ++s) {
    const sepso_batch_scene& c = h->scenes[s];
    for (int g = 0; g < c.G; ++g)
      for (int n0 = 0; n0 < c.N; n0 += tile) {
        const int nl = std::min(tile, c.N - n0);
        t.push_back(make_int4(s, g, n0, nl));
        cost.push_back((double)nl * (c.T + 1) * (std::max(c.O, 1) + 8));
      }
  }
  std::vector<int> order(t.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<int4> sorted(t.size());
  for (size_t i = 0; i < order.size(); ++i) sorted[i] = t[order[i]];
  if ((long long)sorted.size() > h->L.ntiles_max) return bfail(SEPSO_ERANGE, "too many work items");
  BCUDA(cudaMemcpyAsync(h->ws + h->L.tiles, sorted.data(), sorted.size() * sizeof(int4), cudaMemcpyHostToDevice,
                        h->stream));
  BCUDA(cudaStreamSynchronize(h->stream));
  h->ntiles = (int)sorted.size();
  return SEPSO_OK;
}

int apply_shape(sepso_batch_ctx* h, const sepso_batch_shape& sh) {
  if (sh.tile < kMinTile || sh.tile > 256 || (sh.lanes != 0 && sh.lanes != 32) || sh.threads < 64 ||
      sh.threads > 512 || sh.threads % 32)
    return bfail(SEPSO_EINVAL, "bad batch shape (tile %d, threads %d, lanes %d)", sh.tile, sh.threads, sh.lanes);
  const BatchSmem S = BatchSmem::make(h->Omax, sh.tile, h->Dmax, h->Gmax);
  if ((size_t)S.total + 256 > (size_t)h->smem_optin)
    return bfail(SEPSO_ERANGE, "batch shape needs %d B of shared memory", S.total);
  int rc = build_tiles(h, sh.tile);
  if (rc) return rc;
  h->shape = sh;
  h->smem = (size_t)S.total;
  if (h->exec) {
    cudaGraphExecDestroy(h->exec);
    h->exec = nullptr;
  }
  if (h->graph) {
    cudaGraphDestroy(h->graph);
    h->graph = nullptr;
  }
  return SEPSO_OK;
}

// reset + Kmax + 1 iteration launches on the handle's stream.
int enqueue_run(sepso_batch_ctx* h, int upto) {
  const BatchParams p = batch_params(h);
  batch_reset_kernel<<<std::max(1, std::min(1024, (h->n + 255) / 256)), 256, 0, h->stream>>>(p);
  BCUDA(cudaGetLastError());
  for (int j = 1; j <= upto; ++j) {
    batch_kernel<<<h->ntiles, h->shape.threads, h->smem, h->stream>>>(p, j);
    BCUDA(cudaGetLastError());
  }
  return SEPSO_OK;
}

}  // namespace

extern "C" {

const char* sepso_batch_last_error(void) { return g_batch_error.c_str(); }

int sepso_batch_workspace_size(const sepso_batch_scene* scenes, int32_t n, size_t* bytes) {
  int rc = check_scenes(scenes, n);
  if (rc) return rc;
  if (!bytes) return bfail(SEPSO_EINVAL, "bytes is NULL");
  *bytes = batch_layout(scenes, n).total;
  return SEPSO_OK;
}

int sepso_batch_create(const sepso_batch_scene* scenes, int32_t n, float map_w, float map_h, void* d_workspace,
                       size_t bytes, void* stream, sepso_batch_handle* out) {
  int rc = check_scenes(scenes, n);
  if (rc) return rc;
  if (!out) return bfail(SEPSO_EINVAL, "out is NULL");
  *out = nullptr;
  if (!std::isfinite(map_w) || !std::isfinite(map_h) || map_w <= 0 || map_h <= 0)
    return bfail(SEPSO_EINVAL, "map extent must be finite and positive");
  const BatchLayout L = batch_layout(scenes, n);
  if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255u))
    return bfail(SEPSO_ENOSPC, "workspace must be non-NULL and 256-byte aligned");
  if (bytes < L.total) return bfail(SEPSO_ENOSPC, "workspace has %zu bytes, needs %zu", bytes, L.total);
  sepso_batch_ctx* h = new (std::nothrow) sepso_batch_ctx();
  if (!h) return bfail(SEPSO_ENOMEM, "host allocation failed");
  h->scenes.assign(scenes, scenes + n);
  h->n = n;
  h->W = map_w;
  h->H = map_h;
  h->stream = static_cast<cudaStream_t>(stream);
  h->ws = static_cast<char*>(d_workspace);
  h->L = L;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, batch_kernel);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             h->smem_optin - (int)fa.sharedSizeBytes);
  if (e != cudaSuccess) {
    delete h;
    return bfail(SEPSO_ECUDA, "device setup: %s", cudaGetErrorString(e));
  }
  h->smem_optin -= (int)fa.sharedSizeBytes;
  // Scene descriptors.
  long long xo = 0, mo = 0, so = 0, go = 0, to = 0, co = 0, ho = 0, wo = 0, gso = 0;
  h->desc.resize(n);
  for (int s = 0; s < n; ++s) {
    const sepso_batch_scene& c = scenes[s];
    BatchScene& d = h->desc[s];
    d.T = c.T;
    d.D = 2 * c.T;
    d.G = c.G;
    d.N = c.N;
    d.M = c.G * c.N;
    d.O = c.O;
    d.max_iters = c.max_iters;
    d.beta = c.beta;
    d.alpha = c.alpha;
    d.key0 = (uint32_t)(c.seed & 0xffffffffu);
    d.key1 = (uint32_t)(c.seed >> 32);
    d.run_id = c.run_id;
    d.xo = xo; xo += (long long)d.M * d.D;
    d.mo = mo; mo += d.M;
    d.so = so; so += 2LL * d.M * (d.D + 4);
    d.go = go; go += (long long)d.G * d.D;
    d.to = to; to += d.D;
    d.co = co; co += d.O > 0 ? (c.obstacle_kind ? edge_pair_f4(d.O) : pair_block_f4(d.O)) : 0;
    d.ho = ho; ho += 6LL * d.G;
    d.wo = wo; wo += 3LL * d.G;
    d.gso = gso; gso += 2LL * d.G;
    d.j0 = 0;
    d.at_stall = c.stall_iters;
    d.stall_tol = c.stall_tol;
    d.n_pi = c.n_pi;
    d.n_pr = c.n_prior;
    d.pi_h = c.pi_halfwidth;
    d.cycle = c.cycle;
    d.agent = s;  // row of the scene's previous path (PI centre, written by every run)
    d.has_prev = 0;
    d.team0 = s;
    d.nteam = 0;
    d.sep2 = 0.0f;
    d.pad_team = 0;
    d.poly = c.obstacle_kind;
    d.pad_poly = 0;
    // the shared-memory obstacle area holds pair_block_f4(Omax) float4s: E edges
    // need edge_pair_f4(E), which pair_block_f4(2 E) covers
    h->Omax = std::max(h->Omax, c.obstacle_kind ? 2 * c.O : c.O);
    h->Dmax = std::max(h->Dmax, 2 * c.T);
    h->Gmax = std::max(h->Gmax, c.G);
    h->Kmax = std::max(h->Kmax, c.max_iters);
  }
  e = cudaMemsetAsync(h->ws, 0, L.total, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->ws + L.sc, h->desc.data(), h->desc.size() * sizeof(BatchScene), cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    delete h;
    return bfail(SEPSO_ECUDA, "workspace initialisation: %s", cudaGetErrorString(e));
  }
  sepso_batch_shape sh{32, 256, 32, 0};
  rc = apply_shape(h, sh);
  if (rc) {
    sh.tile = 16;
    rc = apply_shape(h, sh);
  }
  if (rc) {
    delete h;
    return rc;
  }
  *out = h;
  return SEPSO_OK;
}

void sepso_batch_destroy(sepso_batch_handle h) { delete h; }

int sepso_batch_set_inputs(sepso_batch_handle h, const float* hyper, const float* points, const float* circles) {
  if (!h || !hyper || !points) return bfail(SEPSO_EINVAL, "NULL argument");
  const BatchLayout& L = h->L;
  for (long long i = 0; i < L.nH; ++i)
    if (!std::isfinite(hyper[i])) return bfail(SEPSO_EINVAL, "hyper[%lld] not finite", i);
  for (int i = 0; i < 4 * h->n; ++i)
    if (!std::isfinite(points[i])) return bfail(SEPSO_EINVAL, "points[%d] not finite", i);
  if (L.nC > 0 && !circles) return bfail(SEPSO_EINVAL, "circles is NULL");
  // circle-pair blocks, or a polygon scene's edge pairs (layouts in sepso_device.cuh)
  std::vector<float4> c4((size_t)std::max(L.nC, 1LL), make_float4(0.0f, 0.0f, 0.0f, 0.0f));
  long long src = 0;  // float offset into circles
  for (int s = 0; s < h->n; ++s) {
    const int O = h->scenes[s].O;
    if (O == 0) continue;
    float4* blk = c4.data() + h->desc[s].co;
    if (h->scenes[s].obstacle_kind) {
      for (int i = 0; i < 4 * O; ++i)
        if (!std::isfinite(circles[src + i])) return bfail(SEPSO_EINVAL, "scene %d: edge %d not finite", s, i / 4);
      pack_edge_pairs(circles + src, O, blk);
      src += 4 * (long long)O;
      continue;
    }
    const int K = circle_pairs(O);
    float* nr2 = reinterpret_cast<float*>(blk + K);
    for (int o = 0; o < O; ++o, src += 3) {
      const float cx = circles[src], cy = circles[src + 1], r = circles[src + 2];
      if (!std::isfinite(cx) || !std::isfinite(cy) || !std::isfinite(r) || r < 0)
        return bfail(SEPSO_EINVAL, "scene %d: circle %d invalid", s, o);
      float* pr = reinterpret_cast<float*>(blk + o / 2);
      pr[o & 1] = cx;
      pr[2 + (o & 1)] = cy;
      nr2[o] = -(r * r);
    }
  }
  BCUDA(cudaMemcpyAsync(h->ws + L.hyper, hyper, (size_t)L.nH * 4, cudaMemcpyHostToDevice, h->stream));
  BCUDA(cudaMemcpyAsync(h->ws + L.pts, points, (size_t)h->n * 16, cudaMemcpyHostToDevice, h->stream));
  if (L.nC > 0)
    BCUDA(cudaMemcpyAsync(h->ws + L.circ, c4.data(), (size_t)L.nC * 16, cudaMemcpyHostToDevice, h->stream));
  BCUDA(cudaStreamSynchronize(h->stream));
  h->inputs = true;
  return SEPSO_OK;
}

int sepso_batch_set_shape(sepso_batch_handle h, const sepso_batch_shape* shape) {
  if (!h || !shape) return bfail(SEPSO_EINVAL, "NULL argument");
  return apply_shape(h, *shape);
}

int sepso_batch_get_shape(sepso_batch_handle h, sepso_batch_shape* shape, int32_t* work_items) {
  if (!h) return bfail(SEPSO_EINVAL, "NULL handle");
  if (shape) *shape = h->shape;
  if (work_items) *work_items = h->ntiles;
  return SEPSO_OK;
}

int sepso_batch_autotune(sepso_batch_handle h, int32_t trial_launches, sepso_batch_shape* best, float* best_ms) {
  if (!h) return bfail(SEPSO_EINVAL, "NULL handle");
  if (!h->inputs) return bfail(SEPSO_ESTATE, "autotune before set_inputs");
  const int trials = std::max(2, std::min((int)trial_launches, h->Kmax + 1));
  const sepso_batch_shape keep = h->shape;
  sepso_batch_shape win = keep;
  float win_ms = INFINITY;
  cudaEvent_t e0, e1;
  BCUDA(cudaEventCreate(&e0));
  BCUDA(cudaEventCreate(&e1));
  const int tiles[] = {8, 16, 32, 64};
  const int threads[] = {128, 256, 512};
  for (int tl : tiles)
    for (int th : threads) {
        sepso_batch_shape sh{tl, th, 32, 0};
        if (apply_shape(h, sh)) continue;
        // time launches 2..trials (update + fitness), after the first (init + fitness)
        if (enqueue_run(h, 1)) continue;
        const BatchParams p = batch_params(h);
        cudaEventRecord(e0, h->stream);
        for (int j = 2; j <= trials; ++j) batch_kernel<<<h->ntiles, th, h->smem, h->stream>>>(p, j);
        cudaEventRecord(e1, h->stream);
        const cudaError_t se = cudaStreamSynchronize(h->stream);
        if (se != cudaSuccess) {  // a device-side fault is sticky: report it here, not at a later call
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return bfail(SEPSO_ECUDA, "autotune trial (tile %d, threads %d): %s", tl, th, cudaGetErrorString(se));
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        h->launches += trials + 1;
        if (ms < win_ms) {
          win_ms = ms;
          win = sh;
        }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  int rc = apply_shape(h, win);
  if (rc) return rc;
  if (best) *best = win;
  if (best_ms) *best_ms = win_ms / (float)(trials - 1);
  (void)keep;
  return SEPSO_OK;
}

int sepso_batch_set_starts(sepso_batch_handle h, const float* prev, const float* prior, int32_t ld,
                           const int32_t* has_prev) {
  if (!h) return bfail(SEPSO_EINVAL, "NULL handle");
  const long long Dm = h->L.Dmax;
  if ((prev || prior) && ld < Dm) return bfail(SEPSO_EINVAL, "ld %d below the largest 2T (%lld)", ld, Dm);
  if (prev)
    BCUDA(cudaMemcpy2DAsync(h->ws + h->L.prevT, (size_t)Dm * 4, prev, (size_t)ld * 4, (size_t)Dm * 4, (size_t)h->n,
                            cudaMemcpyDeviceToDevice, h->stream));
  if (has_prev || prev) {
    for (int s = 0; s < h->n; ++s) h->desc[s].has_prev = has_prev ? (has_prev[s] != 0) : 1;
    BCUDA(cudaMemcpyAsync(h->ws + h->L.sc, h->desc.data(), h->desc.size() * sizeof(BatchScene),
                          cudaMemcpyHostToDevice, h->stream));
  }
  if (prior) {
    BCUDA(cudaMemcpy2DAsync(h->ws + h->L.priorT, (size_t)Dm * 4, prior, (size_t)ld * 4, (size_t)Dm * 4,
                            (size_t)h->n, cudaMemcpyDeviceToDevice, h->stream));
    if (!h->inputs) return bfail(SEPSO_ESTATE, "the prior gate needs the scenes' inputs (set_inputs first)");
    BCUDA(launch_batch_gate(batch_params(h), h->stream));
    ++h->launches;
  } else {
    BCUDA(cudaMemsetAsync(h->ws + h->L.prior_use, 0, (size_t)h->n * 4, h->stream));
  }
  BCUDA(cudaStreamSynchronize(h->stream));
  return SEPSO_OK;
}

int sepso_batch_set_teams(sepso_batch_handle h, const int32_t* team_first, const int32_t* team_size, float sep) {
  if (!h || !team_first || !team_size) return bfail(SEPSO_EINVAL, "NULL argument");
  if (!(sep >= 0.0f) || !std::isfinite(sep)) return bfail(SEPSO_EINVAL, "sep must be finite and >= 0");
  for (int s = 0; s < h->n; ++s) {
    const int f = team_first[s], z = team_size[s];
    if (z < 1 || f < 0 || f > s || s >= f + z || f + z > h->n)
      return bfail(SEPSO_EINVAL, "scene %d: team [%d, %d) does not hold it", s, f, f + z);
    if (team_first[f] != f || team_size[f] != z || h->desc[f].T != h->desc[s].T)
      return bfail(SEPSO_EINVAL, "scene %d: its team must be contiguous with one T", s);
  }
  h->team_size.assign(team_size, team_size + h->n);
  h->sep2 = sep * sep;
  for (int s = 0; s < h->n; ++s) {
    h->desc[s].team0 = team_first[s];
    h->desc[s].nteam = 0;  // the mates' paths count from the first sepso_batch_next_round
    h->desc[s].sep2 = h->sep2;
  }
  BCUDA(cudaMemcpyAsync(h->ws + h->L.sc, h->desc.data(), h->desc.size() * sizeof(BatchScene), cudaMemcpyHostToDevice,
                        h->stream));
  BCUDA(cudaStreamSynchronize(h->stream));
  return SEPSO_OK;
}

int sepso_batch_next_round(sepso_batch_handle h, uint32_t cycle) {
  if (!h) return bfail(SEPSO_EINVAL, "NULL handle");
  if (h->team_size.empty()) return bfail(SEPSO_ESTATE, "no teams (sepso_batch_set_teams first)");
  BCUDA(launch_agent_rows(batch_params(h), h->stream));
  ++h->launches;
  for (int s = 0; s < h->n; ++s) {
    h->desc[s].nteam = h->team_size[s];
    h->desc[s].cycle = cycle;
    h->desc[s].has_prev = 1;  // each run stores its result as the scene's PI centre
  }
  BCUDA(cudaMemcpyAsync(h->ws + h->L.sc, h->desc.data(), h->desc.size() * sizeof(BatchScene), cudaMemcpyHostToDevice,
                        h->stream));
  BCUDA(cudaStreamSynchronize(h->stream));
  return SEPSO_OK;
}

int sepso_batch_prior_used(sepso_batch_handle h, int32_t* n_used) {
  if (!h || !n_used) return bfail(SEPSO_EINVAL, "NULL argument");
  std::vector<int32_t> u((size_t)h->n);
  BCUDA(cudaMemcpyAsync(u.data(), h->ws + h->L.prior_use, u.size() * 4, cudaMemcpyDeviceToHost, h->stream));
  BCUDA(cudaStreamSynchronize(h->stream));
  int32_t c = 0;
  for (int32_t v : u) c += v != 0;
  *n_used = c;
  return SEPSO_OK;
}

int sepso_batch_run_async(sepso_batch_handle h, int32_t use_graph) {
  if (!h) return bfail(SEPSO_EINVAL, "NULL handle");
  if (!h->inputs) return bfail(SEPSO_ESTATE, "run before set_inputs");
  if (!use_graph) {
    const int rc = enqueue_run(h, h->Kmax + 1);
    if (rc) return rc;
    h->launches += h->Kmax + 2;
    return SEPSO_OK;
  }
  if (!h->exec) {
    // Capture the whole run (reset + every iteration launch) once.
    cudaStream_t cap = nullptr;
    BCUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t keep = h->stream;
    h->stream = cap;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    int rc = SEPSO_OK;
    if (e == cudaSuccess) rc = enqueue_run(h, h->Kmax + 1);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    h->stream = keep;
    cudaStreamDestroy(cap);
    if (e != cudaSuccess || e2 != cudaSuccess || rc)
      return rc ? rc : bfail(SEPSO_ECUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    h->graph = g;
    BCUDA(cudaGraphInstantiate(&h->exec, g, 0));
  }
  BCUDA(cudaGraphLaunch(h->exec, h->stream));
  h->launches += h->Kmax + 2;
  return SEPSO_OK;
}

int sepso_batch_read(sepso_batch_handle h, float* waypoints, sepso_result* res) {
  if (!h) return bfail(SEPSO_EINVAL, "NULL handle");
  if (waypoints)
    BCUDA(cudaMemcpyAsync(waypoints, h->ws + h->L.res_wp, (size_t)h->L.nT * 4, cudaMemcpyDeviceToHost, h->stream));
  if (res)
    BCUDA(cudaMemcpyAsync(res, h->ws + h->L.res, (size_t)h->n * sizeof(sepso_result), cudaMemcpyDeviceToHost,
                          h->stream));
  int st[4] = {0, 0, 0, 0};
  BCUDA(cudaMemcpyAsync(st, h->ws + h->L.status, 16, cudaMemcpyDeviceToHost, h->stream));
  BCUDA(cudaStreamSynchronize(h->stream));
  if (st[0])
    return bfail(st[0], "device-side error in the batch (index check %d: scene/item %d, index %d)", st[1], st[2],
                 st[3]);
  return SEPSO_OK;
}

int64_t sepso_batch_launch_count(sepso_batch_handle h) { return h ? h->launches : -1; }

}  // extern "C"
