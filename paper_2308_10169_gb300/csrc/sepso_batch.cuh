// sepso_batch.cuh -- records shared by the batched kernels (sepso_batch.cu) and
// the request server (sepso_server.cu).  Internal to libsepso.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sepso.h"
#include "sepso_device.cuh"

namespace sepso {

struct BatchScene {
  int T, D, G, N, M, O, max_iters, beta;
  float alpha;
  uint32_t key0, key1, run_id;
  long long xo;   // float offset of the scene's rows in X, V, P (M x D)
  long long mo;   // offset in Pfit, PQ (M)
  long long so;   // float offset of the candidate slots (2 x M x (D + 4))
  long long go;   // float offset of the Gbest rows (G x D)
  long long to;   // float offset of the Tbest row and the result row (D)
  long long co;   // float4 offset of the scene's circle-pair block (pair_block_f4(O) float4s)
  long long ho;   // float offset of the hyper-parameters (G x 6)
  long long wo;   // offset of the group words (3 x G)
  long long gso;  // offset of the group scalars Gfit / GQ (2 x G, by parity)
  // Request-slot fields (all zero / -1 for a plain batch run):
  int j0;          // launch index before the scene's first iteration (iteration k runs at j0 + k)
  int at_stall;    // 0: run max_iters; else Auto Truncation by stall counter with this limit
  float stall_tol;
  int n_pi;        // particles per group placed by Priori Initialization (when agent has_prev)
  int n_pr;        // particles per group placed around the learned prior's proposal (when used)
  float pi_h;      // half-width of the PI interval
  uint32_t cycle;  // Philox counter word 2 (low 24 bits): the agent's planning cycle
  int agent;       // row of the warm-start table (-1: none)
  int has_prev;    // the agent has a previous best path
  // Multi-agent teams (a plain batch or a request: nteam = 0):
  int team0;       // first scene of this scene's team (scenes team0 .. team0 + nteam - 1)
  int nteam;       // agents in the team whose paths count, 0 until their first paths exist
  float sep2;      // squared separation below which two agents conflict
  int pad_team;
  int poly;        // 1: the obstacle block holds O polygon edges (x0, y0, x1, y1), not circle pairs
  int pad_poly;
};

struct BatchParams {
  const BatchScene* sc;
  const int4* tiles;   // (scene, group, first particle, particles)
  int ntiles, nscenes;
  float W, H;
  int Omax, Dmax, Gmax, tile;
  float *X, *V, *P, *Pfit;
  int32_t* PQ;
  float* slots;
  float *Gb, *Tb;
  const float4* circ;  // circle-pair blocks of the scenes
  const float* hyper;
  const float* pts;    // 4 per scene: start, target
  unsigned long long* words;
  float* Gfit2;
  int32_t* GQ2;
  float* Tfit2;        // 2 per scene
  int32_t* TQ2;
  float* res_wp;
  sepso_result* res;
  int* status;
  // Request slots (null for a plain batch run):
  int32_t* stall2;     // 2 per scene, by parity
  float* plv2;         // 2 per scene: previous LFV, by parity
  int32_t* done;       // 1 per scene: set when the scene's plan has finished
  float* agent_prevT;  // warm-start table: Dmax floats per agent
  // Learned prior (null for the server):
  const float* prior_path;   // Dmax floats per scene: the prior's proposal
  const int32_t* prior_use;  // 1 per scene: the proposal seeds the scene's first n_pr particles
  // Multi-agent teams (null without teams): per scene its agent's timed path, Dmax + 4
  // floats: x of start, waypoints, target, then the y's (T + 2 each)
  float* agent_rows;
};

// Conflicts of one path with its team mates' timed paths (multi-agent extension):
// all agents leave their starts together and reach one point of their path per
// step, straight in between; in step s the relative position moves on a segment,
// and the pair conflicts when that segment passes closer than sep to the origin.
// The lanes of a warp take (mate, step) items; returns the warp's sum (all lanes).
__device__ __forceinline__ int agent_conflicts(const float* x, int T, float sx, float sy, float tx, float ty,
                                               const float* rows, int ld, int nteam, int self, float sep2,
                                               int lane) {
  const int P = T + 2;
  const int items = nteam * (T + 1);
  int q = 0;
  for (int it = lane; it < items; it += 32) {
    const int b = it / (T + 1);
    const int s = it - b * (T + 1);
    if (b == self) continue;
    const float* w = rows + (long long)b * ld;
    const float ax = (s == 0) ? sx : x[s - 1];
    const float ay = (s == 0) ? sy : x[T + s - 1];
    const float bx = (s == T) ? tx : x[s];
    const float by = (s == T) ? ty : x[T + s];
    const float r0x = ax - w[s], r0y = ay - w[P + s];
    const float dx = (bx - w[s + 1]) - r0x, dy = (by - w[P + s + 1]) - r0y;
    const float L2 = fmaf(dx, dx, dy * dy);
    float t = 0.0f;
    if (L2 > 0.0f) t = fminf(fmaxf(-fmaf(r0x, dx, r0y * dy) / L2, 0.0f), 1.0f);
    const float px = fmaf(t, dx, r0x), py = fmaf(t, dy, r0y);
    q += fmaf(px, px, py * py) < sep2;
  }
  return __reduce_add_sync(0xffffffffu, q);
}

struct BatchSmem {
  int circ, X, V, P, R, G, T, Pfit, PQ, Gfit, GQ, Gsrc, total;
  __host__ __device__ static BatchSmem make(int Omax, int tile, int Dmax, int Gmax) {
    BatchSmem s;
    int off = 0;
    auto al = [](int v) { return (v + 15) / 16 * 16; };
    s.circ = off; off = al(off + pair_block_f4(Omax > 0 ? Omax : 1) * 16);
    s.X = off; off = al(off + tile * Dmax * 4);
    s.V = off; off = al(off + tile * Dmax * 4);
    s.P = off; off = al(off + tile * Dmax * 4);
    s.R = off; off = al(off + tile * 16);
    s.G = off; off = al(off + Dmax * 4);
    s.T = off; off = al(off + Dmax * 4);
    s.Pfit = off; off = al(off + tile * 4);
    s.PQ = off; off = al(off + tile * 4);
    s.Gfit = off; off = al(off + Gmax * 4);
    s.GQ = off; off = al(off + Gmax * 4);
    s.Gsrc = off; off = al(off + Gmax * 4);
    s.total = off;
    return s;
  }
};


cudaError_t batch_configure(int* smem_optin_out);
cudaError_t launch_batch_reset(const BatchParams& p, cudaStream_t s);
cudaError_t launch_batch_iter(const BatchParams& p, int j, int ntiles, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_batch_gate(const BatchParams& p, cudaStream_t s);
// Each scene's current result (with its start and target) becomes its agent's timed path.
cudaError_t launch_agent_rows(const BatchParams& p, cudaStream_t s);

}  // namespace sepso
