// sepso_internal.h -- declarations shared by the kernels and the C-ABI host code.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "sepso.h"

namespace sepso {

struct SwarmParams;
struct RunCtl;

// Shared-memory carve of swarm_kernel (byte offsets); identical on host and device.
struct SmemLayout {
  int pairs, win, X, V, P, R, Gown, Tb, Pfit, PQ, Q, Imp, Len, Gfit, GQ, Gsrc, total;
  __host__ __device__ static SmemLayout make(int obst_f4, int ppc, int D, int T, int G, int tw);
};

// Shared-memory carve of swarm_cluster_kernel: the obstacles, the Auto Truncation
// window, the key slots (two parities x S ranks x ppc particles), the staged
// candidate rows (two parities x ppc particles) and one frame area per particle
// warp.  Its CTAs have one warp per particle plus a control
// warp, at most kClusterMaxThreads threads; rows live in registers, so the form
// takes T + 1 <= 32 segments.
constexpr int kClusterMaxThreads = 512;
struct ClusterLayout {
  int pairs, win, keys, stage, frames, total;
  __host__ __device__ static ClusterLayout make(int obst_f4, int ppc, int T, int tw, int S);
};

struct EvalParams {
  int T, D, n, per_cta, split, O, Omax;
  int poly;            // circ holds O polygon edges (x0, y0, x1, y1) instead of circles
  float alpha;
  int beta;
  const float* X;      // n x D (device)
  const float4* circ;  // Omax x (cx, cy, r, 4 r^2)
  const float* pts;    // start xy, target xy
  float* F;
  int32_t* Q;
  float* len;
  int* status;
};

struct HsefParams {
  int G, HG, HN, HM, E;
  uint32_t key0, key1, run_id;
  float lo[3], hi[3];
  float l_vlimit;
  const float* hhyper;        // device copy, HG x 6
  float *HX, *HV, *HP, *HPfit, *HGb, *HGfit, *HTb, *HTfit;
  float* hyper;               // runs x G x 6 (the L-runs' hyper-parameters)
  RunCtl* ctl;                // runs
  const sepso_result* res;    // runs (the L-runs' LFV)
  float* history;             // E (device) or null
};

cudaError_t configure_swarm_kernel(size_t smem_bytes);
cudaError_t swarm_occupancy(int threads, size_t smem_bytes, int* blocks_per_sm);
cudaError_t launch_swarm(const SwarmParams& p, int grid, int threads, size_t smem, cudaStream_t s);
// The cluster form: clusters of p.cpg CTAs, one per (run, group).
cudaError_t configure_cluster_kernel(size_t smem_bytes);
cudaError_t cluster_max_active(int S, int threads, size_t smem_bytes, int* clusters);
cudaError_t launch_swarm_cluster(const SwarmParams& p, int grid, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_evaluate(const EvalParams& p, cudaStream_t s);
cudaError_t launch_advance(float4* circ, float2* cvel, float* pts, float4* pairs, int O, float W, float H,
                           int steps, cudaStream_t s);
// The same step for polygon obstacles: polygon p (edges poff[p] .. poff[p+1]-1)
// translated by pvel[p], bouncing by its bounding box.
cudaError_t launch_advance_poly(float4* edges, float2* pvel, const int* poff, int P, float* pts, float W, float H,
                                int steps, cudaStream_t s);
// Circle-pair blocks of the scene's circles (after the circles change on the host side).
cudaError_t launch_pairs(const float4* circ, int O, float4* pairs, cudaStream_t s);
cudaError_t launch_hsef_init(const HsefParams& p, cudaStream_t s);
cudaError_t launch_hsef_update(const HsefParams& p, int e, cudaStream_t s);
cudaError_t launch_at_window(const double* win, const int32_t* ns, const int32_t* heads, int count, int tw,
                             float delta, int32_t* out, cudaStream_t s);
cudaError_t launch_philox(const uint4* ctr, long long n, uint64_t seed, uint4* out, int num_sms, cudaStream_t s);
cudaError_t launch_watchdog_selftest(const unsigned int* never, unsigned long long limit_ns, int* fired,
                                     cudaStream_t s);

// The learned prior as the request server uses it (sepso_mlp.cu).  prior_shape:
// the proposal's waypoints, the circles a scene may have, the dataset rows, the map
// and the stream the handle runs on.  prior_propose_device: rasterise n scenes given on the
// device -- circles (cx, cy, r, 0) with n + 1 prefix offsets into circ, points n x 4
// -- into dataset rows [first, first + n) and write their proposals (2 T_p floats
// per row, row stride ld) to out, all on the handle's stream (async).
int prior_shape(const sepso_prior_ctx* h, int* T, int* max_circles, int* capacity, float* map_w, float* map_h,
                cudaStream_t* stream);
int prior_propose_device(sepso_prior_ctx* h, int first, int n, const float4* circ, const int* coff, const float* pts,
                         float* out, int ld);
// Replace the stream the prior's work is issued on; returns the previous one.
cudaStream_t prior_swap_stream(sepso_prior_ctx* h, cudaStream_t s);

}  // namespace sepso
