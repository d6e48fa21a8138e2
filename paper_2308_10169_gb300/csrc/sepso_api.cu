// sepso_api.cu -- host side of the C ABI declared in include/sepso.h.
//
// Argument checking, workspace layout, launch-shape choice and the launches.
// Every step of the planner itself runs in the kernels of sepso_kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "sepso_device.cuh"
#include "sepso_internal.h"

using namespace sepso;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(SEPSO_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CUDA_TRY(expr)                                    \
  do {                                                    \
    cudaError_t e_ = (expr);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr);   \
  } while (0)

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Byte offsets of every array in the caller's workspace.
struct WsLayout {
  size_t circ, pairs, cvel, pts, hyper, X, V, P, Pfit, PQ, Gb, Gfit, GQ, Tb, prevT, res_wp, ctl, res, win,
      gword, counter, crows, grec, poff, hhyper, HX, HV, HP, HPfit, HGb, HGfit, HTb, HTfit, estatus, total;
};

WsLayout make_ws(const sepso_config& c) {
  const size_t R = (size_t)c.runs, G = (size_t)c.G, N = (size_t)c.N, D = 2 * (size_t)c.T;
  const size_t M = G * N, Omax = (size_t)(c.max_obstacles > 0 ? c.max_obstacles : 1);
  const size_t DH = 3 * G;
  WsLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = align256(off);
    const size_t o = off;
    off += bytes;
    return o;
  };
  L.circ = take(Omax * 16);
  L.pairs = take((size_t)pair_block_f4(std::max((int)Omax, 1)) * 16);
  L.cvel = take(Omax * 8);
  L.pts = take(8 * 4);
  L.hyper = take(R * G * 6 * 4);
  L.X = take(R * M * D * 4);
  L.V = take(R * M * D * 4);
  L.P = take(R * M * D * 4);
  L.Pfit = take(R * M * 4);
  L.PQ = take(R * M * 4);
  L.Gb = take(R * G * D * 4);
  L.Gfit = take(R * G * 4);
  L.GQ = take(R * G * 4);
  L.Tb = take(R * D * 4);
  L.prevT = take(R * D * 4);
  L.res_wp = take(R * D * 4);
  L.ctl = take(R * sizeof(RunCtl));
  L.res = take(R * sizeof(sepso_result));
  L.win = take(R * (size_t)c.tw * 8);
  L.gword = take(R * 3 * G * 8);
  L.counter = take(R * sizeof(RunCounter));
  L.crows = take(R * 2 * M * (D + 4) * 4);
  L.grec = take(R * kRecDepth * G * 8);
  L.poff = take((Omax + 1) * 4);  // polygon obstacles: edge offsets of the polygons
  L.hhyper = take(32 * 6 * 4);
  L.HX = take(R * DH * 4);
  L.HV = take(R * DH * 4);
  L.HP = take(R * DH * 4);
  L.HPfit = take(R * 4);
  L.HGb = take(32 * DH * 4);
  L.HGfit = take(32 * 4);
  L.HTb = take(DH * 4);
  L.HTfit = take(4);
  L.estatus = take(4);
  L.total = align256(off);
  return L;
}

bool finite(float v) { return std::isfinite(v); }

int check_config(const sepso_config* c) {
  if (!c) return fail(SEPSO_EINVAL, "config is NULL");
  if (c->T < 1 || c->T > 64) return fail(SEPSO_EINVAL, "T=%d outside [1, 64]", c->T);
  if (c->G < 1 || c->G > 32) return fail(SEPSO_EINVAL, "G=%d outside [1, 32]", c->G);
  if (c->N < 1 || c->N >= (1 << 20)) return fail(SEPSO_EINVAL, "N=%d outside [1, 2^20)", c->N);
  if (c->max_obstacles < 0 || c->max_obstacles > 8192)
    return fail(SEPSO_EINVAL, "max_obstacles=%d outside [0, 8192]", c->max_obstacles);
  if (!finite(c->map_w) || !finite(c->map_h) || c->map_w <= 0 || c->map_h <= 0)
    return fail(SEPSO_EINVAL, "map extent must be finite and positive");
  if (!finite(c->alpha) || c->alpha < 0) return fail(SEPSO_EINVAL, "alpha must be finite and >= 0");
  if (c->beta < 1 || c->beta > 8) return fail(SEPSO_EINVAL, "beta=%d outside [1, 8]", c->beta);
  if (c->max_iters < 1) return fail(SEPSO_EINVAL, "max_iters must be >= 1");
  if (c->at_mode < 0 || c->at_mode > 2) return fail(SEPSO_EINVAL, "at_mode=%d unknown", c->at_mode);
  if (c->tw < 1 || c->tw > 64) return fail(SEPSO_EINVAL, "tw=%d outside [1, 64]", c->tw);
  if (!finite(c->delta) || !finite(c->stall_tol)) return fail(SEPSO_EINVAL, "delta/stall_tol not finite");
  if (c->stall_iters < 0) return fail(SEPSO_EINVAL, "stall_iters must be >= 0");
  if (!finite(c->pi_gamma) || c->pi_gamma < 0 || c->pi_gamma > 1)
    return fail(SEPSO_EINVAL, "pi_gamma outside [0, 1]");
  if (!finite(c->pi_halfwidth) || c->pi_halfwidth < 0) return fail(SEPSO_EINVAL, "pi_halfwidth < 0");
  if (c->runs < 1 || c->runs > 65536) return fail(SEPSO_EINVAL, "runs=%d outside [1, 65536]", c->runs);
  if (c->ctas_per_group < 0) return fail(SEPSO_EINVAL, "ctas_per_group < 0");
  if (c->threads != 0 && (c->threads < 64 || c->threads > 512 || c->threads % 32 != 0))
    return fail(SEPSO_EINVAL, "threads=%d must be 0 or a multiple of 32 in [64, 512]", c->threads);
  if (c->circle_split < 0) return fail(SEPSO_EINVAL, "circle_split < 0");
  if (c->fitness_mode < 0 || c->fitness_mode > 2) return fail(SEPSO_EINVAL, "fitness_mode must be 0, 1 or 2");
  if (c->exchange < 0 || c->exchange > 3) return fail(SEPSO_EINVAL, "exchange must be 0, 1, 2 or 3");
  if (c->obstacle_kind != SEPSO_OBST_CIRCLES && c->obstacle_kind != SEPSO_OBST_POLYGONS)
    return fail(SEPSO_EINVAL, "obstacle_kind=%d unknown", c->obstacle_kind);
  return SEPSO_OK;
}

}  // namespace

struct sepso_ctx {
  sepso_config cfg;
  int device = 0, num_sms = 0;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  WsLayout L{};
  int O = 0;   // circles, or polygon edges
  int P = 0;   // polygons (polygon obstacles)
  bool has_scene = false;
  int cpg = 1, ppc = 1, C = 1, threads = 256, split = 1, lp = 32, grid = 1, items = 0;
  size_t smem = 0;
  // cluster form (one thread-block cluster of cl_S CTAs per group), when it fits
  bool cl_ok = false;
  int cl_S = 1, cl_ppc = 1, cl_threads = 64, cl_grid = 1;
  size_t cl_smem = 0;
  std::vector<char> c3_nonzero;  // per run: some group's C3 is not 0 (the update then needs Tbest)
  bool grec_dirty = false;       // group records not written by the last launches (clear before use)
  int n_pi = 0;
  int64_t launches = 0;
  bool hsef_ready = false;
  int hsef_G = 0;
  float hsef_vlimit = 0.0f;
  float4* staging = nullptr;          // pinned: packed circles then the 8 point floats
  cudaEvent_t staging_free = nullptr; // recorded after each scene copy

  ~sepso_ctx() {
    if (staging_free) cudaEventDestroy(staging_free);
    if (staging) cudaFreeHost(staging);
  }

  template <class T>
  T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
};

namespace {

SwarmParams swarm_params(const sepso_ctx* h, int mode, int step_iters) {
  const sepso_config& c = h->cfg;
  SwarmParams p;
  p.T = c.T;
  p.D = 2 * c.T;
  p.G = c.G;
  p.N = c.N;
  p.M = c.G * c.N;
  p.R = c.runs;
  p.cpg = h->cpg;
  p.C = h->C;
  p.ppc = h->ppc;
  p.split = h->split;
  p.lp = h->lp;
  p.items = h->items;
  p.O = h->O;
  p.Omax = c.max_obstacles;
  p.W = c.map_w;
  p.H = c.map_h;
  p.alpha = c.alpha;
  p.beta = c.beta;
  p.max_iters = c.max_iters;
  p.at_mode = c.at_mode;
  p.tw = c.tw;
  p.delta = c.delta;
  p.stall_iters = c.stall_iters;
  p.stall_tol = c.stall_tol;
  p.use_pi = c.use_pi ? 1 : 0;
  p.n_pi = h->n_pi;
  p.pi_h = c.pi_halfwidth;
  p.key0 = (uint32_t)(c.seed & 0xffffffffu);
  p.key1 = (uint32_t)(c.seed >> 32);
  p.mode = mode;
  p.step_iters = step_iters;
  p.circ = h->at<float4>(h->L.circ);
  p.pairs = h->at<float4>(h->L.pairs);
  p.pts = h->at<float>(h->L.pts);
  p.hyper = h->at<float>(h->L.hyper);
  p.X = h->at<float>(h->L.X);
  p.V = h->at<float>(h->L.V);
  p.P = h->at<float>(h->L.P);
  p.Pfit = h->at<float>(h->L.Pfit);
  p.PQ = h->at<int32_t>(h->L.PQ);
  p.Gb = h->at<float>(h->L.Gb);
  p.Gfit = h->at<float>(h->L.Gfit);
  p.GQ = h->at<int32_t>(h->L.GQ);
  p.Tb = h->at<float>(h->L.Tb);
  p.prevT = h->at<float>(h->L.prevT);
  p.res_wp = h->at<float>(h->L.res_wp);
  p.ctl = h->at<RunCtl>(h->L.ctl);
  p.res = h->at<sepso_result>(h->L.res);
  p.win = h->at<double>(h->L.win);
  p.gword = h->at<unsigned long long>(h->L.gword);
  p.counter = h->at<RunCounter>(h->L.counter);
  p.crows = h->at<float>(h->L.crows);
  p.grec = h->at<unsigned long long>(h->L.grec);
  p.cta_grid = h->C;
  p.poly = c.obstacle_kind == SEPSO_OBST_POLYGONS ? 1 : 0;
  return p;
}

// The cluster form runs when it fits, no run's update needs Tbest (C3 = 0 in every
// group) and the config asks for it: exchange = 2 (required), 3 or 0 (whenever it
// applies).
bool use_cluster(const sepso_ctx* h) {
  if (h->cfg.exchange == 1 || !h->cl_ok) return false;
  for (char nz : h->c3_nonzero)
    if (nz) return false;
  return true;
}

// Launch one swarm kernel for p (plan or step mode) in the form the handle uses.
int launch_plan_kernel(sepso_ctx* h, SwarmParams p) {
  const bool cl = use_cluster(h);
  if (h->cfg.exchange == 2 && !cl)
    return fail(h->cl_ok ? SEPSO_EINVAL : SEPSO_ERANGE,
                h->cl_ok ? "exchange=2 needs C3 = 0 in every group" : "the cluster form does not fit this config");
  if (!cl) {
    CUDA_TRY(launch_swarm(p, h->grid, h->threads, h->smem, h->stream));
    h->grec_dirty = true;
    return SEPSO_OK;
  }
  if (h->grec_dirty) {
    CUDA_TRY(cudaMemsetAsync(h->ws + h->L.grec, 0, (size_t)h->cfg.runs * kRecDepth * h->cfg.G * 8, h->stream));
    h->grec_dirty = false;
  }
  p.cpg = h->cl_S;
  p.C = h->cfg.G * h->cl_S;
  p.ppc = h->cl_ppc;
  CUDA_TRY(launch_swarm_cluster(p, h->cl_grid, h->cl_threads, h->cl_smem, h->stream));
  return SEPSO_OK;
}

// The cluster form: S CTAs per group in one cluster (at most 16), each with one
// warp per particle and a control warp, so ceil(N / S) <= kClusterMaxThreads / 32 - 1
// particles per CTA; rows live in registers, so T + 1 <= 32 and G <= 32.  Every
// cluster of the launch must be resident at once (the groups of a run wait on each
// other's records), which the occupancy query checks.  The most CTAs per group
// first, with one CTA per SM (the shared-memory request is raised above half an
// SM's, so that no two CTAs share an SM's issue slots), then without that rule.
int choose_cluster_shape(sepso_ctx* h, int smem_optin) {
  const sepso_config& c = h->cfg;
  h->cl_ok = false;
  if (c.exchange == 1) return SEPSO_OK;
  const int R = c.runs, G = c.G, N = c.N, T = c.T;
  const int max_ppc = kClusterMaxThreads / 32 - 1;
  auto no_fit = [&](const char* why) {
    return c.exchange == 2 ? fail(SEPSO_ERANGE, "the cluster form does not fit: %s", why) : SEPSO_OK;
  };
  if (T + 1 > 32 || G > 32) return no_fit("it takes T + 1 <= 32 and G <= 32");
  int smem_sm = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device));
  CUDA_TRY(configure_cluster_kernel((size_t)smem_optin));
  const int S_hi = std::min(16, N);
  int S0 = c.ctas_per_group > 0 ? c.ctas_per_group : std::min(S_hi, std::max(1, h->num_sms / std::max(1, R * G)));
  S0 = std::min(S0, S_hi);
  const int S_lo = c.ctas_per_group > 0 ? S0 : 1;
  const bool poly = c.obstacle_kind == SEPSO_OBST_POLYGONS;
  for (int pass = 0; pass < 2; ++pass) {
    for (int S = S0; S >= S_lo; --S) {
      const int ppc = (N + S - 1) / S;
      if (ppc > max_ppc) break;
      if ((N + ppc - 1) / ppc != S) continue;  // no empty CTAs
      const int threads = 32 * (ppc + 1);
      const ClusterLayout Lc = ClusterLayout::make(obstacle_f4(c.max_obstacles, poly ? 1 : 0), ppc, T, c.tw, S);
      size_t smem = (size_t)Lc.total;
      if (pass == 0) smem = std::max(smem, (size_t)smem_sm / 2 + 1024);
      if (smem + 256 > (size_t)smem_optin) continue;
      int nc = 0;
      cudaError_t e = cluster_max_active(S, threads, smem, &nc);
      if (e != cudaSuccess) {
        cudaGetLastError();
        nc = 0;
      }
      if ((long long)nc >= (long long)R * G) {
        h->cl_ok = true;
        h->cl_S = S;
        h->cl_ppc = ppc;
        h->cl_threads = threads;
        h->cl_smem = smem;
        h->cl_grid = R * G * S;
        return SEPSO_OK;
      }
    }
  }
  return no_fit("no cluster size fits every group of every run at once");
}

// Pick CTAs per group, threads and circle split, then check co-residency: the
// cooperative launch needs every CTA resident at once.  Automatic choices start
// from one CTA per SM and back off (fewer threads, then fewer CTAs per group).
int choose_shape(sepso_ctx* h) {
  const sepso_config& c = h->cfg;
  const int R = c.runs, G = c.G, N = c.N, T = c.T, D = 2 * T;
  const int Omax = c.max_obstacles;
  int smem_optin = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
  // Fitness, either one lane group of lp lanes (a power of two, <= 32) per particle
  // taking (segment, circle chunk) items, or (particle, segment, chunk) items spread
  // over all threads of the CTA -- the default from 4 particles per CTA (measured:
  // 3.6% faster on the dynamic workload, 21% on 32 HSEF runs; slower with 2).
  auto items_for = [&](int ppc_) { return c.fitness_mode == 2 || (c.fitness_mode == 0 && ppc_ >= 4) ? 1 : 0; };
  const bool poly = c.obstacle_kind == SEPSO_OBST_POLYGONS;
  const int K = poly ? std::max(Omax, 1) : (std::max(Omax, 1) + 1) / 2;  // edges, or circle pairs
  int split = c.circle_split > 0 ? c.circle_split : 1;
  int lp = 1;
  while (lp < 32 && lp < (T + 1) * split) lp <<= 1;
  // item mode: the split that minimises rounds x (pairs per item + frame setup)
  auto items_split = [&](int thr, int ppc_) {
    if (c.circle_split > 0) return c.circle_split;
    int best = 1;
    long long best_cost = -1;
    for (int sp = 1; sp <= 8; ++sp) {
      const long long rounds = ((long long)ppc_ * (T + 1) * sp + thr - 1) / thr;
      const long long cost = rounds * ((K + sp - 1) / sp + 6);
      if (best_cost < 0 || cost < best_cost) {
        best_cost = cost;
        best = sp;
      }
    }
    return best;
  };
  CUDA_TRY(configure_swarm_kernel((size_t)smem_optin));
  int cpg = c.ctas_per_group > 0 ? c.ctas_per_group : std::max(1, h->num_sms / std::max(1, R * G));
  cpg = std::min(cpg, N);
  size_t smem = 0;
  int bps = 0, threads = 0;
  for (int attempt = 0; attempt < 64; ++attempt) {
    const int ppc = (N + cpg - 1) / cpg;
    cpg = (N + ppc - 1) / ppc;  // no empty CTAs
    const SmemLayout S = SmemLayout::make(obstacle_f4(Omax, poly ? 1 : 0), ppc, D, T, G, c.tw);
    smem = (size_t)S.total;
    const int ppw = 32 / lp;
    const int items = items_for(ppc);
    const int want = items ? 512 : std::min(512, std::max(64, (ppc + ppw - 1) / ppw * 32));
    for (threads = (c.threads ? c.threads : want); threads >= 64; threads -= 64) {
      bps = 0;
      if (smem + 256 <= (size_t)smem_optin) CUDA_TRY(swarm_occupancy(threads, smem, &bps));
      if ((long long)R * G * cpg <= (long long)bps * h->num_sms) {
        h->cpg = cpg;
        h->ppc = ppc;
        h->C = G * cpg;
        h->threads = threads;
        h->split = items ? items_split(threads, ppc) : split;
        h->lp = items ? 32 : lp;
        h->items = items;
        h->smem = smem;
        h->grid = R * G * cpg;
        return choose_cluster_shape(h, smem_optin);
      }
      if (c.threads) break;
    }
    if (c.ctas_per_group > 0) break;
    // Fewer CTAs when the grid is too large; more when one CTA's rows do not fit.
    if (smem + 256 > (size_t)smem_optin && cpg < N) ++cpg;
    else if ((long long)R * G * cpg > (long long)h->num_sms && cpg > 1) cpg = std::max(1, cpg / 2);
    else break;
  }
  return fail(SEPSO_ERANGE,
              "launch does not fit: %d runs x %d groups x %d CTAs, %zu B shared memory per CTA, "
              "%d CTAs per SM on %d SMs",
              R, G, cpg, smem, bps, h->num_sms);
}

int check_handle(sepso_handle h) {
  if (!h) return fail(SEPSO_EINVAL, "handle is NULL");
  return SEPSO_OK;
}

int run_ok(const sepso_ctx* h, int32_t run) {
  if (run < 0 || run >= h->cfg.runs) return fail(SEPSO_EINVAL, "run %d outside [0, %d)", run, h->cfg.runs);
  return SEPSO_OK;
}

// Serialised state layout of one run (see include/sepso.h).
struct StateLayout {
  size_t X, V, P, Pfit, PQ, Gb, Gfit, GQ, Tb, Tfit, TQ, k, cycle, has_prev, prevT, win, win_n, win_head,
      stall, prev_lfv, total;
};

StateLayout state_layout(const sepso_config& c) {
  const size_t G = c.G, N = c.N, D = 2 * (size_t)c.T, M = G * N, tw = c.tw;
  StateLayout s;
  size_t off = 0;
  s.X = off; off += M * D * 4;
  s.V = off; off += M * D * 4;
  s.P = off; off += M * D * 4;
  s.Pfit = off; off += M * 4;
  s.PQ = off; off += M * 4;
  s.Gb = off; off += G * D * 4;
  s.Gfit = off; off += G * 4;
  s.GQ = off; off += G * 4;
  s.Tb = off; off += D * 4;
  s.Tfit = off; off += 4;
  s.TQ = off; off += 4;
  s.k = off; off += 4;
  s.cycle = off; off += 4;
  s.has_prev = off; off += 4;
  s.prevT = off; off += D * 4;
  off = (off + 7) & ~size_t(7);
  s.win = off; off += tw * 8;
  s.win_n = off; off += 4;
  s.win_head = off; off += 4;
  s.stall = off; off += 4;
  s.prev_lfv = off; off += 4;
  s.total = off;
  return s;
}

}  // namespace

extern "C" {

const char* sepso_strerror(int code) {
  switch (code) {
    case SEPSO_OK: return "ok";
    case SEPSO_EINVAL: return "invalid argument";
    case SEPSO_ESTATE: return "call out of order";
    case SEPSO_ENOSPC: return "workspace too small or misaligned";
    case SEPSO_ECUDA: return "CUDA runtime error";
    case SEPSO_ETIMEOUT: return "device-side wait timed out";
    case SEPSO_ENOMEM: return "host allocation failed";
    case SEPSO_ERANGE: return "shape exceeds a kernel limit";
    case SEPSO_EBOUNDS: return "a device-side index check failed";
    default: return "unknown status";
  }
}

const char* sepso_last_error(void) { return g_last_error.c_str(); }

int sepso_workspace_size(const sepso_config* cfg, size_t* bytes) {
  const int rc = check_config(cfg);
  if (rc) return rc;
  if (!bytes) return fail(SEPSO_EINVAL, "bytes is NULL");
  *bytes = make_ws(*cfg).total;
  return SEPSO_OK;
}

int sepso_create(const sepso_config* cfg, void* d_workspace, size_t bytes, void* stream, sepso_handle* out) {
  int rc = check_config(cfg);
  if (rc) return rc;
  if (!out) return fail(SEPSO_EINVAL, "out is NULL");
  *out = nullptr;
  const WsLayout L = make_ws(*cfg);
  if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255u) != 0)
    return fail(SEPSO_ENOSPC, "workspace must be non-NULL and 256-byte aligned");
  if (bytes < L.total) return fail(SEPSO_ENOSPC, "workspace has %zu bytes, needs %zu", bytes, L.total);
  sepso_ctx* h = new (std::nothrow) sepso_ctx();
  if (!h) return fail(SEPSO_ENOMEM, "host allocation failed");
  h->cfg = *cfg;
  h->stream = static_cast<cudaStream_t>(stream);
  h->ws = static_cast<char*>(d_workspace);
  h->ws_bytes = bytes;
  h->L = L;
  {
    const double v = std::ceil((double)cfg->pi_gamma * (double)cfg->N);
    h->n_pi = (int)std::min<double>(std::max(v, 0.0), (double)cfg->N);
  }
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "device query");
  }
  rc = choose_shape(h);
  if (rc) {
    delete h;
    return rc;
  }
  h->c3_nonzero.assign((size_t)cfg->runs, 0);  // the zeroed workspace holds C3 = 0
  e = cudaMallocHost(reinterpret_cast<void**>(&h->staging),
                     ((size_t)std::max(cfg->max_obstacles, 1) + 2) * sizeof(float4));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->staging_free, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "pinned staging buffer");
  }
  // Zero the workspace, then seed each run's control block.
  std::vector<RunCtl> ctl((size_t)cfg->runs);
  for (int r = 0; r < cfg->runs; ++r) {
    std::memset(&ctl[r], 0, sizeof(RunCtl));
    ctl[r].Tfit = INFINITY;
    ctl[r].prev_lfv = INFINITY;
    ctl[r].run_id = cfg->run_id + (uint32_t)r;
  }
  e = cudaMemsetAsync(h->ws, 0, L.total, h->stream);
  if (e == cudaSuccess)  // empty group-best keys
    e = cudaMemsetAsync(h->ws + L.gword, 0xff, (size_t)cfg->runs * 3 * cfg->G * 8, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->ws + L.ctl, ctl.data(), ctl.size() * sizeof(RunCtl), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "workspace initialisation");
  }
  *out = h;
  return SEPSO_OK;
}

void sepso_destroy(sepso_handle h) { delete h; }

int sepso_set_hyper(sepso_handle h, int32_t run, const float* hyper) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!hyper) return fail(SEPSO_EINVAL, "hyper is NULL");
  const int G = h->cfg.G;
  for (int i = 0; i < G * 6; ++i)
    if (!finite(hyper[i])) return fail(SEPSO_EINVAL, "hyper[%d] is not finite", i);
  for (int g = 0; g < G; ++g)
    if (hyper[g * 6 + 5] < 0) return fail(SEPSO_EINVAL, "V_limit of group %d is negative", g);
  const size_t row = (size_t)G * 6 * sizeof(float);
  char nz = 0;
  for (int g = 0; g < G; ++g)
    if (hyper[g * 6 + 2] != 0.0f) nz = 1;
  if (run >= 0) {
    if ((rc = run_ok(h, run))) return rc;
    h->c3_nonzero[run] = nz;
    CUDA_TRY(cudaMemcpyAsync(h->ws + h->L.hyper + run * row, hyper, row, cudaMemcpyHostToDevice, h->stream));
    return SEPSO_OK;
  }
  std::fill(h->c3_nonzero.begin(), h->c3_nonzero.end(), nz);
  std::vector<float> all((size_t)h->cfg.runs * G * 6);
  for (int r = 0; r < h->cfg.runs; ++r) std::memcpy(all.data() + (size_t)r * G * 6, hyper, row);
  CUDA_TRY(cudaMemcpyAsync(h->ws + h->L.hyper, all.data(), all.size() * 4, cudaMemcpyHostToDevice, h->stream));
  return SEPSO_OK;
}

int sepso_set_scene(sepso_handle h, const float* start, const float* target, const float* circles, int32_t O) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (h->cfg.obstacle_kind != SEPSO_OBST_CIRCLES)
    return fail(SEPSO_EINVAL, "this handle plans among polygons: use sepso_set_polygons");
  if (!start || !target) return fail(SEPSO_EINVAL, "start/target is NULL");
  if (O < 0 || O > h->cfg.max_obstacles)
    return fail(SEPSO_EINVAL, "O=%d outside [0, max_obstacles=%d]", O, h->cfg.max_obstacles);
  if (O > 0 && !circles) return fail(SEPSO_EINVAL, "circles is NULL");
  if (!finite(start[0]) || !finite(start[1]) || !finite(target[0]) || !finite(target[1]))
    return fail(SEPSO_EINVAL, "start/target not finite");
  for (int o = 0; o < O; ++o) {
    const float cx = circles[3 * o], cy = circles[3 * o + 1], r = circles[3 * o + 2];
    if (!finite(cx) || !finite(cy) || !finite(r) || r < 0)
      return fail(SEPSO_EINVAL, "circle %d invalid (non-finite or negative radius)", o);
  }
  // the previous scene copy must have left the staging buffer
  CUDA_TRY(cudaEventSynchronize(h->staging_free));
  float4* c4 = h->staging;
  for (int o = 0; o < O; ++o) {
    const float cx = circles[3 * o], cy = circles[3 * o + 1], r = circles[3 * o + 2];
    c4[o] = make_float4(cx, cy, r, 4.0f * (r * r));
  }
  float* pts = reinterpret_cast<float*>(h->staging + std::max(h->cfg.max_obstacles, 1));
  const float pv[8] = {start[0], start[1], target[0], target[1], 0.f, 0.f, 0.f, 0.f};
  std::memcpy(pts, pv, sizeof pv);
  if (O > 0) {
    CUDA_TRY(cudaMemcpyAsync(h->ws + h->L.circ, c4, (size_t)O * 16, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemsetAsync(h->ws + h->L.cvel, 0, (size_t)O * 8, h->stream));
    CUDA_TRY(launch_pairs(h->at<float4>(h->L.circ), O, h->at<float4>(h->L.pairs), h->stream));
    h->launches += 1;
  }
  CUDA_TRY(cudaMemcpyAsync(h->ws + h->L.pts, pts, 8 * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaEventRecord(h->staging_free, h->stream));
  h->O = O;
  h->has_scene = true;
  return SEPSO_OK;
}

int sepso_set_motion(sepso_handle h, const float* circle_vel, const float* start_vel, const float* target_vel) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!h->has_scene) return fail(SEPSO_ESTATE, "set_motion before set_scene");
  const int nv = h->cfg.obstacle_kind == SEPSO_OBST_POLYGONS ? h->P : h->O;  // one velocity per moving body
  if (!start_vel || !target_vel || (nv > 0 && !circle_vel)) return fail(SEPSO_EINVAL, "NULL velocity");
  for (int i = 0; i < 2 * nv; ++i)
    if (!finite(circle_vel[i])) return fail(SEPSO_EINVAL, "obstacle velocity [%d] not finite", i);
  const float vel[4] = {start_vel[0], start_vel[1], target_vel[0], target_vel[1]};
  for (float v : vel)
    if (!finite(v)) return fail(SEPSO_EINVAL, "start/target velocity not finite");
  if (nv > 0)
    CUDA_TRY(cudaMemcpyAsync(h->ws + h->L.cvel, circle_vel, (size_t)nv * 8, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaMemcpyAsync(h->ws + h->L.pts + 16, vel, sizeof vel, cudaMemcpyHostToDevice, h->stream));
  return SEPSO_OK;
}

int sepso_advance_scene(sepso_handle h, int32_t steps) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!h->has_scene) return fail(SEPSO_ESTATE, "advance before set_scene");
  if (steps < 0) return fail(SEPSO_EINVAL, "steps < 0");
  if (steps == 0) return SEPSO_OK;
  if (h->cfg.obstacle_kind == SEPSO_OBST_POLYGONS)
    CUDA_TRY(launch_advance_poly(h->at<float4>(h->L.circ), h->at<float2>(h->L.cvel), h->at<int>(h->L.poff), h->P,
                                 h->at<float>(h->L.pts), h->cfg.map_w, h->cfg.map_h, steps, h->stream));
  else
    CUDA_TRY(launch_advance(h->at<float4>(h->L.circ), h->at<float2>(h->L.cvel), h->at<float>(h->L.pts),
                            h->at<float4>(h->L.pairs), h->O,
                            h->cfg.map_w, h->cfg.map_h, steps, h->stream));
  h->launches += 1;
  return SEPSO_OK;
}

int sepso_get_scene(sepso_handle h, float* start, float* target, float* circles, float* circle_vel) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (h->cfg.obstacle_kind != SEPSO_OBST_CIRCLES)
    return fail(SEPSO_EINVAL, "this handle plans among polygons: use sepso_get_polygons");
  if (!h->has_scene) return fail(SEPSO_ESTATE, "no scene");
  std::vector<float4> c4((size_t)h->O);
  float pts[8];
  if (h->O > 0)
    CUDA_TRY(cudaMemcpyAsync(c4.data(), h->ws + h->L.circ, (size_t)h->O * 16, cudaMemcpyDeviceToHost, h->stream));
  if (circle_vel && h->O > 0)
    CUDA_TRY(cudaMemcpyAsync(circle_vel, h->ws + h->L.cvel, (size_t)h->O * 8, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaMemcpyAsync(pts, h->ws + h->L.pts, sizeof pts, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (start) { start[0] = pts[0]; start[1] = pts[1]; }
  if (target) { target[0] = pts[2]; target[1] = pts[3]; }
  if (circles)
    for (int o = 0; o < h->O; ++o) {
      circles[3 * o] = c4[o].x;
      circles[3 * o + 1] = c4[o].y;
      circles[3 * o + 2] = c4[o].z;
    }
  return SEPSO_OK;
}

int sepso_set_polygons(sepso_handle h, const float* start, const float* target, const float* edges, int32_t E,
                       const int32_t* offsets, int32_t P) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (h->cfg.obstacle_kind != SEPSO_OBST_POLYGONS)
    return fail(SEPSO_EINVAL, "this handle plans among circles (obstacle_kind = 0)");
  if (!start || !target) return fail(SEPSO_EINVAL, "start/target is NULL");
  if (E < 0 || E > h->cfg.max_obstacles)
    return fail(SEPSO_EINVAL, "E=%d outside [0, max_obstacles=%d]", E, h->cfg.max_obstacles);
  if (P < 0 || P > E) return fail(SEPSO_EINVAL, "P=%d outside [0, E=%d]", P, E);
  if ((E > 0 && !edges) || !offsets) return fail(SEPSO_EINVAL, "edges or offsets is NULL");
  if (offsets[0] != 0 || offsets[P] != E) return fail(SEPSO_EINVAL, "offsets must run from 0 to E");
  for (int q = 0; q < P; ++q)
    if (offsets[q + 1] < offsets[q]) return fail(SEPSO_EINVAL, "offsets decrease at polygon %d", q);
  if (!finite(start[0]) || !finite(start[1]) || !finite(target[0]) || !finite(target[1]))
    return fail(SEPSO_EINVAL, "start/target not finite");
  for (int i = 0; i < 4 * E; ++i)
    if (!finite(edges[i])) return fail(SEPSO_EINVAL, "edge %d not finite", i / 4);
  // the previous scene copy must have left the staging buffer
  CUDA_TRY(cudaEventSynchronize(h->staging_free));
  float4* e4 = h->staging;
  for (int e = 0; e < E; ++e) e4[e] = make_float4(edges[4 * e], edges[4 * e + 1], edges[4 * e + 2], edges[4 * e + 3]);
  float* pts = reinterpret_cast<float*>(h->staging + std::max(h->cfg.max_obstacles, 1));
  const float pv[8] = {start[0], start[1], target[0], target[1], 0.f, 0.f, 0.f, 0.f};
  std::memcpy(pts, pv, sizeof pv);
  if (E > 0) CUDA_TRY(cudaMemcpyAsync(h->ws + h->L.circ, e4, (size_t)E * 16, cudaMemcpyHostToDevice, h->stream));
  if (P > 0) CUDA_TRY(cudaMemsetAsync(h->ws + h->L.cvel, 0, (size_t)P * 8, h->stream));
  CUDA_TRY(cudaMemcpyAsync(h->ws + h->L.pts, pts, 8 * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaEventRecord(h->staging_free, h->stream));
  // the offsets come from the caller's (pageable) memory: copied before the return
  CUDA_TRY(cudaMemcpyAsync(h->ws + h->L.poff, offsets, (size_t)(P + 1) * 4, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  h->O = E;
  h->P = P;
  h->has_scene = true;
  return SEPSO_OK;
}

int sepso_get_polygons(sepso_handle h, float* start, float* target, float* edges, float* polygon_vel) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (h->cfg.obstacle_kind != SEPSO_OBST_POLYGONS)
    return fail(SEPSO_EINVAL, "this handle plans among circles (obstacle_kind = 0)");
  if (!h->has_scene) return fail(SEPSO_ESTATE, "no scene");
  float pts[8];
  if (edges && h->O > 0)
    CUDA_TRY(cudaMemcpyAsync(edges, h->ws + h->L.circ, (size_t)h->O * 16, cudaMemcpyDeviceToHost, h->stream));
  if (polygon_vel && h->P > 0)
    CUDA_TRY(cudaMemcpyAsync(polygon_vel, h->ws + h->L.cvel, (size_t)h->P * 8, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaMemcpyAsync(pts, h->ws + h->L.pts, sizeof pts, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (start) { start[0] = pts[0]; start[1] = pts[1]; }
  if (target) { target[0] = pts[2]; target[1] = pts[3]; }
  return SEPSO_OK;
}

int sepso_plan_async(sepso_handle h) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!h->has_scene) return fail(SEPSO_ESTATE, "plan before set_scene");
  if ((rc = launch_plan_kernel(h, swarm_params(h, kModePlan, 0)))) return rc;
  h->launches += 1;
  return SEPSO_OK;
}

int sepso_read_result(sepso_handle h, int32_t run, float* waypoints, sepso_result* res) {
  int rc = check_handle(h);
  if (rc) return rc;
  if ((rc = run_ok(h, run))) return rc;
  const size_t D = 2 * (size_t)h->cfg.T;
  sepso_result tmp;
  if (waypoints)
    CUDA_TRY(cudaMemcpyAsync(waypoints, h->ws + h->L.res_wp + run * D * 4, D * 4, cudaMemcpyDeviceToHost,
                             h->stream));
  CUDA_TRY(cudaMemcpyAsync(&tmp, h->ws + h->L.res + run * sizeof(sepso_result), sizeof tmp,
                           cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (res) *res = tmp;
  if (tmp.status != SEPSO_OK) return fail(tmp.status, "device-side error in run %d", run);
  return SEPSO_OK;
}

int sepso_plan(sepso_handle h, float* waypoints, sepso_result* res) {
  const int rc = sepso_plan_async(h);
  if (rc) return rc;
  return sepso_read_result(h, 0, waypoints, res);
}

int sepso_result_device(sepso_handle h, int32_t run, float** d_waypoints, sepso_result** d_result) {
  int rc = check_handle(h);
  if (rc) return rc;
  if ((rc = run_ok(h, run))) return rc;
  const size_t D = 2 * (size_t)h->cfg.T;
  if (d_waypoints) *d_waypoints = h->at<float>(h->L.res_wp + run * D * 4);
  if (d_result) *d_result = h->at<sepso_result>(h->L.res + run * sizeof(sepso_result));
  return SEPSO_OK;
}

int sepso_step(sepso_handle h, int32_t iters) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!h->has_scene) return fail(SEPSO_ESTATE, "step before set_scene");
  if (iters < 0) return fail(SEPSO_EINVAL, "iters < 0");
  if (iters == 0) return SEPSO_OK;
  if ((rc = launch_plan_kernel(h, swarm_params(h, kModeStep, iters)))) return rc;
  h->launches += 1;
  return SEPSO_OK;
}

int sepso_evaluate(sepso_handle h, const float* d_X, int32_t n, float* d_F, int32_t* d_Q, float* d_len) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!h->has_scene) return fail(SEPSO_ESTATE, "evaluate before set_scene");
  if (n < 0) return fail(SEPSO_EINVAL, "n < 0");
  if (n == 0) return SEPSO_OK;
  if (!d_X) return fail(SEPSO_EINVAL, "d_X is NULL");
  EvalParams p;
  p.T = h->cfg.T;
  p.D = 2 * h->cfg.T;
  p.n = n;
  p.per_cta = std::max(1, 256 / (h->cfg.T + 1));
  p.split = 1;
  p.O = h->O;
  p.poly = h->cfg.obstacle_kind == SEPSO_OBST_POLYGONS ? 1 : 0;
  p.Omax = h->cfg.max_obstacles;
  p.alpha = h->cfg.alpha;
  p.beta = h->cfg.beta;
  p.X = d_X;
  p.circ = h->at<float4>(h->L.circ);
  p.pts = h->at<float>(h->L.pts);
  p.F = d_F;
  p.Q = d_Q;
  p.len = d_len;
  p.status = h->at<int>(h->L.estatus);
  CUDA_TRY(launch_evaluate(p, h->stream));
  h->launches += 1;
  return SEPSO_OK;
}

int sepso_state_size(sepso_handle h, size_t* bytes) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!bytes) return fail(SEPSO_EINVAL, "bytes is NULL");
  *bytes = state_layout(h->cfg).total;
  return SEPSO_OK;
}

namespace {

// One cudaMemcpyAsync per array between the run's workspace slices and a host buffer.
int state_copy(sepso_ctx* h, int32_t run, char* host, bool to_host) {
  const sepso_config& c = h->cfg;
  const StateLayout s = state_layout(c);
  const size_t G = c.G, N = c.N, D = 2 * (size_t)c.T, M = G * N, tw = c.tw;
  const size_t r = (size_t)run;
  const size_t ctl_off = h->L.ctl + r * sizeof(RunCtl);
  struct Piece {
    size_t host_off, dev_off, bytes;
  } pieces[] = {
      {s.X, h->L.X + r * M * D * 4, M * D * 4},
      {s.V, h->L.V + r * M * D * 4, M * D * 4},
      {s.P, h->L.P + r * M * D * 4, M * D * 4},
      {s.Pfit, h->L.Pfit + r * M * 4, M * 4},
      {s.PQ, h->L.PQ + r * M * 4, M * 4},
      {s.Gb, h->L.Gb + r * G * D * 4, G * D * 4},
      {s.Gfit, h->L.Gfit + r * G * 4, G * 4},
      {s.GQ, h->L.GQ + r * G * 4, G * 4},
      {s.Tb, h->L.Tb + r * D * 4, D * 4},
      {s.Tfit, ctl_off + offsetof(RunCtl, Tfit), 4},
      {s.TQ, ctl_off + offsetof(RunCtl, TQ), 4},
      {s.k, ctl_off + offsetof(RunCtl, k), 4},
      {s.cycle, ctl_off + offsetof(RunCtl, cycle), 4},
      {s.has_prev, ctl_off + offsetof(RunCtl, has_prev), 4},
      {s.prevT, h->L.prevT + r * D * 4, D * 4},
      {s.win, h->L.win + r * tw * 8, tw * 8},
      {s.win_n, ctl_off + offsetof(RunCtl, win_n), 4},
      {s.win_head, ctl_off + offsetof(RunCtl, win_head), 4},
      {s.stall, ctl_off + offsetof(RunCtl, stall), 4},
      {s.prev_lfv, ctl_off + offsetof(RunCtl, prev_lfv), 4},
  };
  for (const Piece& pc : pieces) {
    if (to_host)
      CUDA_TRY(cudaMemcpyAsync(host + pc.host_off, h->ws + pc.dev_off, pc.bytes, cudaMemcpyDeviceToHost, h->stream));
    else
      CUDA_TRY(cudaMemcpyAsync(h->ws + pc.dev_off, host + pc.host_off, pc.bytes, cudaMemcpyHostToDevice, h->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return SEPSO_OK;
}

}  // namespace

int sepso_get_state(sepso_handle h, int32_t run, void* host_buf, size_t bytes) {
  int rc = check_handle(h);
  if (rc) return rc;
  if ((rc = run_ok(h, run))) return rc;
  if (!host_buf || bytes < state_layout(h->cfg).total) return fail(SEPSO_EINVAL, "state buffer too small");
  return state_copy(h, run, static_cast<char*>(host_buf), true);
}

int sepso_set_state(sepso_handle h, int32_t run, const void* host_buf, size_t bytes) {
  int rc = check_handle(h);
  if (rc) return rc;
  if ((rc = run_ok(h, run))) return rc;
  const StateLayout s = state_layout(h->cfg);
  if (!host_buf || bytes < s.total) return fail(SEPSO_EINVAL, "state buffer too small");
  const char* b = static_cast<const char*>(host_buf);
  int32_t win_n, win_head;
  std::memcpy(&win_n, b + s.win_n, 4);
  std::memcpy(&win_head, b + s.win_head, 4);
  if (win_n < 0 || win_n > h->cfg.tw || win_head < 0 || win_head >= h->cfg.tw)
    return fail(SEPSO_EINVAL, "AT window counters out of range");
  return state_copy(h, run, const_cast<char*>(b), false);
}

int sepso_hsef(sepso_handle h, const sepso_hsef_config* hc, float* d_history) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!hc) return fail(SEPSO_EINVAL, "hsef config is NULL");
  if (!h->has_scene) return fail(SEPSO_ESTATE, "hsef before set_scene");
  const sepso_config& c = h->cfg;
  if (hc->HG < 1 || hc->HG > 32 || hc->HN < 1 || hc->HG * hc->HN != c.runs)
    return fail(SEPSO_EINVAL, "HG*HN must equal runs (%d), 1 <= HG <= 32", c.runs);
  if (hc->E < 1) return fail(SEPSO_EINVAL, "E must be >= 1");
  for (int i = 0; i < 3; ++i)
    if (!finite(hc->lo[i]) || !finite(hc->hi[i]) || hc->hi[i] < hc->lo[i])
      return fail(SEPSO_EINVAL, "bad (w, C1, C2) box");
  for (int i = 0; i < hc->HG * 6; ++i)
    if (!finite(hc->hhyper[i])) return fail(SEPSO_EINVAL, "hhyper not finite");
  HsefParams p;
  p.G = c.G;
  p.HG = hc->HG;
  p.HN = hc->HN;
  p.HM = c.runs;
  p.E = hc->E;
  p.key0 = (uint32_t)(hc->hseed & 0xffffffffu);
  p.key1 = (uint32_t)(hc->hseed >> 32);
  p.run_id = c.run_id;
  for (int i = 0; i < 3; ++i) {
    p.lo[i] = hc->lo[i];
    p.hi[i] = hc->hi[i];
  }
  p.l_vlimit = hc->l_vlimit;
  p.hhyper = h->at<float>(h->L.hhyper);
  p.HX = h->at<float>(h->L.HX);
  p.HV = h->at<float>(h->L.HV);
  p.HP = h->at<float>(h->L.HP);
  p.HPfit = h->at<float>(h->L.HPfit);
  p.HGb = h->at<float>(h->L.HGb);
  p.HGfit = h->at<float>(h->L.HGfit);
  p.HTb = h->at<float>(h->L.HTb);
  p.HTfit = h->at<float>(h->L.HTfit);
  p.hyper = h->at<float>(h->L.hyper);
  p.ctl = h->at<RunCtl>(h->L.ctl);
  p.res = h->at<sepso_result>(h->L.res);
  p.history = d_history;
  CUDA_TRY(cudaMemcpyAsync(h->ws + h->L.hhyper, hc->hhyper, (size_t)hc->HG * 6 * 4, cudaMemcpyHostToDevice,
                           h->stream));
  CUDA_TRY(launch_hsef_init(p, h->stream));
  h->launches += 1;
  SwarmParams sp = swarm_params(h, kModePlan, 0);
  sp.at_mode = SEPSO_AT_OFF;  // an L-run maps hyper-parameters to the LFV after max_iters
  sp.use_pi = 0;
  std::fill(h->c3_nonzero.begin(), h->c3_nonzero.end(), 0);  // the L-runs' hyper-parameters have C3 = 0
  for (int e = 1; e <= hc->E; ++e) {
    if ((rc = launch_plan_kernel(h, sp))) return rc;
    CUDA_TRY(launch_hsef_update(p, e, h->stream));
    h->launches += 2;
  }
  h->hsef_ready = true;
  h->hsef_G = c.G;
  h->hsef_vlimit = hc->l_vlimit;
  return SEPSO_OK;
}

int sepso_hsef_best(sepso_handle h, float* hyper_out, float* best_lfv) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!h->hsef_ready) return fail(SEPSO_ESTATE, "no HSEF run yet");
  const int G = h->cfg.G;
  std::vector<float> tb((size_t)3 * G);
  float tf = 0.0f;
  CUDA_TRY(cudaMemcpyAsync(tb.data(), h->ws + h->L.HTb, tb.size() * 4, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaMemcpyAsync(&tf, h->ws + h->L.HTfit, 4, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (hyper_out)
    for (int g = 0; g < G; ++g) {
      hyper_out[g * 6 + 0] = tb[G + g];
      hyper_out[g * 6 + 1] = tb[2 * G + g];
      hyper_out[g * 6 + 2] = 0.0f;
      hyper_out[g * 6 + 3] = tb[g];
      hyper_out[g * 6 + 4] = tb[g];
      hyper_out[g * 6 + 5] = h->hsef_vlimit;
    }
  if (best_lfv) *best_lfv = tf;
  return SEPSO_OK;
}

int sepso_sync(sepso_handle h) {
  int rc = check_handle(h);
  if (rc) return rc;
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  std::vector<RunCtl> ctl((size_t)h->cfg.runs);
  int estatus = 0;
  CUDA_TRY(cudaMemcpy(ctl.data(), h->ws + h->L.ctl, ctl.size() * sizeof(RunCtl), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(&estatus, h->ws + h->L.estatus, 4, cudaMemcpyDeviceToHost));
  int first = estatus;
  bool dirty = estatus != 0;
  for (auto& c : ctl)
    if (c.status != 0) {
      if (first == 0) first = c.status;
      c.status = 0;
      dirty = true;
    }
  if (dirty) {
    // Clear the error words.  A wait that gave up leaves the barrier counters and
    // group words of its run inconsistent: rebuild them from the iteration counts.
    std::vector<RunCounter> cnt(ctl.size());
    for (size_t r = 0; r < ctl.size(); ++r) {
      std::memset(&cnt[r], 0, sizeof(RunCounter));
      cnt[r].count = (unsigned int)h->C * (unsigned int)ctl[r].iters_total;
      ctl[r].fin_launches = 0;
    }
    h->grec_dirty = true;
    CUDA_TRY(cudaMemcpy(h->ws + h->L.ctl, ctl.data(), ctl.size() * sizeof(RunCtl), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(h->ws + h->L.counter, cnt.data(), cnt.size() * sizeof(RunCounter), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemset(h->ws + h->L.gword, 0xff, ctl.size() * 3 * h->cfg.G * 8));
    CUDA_TRY(cudaMemset(h->ws + h->L.estatus, 0, 4));
    return fail(first, "device-side error: %s", sepso_strerror(first));
  }
  return SEPSO_OK;
}

int sepso_launch_shape(sepso_handle h, int32_t* ctas_per_group, int32_t* threads, int32_t* circle_split,
                       int32_t* grid) {
  int rc = check_handle(h);
  if (rc) return rc;
  const bool cl = use_cluster(h);
  if (ctas_per_group) *ctas_per_group = cl ? h->cl_S : h->cpg;
  if (threads) *threads = cl ? h->cl_threads : h->threads;
  if (circle_split) *circle_split = cl ? 1 : h->split;
  if (grid) *grid = cl ? h->cl_grid : h->grid;
  return SEPSO_OK;
}

int sepso_exchange_form(sepso_handle h) {
  int rc = check_handle(h);
  if (rc) return rc;
  return use_cluster(h) ? 2 : 1;
}

int sepso_counters(sepso_handle h, int32_t run, int64_t* plans, int64_t* iterations) {
  int rc = check_handle(h);
  if (rc) return rc;
  if ((rc = run_ok(h, run))) return rc;
  long long v[2] = {0, 0};
  const size_t off = h->L.ctl + (size_t)run * sizeof(RunCtl) + offsetof(RunCtl, plans_total);
  CUDA_TRY(cudaMemcpyAsync(v, h->ws + off, sizeof v, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (plans) *plans = v[0];
  if (iterations) *iterations = v[1];
  return SEPSO_OK;
}

int64_t sepso_launch_count(sepso_handle h) { return h ? h->launches : -1; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Watchdog self-test: the kernels' bounded waits, left to run out on purpose.
// ---------------------------------------------------------------------------
namespace {
__device__ unsigned int g_wd_never;  // nothing ever increments it
__device__ int g_wd_fired;
}  // namespace

extern "C" int sepso_watchdog_selftest(int32_t limit_us, int32_t* fired, void* stream) {
  if (!fired || limit_us < 1 || limit_us > 1000000) return fail(SEPSO_EINVAL, "limit_us must be in [1, 1e6]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* never = nullptr;
  void* out = nullptr;
  CUDA_TRY(cudaGetSymbolAddress(&never, g_wd_never));
  CUDA_TRY(cudaGetSymbolAddress(&out, g_wd_fired));
  CUDA_TRY(cudaMemsetAsync(never, 0, sizeof(unsigned int), s));
  CUDA_TRY(cudaMemsetAsync(out, 0xff, sizeof(int), s));
  CUDA_TRY(launch_watchdog_selftest(static_cast<const unsigned int*>(never), (unsigned long long)limit_us * 1000ull,
                                    static_cast<int*>(out), s));
  int f = -1;
  CUDA_TRY(cudaMemcpyAsync(&f, out, sizeof f, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  *fired = f;
  return SEPSO_OK;
}

// ---------------------------------------------------------------------------
// The planner's Philox4x32-10 on caller-given counters (device arrays).
// ---------------------------------------------------------------------------
extern "C" int sepso_philox(const uint32_t* ctr, int64_t n, uint64_t seed, uint32_t* out, void* stream) {
  if (n < 0) return fail(SEPSO_EINVAL, "n=%lld is negative", (long long)n);
  if (n == 0) return SEPSO_OK;
  if (!ctr || !out) return fail(SEPSO_EINVAL, "NULL counter or output array");
  if ((reinterpret_cast<uintptr_t>(ctr) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
    return fail(SEPSO_EINVAL, "counter and output arrays must be 16-byte aligned");
  int dev = 0, sms = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CUDA_TRY(launch_philox(reinterpret_cast<const uint4*>(ctr), (long long)n, seed, reinterpret_cast<uint4*>(out), sms,
                         static_cast<cudaStream_t>(stream)));
  return SEPSO_OK;
}

// ---------------------------------------------------------------------------
// The Auto Truncation window criterion, evaluated on the device by the planner's code.
// ---------------------------------------------------------------------------
extern "C" int sepso_at_window_test(const double* win, const int32_t* ns, const int32_t* heads, int32_t count,
                                    int32_t tw, float delta, int32_t* out, void* stream) {
  if (count < 0 || (count > 0 && (!win || !ns || !heads || !out)))
    return fail(SEPSO_EINVAL, "null argument or negative count");
  if (tw < 1 || tw > 64) return fail(SEPSO_EINVAL, "tw=%d outside [1, 64]", tw);
  if (count > (1 << 20)) return fail(SEPSO_EINVAL, "count=%d above 2^20", count);
  for (int32_t i = 0; i < count; ++i) {
    if (ns[i] < 1 || ns[i] > tw) return fail(SEPSO_EINVAL, "ns[%d]=%d outside [1, tw]", i, ns[i]);
    if (heads[i] < 0 || heads[i] >= tw) return fail(SEPSO_EINVAL, "heads[%d]=%d outside [0, tw)", i, heads[i]);
  }
  if (count == 0) return SEPSO_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t wb = (size_t)count * tw * sizeof(double), ib = (size_t)count * sizeof(int32_t);
  char* d = nullptr;
  CUDA_TRY(cudaMalloc(&d, wb + 3 * ib));
  double* dw = reinterpret_cast<double*>(d);
  int32_t* dn = reinterpret_cast<int32_t*>(d + wb);
  int32_t* dh = dn + count;
  int32_t* dout = dh + count;
  cudaError_t e = cudaMemcpyAsync(dw, win, wb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dn, ns, ib, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dh, heads, ib, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_at_window(dw, dn, dh, count, tw, delta, dout, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, ib, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  CUDA_TRY(e);
  return SEPSO_OK;
}

// ---------------------------------------------------------------------------
// Planning without any device allocation.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// framework's memory pool, plugins whose host application forbids allocations
// after start-up, or real-time loops where an allocation could block.  For
// them, sepso_plan_static keeps its workspace in the file-scope device array
// below instead of caller-provided memory.  The array is part of the library
// image, so every GPU that loads libsepso holds these bytes until the process
// exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchBytes = size_t(8) << 20;  // 8 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::once_flag g_scratch_once[kMaxDevices];
void* g_scratch_addr[kMaxDevices];
cudaError_t g_scratch_err[kMaxDevices];

// The array's name is only a host-side stand-in in host code; its device
// address must be looked up once per device with that device current.
int static_scratch(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return fail(SEPSO_EINVAL, "device %d out of range", device);
  std::call_once(g_scratch_once[device], [device] {
    g_scratch_err[device] = cudaGetSymbolAddress(&g_scratch_addr[device], g_static_scratch);
  });
  if (g_scratch_err[device] != cudaSuccess) return cuda_fail(g_scratch_err[device], "cudaGetSymbolAddress");
  *out = g_scratch_addr[device];
  return SEPSO_OK;
}

}  // namespace

extern "C" int sepso_plan_static(const sepso_config* cfg, const float* hyper, const float* start,
                                 const float* target, const float* circles, int32_t O, float* waypoints,
                                 sepso_result* res, void* stream) {
  int rc = check_config(cfg);
  if (rc) return rc;
  if (cfg->runs != 1) return fail(SEPSO_EINVAL, "sepso_plan_static plans one run (runs=%d)", cfg->runs);
  if (cfg->obstacle_kind != SEPSO_OBST_CIRCLES) return fail(SEPSO_EINVAL, "sepso_plan_static plans among circles");
  if (!hyper || !start || !target || (O > 0 && !circles))
    return fail(SEPSO_EINVAL, "NULL input to sepso_plan_static");
  if (O < 0 || O > cfg->max_obstacles)
    return fail(SEPSO_EINVAL, "O=%d outside [0, max_obstacles=%d]", O, cfg->max_obstacles);
  for (int i = 0; i < cfg->G * 6; ++i)
    if (!finite(hyper[i])) return fail(SEPSO_EINVAL, "hyper[%d] is not finite", i);
  for (int g = 0; g < cfg->G; ++g)  // the same rule as sepso_set_hyper
    if (hyper[g * 6 + 5] < 0) return fail(SEPSO_EINVAL, "V_limit of group %d is negative", g);
  if (!finite(start[0]) || !finite(start[1]) || !finite(target[0]) || !finite(target[1]))
    return fail(SEPSO_EINVAL, "start/target not finite");
  for (int o = 0; o < O; ++o) {
    const float r = circles[3 * o + 2];
    if (!finite(circles[3 * o]) || !finite(circles[3 * o + 1]) || !finite(r) || r < 0)
      return fail(SEPSO_EINVAL, "circle %d invalid (non-finite or negative radius)", o);
  }
  const WsLayout L = make_ws(*cfg);
  if (L.total > kStaticScratchBytes)
    return fail(SEPSO_ENOSPC,
                "sepso_plan_static: this configuration needs %zu bytes of workspace; the static "
                "scratch holds %zu bytes (use sepso_create with caller memory instead)",
                L.total, kStaticScratchBytes);

  // A handle on the stack: no host or device allocation.
  sepso_ctx h;
  h.cfg = *cfg;
  h.stream = static_cast<cudaStream_t>(stream);
  h.L = L;
  h.O = O;
  h.has_scene = true;
  {
    const double v = std::ceil((double)cfg->pi_gamma * (double)cfg->N);
    h.n_pi = (int)std::min<double>(std::max(v, 0.0), (double)cfg->N);
  }
  CUDA_TRY(cudaGetDevice(&h.device));
  CUDA_TRY(cudaDeviceGetAttribute(&h.num_sms, cudaDevAttrMultiProcessorCount, h.device));
  void* scratch = nullptr;
  if ((rc = static_scratch(h.device, &scratch))) return rc;
  h.ws = static_cast<char*>(scratch);
  h.ws_bytes = kStaticScratchBytes;
  if ((rc = choose_shape(&h))) return rc;

  // Each call starts from zeroed scratch (barrier counter, bests, counters) with
  // empty group-best keys, then writes its inputs.  Host inputs are copied from the caller's (pageable)
  // memory, so they may be reused as soon as this call returns.
  CUDA_TRY(cudaMemsetAsync(h.ws, 0, L.total, h.stream));
  CUDA_TRY(cudaMemsetAsync(h.ws + L.gword, 0xff, (size_t)3 * cfg->G * 8, h.stream));  // empty keys
  RunCtl ctl;
  std::memset(&ctl, 0, sizeof ctl);
  ctl.Tfit = INFINITY;
  ctl.prev_lfv = INFINITY;
  ctl.run_id = cfg->run_id;
  CUDA_TRY(cudaMemcpyAsync(h.ws + L.ctl, &ctl, sizeof ctl, cudaMemcpyHostToDevice, h.stream));
  CUDA_TRY(cudaMemcpyAsync(h.ws + L.hyper, hyper, (size_t)cfg->G * 6 * 4, cudaMemcpyHostToDevice, h.stream));
  float4 chunk[128];
  for (int o0 = 0; o0 < O; o0 += 128) {
    const int n = std::min(128, O - o0);
    for (int i = 0; i < n; ++i) {
      const float* c = circles + 3 * (o0 + i);
      chunk[i] = make_float4(c[0], c[1], c[2], 4.0f * (c[2] * c[2]));
    }
    CUDA_TRY(cudaMemcpyAsync(h.ws + L.circ + (size_t)o0 * 16, chunk, (size_t)n * 16, cudaMemcpyHostToDevice,
                             h.stream));
    // the copy reads the stack buffer: let it finish before the buffer is refilled
    if (o0 + 128 < O) CUDA_TRY(cudaStreamSynchronize(h.stream));
  }
  const float pts[8] = {start[0], start[1], target[0], target[1], 0.f, 0.f, 0.f, 0.f};
  CUDA_TRY(cudaMemcpyAsync(h.ws + L.pts, pts, sizeof pts, cudaMemcpyHostToDevice, h.stream));
  CUDA_TRY(launch_pairs(h.at<float4>(L.circ), O, h.at<float4>(L.pairs), h.stream));

  h.c3_nonzero.assign(1, 0);
  for (int g = 0; g < cfg->G; ++g)
    if (hyper[g * 6 + 2] != 0.0f) h.c3_nonzero[0] = 1;
  if ((rc = launch_plan_kernel(&h, swarm_params(&h, kModePlan, 0)))) return rc;

  sepso_result tmp;
  if (waypoints)
    CUDA_TRY(cudaMemcpyAsync(waypoints, h.ws + L.res_wp, (size_t)2 * cfg->T * 4, cudaMemcpyDeviceToHost,
                             h.stream));
  CUDA_TRY(cudaMemcpyAsync(&tmp, h.ws + L.res, sizeof tmp, cudaMemcpyDeviceToHost, h.stream));
  CUDA_TRY(cudaStreamSynchronize(h.stream));
  if (res) *res = tmp;
  if (tmp.status != SEPSO_OK) return fail(tmp.status, "device-side error in sepso_plan_static");
  return SEPSO_OK;
}
