// sepso_server.cu -- continuous-batching request server for SEPSO planning on
// GB300 (sm_103a).
//
// Agents submit planning requests (their current scene).  The server keeps up to
// S request slots on the device and advances every occupied slot by one iteration
// of Algorithm 1 per "tick" (one launch of the batched kernel over the slots'
// work items).  A request runs Priori Initialization from its agent's previous
// best path (kept in a device table, Sec. 3.3.3) and ends by Auto Truncation
// (stall counter, Sec. 3.3.4) or the cap; its slot is then freed and a queued
// request is admitted at the next tick, so requests that arrive while others are
// on the GPU join the running batch.  The number of slots is bounded by a device
// memory budget.  Between ticks the host (1) launches the tick, (2) queues the
// read-back of done flags and results, (3) retires the slots that finished in the
// previous tick, (4) admits queued requests with one upload and one scatter
// launch, (5) uploads the new work-item list -- all stream-ordered after the
// running tick, so the GPU keeps working while the host does this.  An agent has
// at most one request in flight (the next one needs its warm start).  A request's
// random streams are keyed by (agent, cycle), so its result is the same alone and
// in any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <new>
#include <string>
#include <vector>

#include "sepso_batch.cuh"
#include "sepso_device.cuh"
#include "sepso_internal.h"

using namespace sepso;

namespace {

thread_local std::string g_server_error;

int sfail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int sfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_server_error = buf;
  return code;
}

#define SCUDA(expr)                                                                                \
  do {                                                                                             \
    cudaError_t e_ = (expr);                                                                       \
    if (e_ != cudaSuccess) return sfail(SEPSO_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));    \
  } while (0)

size_t a256(size_t v) { return (v + 255) & ~size_t(255); }

// One admission: the slot, its scene record and its points; its circles follow in
// the circle staging area at slot-independent offset `c0`.
struct Admit {
  BatchScene desc;
  float pts[4];
  int slot;
  int c0;
  int pad[2];
};

struct ServerLayout {
  size_t sc, tiles, X, V, P, Pfit, PQ, slots, Gb, Tb, circ, hyper, pts, words, Gfit2, GQ2, Tfit2, TQ2, stall2, plv2,
      done, res_wp, res, prevT, admits, admit_circ, status, priorT, prior_use, praw, rcirc, rcoff, rpts, total;
};

constexpr int kPriorMaxT = 64;  // largest proposal of an attached prior (waypoints)

ServerLayout server_layout(const sepso_server_config& c, int S) {
  const size_t G = c.G, N = c.N, M = G * N, Dm = 2 * (size_t)c.Tmax, Om = std::max(c.Omax, 1);
  const size_t tiles_per_slot = G * ((N + 7) / 8);
  ServerLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = a256(off);
    const size_t o = off;
    off += bytes;
    return o;
  };
  L.sc = take(S * sizeof(BatchScene));
  L.tiles = take(S * tiles_per_slot * sizeof(int4));
  L.X = take(S * M * Dm * 4);
  L.V = take(S * M * Dm * 4);
  L.P = take(S * M * Dm * 4);
  L.Pfit = take(S * M * 4);
  L.PQ = take(S * M * 4);
  L.slots = take(S * 2 * M * (Dm + 4) * 4);
  L.Gb = take(S * G * Dm * 4);
  L.Tb = take(S * Dm * 4);
  L.circ = take(S * (size_t)pair_block_f4((int)Om) * 16);
  L.hyper = take((size_t)c.n_agents * G * 6 * 4);
  L.pts = take(S * 16);
  L.words = take(S * 3 * G * 8);
  L.Gfit2 = take(S * 2 * G * 4);
  L.GQ2 = take(S * 2 * G * 4);
  L.Tfit2 = take(S * 2 * 4);
  L.TQ2 = take(S * 2 * 4);
  L.stall2 = take(S * 2 * 4);
  L.plv2 = take(S * 2 * 4);
  L.done = take(S * 4);
  L.res_wp = take(S * Dm * 4);
  L.res = take(S * sizeof(sepso_result));
  L.prevT = take((size_t)c.n_agents * Dm * 4);
  L.admits = take(S * sizeof(Admit));
  L.admit_circ = take(S * (size_t)pair_block_f4((int)Om) * 16);
  L.status = take(16);  // status, then the first failed index check of the batch kernel
  // learned prior (used once one is attached): the slots' proposals at their own T,
  // the gate flags, the raw proposals of one admission batch, and its scenes as the
  // rasteriser reads them
  L.priorT = take(S * Dm * 4);
  L.prior_use = take(S * 4);
  L.praw = take(2 * S * 2 * (size_t)kPriorMaxT * 4);  // by tick parity
  L.rcirc = take(S * Om * 16);
  L.rcoff = take((S + 1) * 4);
  L.rpts = take(S * 16);
  L.total = a256(off);
  return L;
}

int check_server_config(const sepso_server_config* c) {
  if (!c) return sfail(SEPSO_EINVAL, "config is NULL");
  if (c->n_agents < 1 || c->max_slots < 1 || c->G < 1 || c->G > 32 || c->N < 1 || c->N >= (1 << 20) ||
      c->Tmax < 1 || c->Tmax > 64 || c->Omax < 0 || c->Omax > 8192 || c->max_iters < 1 || c->stall_iters < 0 ||
      c->beta < 1 || c->beta > 8 || !std::isfinite(c->alpha) || c->alpha < 0 || !std::isfinite(c->map_w) ||
      !std::isfinite(c->map_h) || c->map_w <= 0 || c->map_h <= 0 || !(c->pi_gamma >= 0 && c->pi_gamma <= 1) ||
      !(c->pi_halfwidth >= 0) || !std::isfinite(c->stall_tol))
    return sfail(SEPSO_EINVAL, "bad server configuration");
  if (c->tile < 0 || c->tile > 256 || c->threads < 0 || c->threads > 512 || c->threads % 32)
    return sfail(SEPSO_EINVAL, "bad launch shape");
  return SEPSO_OK;
}

// Slots that fit: at most max_slots, and (when a budget is given) within it.
int server_slots(const sepso_server_config& c) {
  int S = c.max_slots;
  if (c.mem_budget > 0) {
    while (S > 1 && server_layout(c, S).total > c.mem_budget) S = std::max(1, S * 7 / 8);
  }
  return S;
}

// Scatter the admissions into their slots and reset the slots' bests.
__global__ void server_admit_kernel(BatchParams p, const Admit* admits, const float4* admit_circ, int n,
                                    int Omax) {
  const int a = blockIdx.x;
  if (a >= n) return;
  const Admit A = admits[a];
  const int s = A.slot;
  const BatchScene& S = A.desc;
  if (threadIdx.x == 0) {
    const_cast<BatchScene*>(p.sc)[s] = S;
    float* pts = const_cast<float*>(p.pts);
    for (int i = 0; i < 4; ++i) pts[4 * s + i] = A.pts[i];
    p.Tfit2[2 * s] = p.Tfit2[2 * s + 1] = INFINITY;
    p.TQ2[2 * s] = p.TQ2[2 * s + 1] = 0;
    p.stall2[2 * s] = p.stall2[2 * s + 1] = 0;
    p.plv2[2 * s] = p.plv2[2 * s + 1] = INFINITY;
    p.done[s] = 0;
  }
  // the request's circle-pair block, staged by the host in the same layout
  float4* circ = const_cast<float4*>(p.circ) + S.co;
  const int nf4 = S.O > 0 ? (S.poly ? edge_pair_f4(S.O) : pair_block_f4(S.O)) : 0;
  for (int o = threadIdx.x; o < nf4; o += blockDim.x) circ[o] = admit_circ[A.c0 + o];
  for (int g = threadIdx.x; g < 2 * S.G; g += blockDim.x) {
    p.Gfit2[S.gso + g] = INFINITY;
    p.GQ2[S.gso + g] = 0;
  }
  for (int g = threadIdx.x; g < 3 * S.G; g += blockDim.x) p.words[S.wo + g] = kKeyEmpty;
}

// Learned-prior seeds of one admission batch (an extension: the paper has no learned
// component), one warp per admitted request.  Its proposal (Tp waypoints, row a of
// praw) becomes the slot's row at the request's T: the proposal itself when T = Tp,
// else the T points at arc-length fractions 1/(T+1), ..., T/(T+1) of the polyline
// start -> proposal -> target (FP32, lengths summed in order on lane 0).  Then the
// batch planner's gate: the proposal seeds the slot only when its fitness (Sec.
// 3.3.2, FP32) on the request's scene is below that of the agent's previous path, or
// the agent has none.  The slot's circles are in place (server_admit_kernel ran).
__global__ void server_prior_kernel(BatchParams p, const Admit* admits, int n, const float* praw, int Tp) {
  __shared__ float cum[kPriorMaxT + 2];
  const int a = blockIdx.x, lane = threadIdx.x;
  if (a >= n) return;
  const BatchScene S = admits[a].desc;
  const int s = admits[a].slot, T = S.T;
  const float sx = admits[a].pts[0], sy = admits[a].pts[1], tx = admits[a].pts[2], ty = admits[a].pts[3];
  const float* P = praw + (size_t)a * 2 * Tp;
  float* out = const_cast<float*>(p.prior_path) + (size_t)s * p.Dmax;
  if (T == Tp) {
    for (int j = lane; j < 2 * T; j += 32) out[j] = P[j];
  } else {
    auto px = [&](int k) { return k == 0 ? sx : (k == Tp + 1 ? tx : P[k - 1]); };
    auto py = [&](int k) { return k == 0 ? sy : (k == Tp + 1 ? ty : P[Tp + k - 1]); };
    if (lane == 0) {
      float c = 0.0f;
      cum[0] = 0.0f;
      for (int k = 0; k <= Tp; ++k) {
        const float dx = px(k + 1) - px(k), dy = py(k + 1) - py(k);
        c += sqrtf(fmaf(dx, dx, dy * dy));
        cum[k + 1] = c;
      }
    }
    __syncwarp();
    const float total = cum[Tp + 1];
    for (int i = lane; i < T; i += 32) {
      const float t = total * ((float)(i + 1) / (float)(T + 1));
      int k = 0;
      while (k < Tp && cum[k + 1] < t) ++k;  // segment k holds arc length t
      const float L = cum[k + 1] - cum[k];
      const float f = L > 0.0f ? fminf(fmaxf((t - cum[k]) / L, 0.0f), 1.0f) : 0.0f;
      out[i] = fmaf(f, px(k + 1) - px(k), px(k));
      out[T + i] = fmaf(f, py(k + 1) - py(k), py(k));
    }
  }
  __syncwarp();
  const int K = circle_pairs(S.O);
  const int split = warp_split(T, K);
  const float4* cxy = p.circ + S.co;
  const float2* nr2 = reinterpret_cast<const float2*>(cxy + K);
  float len;
  int q;
  group_fitness_pairs(out, true, 32, T, split, K, sx, sy, tx, ty, cxy, nr2, &len, &q);
  const float f_prior = len + S.alpha * powi((float)q, S.beta);
  int ok = 1;
  if (S.has_prev && S.n_pi > 0) {
    group_fitness_pairs(p.agent_prevT + (size_t)S.agent * p.Dmax, true, 32, T, split, K, sx, sy, tx, ty, cxy, nr2,
                        &len, &q);
    ok = f_prior < len + S.alpha * powi((float)q, S.beta);
  }
  if (lane == 0) const_cast<int32_t*>(p.prior_use)[s] = ok;
}

struct Request {
  int agent, T, O;
  bool poly = false;        // O polygon edges instead of circles
  float pts[4];
  std::vector<float> circ;  // O x 3 (circles) or O x 4 (edges)
  long long tag;
  double arrival;           // server clock (s); admitted once the clock passes it
};

struct Slot {
  bool busy = false;
  int agent = -1, T = 0, O = 0;
  bool poly = false;
  long long tag = 0;
  long long start_tick = 0;  // tick of the first iteration
  double arrival = 0.0;
};

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct sepso_server_ctx {
  sepso_server_config cfg{};
  int S = 0, Dm = 0, Om = 0, tiles_per_slot = 0;
  ServerLayout L{};
  char* ws = nullptr;
  cudaStream_t stream = nullptr;
  int smem_optin = 0, tile = 32, threads = 128;
  size_t smem = 0;
  std::vector<Slot> slots;
  std::vector<int> order;  // occupied slots by cost (scratch of upload_tiles)
  std::deque<Request> queue;
  std::vector<int> agent_cycle;
  std::vector<char> agent_busy;
  std::vector<sepso_server_done> done_list;
  std::vector<float> done_wp;
  long long tick = 0;
  // pinned staging, by tick parity
  int32_t* rb_done[2] = {nullptr, nullptr};
  sepso_result* rb_res[2] = {nullptr, nullptr};
  float* rb_wp[2] = {nullptr, nullptr};
  int rb_hw[2] = {0, 0};
  long long rb_tick[2] = {0, 0};
  bool rb_pending[2] = {false, false};
  cudaEvent_t rb_ev[2] = {nullptr, nullptr};
  Admit* h_admit[2] = {nullptr, nullptr};
  float4* h_acirc[2] = {nullptr, nullptr};
  int4* h_tiles[2] = {nullptr, nullptr};
  bool tiles_dirty = false;
  int ntiles = 0;
  long long admitted = 0, completed = 0, launches = 0;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  // learned prior (sepso_server_set_prior): its handle, seeds per group, first
  // dataset row, proposal waypoints, and the admissions' scenes staged for its
  // rasteriser (pinned, by tick parity)
  sepso_prior_ctx* prior = nullptr;
  int n_prior = 0, prior_first = 0, prior_T = 0;
  // the prior's work runs on a side stream beside the tick's batch kernel: it waits
  // for ev_tick (main stream, before the tick's launch), the main stream waits for
  // ev_prop before the seed / gate kernel
  cudaStream_t pside = nullptr;
  cudaEvent_t ev_tick = nullptr, ev_prop = nullptr;
  // The seeds of a tick's admissions are applied in the next tick, after that tick's
  // batch launch: the proposals then run beside it instead of holding up the main
  // stream, and the admitted slots start one tick later.  Pending: the tick parity
  // of the admissions, their number and the proposals' waypoint count.
  bool seed_pending = false;
  int seed_b = 0, seed_n = 0, seed_T = 0;
  float4* h_rcirc[2] = {nullptr, nullptr};
  int* h_rcoff[2] = {nullptr, nullptr};
  float* h_rpts[2] = {nullptr, nullptr};

  ~sepso_server_ctx() {
    for (int i = 0; i < 2; ++i) {
      if (rb_ev[i]) cudaEventDestroy(rb_ev[i]);
      if (rb_done[i]) cudaFreeHost(rb_done[i]);
      if (rb_res[i]) cudaFreeHost(rb_res[i]);
      if (rb_wp[i]) cudaFreeHost(rb_wp[i]);
      if (h_admit[i]) cudaFreeHost(h_admit[i]);
      if (h_acirc[i]) cudaFreeHost(h_acirc[i]);
      if (h_tiles[i]) cudaFreeHost(h_tiles[i]);
      if (h_rcirc[i]) cudaFreeHost(h_rcirc[i]);
      if (h_rcoff[i]) cudaFreeHost(h_rcoff[i]);
      if (h_rpts[i]) cudaFreeHost(h_rpts[i]);
    }
    if (ev_tick) cudaEventDestroy(ev_tick);
    if (ev_prop) cudaEventDestroy(ev_prop);
    if (pside) cudaStreamDestroy(pside);
  }
  template <class T>
  T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }

  BatchParams params() const {
    BatchParams p;
    p.sc = at<BatchScene>(L.sc);
    p.tiles = at<int4>(L.tiles);
    p.ntiles = ntiles;
    p.nscenes = S;
    p.W = cfg.map_w;
    p.H = cfg.map_h;
    p.Omax = Om;
    p.Dmax = Dm;
    p.Gmax = cfg.G;
    p.tile = tile;
    p.X = at<float>(L.X);
    p.V = at<float>(L.V);
    p.P = at<float>(L.P);
    p.Pfit = at<float>(L.Pfit);
    p.PQ = at<int32_t>(L.PQ);
    p.slots = at<float>(L.slots);
    p.Gb = at<float>(L.Gb);
    p.Tb = at<float>(L.Tb);
    p.circ = at<float4>(L.circ);
    p.hyper = at<float>(L.hyper);
    p.pts = at<float>(L.pts);
    p.words = at<unsigned long long>(L.words);
    p.Gfit2 = at<float>(L.Gfit2);
    p.GQ2 = at<int32_t>(L.GQ2);
    p.Tfit2 = at<float>(L.Tfit2);
    p.TQ2 = at<int32_t>(L.TQ2);
    p.res_wp = at<float>(L.res_wp);
    p.res = at<sepso_result>(L.res);
    p.status = at<int>(L.status);
    p.stall2 = at<int32_t>(L.stall2);
    p.plv2 = at<float>(L.plv2);
    p.done = at<int32_t>(L.done);
    p.agent_prevT = at<float>(L.prevT);
    p.prior_path = prior ? at<float>(L.priorT) : nullptr;
    p.agent_rows = nullptr;
    p.prior_use = prior ? at<int32_t>(L.prior_use) : nullptr;
    return p;
  }
};

namespace {

// Slots that finished in the tick whose read-back sits in buffer b.
void retire(sepso_server_ctx* h, int b) {
  for (int i = 0; i < h->rb_hw[b]; ++i) {
    Slot& sl = h->slots[i];
    if (!sl.busy || sl.start_tick > h->rb_tick[b] || !h->rb_done[b][i]) continue;
    sepso_server_done d;
    d.tag = sl.tag;
    d.agent = sl.agent;
    d.T = sl.T;
    d.res = h->rb_res[b][i];
    d.arrival_s = sl.arrival;
    d.finish_s = now_s(h->t0);
    h->done_list.push_back(d);
    const float* wp = h->rb_wp[b] + (size_t)i * h->Dm;
    h->done_wp.insert(h->done_wp.end(), wp, wp + h->Dm);
    h->agent_cycle[sl.agent] += 1;
    h->agent_busy[sl.agent] = 0;
    sl.busy = false;
    h->tiles_dirty = true;
    ++h->completed;
  }
}

// The previous tick's seeds (resampling and gate of each admitted slot's proposal),
// on the main stream once its proposals are done; the admissions' descriptors are
// still in the device buffer (this tick's upload comes after).
int flush_seeds(sepso_server_ctx* h) {
  if (!h->seed_pending) return SEPSO_OK;
  h->seed_pending = false;
  float* praw = h->at<float>(h->L.praw) + (size_t)h->seed_b * h->S * 2 * kPriorMaxT;
  SCUDA(cudaStreamWaitEvent(h->stream, h->ev_prop, 0));
  server_prior_kernel<<<h->seed_n, 32, 0, h->stream>>>(h->params(), h->at<Admit>(h->L.admits), h->seed_n, praw,
                                                         h->seed_T);
  SCUDA(cudaGetLastError());
  ++h->launches;
  return SEPSO_OK;
}

int admit(sepso_server_ctx* h, int b) {
  const sepso_server_config& c = h->cfg;
  {
    const int rc = flush_seeds(h);
    if (rc) return rc;
  }
  // with a prior, a slot's first iteration waits one more tick for its seed
  const int defer = h->prior ? 1 : 0;
  int n = 0, c0 = 0, rc0 = 0;
  size_t free_slot = 0;
  const double now = now_s(h->t0);
  for (auto it = h->queue.begin(); it != h->queue.end();) {
    if (it->arrival > now) break;  // the queue is in arrival order
    if (h->agent_busy[it->agent]) {
      ++it;
      continue;
    }
    while (free_slot < h->slots.size() && h->slots[free_slot].busy) ++free_slot;
    if (free_slot >= h->slots.size()) break;
    const Request& r = *it;
    const int i = (int)free_slot;
    Admit& A = h->h_admit[b][n];
    std::memset(&A, 0, sizeof A);
    BatchScene& d = A.desc;
    const long long M = (long long)c.G * c.N;
    d.T = r.T;
    d.D = 2 * r.T;
    d.G = c.G;
    d.N = c.N;
    d.M = (int)M;
    d.O = r.O;
    d.max_iters = c.max_iters;
    d.beta = c.beta;
    d.alpha = c.alpha;
    d.key0 = (uint32_t)(c.seed & 0xffffffffu);
    d.key1 = (uint32_t)(c.seed >> 32);
    d.run_id = (uint32_t)r.agent;
    d.xo = (long long)i * M * h->Dm;
    d.mo = (long long)i * M;
    d.so = (long long)i * 2 * M * (h->Dm + 4);
    d.go = (long long)i * c.G * h->Dm;
    d.to = (long long)i * h->Dm;
    d.co = (long long)i * pair_block_f4(h->Om);
    d.ho = (long long)r.agent * c.G * 6;
    d.wo = (long long)i * 3 * c.G;
    d.gso = (long long)i * 2 * c.G;
    d.j0 = (int)h->tick + defer;  // its first iteration is the next launch (with a prior, the one after)
    d.at_stall = c.stall_iters;
    d.stall_tol = c.stall_tol;
    d.n_pi = (int)std::min<double>(std::max(std::ceil((double)c.pi_gamma * c.N), 0.0), (double)c.N);
    d.n_pr = h->prior ? h->n_prior : 0;
    d.pi_h = c.pi_halfwidth;
    d.cycle = (uint32_t)h->agent_cycle[r.agent];
    d.agent = r.agent;
    d.has_prev = h->agent_cycle[r.agent] > 0;
    std::memcpy(A.pts, r.pts, sizeof A.pts);
    A.slot = i;
    A.c0 = c0;
    d.poly = r.poly ? 1 : 0;
    d.pad_poly = 0;
    if (r.poly) {
      d.n_pr = 0;  // no learned prior for a polygon request
      pack_edge_pairs(r.circ.data(), r.O, h->h_acirc[b] + c0);
      c0 += edge_pair_f4(r.O);
    } else if (r.O > 0) {
      // circle-pair block (layout in sepso_device.cuh)
      const int K = circle_pairs(r.O), nf4 = pair_block_f4(r.O);
      float4* blk = h->h_acirc[b] + c0;
      for (int q = 0; q < nf4; ++q) blk[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      float* nr2 = reinterpret_cast<float*>(blk + K);
      for (int o = 0; o < r.O; ++o) {
        const float rr = r.circ[3 * o + 2];
        float* pr = reinterpret_cast<float*>(blk + o / 2);
        pr[o & 1] = r.circ[3 * o];
        pr[2 + (o & 1)] = r.circ[3 * o + 1];
        nr2[o] = -(rr * rr);
      }
      c0 += nf4;
    }
    if (h->prior) {  // the scene as the prior's rasteriser reads it
      float4* rc = h->h_rcirc[b] + rc0;
      for (int o = 0; o < r.O; ++o) rc[o] = make_float4(r.circ[3 * o], r.circ[3 * o + 1], r.circ[3 * o + 2], 0.0f);
      h->h_rcoff[b][n] = rc0;
      std::memcpy(h->h_rpts[b] + 4 * n, r.pts, sizeof r.pts);
      rc0 += r.O;
    }
    Slot& sl = h->slots[i];
    sl.busy = true;
    sl.agent = r.agent;
    sl.T = r.T;
    sl.O = r.O;
    sl.poly = r.poly;
    sl.tag = r.tag;
    sl.start_tick = h->tick + 1 + defer;
    sl.arrival = r.arrival;
    h->agent_busy[r.agent] = 1;
    ++n;
    ++h->admitted;
    h->tiles_dirty = true;
    it = h->queue.erase(it);
  }
  if (n == 0) return SEPSO_OK;
  SCUDA(cudaMemcpyAsync(h->ws + h->L.admits, h->h_admit[b], (size_t)n * sizeof(Admit), cudaMemcpyHostToDevice,
                        h->stream));
  if (c0 > 0)
    SCUDA(cudaMemcpyAsync(h->ws + h->L.admit_circ, h->h_acirc[b], (size_t)c0 * 16, cudaMemcpyHostToDevice,
                          h->stream));
  server_admit_kernel<<<n, 128, 0, h->stream>>>(h->params(), h->at<Admit>(h->L.admits),
                                                h->at<float4>(h->L.admit_circ), n, h->Om);
  SCUDA(cudaGetLastError());
  ++h->launches;
  if (h->prior) {
    // The prior's proposals for the admitted scenes on the side stream, beside the
    // running tick and the next one (they touch only the prior's rows and this
    // parity's staging); each slot's seed row and gate follow in the next tick.
    h->h_rcoff[b][n] = rc0;
    const cudaStream_t ps = h->pside;
    float* praw = h->at<float>(h->L.praw) + (size_t)b * h->S * 2 * kPriorMaxT;
    SCUDA(cudaStreamWaitEvent(ps, h->ev_tick, 0));
    if (rc0 > 0) SCUDA(cudaMemcpyAsync(h->ws + h->L.rcirc, h->h_rcirc[b], (size_t)rc0 * 16, cudaMemcpyHostToDevice, ps));
    SCUDA(cudaMemcpyAsync(h->ws + h->L.rcoff, h->h_rcoff[b], (size_t)(n + 1) * 4, cudaMemcpyHostToDevice, ps));
    SCUDA(cudaMemcpyAsync(h->ws + h->L.rpts, h->h_rpts[b], (size_t)n * 16, cudaMemcpyHostToDevice, ps));
    const long long l0 = sepso_prior_launch_count(h->prior);
    const cudaStream_t keep = prior_swap_stream(h->prior, ps);
    const int rc = prior_propose_device(h->prior, h->prior_first, n, h->at<float4>(h->L.rcirc),
                                        h->at<int>(h->L.rcoff), h->at<float>(h->L.rpts), praw, 2 * h->prior_T);
    prior_swap_stream(h->prior, keep);
    if (rc) return sfail(rc, "learned prior: %s", sepso_prior_last_error());
    h->launches += sepso_prior_launch_count(h->prior) - l0;
    SCUDA(cudaEventRecord(h->ev_prop, ps));
    h->seed_pending = true;
    h->seed_b = b;
    h->seed_n = n;
    h->seed_T = h->prior_T;
  }
  return SEPSO_OK;
}

// Work items of the occupied slots, costliest first (segments x circles), so that
// each launch ends with its cheapest items.
int upload_tiles(sepso_server_ctx* h, int b) {
  if (!h->tiles_dirty) return SEPSO_OK;
  h->order.clear();
  for (size_t i = 0; i < h->slots.size(); ++i)
    if (h->slots[i].busy) h->order.push_back((int)i);
  std::stable_sort(h->order.begin(), h->order.end(), [h](int a, int c) {
    const Slot &x = h->slots[a], &y = h->slots[c];
    return (long long)(x.T + 1) * (std::max(x.O, 1) + 8) > (long long)(y.T + 1) * (std::max(y.O, 1) + 8);
  });
  int n = 0;
  for (int i : h->order)
    for (int g = 0; g < h->cfg.G; ++g)
      for (int n0 = 0; n0 < h->cfg.N; n0 += h->tile)
        h->h_tiles[b][n++] = make_int4(i, g, n0, std::min(h->tile, h->cfg.N - n0));
  if (n > 0)
    SCUDA(cudaMemcpyAsync(h->ws + h->L.tiles, h->h_tiles[b], (size_t)n * sizeof(int4), cudaMemcpyHostToDevice,
                          h->stream));
  h->ntiles = n;
  h->tiles_dirty = false;
  return SEPSO_OK;
}

}  // namespace

extern "C" {

const char* sepso_server_last_error(void) { return g_server_error.c_str(); }

int sepso_server_workspace_size(const sepso_server_config* cfg, size_t* bytes, int32_t* slots) {
  int rc = check_server_config(cfg);
  if (rc) return rc;
  const int S = server_slots(*cfg);
  if (bytes) *bytes = server_layout(*cfg, S).total;
  if (slots) *slots = S;
  return SEPSO_OK;
}

int sepso_server_create(const sepso_server_config* cfg, void* d_workspace, size_t bytes, void* stream,
                        sepso_server_handle* out) {
  int rc = check_server_config(cfg);
  if (rc) return rc;
  if (!out) return sfail(SEPSO_EINVAL, "out is NULL");
  *out = nullptr;
  const int S = server_slots(*cfg);
  const ServerLayout L = server_layout(*cfg, S);
  if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255u))
    return sfail(SEPSO_ENOSPC, "workspace must be non-NULL and 256-byte aligned");
  if (bytes < L.total) return sfail(SEPSO_ENOSPC, "workspace has %zu bytes, needs %zu", bytes, L.total);
  sepso_server_ctx* h = new (std::nothrow) sepso_server_ctx();
  if (!h) return sfail(SEPSO_ENOMEM, "host allocation failed");
  h->cfg = *cfg;
  h->S = S;
  h->Dm = 2 * cfg->Tmax;
  h->Om = std::max(cfg->Omax, 1);
  h->L = L;
  h->ws = static_cast<char*>(d_workspace);
  h->stream = static_cast<cudaStream_t>(stream);
  h->tile = cfg->tile > 0 ? std::max(8, cfg->tile) : 32;
  h->threads = cfg->threads > 0 ? cfg->threads : 128;
  h->slots.resize(S);
  h->agent_cycle.assign(cfg->n_agents, 0);
  h->agent_busy.assign(cfg->n_agents, 0);
  const size_t tps = (size_t)cfg->G * ((cfg->N + 7) / 8);
  cudaError_t e = batch_configure(&h->smem_optin);
  h->smem = (size_t)BatchSmem::make(h->Om, h->tile, h->Dm, cfg->G).total;
  if (e == cudaSuccess && h->smem > (size_t)h->smem_optin) {
    const size_t need = h->smem;
    delete h;
    return sfail(SEPSO_ERANGE, "a work item needs %zu B of shared memory", need);
  }
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaMallocHost(reinterpret_cast<void**>(&h->rb_done[i]), (size_t)S * 4);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&h->rb_res[i]), (size_t)S * sizeof(sepso_result));
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&h->rb_wp[i]), (size_t)S * h->Dm * 4);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&h->h_admit[i]), (size_t)S * sizeof(Admit));
    if (e == cudaSuccess)
      e = cudaMallocHost(reinterpret_cast<void**>(&h->h_acirc[i]), (size_t)S * pair_block_f4(h->Om) * 16);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&h->h_tiles[i]), (size_t)S * tps * sizeof(int4));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->rb_ev[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->ws, 0, L.total, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    delete h;
    return sfail(SEPSO_ECUDA, "server set-up: %s", cudaGetErrorString(e));
  }
  *out = h;
  return SEPSO_OK;
}

void sepso_server_destroy(sepso_server_handle h) {
  if (h) cudaStreamSynchronize(h->stream);
  delete h;
}

int sepso_server_set_hyper(sepso_server_handle h, int32_t agent, const float* hyper) {
  if (!h || !hyper) return sfail(SEPSO_EINVAL, "NULL argument");
  const int G = h->cfg.G;
  for (int i = 0; i < 6 * G; ++i)
    if (!std::isfinite(hyper[i])) return sfail(SEPSO_EINVAL, "hyper[%d] not finite", i);
  if (agent >= h->cfg.n_agents) return sfail(SEPSO_EINVAL, "agent %d out of range", agent);
  const int a0 = agent < 0 ? 0 : agent, a1 = agent < 0 ? h->cfg.n_agents : agent + 1;
  std::vector<float> all((size_t)(a1 - a0) * G * 6);
  for (int a = a0; a < a1; ++a) std::memcpy(all.data() + (size_t)(a - a0) * G * 6, hyper, (size_t)G * 6 * 4);
  SCUDA(cudaMemcpyAsync(h->ws + h->L.hyper + (size_t)a0 * G * 6 * 4, all.data(), all.size() * 4,
                        cudaMemcpyHostToDevice, h->stream));
  SCUDA(cudaStreamSynchronize(h->stream));
  return SEPSO_OK;
}

int sepso_server_set_prior(sepso_server_handle h, sepso_prior_handle prior, int32_t n_prior, int32_t first_row) {
  if (!h) return sfail(SEPSO_EINVAL, "NULL handle");
  {
    const int rc = flush_seeds(h);  // seeds of admissions made under the previous setting
    if (rc) return rc;
  }
  if (!prior) {
    h->prior = nullptr;
    h->n_prior = 0;
    return SEPSO_OK;
  }
  for (const Request& r : h->queue)
    if (r.poly) return sfail(SEPSO_EINVAL, "polygon requests queued: the prior rasterises circles only");
  for (const Slot& sl : h->slots)
    if (sl.busy && sl.poly) return sfail(SEPSO_EINVAL, "polygon requests in flight: the prior rasterises circles only");
  int T = 0, mc = 0, cap = 0;
  float W = 0.0f, H = 0.0f;
  cudaStream_t st = nullptr;
  if (prior_shape(prior, &T, &mc, &cap, &W, &H, &st) != SEPSO_OK) return sfail(SEPSO_EINVAL, "bad prior handle");
  if (T < 1 || T > kPriorMaxT) return sfail(SEPSO_EINVAL, "the prior proposes %d waypoints (1..%d)", T, kPriorMaxT);
  if (n_prior < 0 || n_prior > h->cfg.N) return sfail(SEPSO_EINVAL, "n_prior %d outside [0, N=%d]", n_prior, h->cfg.N);
  if (mc < h->cfg.Omax)
    return sfail(SEPSO_EINVAL, "the prior rasterises at most %d circles, requests have up to %d", mc, h->cfg.Omax);
  if (first_row < 0 || (long long)first_row + h->S > cap)
    return sfail(SEPSO_EINVAL, "rows [%d, %d) outside the prior's %d", first_row, first_row + h->S, cap);
  if (W != h->cfg.map_w || H != h->cfg.map_h) return sfail(SEPSO_EINVAL, "the prior's map differs from the server's");
  if (st != h->stream) return sfail(SEPSO_EINVAL, "the prior must run on the server's stream");
  if (!h->pside) SCUDA(cudaStreamCreateWithFlags(&h->pside, cudaStreamNonBlocking));
  if (!h->ev_tick) SCUDA(cudaEventCreateWithFlags(&h->ev_tick, cudaEventDisableTiming));
  if (!h->ev_prop) SCUDA(cudaEventCreateWithFlags(&h->ev_prop, cudaEventDisableTiming));
  for (int i = 0; i < 2; ++i) {
    if (!h->h_rcirc[i]) SCUDA(cudaMallocHost(reinterpret_cast<void**>(&h->h_rcirc[i]), (size_t)h->S * h->Om * 16));
    if (!h->h_rcoff[i]) SCUDA(cudaMallocHost(reinterpret_cast<void**>(&h->h_rcoff[i]), (size_t)(h->S + 1) * 4));
    if (!h->h_rpts[i]) SCUDA(cudaMallocHost(reinterpret_cast<void**>(&h->h_rpts[i]), (size_t)h->S * 16));
  }
  h->prior = prior;
  h->n_prior = n_prior;
  h->prior_first = first_row;
  h->prior_T = T;
  return SEPSO_OK;
}

int sepso_server_submit_at(sepso_server_handle h, int32_t agent, int32_t T, const float* start,
                           const float* target, const float* circles, int32_t O, int64_t tag, double arrival_s) {
  if (!h || !start || !target) return sfail(SEPSO_EINVAL, "NULL argument");
  if (agent < 0 || agent >= h->cfg.n_agents) return sfail(SEPSO_EINVAL, "agent %d out of range", agent);
  if (T < 1 || T > h->cfg.Tmax) return sfail(SEPSO_EINVAL, "T=%d outside [1, Tmax=%d]", T, h->cfg.Tmax);
  if (O < 0 || O > h->cfg.Omax || (O > 0 && !circles)) return sfail(SEPSO_EINVAL, "O=%d invalid", O);
  Request r;
  r.agent = agent;
  r.T = T;
  r.O = O;
  r.pts[0] = start[0];
  r.pts[1] = start[1];
  r.pts[2] = target[0];
  r.pts[3] = target[1];
  for (float v : r.pts)
    if (!std::isfinite(v)) return sfail(SEPSO_EINVAL, "start/target not finite");
  r.circ.assign(circles, circles + 3 * (size_t)O);
  for (int o = 0; o < O; ++o)
    if (!std::isfinite(r.circ[3 * o]) || !std::isfinite(r.circ[3 * o + 1]) || !std::isfinite(r.circ[3 * o + 2]) ||
        r.circ[3 * o + 2] < 0)
      return sfail(SEPSO_EINVAL, "circle %d invalid", o);
  r.tag = tag;
  r.arrival = arrival_s;
  if (!h->queue.empty() && arrival_s < h->queue.back().arrival)
    return sfail(SEPSO_EINVAL, "requests must be submitted in arrival order");
  h->queue.push_back(std::move(r));
  return SEPSO_OK;
}

int sepso_server_submit_polygons(sepso_server_handle h, int32_t agent, int32_t T, const float* start,
                                 const float* target, const float* edges, int32_t E, int64_t tag, double arrival_s) {
  if (!h || !start || !target) return sfail(SEPSO_EINVAL, "NULL argument");
  if (h->prior) return sfail(SEPSO_EINVAL, "polygon requests are served without the learned prior: detach it");
  if (agent < 0 || agent >= h->cfg.n_agents) return sfail(SEPSO_EINVAL, "agent %d out of range", agent);
  if (T < 1 || T > h->cfg.Tmax) return sfail(SEPSO_EINVAL, "T=%d outside [1, Tmax=%d]", T, h->cfg.Tmax);
  const int cap = std::min(h->Om, pair_block_f4(h->Om) & ~1);  // the edge pairs fill the circle block
  if (E < 0 || E > cap || (E > 0 && !edges)) return sfail(SEPSO_EINVAL, "E=%d edges invalid (at most %d)", E, cap);
  Request r;
  r.agent = agent;
  r.T = T;
  r.O = E;
  r.poly = true;
  r.pts[0] = start[0];
  r.pts[1] = start[1];
  r.pts[2] = target[0];
  r.pts[3] = target[1];
  for (float v : r.pts)
    if (!std::isfinite(v)) return sfail(SEPSO_EINVAL, "start/target not finite");
  r.circ.assign(edges, edges + 4 * (size_t)E);
  for (float v : r.circ)
    if (!std::isfinite(v)) return sfail(SEPSO_EINVAL, "edge coordinate not finite");
  r.tag = tag;
  if (arrival_s < 0.0) {
    const double now = now_s(h->t0);
    arrival_s = h->queue.empty() ? now : std::max(now, h->queue.back().arrival);
  }
  r.arrival = arrival_s;
  if (!h->queue.empty() && arrival_s < h->queue.back().arrival)
    return sfail(SEPSO_EINVAL, "requests must be submitted in arrival order");
  h->queue.push_back(std::move(r));
  return SEPSO_OK;
}

int sepso_server_submit(sepso_server_handle h, int32_t agent, int32_t T, const float* start, const float* target,
                        const float* circles, int32_t O, int64_t tag) {
  if (!h) return sfail(SEPSO_EINVAL, "NULL handle");
  const double now = now_s(h->t0);
  const double last = h->queue.empty() ? now : std::max(now, h->queue.back().arrival);
  return sepso_server_submit_at(h, agent, T, start, target, circles, O, tag, last);
}

double sepso_server_clock(sepso_server_handle h, int32_t restart) {
  if (!h) return -1.0;
  if (restart) h->t0 = std::chrono::steady_clock::now();
  return now_s(h->t0);
}

int sepso_server_tick(sepso_server_handle h, int32_t* active, int32_t* queued) {
  if (!h) return sfail(SEPSO_EINVAL, "NULL handle");
  const long long j = ++h->tick;
  const int b = (int)(j & 1);
  // (1) one iteration of every occupied slot (after the point the prior's work of this
  // tick's admissions may start from)
  if (h->prior) SCUDA(cudaEventRecord(h->ev_tick, h->stream));
  if (h->ntiles > 0) {
    SCUDA(launch_batch_iter(h->params(), (int)j, h->ntiles, h->threads, h->smem, h->stream));
    ++h->launches;
  }
  // (2) read back done flags and results of the occupied slots
  int hw = 0;
  for (int i = 0; i < h->S; ++i)
    if (h->slots[i].busy) hw = i + 1;
  if (hw > 0) {
    SCUDA(cudaMemcpyAsync(h->rb_done[b], h->ws + h->L.done, (size_t)hw * 4, cudaMemcpyDeviceToHost, h->stream));
    SCUDA(cudaMemcpyAsync(h->rb_res[b], h->ws + h->L.res, (size_t)hw * sizeof(sepso_result), cudaMemcpyDeviceToHost,
                          h->stream));
    SCUDA(cudaMemcpyAsync(h->rb_wp[b], h->ws + h->L.res_wp, (size_t)hw * h->Dm * 4, cudaMemcpyDeviceToHost,
                          h->stream));
  }
  SCUDA(cudaEventRecord(h->rb_ev[b], h->stream));
  h->rb_hw[b] = hw;
  h->rb_tick[b] = j;
  h->rb_pending[b] = true;
  // (3) retire what finished in the previous tick
  const int pb = b ^ 1;
  if (h->rb_pending[pb]) {
    SCUDA(cudaEventSynchronize(h->rb_ev[pb]));
    retire(h, pb);
    h->rb_pending[pb] = false;
  }
  // (4) admit, (5) the work items of the next tick
  int rc = admit(h, b);
  if (rc) return rc;
  rc = upload_tiles(h, b);
  if (rc) return rc;
  int act = 0;
  for (const Slot& sl : h->slots) act += sl.busy;
  if (active) *active = act;
  if (queued) *queued = (int32_t)h->queue.size();
  return SEPSO_OK;
}

int sepso_server_poll(sepso_server_handle h, sepso_server_done* out, float* waypoints, int32_t max_n, int32_t* n) {
  if (!h || !n) return sfail(SEPSO_EINVAL, "NULL argument");
  const int k = std::min<int>(max_n, (int)h->done_list.size());
  for (int i = 0; i < k; ++i) {
    if (out) out[i] = h->done_list[i];
    if (waypoints) std::memcpy(waypoints + (size_t)i * h->Dm, h->done_wp.data() + (size_t)i * h->Dm, (size_t)h->Dm * 4);
  }
  h->done_list.erase(h->done_list.begin(), h->done_list.begin() + k);
  h->done_wp.erase(h->done_wp.begin(), h->done_wp.begin() + (size_t)k * h->Dm);
  *n = k;
  return SEPSO_OK;
}

int sepso_server_drain(sepso_server_handle h, int64_t max_ticks) {
  if (!h) return sfail(SEPSO_EINVAL, "NULL handle");
  for (int64_t t = 0; t < max_ticks; ++t) {
    int act = 0;
    for (const Slot& sl : h->slots) act += sl.busy;
    if (act == 0 && h->queue.empty()) {
      for (int b = 0; b < 2; ++b)
        if (h->rb_pending[b]) {
          SCUDA(cudaEventSynchronize(h->rb_ev[b]));
          h->rb_pending[b] = false;
        }
      return SEPSO_OK;
    }
    const int rc = sepso_server_tick(h, nullptr, nullptr);
    if (rc) return rc;
  }
  return sfail(SEPSO_ETIMEOUT, "requests still active after %lld ticks", (long long)max_ticks);
}

int sepso_server_run(sepso_server_handle h, int64_t max_ticks) {
  if (!h) return sfail(SEPSO_EINVAL, "NULL handle");
  for (int64_t t = 0; t < max_ticks; ++t) {
    int act = 0;
    for (const Slot& sl : h->slots) act += sl.busy;
    if (act == 0) {
      if (h->queue.empty()) return sepso_server_drain(h, max_ticks);
      // idle until the next arrival
      while (now_s(h->t0) < h->queue.front().arrival) {
      }
    }
    const int rc = sepso_server_tick(h, nullptr, nullptr);
    if (rc) return rc;
  }
  return sfail(SEPSO_ETIMEOUT, "requests still pending after %lld ticks", (long long)max_ticks);
}

int sepso_server_stats(sepso_server_handle h, int32_t* slots, int64_t* admitted, int64_t* completed,
                       int64_t* ticks, int64_t* launches) {
  if (!h) return sfail(SEPSO_EINVAL, "NULL handle");
  if (slots) *slots = h->S;
  if (admitted) *admitted = h->admitted;
  if (completed) *completed = h->completed;
  if (ticks) *ticks = h->tick;
  if (launches) *launches = h->launches;
  return SEPSO_OK;
}

}  // extern "C"
