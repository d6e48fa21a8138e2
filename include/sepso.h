/*
 * sepso.h -- C ABI of the GB300 (sm_103a) SEPSO planner library (libsepso.so).
 *
 * SEPSO: Self-Evolving Particle Swarm Optimization for real-time path planning
 * (Xin, Li, Zhang, Li; arXiv 2308.10169).  The library runs the grouped,
 * tensor-form PSO (DTPSO, Sec. 3.1, Algorithm 1) over a swarm X[G][N][D=2T] of
 * waypoint paths, scores paths with Eqs. path_fit / lenth / penalty
 * (Sec. 3.3.2) against circular obstacles, and wraps the loop with Priori
 * Initialization (Sec. 3.3.3), Auto Truncation (Sec. 3.3.4) and the
 * hierarchical self-evolving framework HSEF (Sec. 3.2.1, Eq. fit_h).
 *
 * Conventions for every call:
 *   - Return value: SEPSO_OK (0) or a negative SEPSO_E* code; nothing aborts.
 *     sepso_strerror() names the code; sepso_last_error() gives a message.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA global
 *     memory of the device that was current at sepso_create().  All input arrays
 *     are read during the call (host) or before the enqueued work completes
 *     (device); the caller keeps ownership of everything it passes.
 *   - The caller owns the workspace (device memory of sepso_workspace_size()
 *     bytes, 256-byte aligned) and the CUDA stream; all device work of a handle
 *     is enqueued on that stream.  Calls marked "async" return once the work is
 *     enqueued; calls marked "sync" wait for the stream.
 *   - Layouts: a particle / path is D = 2T floats [x_1..x_T, y_1..y_T]
 *     (Eq. coordinate); hyper-parameters are G rows of
 *     (C1, C2, C3, w_init, w_end, V_limit) (Table hyper8 layout);
 *     circles are O rows of (cx, cy, r).
 *   - A handle is not thread-safe; distinct handles may be used concurrently.
 */
#ifndef SEPSO_H
#define SEPSO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define SEPSO_OK 0
#define SEPSO_EINVAL (-1)   /* bad argument: size, NaN/Inf, O > max, ...        */
#define SEPSO_ESTATE (-2)   /* call out of order (e.g. plan before a scene)      */
#define SEPSO_ENOSPC (-3)   /* workspace too small or misaligned                 */
#define SEPSO_ECUDA (-4)    /* a CUDA runtime call failed                        */
#define SEPSO_ETIMEOUT (-5) /* a device-side wait gave up (bounded spin)         */
#define SEPSO_ENOMEM (-6)   /* host allocation failed                            */
#define SEPSO_ERANGE (-7)   /* shape exceeds a kernel limit (shared memory etc.) */
#define SEPSO_EBOUNDS (-8)  /* a device-side index check failed (access skipped)  */

/* Auto Truncation modes (Sec. 3.3.4). */
#define SEPSO_AT_OFF 0          /* run to max_iters                                  */
#define SEPSO_AT_STD_WINDOW 1   /* std of the LFV over the last TW iterations < delta,
                                   and the best path collision-free                  */
#define SEPSO_AT_STALL 2        /* LFV not improved (by more than stall_tol) for
                                   stall_iters iterations, and the best path
                                   collision-free                                    */

/* Obstacle kinds (sepso_config.obstacle_kind). */
#define SEPSO_OBST_CIRCLES 0    /* Q = (path segment, circle) pairs closer than r    */
#define SEPSO_OBST_POLYGONS 1   /* Q = (path segment, polygon edge) pairs crossing
                                   properly (Sec. 3.3.1's map model: bounding boxes
                                   or outlines, Eq. penalty)                         */

typedef struct sepso_ctx* sepso_handle;

/* Fixed at sepso_create().  Fields follow Algorithm 1 and Tables params_path /
 * hyper8; "runs" swarms share one scene (used by HSEF, whose H-particles each
 * own one L-run). */
typedef struct {
  int32_t T;              /* waypoints per path; D = 2T, 1 <= T <= 64            */
  int32_t G;              /* groups, 1 <= G <= 32                                */
  int32_t N;              /* particles per group, 1 <= N < 2^20                  */
  int32_t max_obstacles;  /* capacity for circles, >= 0                          */
  float map_w, map_h;     /* X_range: x in [0, map_w], y in [0, map_h]           */
  float alpha;            /* Eq. penalty: alpha * Q^beta                         */
  int32_t beta;           /* integer exponent, 1..8                              */
  int32_t max_iters;      /* cap; also T of Eq. TOF_omega                        */
  int32_t at_mode;        /* SEPSO_AT_*                                          */
  int32_t tw;             /* truncation window TW (mode 1), 1..64                */
  float delta;            /* std threshold (mode 1)                              */
  int32_t stall_iters;    /* mode 2 limit                                        */
  float stall_tol;        /* mode 2: improvement must exceed this                */
  int32_t use_pi;         /* Priori Initialization on/off                        */
  float pi_gamma;         /* fraction of each group placed by PI, [0, 1]         */
  float pi_halfwidth;     /* half-width of the PI interval around the last best  */
  uint64_t seed;          /* Philox4x32-10 key                                   */
  uint32_t run_id;        /* Philox counter word 3 of run 0 (run r: run_id + r)  */
  int32_t runs;           /* independent swarms on the same scene, >= 1          */
  int32_t ctas_per_group; /* 0 = automatic; else CTAs cooperating on one group   */
  int32_t threads;        /* 0 = automatic; else 64..512, a multiple of 32       */
  int32_t circle_split;   /* 0 = automatic; else circle chunks per segment        */
  int32_t fitness_mode;   /* 0 = automatic; 1 = a lane group per particle; 2 =
                             (particle, segment, circle chunk) items spread over
                             all threads of a CTA                                  */
  int32_t exchange;       /* how the CTAs of a run trade their bests each
                             iteration: 1 = grid-wide: one barrier of all the
                             run's CTAs per iteration; 2 = cluster form: the CTAs
                             of a group form one thread-block cluster (one warp
                             per particle, rows in registers) and trade through
                             distributed shared memory, groups trade only
                             (Gfit, Q) through global memory, read two
                             iterations later (needs C3 = 0 in every group: Eq.
                             TOF_V then uses the own group's Gbest alone, and a
                             config that fits: T + 1 <= 32, G <= 32, at most 15
                             particles per CTA of at most 16 per group, every
                             group resident at once).  Both forms give identical
                             results.  0 (automatic) and 3 = the cluster form
                             whenever every group's C3 is 0 and it fits, else
                             grid-wide.                                          */
  int32_t obstacle_kind;  /* SEPSO_OBST_*: circles (sepso_set_scene) or polygon
                             edges (sepso_set_polygons); for polygons
                             max_obstacles is the edge capacity                   */
} sepso_config;

/* Outcome of one planning cycle of one run. */
typedef struct {
  float cost;     /* F(Tbest) = length + alpha * Q^beta                          */
  float length;   /* Eq. lenth of Tbest                                          */
  int32_t Q;      /* collision count of Tbest                                    */
  int32_t iters;  /* iterations run (k at exit)                                  */
  int32_t status; /* SEPSO_OK or the device-side error of the run                */
} sepso_result;

/* ---- lifetime ----------------------------------------------------------- */

/* Bytes of device workspace a config needs.  Errors: EINVAL on a bad config. */
int sepso_workspace_size(const sepso_config* cfg, size_t* bytes);

/* Validate cfg, lay out the caller's workspace (d_workspace, bytes; device,
 * 256-byte aligned, not freed before sepso_destroy) and pick launch shapes for
 * the current device.  stream: a cudaStream_t (NULL = legacy default stream).
 * Zeroes the workspace (async on the stream).  Errors: EINVAL, ENOSPC,
 * ERANGE (shape does not fit the kernel), ECUDA, ENOMEM. */
int sepso_create(const sepso_config* cfg, void* d_workspace, size_t bytes, void* stream,
                 sepso_handle* out);

/* Release the host context.  Does not free the workspace or the stream. */
void sepso_destroy(sepso_handle h);

/* ---- inputs ------------------------------------------------------------- */

/* Hyper-parameters (host, G x 6 floats, Table hyper8 layout) for run `run`,
 * or for every run when run < 0.  Copied to the device (async).
 * Errors: EINVAL (non-finite value, V_limit < 0, run out of range). */
int sepso_set_hyper(sepso_handle h, int32_t run, const float* hyper);

/* Scene (host): start[2], target[2], circles O x 3 (cx, cy, r), 0 <= O <=
 * max_obstacles, r >= 0.  Packed into the handle's pinned staging buffer and
 * copied to the device (async DMA; the call first waits for the previous
 * scene copy to leave the staging buffer); circle velocities are reset to
 * zero.  Errors: EINVAL. */
int sepso_set_scene(sepso_handle h, const float* start, const float* target,
                    const float* circles, int32_t O);

/* Per-cycle velocities for the dynamic scene (host): circle_vel O x 2 (for
 * polygon obstacles: P x 2, one per polygon), start_vel[2], target_vel[2].
 * Errors: EINVAL, ESTATE (no scene yet). */
int sepso_set_motion(sepso_handle h, const float* circle_vel, const float* start_vel,
                     const float* target_vel);

/* Advance the dynamic scene `steps` times on the device (async): every circle and
 * the start/target move by their velocity; a velocity component flips when the
 * disk crosses the border it moves towards (Fig. PP caption).  Polygon obstacles
 * move rigidly (all edges of a polygon by its velocity) and bounce by their
 * bounding box: a component flips when the box lies past the border it moves
 * towards.  Errors: ESTATE, EINVAL (steps < 0). */
int sepso_advance_scene(sepso_handle h, int32_t steps);

/* Read the current scene back (host outputs, sync): start[2], target[2],
 * circles O x 3, circle_vel O x 2 (any output may be NULL). */
int sepso_get_scene(sepso_handle h, float* start, float* target, float* circles,
                    float* circle_vel);

/* Scene among polygon obstacles (Sec. 3.3.1: obstacles are bounding boxes or
 * outlines given by their edges; Q of Eq. penalty counts the (path segment, edge)
 * pairs that cross properly -- each segment's endpoints strictly on opposite
 * sides of the other's line -- so touching and collinear contacts do not count,
 * and a path wholly inside an obstacle crosses nothing).  Host inputs: start[2],
 * target[2], edges E x 4 (x0, y0, x1, y1), 0 <= E <= max_obstacles; offsets
 * P + 1 int32: polygon p owns edges [offsets[p], offsets[p+1]) (offsets[0] = 0,
 * offsets[P] = E, non-decreasing), so that it moves as one body.  Polygon
 * velocities are reset to zero (sepso_set_motion sets them, one per polygon).
 * Only on a handle with obstacle_kind = SEPSO_OBST_POLYGONS.  Sync.
 * Errors: EINVAL. */
int sepso_set_polygons(sepso_handle h, const float* start, const float* target, const float* edges,
                       int32_t E, const int32_t* offsets, int32_t P);

/* Read a polygon scene back (host outputs, sync; any may be NULL): start[2],
 * target[2], edges E x 4, polygon velocities P x 2.  Errors: EINVAL, ESTATE. */
int sepso_get_polygons(sepso_handle h, float* start, float* target, float* edges, float* polygon_vel);

/* ---- the hot path ------------------------------------------------------- */

/* One planning cycle of every run (async): initialise the swarm (uniform over
 * X_range, V uniform in +-V_range; with PI and a previous path, the first
 * ceil(pi_gamma * N) particles of each group uniform in prevT +- pi_halfwidth,
 * clipped), then iterate Algorithm 1 until Auto Truncation or max_iters, then
 * store the result and the warm-start state (previous best path, AT window,
 * cycle counter).  One cooperative persistent kernel launch.
 * Errors: ESTATE (no scene), ECUDA (launch). Device-side errors are reported by
 * sepso_read_result / sepso_sync. */
int sepso_plan_async(sepso_handle h);

/* sepso_plan_async, then read run 0's result (sync).  waypoints: host, D floats
 * (may be NULL); res: host (may be NULL). */
int sepso_plan(sepso_handle h, float* waypoints, sepso_result* res);

/* Copy the last result of run `run` to the host (sync). */
int sepso_read_result(sepso_handle h, int32_t run, float* waypoints, sepso_result* res);

/* Device address of run `run`'s result waypoints (D floats) and of its
 * sepso_result record, valid while the handle lives (for device-side consumers). */
int sepso_result_device(sepso_handle h, int32_t run, float** d_waypoints,
                        sepso_result** d_result);

/* Continue the current swarm of every run for `iters` full iterations of
 * Algorithm 1 (no re-initialisation, no truncation check, no cap) (async). */
int sepso_step(sepso_handle h, int32_t iters);

/* Fitness of n paths on the current scene (async): d_X device n x D floats;
 * outputs device (any may be NULL): d_F fitness, d_Q collision counts,
 * d_len lengths.  Errors: ESTATE, EINVAL. */
int sepso_evaluate(sepso_handle h, const float* d_X, int32_t n, float* d_F, int32_t* d_Q,
                   float* d_len);

/* ---- state (checkpoint / parity) ---------------------------------------- */

/* Bytes of one run's serialised state.  Layout, in order (floats unless noted):
 *   X[M*D] V[M*D] P[M*D] Pfit[M] PQ[M](int32) Gb[G*D] Gfit[G] GQ[G](int32)
 *   Tb[D] Tfit[1] TQ[1](int32) k[1](int32) cycle[1](int32) has_prev[1](int32)
 *   prevT[D] win[TW](double) win_n[1](int32) win_head[1](int32) stall[1](int32)
 *   prev_lfv[1]
 * with M = G*N; the double block starts 8-byte aligned (zero padding before it
 * when needed). */
int sepso_state_size(sepso_handle h, size_t* bytes);

/* Copy run `run`'s state to/from host memory (sync). */
int sepso_get_state(sepso_handle h, int32_t run, void* host_buf, size_t bytes);
int sepso_set_state(sepso_handle h, int32_t run, const void* host_buf, size_t bytes);

/* ---- HSEF (Sec. 3.2.1) -------------------------------------------------- */

/* The evolution phase.  The handle's runs are the H-particles (runs = HG * HN);
 * each H-particle is a per-group (w, C1, C2) vector; its fitness is the LFV
 * (Eq. fit_h) of an L-run of max_iters iterations with C3 = 0,
 * w_init = w_end = w and V_limit = l_vlimit, AT and PI off, all L-runs of one
 * evolution on the same random streams (run id cfg.run_id, cycle = evolution-1).
 * The H-swarm is DTPSO with hhyper (HG x 6, Table hyper8) and omega schedule
 * over E evolutions, inside the box [lo, hi] of (w, C1, C2). */
typedef struct {
  int32_t HG, HN;     /* H-swarm groups and particles per group                */
  int32_t E;          /* evolutions                                            */
  float hhyper[32 * 6]; /* HG rows, Table hyper8 layout                        */
  float lo[3], hi[3]; /* box of (w, C1, C2)                                    */
  float l_vlimit;     /* V_limit of the L-runs                                 */
  uint64_t hseed;     /* Philox key of the H-swarm                             */
} sepso_hsef_config;

/* Run E evolutions (async; 2 launches per evolution).  d_history: device, E
 * floats (may be NULL), receives the best LFV after each evolution.
 * Errors: EINVAL (runs != HG*HN, HG > 32, 3G > 96), ESTATE. */
int sepso_hsef(sepso_handle h, const sepso_hsef_config* hc, float* d_history);

/* Best H-position found so far as G hyper rows (C1, C2, 0, w, w, l_vlimit)
 * and its LFV (host outputs, sync). */
int sepso_hsef_best(sepso_handle h, float* hyper_out, float* best_lfv);

/* ---- many scenes of uneven size in one batch ------------------------------ */

/* One independent DTPSO run per scene (Algorithm 1 with the path fitness of
 * Sec. 3.3.2).  Each launch advances every unfinished scene by one iteration;
 * the whole run is one CUDA graph.  Scenes may differ in T, G, N, O, max_iters,
 * alpha, beta, seed and truncation; the map extent is shared.  Optional per
 * scene: Auto Truncation by stall counter (Sec. 3.3.4) and warm starts
 * (sepso_batch_set_starts): Priori Initialization around the scene's previous
 * path (Sec. 3.3.3) and a second seed of the same kind around a learned prior's
 * proposal.  A scene's result does not depend on the rest of the batch (its
 * random streams are keyed by its seed, run id and cycle). */
typedef struct sepso_batch_ctx* sepso_batch_handle;

typedef struct {
  int32_t T, G, N, O;   /* waypoints (1..64), groups (1..32), particles per group, circles */
  int32_t max_iters;    /* iterations of this scene (>= 1)                              */
  float alpha;          /* Eq. penalty                                                  */
  int32_t beta;         /* 1..8                                                         */
  uint64_t seed;        /* Philox key                                                   */
  uint32_t run_id;      /* Philox counter word 3                                        */
  int32_t stall_iters;  /* 0: run max_iters; else Auto Truncation (Sec. 3.3.4): stop
                           once Tbest is collision-free and its fitness has not dropped
                           by more than stall_tol for stall_iters iterations            */
  float stall_tol;
  int32_t n_pi;         /* particles per group started around the previous path (PI) */
  int32_t n_prior;      /* particles per group started around the prior's proposal   */
  float pi_halfwidth;   /* half-width of both start intervals                         */
  uint32_t cycle;       /* Philox counter word 2 (low 24 bits): the planning cycle    */
  int32_t obstacle_kind; /* 0: O circles; 1: O polygon edges (Sec. 3.3.1: Q = the
                            number of proper crossings of path segments and edges) */
} sepso_batch_scene;

/* Launch shape: particles per work item (8..256), threads per CTA (64..512, a
 * multiple of 32); lanes is 32 (a warp per particle; 0 is accepted); reserved
 * must be 0.  The shape changes speed only, never results. */
typedef struct {
  int32_t tile, threads, lanes, reserved;
} sepso_batch_shape;

/* Bytes of device workspace for n scenes.  Errors: EINVAL. */
int sepso_batch_workspace_size(const sepso_batch_scene* scenes, int32_t n, size_t* bytes);

/* Lay out the batch in the caller's workspace (device, 256-byte aligned, owned by
 * the caller), on the caller's stream; the map is [0, map_w] x [0, map_h].
 * Errors: EINVAL, ENOSPC, ECUDA, ENOMEM, ERANGE. */
int sepso_batch_create(const sepso_batch_scene* scenes, int32_t n, float map_w, float map_h,
                       void* d_workspace, size_t bytes, void* stream, sepso_batch_handle* out);
void sepso_batch_destroy(sepso_batch_handle h);

/* Inputs (host, copied; sync): hyper = the scenes' G x 6 rows back to back (Table
 * hyper8 layout), points = n x 4 (start x, y, target x, y), circles = the scenes'
 * obstacle rows back to back: O x 3 (cx, cy, r) for a circle scene, O x 4 (x0, y0,
 * x1, y1; a closed polygon lists each side once) for a polygon scene.
 * Errors: EINVAL. */
int sepso_batch_set_inputs(sepso_batch_handle h, const float* hyper, const float* points,
                           const float* circles);

/* Set or read the launch shape (work_items: number of CTAs per launch). */
int sepso_batch_set_shape(sepso_batch_handle h, const sepso_batch_shape* shape);
int sepso_batch_get_shape(sepso_batch_handle h, sepso_batch_shape* shape, int32_t* work_items);

/* Time the candidate shapes (tile 8..64, threads 128..512) over
 * trial_launches iteration launches on the loaded batch and keep the fastest
 * (sync).  best_ms: time of one iteration launch with it.  The batch state is
 * overwritten (a later run starts from scratch), the stored previous paths
 * included: call it before sepso_batch_set_starts. */
int sepso_batch_autotune(sepso_batch_handle h, int32_t trial_launches, sepso_batch_shape* best,
                         float* best_ms);

/* Warm starts of the next run (sync).  prev, prior: device arrays of row stride
 * ld floats (ld >= the batch's largest 2T), row s for scene s, waypoint layout
 * x_0..x_{T-1}, y_0..y_{T-1}; either may be NULL.  prev: the scenes' previous
 * best paths, the centres of PI (NULL keeps the stored paths: every run stores
 * each scene's result there, the next cycle's PI centre); n rows of ld floats.  has_prev: n host flags
 * (a scene without a previous path starts without PI), or NULL (all 1 when prev
 * is given, else unchanged).  prior: proposals of the learned prior (NULL: none).
 * A scene's n_prior particles start around its proposal only when the proposal's
 * fitness (Sec. 3.3.2, FP32) on the scene is below that of its previous path, or
 * it has none; otherwise the scene starts from PI alone.  The decision is taken
 * on the device at this call.  Errors: EINVAL, ECUDA. */
int sepso_batch_set_starts(sepso_batch_handle h, const float* prev, const float* prior, int32_t ld,
                           const int32_t* has_prev);

/* Multi-agent teams (the paper names multi-agent planning as future work; this is
 * an extension).  Scenes [team_first[s], team_first[s] + team_size[s]) form scene
 * s's team: agents sharing a map, contiguous, with one T.  All agents of a team
 * leave their starts together and reach one point of their path per time step
 * (start, T waypoints, target), straight in between; in each step, a pair whose
 * relative position passes closer than sep to the origin (the relative motion is a
 * segment) is one conflict, added to Q of Eq. penalty.  An agent's fitness counts
 * its conflicts with its mates' current paths: moving obstacles.  Host arrays of n
 * int32; sync.  The mates' paths count from the first sepso_batch_next_round.
 * Errors: EINVAL. */
int sepso_batch_set_teams(sepso_batch_handle h, const int32_t* team_first, const int32_t* team_size, float sep);

/* Start the next round of best responses: every scene's last result (with its
 * start and target) becomes its agent's path as its mates see it, and the centre
 * of its own Priori Initialization; every scene's Philox cycle becomes `cycle`.
 * The next sepso_batch_run_async then plans every agent against its mates' paths
 * of the round before (device copies; sync).  Errors: ESTATE (no teams), ECUDA. */
int sepso_batch_next_round(sepso_batch_handle h, uint32_t cycle);

/* Number of scenes that will use their prior proposal (host output, sync). */
int sepso_batch_prior_used(sepso_batch_handle h, int32_t* n_used);

/* Run every scene from initialisation to its max_iters (async).  use_graph != 0
 * replays a CUDA graph of the run (captured at the first call after a shape
 * change); 0 launches the kernels directly.  Errors: ESTATE, ECUDA. */
int sepso_batch_run_async(sepso_batch_handle h, int32_t use_graph);

/* Results (host, sync): waypoints = the scenes' 2T floats back to back, res = n
 * records.  Either may be NULL. */
int sepso_batch_read(sepso_batch_handle h, float* waypoints, sepso_result* res);

int64_t sepso_batch_launch_count(sepso_batch_handle h);
const char* sepso_batch_last_error(void);

/* ---- serving: continuous batching of planning requests -------------------- */

/* Agents submit planning requests (their current scene).  Up to S requests are
 * on the device at once, each in a slot; every tick advances every occupied slot
 * by one iteration of Algorithm 1 (one launch).  A request starts with Priori
 * Initialization (Sec. 3.3.3) around its agent's previous best path, kept on the
 * device, and ends by Auto Truncation with the stall counter (Sec. 3.3.4) or at
 * max_iters; its slot then takes the next queued request at the following tick.
 * S is max_slots, lowered to fit mem_budget (admission by device memory).  An
 * agent has at most one request on the device; its later requests wait in the
 * queue.  Random streams are keyed by (seed, agent, the agent's request count),
 * so a result does not depend on the other requests in flight. */
typedef struct sepso_server_ctx* sepso_server_handle;

typedef struct {
  int32_t n_agents;      /* rows of the warm-start table                          */
  int32_t max_slots;     /* requests on the device at most                        */
  size_t mem_budget;     /* workspace bytes the slots may use (0: no bound)       */
  int32_t G, N;          /* swarm of every request                                */
  int32_t Tmax, Omax;    /* largest request: waypoints, circles                   */
  int32_t max_iters;     /* cap per request                                       */
  int32_t stall_iters;   /* AT stall limit (0: run to the cap)                    */
  float stall_tol;
  float alpha;           /* Eq. penalty                                           */
  int32_t beta;
  float pi_gamma, pi_halfwidth;
  float map_w, map_h;
  uint64_t seed;         /* Philox key                                            */
  int32_t tile, threads; /* launch shape (0: 32 particles, 128 threads)           */
} sepso_server_config;

/* A finished request. */
typedef struct {
  int64_t tag;           /* the caller's tag from sepso_server_submit             */
  int32_t agent, T;
  sepso_result res;
  double arrival_s;      /* server clock at arrival                               */
  double finish_s;       /* server clock when its completion was collected        */
} sepso_server_done;

/* Bytes of workspace and the number of slots S a config gets.  Errors: EINVAL. */
int sepso_server_workspace_size(const sepso_server_config* cfg, size_t* bytes, int32_t* slots);
/* Create on the caller's workspace and stream (as sepso_create).  Allocates pinned
 * host staging buffers.  Errors: EINVAL, ENOSPC, ERANGE, ECUDA, ENOMEM. */
int sepso_server_create(const sepso_server_config* cfg, void* d_workspace, size_t bytes, void* stream,
                        sepso_server_handle* out);
void sepso_server_destroy(sepso_server_handle h);
/* Hyper-parameters (host G x 6) of one agent, or of all when agent < 0 (sync). */
int sepso_server_set_hyper(sepso_server_handle h, int32_t agent, const float* hyper);
/* Attach a learned prior (sepso_prior_*; an extension: the paper has no learned
 * component) to the server, or detach it (prior NULL).  From the next admission on,
 * each admitted request's scene is rasterised into the prior's dataset rows
 * [first_row, first_row + S) (S = the server's slots; they are overwritten), the
 * prior proposes a path of its own T_p waypoints, and that path becomes the
 * request's: itself when T = T_p, else the T points at arc-length fractions
 * 1/(T+1) .. T/(T+1) of the polyline start -> proposal -> target.  The first n_prior
 * particles of every group then start around it (the PI half-width), before the PI
 * particles, when its fitness (Sec. 3.3.2, FP32) on the request's scene is below
 * that of the agent's previous path, or the agent has none -- the gate of
 * sepso_batch_set_starts.  All of it runs on the device: the rasteriser and the
 * network on a side stream of the server, beside the tick that is running and the
 * next one, the resampling and the gate on the server's stream in the next tick;
 * a request admitted with a prior attached therefore starts one tick later than
 * without (its first iteration is the second launch after its admission).  The prior
 * must have been created on the server's stream and map, with max_circles >= Omax,
 * T_p <= 64 and capacity >= first_row + S; it must outlive its attachment, and the
 * caller must not use it while it is attached.  The server does not train it.
 * Errors: EINVAL, ECUDA (pinned staging). */
struct sepso_prior_ctx; /* sepso_prior_handle, below */
int sepso_server_set_prior(sepso_server_handle h, struct sepso_prior_ctx* prior, int32_t n_prior, int32_t first_row);
/* Queue a request (host inputs, copied): T waypoints (<= Tmax), start[2],
 * target[2], circles O x 3 (O <= Omax).  Errors: EINVAL. */
int sepso_server_submit(sepso_server_handle h, int32_t agent, int32_t T, const float* start,
                        const float* target, const float* circles, int32_t O, int64_t tag);
/* As sepso_server_submit for a request that arrives at arrival_s on the server
 * clock (seconds); it is admitted only once the clock has passed it.  Requests
 * must be submitted in arrival order.  Errors: EINVAL. */
int sepso_server_submit_at(sepso_server_handle h, int32_t agent, int32_t T, const float* start,
                           const float* target, const float* circles, int32_t O, int64_t tag,
                           double arrival_s);
/* As sepso_server_submit_at for a request among polygon obstacles (Sec. 3.3.1 map
 * model): edges E x 4 (x0, y0, x1, y1; a closed polygon lists each side once), Q =
 * the number of proper crossings of path segments and edges.  A slot holds at most
 * min(Omax, the float4 records of its circle block rounded down to even) edges (two
 * edges take two float4s).  Polygon requests are served without the learned prior (its
 * raster reads circles): while a prior is attached they are refused, and a prior
 * cannot be attached while polygon requests are queued or in flight.
 * arrival_s < 0: now (as sepso_server_submit).  Errors: EINVAL. */
int sepso_server_submit_polygons(sepso_server_handle h, int32_t agent, int32_t T, const float* start,
                                 const float* target, const float* edges, int32_t E, int64_t tag, double arrival_s);
/* The server clock (s since creation or the last restart); restart != 0 resets it. */
double sepso_server_clock(sepso_server_handle h, int32_t restart);
/* Tick natively until every submitted request (including future arrivals) has
 * finished, waiting for arrivals when the device is idle (at most max_ticks). */
int sepso_server_run(sepso_server_handle h, int64_t max_ticks);
/* One tick: launch one iteration of every occupied slot, collect the requests
 * that finished in the previous tick, admit queued requests into free slots.
 * active / queued (may be NULL): slots occupied and requests waiting after it. */
int sepso_server_tick(sepso_server_handle h, int32_t* active, int32_t* queued);
/* Move up to max_n finished requests to out (and their 2 * Tmax waypoint floats,
 * padded, to waypoints; either may be NULL); n = how many. */
int sepso_server_poll(sepso_server_handle h, sepso_server_done* out, float* waypoints, int32_t max_n,
                      int32_t* n);
/* Tick until nothing is queued or on the device (at most max_ticks; ETIMEOUT). */
int sepso_server_drain(sepso_server_handle h, int64_t max_ticks);
int sepso_server_stats(sepso_server_handle h, int32_t* slots, int64_t* admitted, int64_t* completed,
                       int64_t* ticks, int64_t* launches);
const char* sepso_server_last_error(void);

/* ---- planning without device allocation ---------------------------------- */

/* One planning cycle, like a fresh handle's sepso_plan, for callers that cannot
 * allocate device memory (code running inside another framework's memory pool,
 * plugins whose host forbids allocations after start-up, real-time loops where
 * an allocation may block).  The paper has no counterpart; this is a deployment
 * convenience.
 *
 * The workspace is a static device array inside the library: 8 MiB per GPU that
 * loads libsepso.so, held until the process exits.  The call allocates no device
 * or pinned memory and creates no handle.  Inputs are host pointers (cfg;
 * hyper G x 6; start[2]; target[2]; circles O x 3), copied during the call;
 * outputs are host pointers (waypoints D floats, res; either may be NULL).
 * stream: cudaStream_t (NULL = legacy default stream).  Sync.
 *
 * Limits: cfg->runs must be 1 and the configuration's workspace
 * (sepso_workspace_size) must fit in the 8 MiB, else SEPSO_ENOSPC with a message.
 * Every call starts from zeroed scratch, so no warm-start state (PI, AT window)
 * carries over between calls.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any CUDA
 * stream capture.  All calls on a device share the one array: calls that
 * overlap on the GPU (other threads, other streams) race and corrupt each
 * other; serialise them.
 * Errors: EINVAL, ENOSPC, ERANGE, ECUDA, and device-side errors (ETIMEOUT). */
int sepso_plan_static(const sepso_config* cfg, const float* hyper, const float* start,
                      const float* target, const float* circles, int32_t O, float* waypoints,
                      sepso_result* res, void* stream);

/* ---- learned prior: an MLP proposing a cycle's initial waypoints ---------- */

/* The paper seeds each cycle with Priori Initialization (Sec. 3.3.3): part of each
 * group starts around the previous cycle's best path.  The learned prior is a
 * second seed of that kind: a network maps the scene to a proposed path of T
 * waypoints, and a batch scene with n_prior > 0 starts that many particles per
 * group around it (sepso_batch_set_starts).  The paper has no learned component.
 *
 * Features of a scene (K = g*g + 4 rounded up to a multiple of 8): the g x g
 * occupancy raster of [0, W] x [0, H] (cell (i, j), row i along y, is 1 when its
 * centre ((j + 1/2) W / g, (i + 1/2) H / g) lies in a closed disk; decided in
 * FP32), then start x / W, start y / H, target x / W, target y / H, then zeros.
 * Label of a path (2T values, layout x_0..x_{T-1}, y_0..y_{T-1}): each waypoint's
 * offset from the straight start-target line point at fraction (k + 1) / (T + 1),
 * over the extent.  Network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2),
 * y = W3 h2 + b3 with BF16 weights and activations on the tensor cores (tcgen05,
 * FP32 accumulation) and FP32 master weights; loss (1/2B) sum (y - t)^2; Adam
 * (Kingma and Ba, 2015).  Parameters as one flat FP32 vector: W1 (H1 x K,
 * row-major), b1, W2 (H2 x H1), b2, W3 (2T x H2), b3.
 *
 * The dataset (features, labels, start/target) lives in the workspace: rows
 * [0, capacity).  Calls are ordered on the handle's stream; those marked sync
 * wait for it. */
typedef struct sepso_prior_ctx* sepso_prior_handle;

typedef struct {
  int32_t T;            /* waypoints of a proposal (1..64); 2T outputs            */
  int32_t grid;         /* raster side g (8..256)                                 */
  int32_t hidden1;      /* H1 (multiple of 8)                                     */
  int32_t hidden2;      /* H2 (multiple of 8)                                     */
  int32_t max_batch;    /* rows per step / per inference chunk (multiple of 8)    */
  int32_t capacity;     /* dataset rows                                           */
  int32_t max_circles;  /* circles per scene at most (add_scenes)                 */
  float map_w, map_h;
  float lr, beta1, beta2, eps; /* Adam                                            */
} sepso_prior_config;

/* Bytes of device workspace.  Errors: EINVAL. */
int sepso_prior_workspace_size(const sepso_prior_config* cfg, size_t* bytes);

/* Lay out the prior in the caller's workspace (device, 256-byte aligned, owned by
 * the caller, at least sepso_prior_workspace_size bytes) on the caller's stream
 * (cudaStream_t).  Parameters start at zero.  The handle also owns a second,
 * non-blocking stream and three events (created here, destroyed by
 * sepso_prior_destroy): training forks work onto that stream from the caller's
 * stream and joins it back before each call's work ends on the caller's stream,
 * so the caller sees one ordered stream.  Errors: EINVAL, ENOSPC, ECUDA, ENOMEM. */
int sepso_prior_create(const sepso_prior_config* cfg, void* d_workspace, size_t bytes, void* stream,
                       sepso_prior_handle* out);
void sepso_prior_destroy(sepso_prior_handle h);

/* Length of the flat parameter vector. */
int64_t sepso_prior_num_params(sepso_prior_handle h);

/* Set (host, copied; resets Adam's moments and step count) or read (host, sync)
 * the FP32 parameters.  Errors: EINVAL, ECUDA. */
int sepso_prior_set_params(sepso_prior_handle h, const float* params);
int sepso_prior_get_params(sepso_prior_handle h, float* params);

/* Rasterise n scenes into dataset rows [first, first + n) (host inputs, copied;
 * sync): points n x 4 (start x, y, target x, y), counts n circle counts (each <=
 * max_circles), circles = the scenes' (cx, cy, r) rows back to back, waypoints
 * n x 2T labels' paths or NULL (rows keep their old labels).
 * Errors: EINVAL (range, counts), ECUDA. */
int sepso_prior_add_scenes(sepso_prior_handle h, int32_t first, int32_t n, const float* points,
                           const int32_t* counts, const float* circles, const float* waypoints);

/* Replace the labels of rows [first, first + n) (already added) by the paths in
 * the device array d_waypoints (n rows of stride ld >= 2T), encoded on the
 * device (async).  Errors: EINVAL, ECUDA. */
int sepso_prior_set_labels(sepso_prior_handle h, int32_t first, int32_t n, const float* d_waypoints, int32_t ld);

/* Read dataset rows back (host outputs, sync; either may be NULL): features as
 * FP32 (n x K), labels (n x 2T).  Errors: EINVAL, ECUDA. */
int sepso_prior_get_rows(sepso_prior_handle h, int32_t first, int32_t n, float* features, float* labels);

/* Network outputs y (normalised, n x 2T, host, sync) of rows [first, first + n).
 * Errors: EINVAL, ECUDA, ETIMEOUT. */
int sepso_prior_forward(sepso_prior_handle h, int32_t first, int32_t n, float* y);

/* Loss and its gradient (flat, host, sync) on rows [first, first + n), n a
 * multiple of 8 and <= max_batch; no update.  Errors: EINVAL, ECUDA, ETIMEOUT. */
int sepso_prior_grad(sepso_prior_handle h, int32_t first, int32_t n, float* grad, float* loss);

/* Training: `steps` Adam steps (async unless losses is given).  rows < 0: minibatches of `batch` rows
 * drawn with replacement from dataset rows [0, n_rows) by Philox keyed by seed
 * (counter: the handle's step count); first >= 0: every step uses rows
 * [first, first + batch).  batch: a multiple of 8, <= max_batch.  losses: host
 * array of `steps` (<= 65536) floats, the minibatch loss of each step, filled
 * before the call returns (it then waits for the stream), or NULL.
 * Errors: EINVAL, ECUDA. */
int sepso_prior_train(sepso_prior_handle h, int32_t n_rows, int32_t first, int32_t steps, int32_t batch,
                      uint64_t seed, float* losses);

/* Proposals of rows [first, first + n): waypoints (2T floats per row, the row
 * stride ld >= 2T) written to the device array out on the handle's stream
 * (async).  Errors: EINVAL, ECUDA. */
int sepso_prior_infer(sepso_prior_handle h, int32_t first, int32_t n, float* d_out, int32_t ld);

/* Wait for the handle's stream and return the first device-side error (ETIMEOUT
 * of a tensor-core wait), else OK; clears it. */
int sepso_prior_sync(sepso_prior_handle h);

/* Kernel launches issued so far. */
int64_t sepso_prior_launch_count(sepso_prior_handle h);
const char* sepso_prior_last_error(void);

/* The tensor-core GEMM used by the prior, exposed for testing and benchmarking:
 * C[m][n] = epilogue(alpha * sum_k A[m][k] * B[n][k]) for m < M, n < N, with A
 * (M x K, row stride lda) and B (N x K, row stride ldb) BF16 device arrays, K,
 * lda and ldb multiples of 8, A and B 16-byte aligned.  Epilogue: + bias[n]
 * (device FP32, or NULL), then max(., 0) if relu, then 0 where mask[m][n] (BF16,
 * row stride ldm, or NULL) is not > 0.  Outputs: Cf (FP32, row stride ldcf)
 * and/or Cb (BF16, ldcb), device, either may be NULL.  tile_n: 64, 128 or 256
 * columns per 128-row tile on persistent CTAs (each loops over tiles, the
 * epilogue of one overlapping the main loop of the next), -64 / -128 / -256 the
 * same widths with one tile per CTA, 0 = chosen from the grid it gives.  Async on
 * stream; a device-side timeout is reported by the next sepso_gemm_bf16_sync.
 * Errors: EINVAL, ECUDA. */
int sepso_gemm_bf16(const void* A, const void* B, int32_t M, int32_t N, int32_t K, int32_t lda, int32_t ldb,
                    float alpha, const float* bias, int32_t relu, const void* mask, int32_t ldm, float* Cf,
                    int32_t ldcf, void* Cb, int32_t ldcb, int32_t tile_n, void* stream);
int sepso_gemm_bf16_sync(void* stream);

/* Outputs of sepso_gemm_bf16_ex beyond those of sepso_gemm_bf16 (the backward
 * pass of the learned prior uses all three). */
typedef struct {
  void* Ct;               /* BF16 copy of the output transposed, Ct[n * ldct + m] (device), or NULL */
  int32_t ldct;           /* >= M */
  float* colsum;          /* colsum[n] = sum over m of the output (device FP32, N floats), or NULL;
                             summed per 32-row slab in row order, then over the slabs in order */
  int32_t ksplit;         /* 0 or 1: one pass over K.  S > 1: K in S slices of whole 64-deep blocks
                             (fewer when K has fewer blocks), one CTA per tile and slice, the slices'
                             FP32 products summed in slice order before the epilogue; Cf/Cb only */
  void* workspace;        /* device scratch, 16-byte aligned, caller-owned: */
  size_t workspace_bytes; /* >= sepso_gemm_bf16_ex_workspace(M, N, ksplit, colsum != NULL) */
} sepso_gemm_extra;

/* Scratch bytes sepso_gemm_bf16_ex needs: S M N 4 for a K split in S slices,
 * else ceil(M / 32) N 4 with column sums, else 0.  Errors: EINVAL. */
int sepso_gemm_bf16_ex_workspace(int32_t M, int32_t N, int32_t ksplit, int32_t colsum, size_t* bytes);

/* sepso_gemm_bf16 with the outputs of `extra` (NULL: none).  The epilogue's
 * values (after bias, ReLU and mask) are what Ct and colsum receive.  A K split
 * uses the one-tile-per-CTA kernel with width |tile_n| (0: 128) and a second
 * launch for the sum and the epilogue.  Errors: EINVAL (also a K split with Ct
 * or colsum), ENOSPC (workspace), ECUDA. */
int sepso_gemm_bf16_ex(const void* A, const void* B, int32_t M, int32_t N, int32_t K, int32_t lda, int32_t ldb,
                       float alpha, const float* bias, int32_t relu, const void* mask, int32_t ldm, float* Cf,
                       int32_t ldcf, void* Cb, int32_t ldcb, const sepso_gemm_extra* extra, int32_t tile_n,
                       void* stream);

/* ---- misc --------------------------------------------------------------- */

/* Wait for the handle's stream; returns the first device-side error of any run
 * (e.g. SEPSO_ETIMEOUT), else SEPSO_OK, and clears it. */
int sepso_sync(sepso_handle h);

/* Launch shape chosen at create, of the form the next plan or step launches
 * (see sepso_exchange_form): CTAs per group, threads, circle split (1 in the
 * cluster form: each lane tests whole obstacles), grid. */
int sepso_launch_shape(sepso_handle h, int32_t* ctas_per_group, int32_t* threads,
                       int32_t* circle_split, int32_t* grid);

/* The form of the exchange the next plan or step launches: 2 = one thread-block
 * cluster per group (exchange 0, 2 or 3, every group's C3 is 0 and the cluster
 * form fits), 1 = the grid-wide barrier.  Negative on a bad handle. */
int sepso_exchange_form(sepso_handle h);

/* Cumulative counters of run `run` (host outputs, sync): planning cycles
 * finished and iterations of Algorithm 1 executed (plans and steps). */
int sepso_counters(sepso_handle h, int32_t run, int64_t* plans, int64_t* iterations);

/* Number of kernel launches this handle has issued so far. */
int64_t sepso_launch_count(sepso_handle h);

const char* sepso_strerror(int code);
const char* sepso_last_error(void);

/* ------------------------------------------------------------------------- */
/* Benchmark functions (Table BFs; Secs. 4.1.1 and 4.1.2): DTPSO with the     */
/* objective BF1 Sphere, BF2 Rosenbrock, BF3 Rastrigin or BF4 Griewank over   */
/* the box [lo, hi]^D.  The iteration is the planner's (Algorithm 1: fitness, */
/* Pbest/Gbest/Tbest with the strictly-better rule and lowest-index ties,     */
/* Eq. TOF_omega over max_iters, Eq. TOF_V with C3 and clipping to            */
/* V_range = V_limit (hi - lo), Eq. TOF_X clipped to the box); no PI, no AT.  */
/* Textbook definitions, index i = 1..D:                                      */
/*   BF1 sum x_i^2;  BF2 sum_{i<D} 100 (x_{i+1} - x_i^2)^2 + (x_i - 1)^2;     */
/*   BF3 10 D + sum x_i^2 - 10 cos(2 pi x_i);                                  */
/*   BF4 1 + sum x_i^2 / 4000 - prod cos(x_i / sqrt i).                        */
/* ------------------------------------------------------------------------- */
typedef struct sepso_bf_config {
  int32_t fn;         /* 1..4: BF1..BF4; 5: a path among polygons; 6: a 3D path */
                      /* among spheres (both below)                             */
  int32_t D;          /* coordinates per particle, 1..16384                     */
  int32_t G;          /* groups, 1..32                                          */
  int32_t N;          /* particles per group (G x N + G + 1 < 2^30)             */
  float lo, hi;       /* X_range per coordinate, lo < hi, finite                */
  int32_t max_iters;  /* iterations of sepso_bf_run_async; T of Eq. TOF_omega   */
  int32_t runs;       /* independent swarms (trials); runs x G <= 4096          */
  uint64_t seed;      /* Philox key                                             */
  uint32_t run_id;    /* Philox counter word 3 of run 0; run r uses run_id + r  */
  /* objective 5 only (lo and hi are then unused): D = 2T waypoint coordinates,  */
  /* x in [0, map_w], y in [0, map_h]; fitness = Eq. lenth + alpha * Q^beta     */
  float map_w, map_h; /* > 0                                                     */
  float alpha;        /* >= 0                                                    */
  int32_t beta;       /* 1..8                                                    */
  int32_t max_edges;  /* capacity for obstacle edges, 0..4096                    */
  /* objective 6 only (the Conclusion's extension from 2D to 3D planning): D = 3T */
  /* coordinates [x1..xT, y1..yT, z1..zT], x in [0, map_w], y in [0, map_h], z   */
  /* in [0, map_d]; fitness = 3D length + alpha * Q^beta (alpha, beta as above)  */
  float map_d;        /* > 0                                                     */
  int32_t max_spheres; /* capacity for spheres, 0..4096                          */
  /* objectives 5 and 6: Auto Truncation (Sec. 3.3.4, stall-counter reading): a   */
  /* run stops after at_stall iterations in which its Tbest fitness did not drop  */
  /* by more than stall_tol while its Tbest path collides with nothing; it then   */
  /* keeps Tbest of the stopping iteration and moves no particle after it (a      */
  /* loaded state counts as colliding until a particle of the swarm holds Tbest). */
  /* 0 = off (max_iters iterations).                                              */
  int32_t at_stall;   /* >= 0                                                    */
  float stall_tol;    /* >= 0, finite                                            */
} sepso_bf_config;

typedef struct sepso_bf_ctx* sepso_bf_handle;

/* Device workspace for a configuration: about runs x G x N x D x 20 bytes (X, V
 * and two Pbest buffers, FP32) plus small tables.  Errors: EINVAL. */
int sepso_bf_workspace_size(const sepso_bf_config* c, size_t* bytes);
/* Create a handle on a caller-owned device workspace (256-byte aligned, at least
 * sepso_bf_workspace_size bytes; cleared here) and stream.  The caller keeps both
 * alive until sepso_bf_destroy.  Errors: EINVAL, ENOSPC (size or alignment),
 * ERANGE (the iteration kernel does not fit an SM), ECUDA, ENOMEM. */
int sepso_bf_create(const sepso_bf_config* c, void* workspace, size_t bytes, void* stream, sepso_bf_handle* out);
int sepso_bf_destroy(sepso_bf_handle h);
/* hyper: host G x 6 rows (C1, C2, C3, w_init, w_end, V_limit), Table hyper8
 * layout, for one run or (run = -1) for every run; finite, V_limit >= 0.  Syncs
 * the stream.  Errors: EINVAL, ECUDA. */
int sepso_bf_set_hyper(sepso_bf_handle h, const float* hyper, int32_t run);
/* One whole run of every swarm on the stream: initialisation (X uniform over the
 * box, V uniform in +-V_range; Philox streams as the planner's), max_iters
 * iterations, then the bests.  use_graph != 0 captures the launches once into a
 * CUDA graph and replays it.  Errors: ESTATE (no hyper-parameters), ECUDA. */
int sepso_bf_run_async(sepso_bf_handle h, int32_t use_graph);
/* Objective 5 (Sec. 3.3.1 map model): obstacles are polygons given by their edges
 * (host float[E*4]: x0, y0, x1, y1; a closed polygon lists each side once, convex
 * or not), start and target host float[2].  Q = the number of (path segment,
 * edge) pairs that cross properly (the endpoints of each strictly on opposite
 * sides of the other; touching and collinear contacts do not count).  Required
 * before sepso_bf_run_async; a new edge count re-captures the graph.  Syncs.
 * Errors: EINVAL (objective, E > max_edges, non-finite values), ECUDA. */
int sepso_bf_set_polygons(sepso_bf_handle h, const float* start, const float* target, const float* edges,
                          int32_t E);
/* Objective 5 of n paths X (device, row pitch ldx >= 2T floats: x of the T
 * waypoints, then y) among E device edges (float4 x0, y0, x1, y1; 16-byte
 * aligned): fitness into device F[n] and, if Q is not NULL, the crossing counts
 * into device Q[n].  start/target: host float[2].  On stream.
 * Errors: EINVAL, ECUDA. */
int sepso_poly_evaluate(int32_t T, int32_t n, const float* X, int32_t ldx, const float* start, const float* target,
                        const float* edges, int32_t E, float alpha, int32_t beta, float* F, int32_t* Q,
                        void* stream);
/* Objective 6, a path in three dimensions among spheres (the paper's Conclusion
 * names the extension from 2D to 3D planning as future work; this is Eqs.
 * path_fit, lenth and penalty with a third coordinate).  spheres: host
 * float[S*4] (cx, cy, cz, r; r >= 0), start and target host float[3].  Q = the
 * number of (path segment, sphere) pairs whose distance is below the radius (the
 * circles' rule of Sec. 3.3.2 in 3D; a segment inside a sphere counts).  Required
 * before sepso_bf_run_async; a new sphere count re-captures the graph.  Syncs.
 * Errors: EINVAL (objective, S > max_spheres, non-finite values, negative radius),
 * ECUDA. */
int sepso_bf_set_spheres(sepso_bf_handle h, const float* start, const float* target, const float* spheres,
                         int32_t S);
/* Priori Initialization for the path objectives 5 and 6 (Sec. 3.3.3): the next
 * run initialises the first ceil(pi_gamma N) particles of each group (computed in
 * double precision) around that run's previous best path, X = clip(prevT +
 * (2u - 1) pi_h) with u from the PI stream, and every Philox counter of the run
 * carries `cycle` (the planning cycle, < 2^24) as the planner's do.  prevT: host
 * float[runs*D], one previous path per run, or NULL with pi_gamma = 0 (a cold start
 * that still sets the cycle).  The values live in the workspace, so a captured
 * run graph stays valid.  Syncs.  Errors: EINVAL (objective, gamma outside [0, 1],
 * negative or non-finite pi_h, non-finite prevT, cycle too large), ECUDA. */
int sepso_bf_set_warm_start(sepso_bf_handle h, const float* prevT, float pi_gamma, float pi_h, uint32_t cycle);
/* Objective 6 of n paths X (device, row pitch ldx >= 3T floats: x of the T
 * waypoints, then y, then z) among S device spheres (float4 cx, cy, cz, r;
 * 16-byte aligned): fitness into device F[n] and, if Q is not NULL, the collision
 * counts into device Q[n].  start/target: host float[3].  On stream.
 * Errors: EINVAL, ECUDA. */
int sepso_sphere_evaluate(int32_t T, int32_t n, const float* X, int32_t ldx, const float* start, const float* target,
                          const float* spheres, int32_t S, float alpha, int32_t beta, float* F, int32_t* Q,
                          void* stream);
/* Continue every swarm for iters more iterations (after a run or a loaded state). */
int sepso_bf_step(sepso_bf_handle h, int32_t iters);
int sepso_bf_sync(sepso_bf_handle h);
/* Tbest of a run: best_x host float[D] (or NULL), best_fit host float (or NULL),
 * iterations done (with Auto Truncation, the run's stopping iteration if it
 * stopped).  Syncs the stream.  Errors: EINVAL, ESTATE, ECUDA. */
int sepso_bf_read(sepso_bf_handle h, int32_t run, float* best_x, float* best_fit, int32_t* iters);
/* Tbest fitness after each of the first max_iters iterations: host float[max_iters]. */
int sepso_bf_history(sepso_bf_handle h, int32_t run, float* hist);
/* Swarm state of one run in host arrays (any may be NULL): X, V, P float[G*N*D]
 * (particle-major), Pfit float[G*N], Gb float[G*D], Gfit float[G], Tb float[D],
 * Tfit float[1], k = iterations done.  Syncs.  Errors: EINVAL, ESTATE, ECUDA. */
int sepso_bf_get_state(sepso_bf_handle h, int32_t run, float* X, float* V, float* P, float* Pfit, float* Gb,
                       float* Gfit, float* Tb, float* Tfit, int32_t* k);
/* Load the same arrays (all required; X, V, P finite, no NaN fitness) as the state
 * after k iterations; with several runs, k must match theirs.  The next step
 * continues with iteration k + 1.  Syncs.  Errors: EINVAL, ECUDA. */
int sepso_bf_set_state(sepso_bf_handle h, int32_t run, const float* X, const float* V, const float* P,
                       const float* Pfit, const float* Gb, const float* Gfit, const float* Tb, const float* Tfit,
                       int32_t k);
/* Fitness of n rows of a device array X (row pitch ldx >= D floats) into device
 * F[n], on stream.  Errors: EINVAL, ECUDA. */
int sepso_bf_evaluate(int32_t fn, int32_t D, int32_t n, const float* X, int32_t ldx, float* F, void* stream);
int64_t sepso_bf_launch_count(sepso_bf_handle h);
/* Name of the kernels this handle launches: bf_iter_kernel<fn> (a launch per
 * iteration, a warp per particle); poly_lane_kernel or sphere_lane_kernel
 * (objective 5 or 6, D <= 64, at least 256 particles per SM: a lane per
 * particle); or, for benchmark-function
 * swarms of at most 8192 coordinates (G x N x D), bf_small_kernel for whole runs
 * (one CTA per run, the swarm in shared memory) with bf_iter_kernel for steps.
 * Static string. */
const char* sepso_bf_kernel_name(sepso_bf_handle h);
const char* sepso_bf_last_error(void);

/* The planner's random numbers on their own, for checking: Philox4x32-10 (Salmon,
 * Moraes, Dror and Shaw, SC'11: ten rounds of the two multipliers 0xD2511F53 and
 * 0xCD9E8D57 with the Weyl key increments 0x9E3779B9 and 0xBB67AE85) of n counters
 * under the key (seed low word, seed high word), computed on the device by the
 * function the kernels draw with.  The planner's counters are (iteration or
 * coordinate chunk, particle, stream << 24 | cycle, run); its uniforms are
 * (word >> 8) 2^-24, and R1, R2, R3 of Eq. TOF_V are words 0, 1, 2 of counter
 * (k, g N + n, 0 << 24 | cycle, run).  ctr, out: device uint32[n][4] (16-byte
 * aligned, caller-owned; they may not overlap).  Async on stream; allocates nothing.
 * Errors: EINVAL (n < 0, NULL or misaligned arrays), ECUDA. */
int sepso_philox(const uint32_t* ctr, int64_t n, uint64_t seed, uint32_t* out, void* stream);

/* Auto Truncation window criterion (Sec. 3.3.4, first criterion) on its own, for
 * checking: for each of `count` windows, whether the population standard deviation
 * of the ns[i] newest entries of the ring win[i*tw .. i*tw+tw) (head heads[i], the
 * slot the next entry would take; entries oldest first at (head - n + j) mod tw)
 * is below delta, as a two-pass FP64 computation decides it.  Evaluated on the
 * device by the code sepso_plan runs (an FP32 warp pass with a rounding-error
 * bound, FP64 sums near the threshold or for entries that are not FP32 values).
 * win: host double[count*tw]; ns, heads: host int32[count] with 1 <= ns[i] <= tw,
 * 0 <= heads[i] < tw; tw in [1, 64]; out: host int32[count] gets 1 (below) or 0.
 * delta <= 0 or NaN gives 0.  Allocates and frees a device buffer; syncs stream.
 * Errors: EINVAL (counts, ranges, null pointers), ECUDA. */
int sepso_at_window_test(const double* win, const int32_t* ns, const int32_t* heads, int32_t count,
                         int32_t tw, float delta, int32_t* out, void* stream);

/* Watchdog self-test (failure detection without a fault): one kernel runs the two
 * kinds of bounded wait the library's kernels use -- an mbarrier that no copy
 * completes, and the inter-CTA counter that no CTA increments -- with a limit of
 * limit_us microseconds (1..1e6) instead of 2 s.  Both give up, the kernel
 * returns normally and *fired gets bit 0 (mbarrier) and bit 1 (counter) set, so a
 * healthy build reports 3 and leaves the context usable.  The paper has no
 * counterpart.  Sync on stream.  Errors: EINVAL, ECUDA. */
int sepso_watchdog_selftest(int32_t limit_us, int32_t* fired, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SEPSO_H */
