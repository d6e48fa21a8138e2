/*
 * sepso_oracle.c -- plain, slow, FP64 CPU oracle for the SEPSO planner's hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load this library.  The product path (the CUDA
 * library under paper_2308_10169_gb300/) never calls it and shares no code,
 * header, table or constant generator with it.
 *
 * Paper: J. Xin, Z. Li, Y. Zhang, N. Li, "Efficient Real-time Path Planning with
 * Self-evolving Particle Swarm Optimization in Dynamic Scenarios" (arXiv 2308.10169).
 *
 * Everything here is scalar double precision, written as the paper states it,
 * with no blocking, fusion or reordering:
 *   - Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11),
 *     written from its published definition; it supplies R1, R2, R3 (Table
 *     EXP_TOF: one scalar per particle per iteration) and the initial draws.
 *   - Path fitness, Eqs. path_fit / lenth / penalty (Sec. 3.3.2), with the
 *     collision count Q over circular obstacles (reading: a (segment, circle)
 *     pair counts once when the segment passes strictly inside the disk).
 *   - One DTPSO iteration, Algorithm 1 with Eqs. TOF_omega / TOF_V / TOF_X
 *     (Sec. 3.1), equal to Eqs. DPPSO_V / DPPSO_X with the per-group omega.
 *   - Priori Initialization (Sec. 3.3.3) and Auto Truncation (Sec. 3.3.4).
 *   - The hierarchical self-evolving framework (Sec. 3.2.1, Eq. fit_h).
 *   - The dynamic scene step of the simulator (Fig. PP caption: obstacles
 *     reverse velocity at the map border; start/target move vertically).
 *   - The paper's stated extension from 2D to 3D planning (Conclusion, item
 *     (iii)): the same fitness for a path of T waypoints in a box among
 *     spheres, Q counting the (segment, sphere) pairs closer than the radius.
 *
 * Compile with -ffp-contract=off so that x86 and Arm give identical results.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11, "Parallel random numbers: as easy as  */
/* 1, 2, 3").  Ten rounds of the 4x32 S-P network; each round multiplies     */
/* counter words 0 and 2 by the two published multipliers, swaps the words   */
/* and xors the key in; the key is bumped by the two Weyl constants between  */
/* rounds.                                                                   */
/* ------------------------------------------------------------------------- */
#define SO_PHILOX_M0 0xD2511F53u
#define SO_PHILOX_M1 0xCD9E8D57u
#define SO_PHILOX_W0 0x9E3779B9u
#define SO_PHILOX_W1 0xBB67AE85u

/* Random stream identifiers, carried in the top byte of counter word 2. */
enum { SO_STREAM_VEL = 0, SO_STREAM_INIT_X = 1, SO_STREAM_INIT_V = 2, SO_STREAM_PI = 3,
       SO_STREAM_PRIOR = 4, SO_STREAM_H_INIT_X = 5, SO_STREAM_H_INIT_V = 6, SO_STREAM_H_VEL = 7 };

void so_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += SO_PHILOX_W0;
      k1 += SO_PHILOX_W1;
    }
    uint64_t prod0 = (uint64_t)SO_PHILOX_M0 * (uint64_t)x0;
    uint64_t prod1 = (uint64_t)SO_PHILOX_M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Batch form for tests: n counters (n x 4 words) under one 64-bit key. */
void so_philox_batch(int32_t n, const uint32_t* ctr, uint64_t seed, uint32_t* out) {
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  for (int32_t i = 0; i < n; ++i) so_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* Uniform on [0,1): the top 24 bits of a word, times 2^-24 (exact in FP32 too). */
double so_u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

/* Draw the four uniforms of counter (c0, p, stream|cycle, run). */
static void so_draw4(uint64_t seed, uint32_t c0, uint32_t p, uint32_t stream, uint32_t cycle,
                     uint32_t run, double u[4]) {
  uint32_t ctr[4] = {c0, p, (stream << 24) | (cycle & 0x00ffffffu), run};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t o[4];
  so_philox4x32_10(ctr, key, o);
  for (int i = 0; i < 4; ++i) u[i] = so_u01(o[i]);
}

/* ------------------------------------------------------------------------- */
/* Configuration, scene and state.                                           */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t T, G, N;       /* waypoints (D = 2T), groups, particles per group   */
  double W, H;           /* map: x in [0,W], y in [0,H] (X_range)            */
  double alpha;          /* Eq. penalty: alpha * Q^beta                       */
  int32_t beta;
  int32_t max_iters;     /* iteration cap, also the T of Eq. TOF_omega        */
  int32_t at_mode;       /* 0 off, 1 std window (Sec. 3.3.4), 2 stall counter */
  int32_t tw;            /* truncation window TW                              */
  double delta;          /* std threshold                                     */
  int32_t stall_iters;   /* stall-counter limit                               */
  double stall_tol;
  int32_t use_pi;        /* Priori Initialization on/off                      */
  double pi_gamma;       /* fraction of each group initialised by PI          */
  double pi_h;           /* half-width of the PI interval                     */
  uint64_t seed;         /* Philox key                                        */
  uint32_t run_id;       /* Philox counter word 3                             */
  /* The objective: 0 = path planning among circles (Sec. 3.3: D = 2T waypoint
   * coordinates in the map); 1..4 = benchmark functions BF1..BF4 (Table BFs:
   * Sphere, Rosenbrock, Rastrigin, Griewank) over the box [lo, hi]^D, D = Dbf;
   * 5 = path planning among polygons (Sec. 3.3.1: Q counts crossings of path
   * segments with obstacle edges); 6 = path planning in three dimensions among
   * spheres (the 3D extension of the Conclusion: D = 3T coordinates
   * [x1..xT, y1..yT, z1..zT] in [0,W] x [0,H] x [0,Z]).                     */
  int32_t problem;
  int32_t Dbf;
  double lo, hi;
  double Z;              /* problem 6: depth of the box (z in [0,Z])          */
} so_config;

typedef struct {
  double sx, sy, tx, ty; /* start and target                                 */
  int32_t O;             /* number of circles                                 */
  const double* circ;    /* O x 3: cx, cy, r                                  */
  int32_t E;             /* polygon edges (problem 5)                         */
  const double* edges;   /* E x 4: x0, y0, x1, y1                             */
  /* Other agents sharing the scene (multi-agent extension): A timed paths of
   * T + 2 points each, A x (2 (T + 2)): x_0..x_{T+1}, then y_0..y_{T+1} (their
   * start, their T waypoints, their target), and the separation below which two
   * agents conflict. */
  int32_t A;
  const double* agents;
  double sep;
  /* Problem 6: the z of start and target, and S spheres (S x 4: cx, cy, cz, r). */
  double sz, tz;
  int32_t S;
  const double* spheres;
} so_scene;

typedef struct {
  double *X, *V, *P, *Pfit;   /* (G*N*D), (G*N*D), (G*N*D), (G*N)             */
  int32_t *PQ;                /* (G*N) collision count of each Pbest          */
  double *Gb, *Gfit;          /* (G*D), (G)                                   */
  int32_t *GQ;                /* (G)                                          */
  double *Tb, *Tfit;          /* (D), (1)                                     */
  int32_t *TQ, *k;            /* (1), (1)                                     */
  /* state carried from one planning cycle to the next */
  int32_t *cycle, *has_prev;  /* (1), (1)                                     */
  double *prevT;              /* (D) previous cycle's Tbest, centre of PI     */
  double *win;                /* (TW) LFV ring buffer for AT mode 1           */
  int32_t *win_n, *win_head;  /* (1), (1)                                     */
  int32_t *stall;             /* (1) stall counter for AT mode 2              */
  double *prev_lfv;           /* (1)                                          */
  /* optional second seed of the initialisation (a learned prior's proposal) */
  int32_t *n_prior;           /* (1) particles per group around priorT, or NULL */
  double *priorT;             /* (D) or NULL                                  */
} so_state;

/* ------------------------------------------------------------------------- */
/* Fitness, Sec. 3.3.2.                                                      */
/* ------------------------------------------------------------------------- */

/* Euclidean distance from point c to the closed segment [a, b]: the closest
 * point is a + t (b - a) with t the projection parameter clamped to [0, 1]. */
double so_seg_point_dist(double ax, double ay, double bx, double by, double cx, double cy) {
  double dx = bx - ax, dy = by - ay;
  double L2 = dx * dx + dy * dy;
  double t = 0.0;
  if (L2 > 0.0) {
    t = ((cx - ax) * dx + (cy - ay) * dy) / L2;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
  }
  double px = ax + t * dx - cx, py = ay + t * dy - cy;
  return sqrt(px * px + py * py);
}

static double so_pow_int(double q, int32_t beta) {
  double r = 1.0;
  for (int32_t i = 0; i < beta; ++i) r *= q;
  return r;
}

/* Eq. lenth: the internal segments d = 2..D/2, then start->w1, then wT->target.
 * X rows follow Eq. coordinate: [x1..xT, y1..yT]. */
static double so_length(int32_t T, const double* x, double sx, double sy, double tx, double ty) {
  double len = 0.0;
  for (int32_t d = 1; d < T; ++d) {
    double ddx = x[d] - x[d - 1], ddy = x[T + d] - x[T + d - 1];
    len += sqrt(ddx * ddx + ddy * ddy);
  }
  len += sqrt((sx - x[0]) * (sx - x[0]) + (sy - x[T]) * (sy - x[T]));
  len += sqrt((tx - x[T - 1]) * (tx - x[T - 1]) + (ty - x[2 * T - 1]) * (ty - x[2 * T - 1]));
  return len;
}

/* Orientation of r relative to the directed line p -> q (twice the signed area). */
static double so_orient(double px, double py, double qx, double qy, double rx, double ry) {
  return (qx - px) * (ry - py) - (qy - py) * (rx - px);
}

/* Segments ab and cd cross properly: c and d strictly on opposite sides of line
 * ab, and a and b strictly on opposite sides of line cd (touching and collinear
 * contacts are not crossings). */
int32_t so_seg_cross(double ax, double ay, double bx, double by, double cx, double cy, double dx, double dy) {
  const double o1 = so_orient(ax, ay, bx, by, cx, cy), o2 = so_orient(ax, ay, bx, by, dx, dy);
  const double o3 = so_orient(cx, cy, dx, dy, ax, ay), o4 = so_orient(cx, cy, dx, dy, bx, by);
  return (o1 * o2 < 0.0) && (o3 * o4 < 0.0);
}

/* Q among polygons (Sec. 3.3.1, Eq. penalty): the number of (path segment,
 * obstacle edge) pairs that cross. */
static int32_t so_poly_crossings(int32_t T, const double* x, const so_scene* sc) {
  int32_t q = 0;
  for (int32_t s = 0; s <= T; ++s) {
    const double ax = (s == 0) ? sc->sx : x[s - 1];
    const double ay = (s == 0) ? sc->sy : x[T + s - 1];
    const double bx = (s == T) ? sc->tx : x[s];
    const double by = (s == T) ? sc->ty : x[T + s];
    for (int32_t e = 0; e < sc->E; ++e) {
      const double* d = sc->edges + 4 * e;
      q += so_seg_cross(ax, ay, bx, by, d[0], d[1], d[2], d[3]);
    }
  }
  return q;
}

/* For the parity tests: per particle, how far its crossing decisions are from
 * flipping -- the smallest |orientation| / (|ab| |cd|) over the pairs whose result
 * hangs on a near-zero orientation (a pair decided by a clear "no" of the other
 * side test, at 1e-3, does not count). */
void so_poly_margin(const so_config* cfg, const so_scene* sc, int32_t n, const double* X, double* margin) {
  const int32_t T = cfg->T, D = 2 * T;
  for (int32_t p = 0; p < n; ++p) {
    const double* x = X + (int64_t)p * D;
    double m = INFINITY;
    for (int32_t s = 0; s <= T; ++s) {
      const double ax = (s == 0) ? sc->sx : x[s - 1];
      const double ay = (s == 0) ? sc->sy : x[T + s - 1];
      const double bx = (s == T) ? sc->tx : x[s];
      const double by = (s == T) ? sc->ty : x[T + s];
      for (int32_t e = 0; e < sc->E; ++e) {
        const double* d = sc->edges + 4 * e;
        const double L = sqrt((bx - ax) * (bx - ax) + (by - ay) * (by - ay)) *
                         sqrt((d[2] - d[0]) * (d[2] - d[0]) + (d[3] - d[1]) * (d[3] - d[1]));
        if (!(L > 0.0)) {
          m = 0.0;
          continue;
        }
        const double o1 = so_orient(ax, ay, bx, by, d[0], d[1]), o2 = so_orient(ax, ay, bx, by, d[2], d[3]);
        const double o3 = so_orient(d[0], d[1], d[2], d[3], ax, ay), o4 = so_orient(d[0], d[1], d[2], d[3], bx, by);
        const double m12 = fmin(fabs(o1), fabs(o2)) / L, m34 = fmin(fabs(o3), fabs(o4)) / L;
        if ((m12 >= 1e-3 && o1 * o2 > 0.0) || (m34 >= 1e-3 && o3 * o4 > 0.0)) continue;
        m = fmin(m, fmin(m12, m34));
      }
    }
    margin[p] = m;
  }
}

/* Conflicts with the other agents of the scene (the multi-agent extension the
 * paper names as future work): all agents leave their starts together and reach
 * one point of their path per time step (start, T waypoints, target), moving
 * straight in between.  During step s the position of this path relative to agent
 * b's moves on a straight line, so their closest approach in that step is the
 * distance of the origin to the segment rel(s) -> rel(s + 1), rel = own point -
 * b's point; each (agent, step) with a closest approach below sep is one conflict,
 * added to Q of Eq. penalty. */
static int32_t so_agent_conflicts(int32_t T, const double* x, const so_scene* sc) {
  int32_t q = 0;
  const int32_t P = T + 2;
  for (int32_t b = 0; b < sc->A; ++b) {
    const double* w = sc->agents + (int64_t)b * 2 * P;
    for (int32_t s = 0; s <= T; ++s) {
      const double ax = (s == 0) ? sc->sx : x[s - 1];
      const double ay = (s == 0) ? sc->sy : x[T + s - 1];
      const double bx = (s == T) ? sc->tx : x[s];
      const double by = (s == T) ? sc->ty : x[T + s];
      const double r0x = ax - w[s], r0y = ay - w[P + s];
      const double r1x = bx - w[s + 1], r1y = by - w[P + s + 1];
      if (so_seg_point_dist(r0x, r0y, r1x, r1y, 0.0, 0.0) < sc->sep) ++q;
    }
  }
  return q;
}

/* Q: number of (path segment, circle) pairs whose distance is below the radius. */
static int32_t so_collisions(int32_t T, const double* x, const so_scene* sc) {
  int32_t q = 0;
  for (int32_t s = 0; s <= T; ++s) {
    double ax = (s == 0) ? sc->sx : x[s - 1];
    double ay = (s == 0) ? sc->sy : x[T + s - 1];
    double bx = (s == T) ? sc->tx : x[s];
    double by = (s == T) ? sc->ty : x[T + s];
    for (int32_t o = 0; o < sc->O; ++o) {
      const double* c = sc->circ + 3 * o;
      if (so_seg_point_dist(ax, ay, bx, by, c[0], c[1]) < c[2]) ++q;
    }
  }
  return q;
}

/* For the parity tests: per particle, the smallest |dist - r| over all of its
 * (segment, circle) pairs; pairs this close to tangency may flip in FP32. */
void so_tangency_margin(const so_config* cfg, const so_scene* sc, int32_t n, const double* X,
                        double* margin) {
  const int32_t T = cfg->T, D = 2 * T;
  for (int32_t p = 0; p < n; ++p) {
    const double* x = X + (int64_t)p * D;
    double m = INFINITY;
    for (int32_t s = 0; s <= T; ++s) {
      double ax = (s == 0) ? sc->sx : x[s - 1];
      double ay = (s == 0) ? sc->sy : x[T + s - 1];
      double bx = (s == T) ? sc->tx : x[s];
      double by = (s == T) ? sc->ty : x[T + s];
      for (int32_t o = 0; o < sc->O; ++o) {
        const double* c = sc->circ + 3 * o;
        double d = fabs(so_seg_point_dist(ax, ay, bx, by, c[0], c[1]) - c[2]);
        if (d < m) m = d;
      }
    }
    margin[p] = m;
  }
}


/* ------------------------------------------------------------------------- */
/* Three dimensions (the Conclusion's extension from 2D to 3D planning): the */
/* fitness of Eqs. path_fit / lenth / penalty for a path start -> T          */
/* waypoints -> target in a box, with spheres as obstacles.  A row holds     */
/* [x1..xT, y1..yT, z1..zT].                                                 */
/* ------------------------------------------------------------------------- */

/* Euclidean distance from point c to the closed segment [a, b] in 3D: the
 * closest point is a + t (b - a), t the projection parameter clamped to [0, 1]
 * (t = 0 for a zero-length segment). */
double so_seg_point_dist3(const double* a, const double* b, const double* c) {
  const double dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
  const double L2 = dx * dx + dy * dy + dz * dz;
  double t = 0.0;
  if (L2 > 0.0) {
    t = ((c[0] - a[0]) * dx + (c[1] - a[1]) * dy + (c[2] - a[2]) * dz) / L2;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
  }
  const double px = a[0] + t * dx - c[0], py = a[1] + t * dy - c[1], pz = a[2] + t * dz - c[2];
  return sqrt(px * px + py * py + pz * pz);
}

/* Point s of the path (s = 0: start, 1..T: waypoint s, T + 1: target). */
static void so_point3(int32_t T, const double* x, const so_scene* sc, int32_t s, double* out) {
  if (s == 0) {
    out[0] = sc->sx;
    out[1] = sc->sy;
    out[2] = sc->sz;
  } else if (s == T + 1) {
    out[0] = sc->tx;
    out[1] = sc->ty;
    out[2] = sc->tz;
  } else {
    out[0] = x[s - 1];
    out[1] = x[T + s - 1];
    out[2] = x[2 * T + s - 1];
  }
}

/* Eq. lenth in 3D: the T + 1 segment lengths in path order. */
static double so_length3(int32_t T, const double* x, const so_scene* sc) {
  double len = 0.0;
  for (int32_t s = 0; s <= T; ++s) {
    double a[3], b[3];
    so_point3(T, x, sc, s, a);
    so_point3(T, x, sc, s + 1, b);
    len += sqrt((b[0] - a[0]) * (b[0] - a[0]) + (b[1] - a[1]) * (b[1] - a[1]) + (b[2] - a[2]) * (b[2] - a[2]));
  }
  return len;
}

/* Q in 3D: the number of (path segment, sphere) pairs whose distance is below
 * the radius (the circles' reading with a third coordinate). */
static int32_t so_sphere_collisions(int32_t T, const double* x, const so_scene* sc) {
  int32_t q = 0;
  for (int32_t s = 0; s <= T; ++s) {
    double a[3], b[3];
    so_point3(T, x, sc, s, a);
    so_point3(T, x, sc, s + 1, b);
    for (int32_t o = 0; o < sc->S; ++o) {
      const double* c = sc->spheres + 4 * o;
      if (so_seg_point_dist3(a, b, c) < c[3]) ++q;
    }
  }
  return q;
}

/* For the parity tests: per path, the smallest |dist - r| over its (segment,
 * sphere) pairs; pairs this close to tangency may flip in FP32. */
void so_sphere_margin(const so_config* cfg, const so_scene* sc, int32_t n, const double* X, double* margin) {
  const int32_t T = cfg->T, D = 3 * T;
  for (int32_t p = 0; p < n; ++p) {
    const double* x = X + (int64_t)p * D;
    double m = INFINITY;
    for (int32_t s = 0; s <= T; ++s) {
      double a[3], b[3];
      so_point3(T, x, sc, s, a);
      so_point3(T, x, sc, s + 1, b);
      for (int32_t o = 0; o < sc->S; ++o) {
        const double* c = sc->spheres + 4 * o;
        const double d = fabs(so_seg_point_dist3(a, b, c) - c[3]);
        if (d < m) m = d;
      }
    }
    margin[p] = m;
  }
}

/* Eq. path_fit = Length + alpha * Q^beta for n particles (rows of X). */
/* ------------------------------------------------------------------------- */
/* Benchmark functions BF1-BF4 (Table BFs), their textbook definitions with  */
/* 1-based coordinate index i = 1..D:                                        */
/*   Sphere      sum x_i^2                                                   */
/*   Rosenbrock  sum_{i<D} 100 (x_{i+1} - x_i^2)^2 + (x_i - 1)^2             */
/*   Rastrigin   10 D + sum x_i^2 - 10 cos(2 pi x_i)                         */
/*   Griewank    1 + sum x_i^2 / 4000 - prod cos(x_i / sqrt(i))              */
/* All four have minimum 0 (at x = 0; Rosenbrock at x = 1).                  */
/* ------------------------------------------------------------------------- */
double so_bf_value(int32_t fn, int32_t D, const double* x) {
  const double two_pi = 6.283185307179586476925286766559;
  double s = 0.0;
  if (fn == 1) {
    for (int32_t i = 0; i < D; ++i) s += x[i] * x[i];
    return s;
  }
  if (fn == 2) {
    for (int32_t i = 0; i + 1 < D; ++i) {
      const double a = x[i + 1] - x[i] * x[i], b = x[i] - 1.0;
      s += 100.0 * a * a + b * b;
    }
    return s;
  }
  if (fn == 3) {
    for (int32_t i = 0; i < D; ++i) s += x[i] * x[i] - 10.0 * cos(two_pi * x[i]);
    return 10.0 * (double)D + s;
  }
  if (fn == 4) {
    double prod = 1.0;
    for (int32_t i = 0; i < D; ++i) {
      s += x[i] * x[i];
      prod *= cos(x[i] / sqrt((double)(i + 1)));
    }
    return 1.0 + s / 4000.0 - prod;
  }
  return NAN;
}

static int32_t so_is_bf(const so_config* cfg) { return cfg->problem >= 1 && cfg->problem <= 4; }
static int32_t so_dim(const so_config* cfg) {
  if (so_is_bf(cfg)) return cfg->Dbf;
  return cfg->problem == 6 ? 3 * cfg->T : 2 * cfg->T;
}

/* Eq. lenth of one row, in the problem's dimension. */
static double so_path_length(const so_config* cfg, const so_scene* sc, const double* x) {
  if (cfg->problem == 6) return so_length3(cfg->T, x, sc);
  return so_length(cfg->T, x, sc->sx, sc->sy, sc->tx, sc->ty);
}

void so_evaluate(const so_config* cfg, const so_scene* sc, int32_t n, const double* X, double* F,
                 int32_t* Q, double* len) {
  const int32_t T = cfg->T, D = so_dim(cfg);
  if (so_is_bf(cfg)) {
    for (int32_t p = 0; p < n; ++p) {
      if (F) F[p] = so_bf_value(cfg->problem, D, X + (int64_t)p * D);
      if (Q) Q[p] = 0;
      if (len) len[p] = 0.0;
    }
    return;
  }
  if (cfg->problem == 6) {
    for (int32_t p = 0; p < n; ++p) {
      const double* x = X + (int64_t)p * D;
      const double l = so_length3(T, x, sc);
      const int32_t q = so_sphere_collisions(T, x, sc);
      if (F) F[p] = l + cfg->alpha * so_pow_int((double)q, cfg->beta);
      if (Q) Q[p] = q;
      if (len) len[p] = l;
    }
    return;
  }
  if (cfg->problem == 5) {
    for (int32_t p = 0; p < n; ++p) {
      const double* x = X + (int64_t)p * D;
      const double l = so_length(T, x, sc->sx, sc->sy, sc->tx, sc->ty);
      const int32_t q = so_poly_crossings(T, x, sc) + (sc->A > 0 ? so_agent_conflicts(T, x, sc) : 0);
      if (F) F[p] = l + cfg->alpha * so_pow_int((double)q, cfg->beta);
      if (Q) Q[p] = q;
      if (len) len[p] = l;
    }
    return;
  }
  for (int32_t p = 0; p < n; ++p) {
    const double* x = X + (int64_t)p * D;
    double l = so_length(T, x, sc->sx, sc->sy, sc->tx, sc->ty);
    int32_t q = so_collisions(T, x, sc) + (sc->A > 0 ? so_agent_conflicts(T, x, sc) : 0);
    if (F) F[p] = l + cfg->alpha * so_pow_int((double)q, cfg->beta);
    if (Q) Q[p] = q;
    if (len) len[p] = l;
  }
}

/* ------------------------------------------------------------------------- */
/* Initialisation with Priori Initialization, Sec. 3.3.3 / Algorithm 1.      */
/* ------------------------------------------------------------------------- */

/* Number of PI particles per group: ceil(gamma * N), computed on the host. */
int32_t so_pi_count(double gamma, int32_t N) {
  double v = ceil(gamma * (double)N);
  if (v < 0) v = 0;
  if (v > N) v = N;
  return (int32_t)v;
}

/* X_range of coordinate j: [so_lo, so_lo + so_extent]; the map for a path. */
static double so_extent(const so_config* cfg, int32_t j) {
  if (so_is_bf(cfg)) return cfg->hi - cfg->lo;
  if (j < cfg->T) return cfg->W;
  return (cfg->problem == 6 && j >= 2 * cfg->T) ? cfg->Z : cfg->H;
}
static double so_lo(const so_config* cfg) { return so_is_bf(cfg) ? cfg->lo : 0.0; }
static double so_hi(const so_config* cfg, int32_t j) { return so_is_bf(cfg) ? cfg->hi : so_extent(cfg, j); }

static double so_clip(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* hyper: G x 6 rows (C1, C2, C3, w_init, w_end, V_limit), Table hyper8 layout. */
void so_init_swarm(const so_config* cfg, const double* hyper, so_state* st) {
  const int32_t G = cfg->G, N = cfg->N, D = so_dim(cfg);
  const uint32_t cyc = (uint32_t)*st->cycle;
  const int32_t n_pi = (cfg->use_pi && *st->has_prev) ? so_pi_count(cfg->pi_gamma, N) : 0;
  /* A second seed of the same kind as PI (the learned prior's proposal) takes the
   * first n_pr particles of each group; PI's particles follow it. */
  const int32_t n_pr = (st->n_prior != NULL && st->priorT != NULL) ? *st->n_prior : 0;
  for (int32_t g = 0; g < G; ++g) {
    const double vlim = hyper[6 * g + 5];
    for (int32_t n = 0; n < N; ++n) {
      const int32_t p = g * N + n;
      for (int32_t j = 0; j < D; ++j) {
        const double ext = so_extent(cfg, j);
        double u[4];
        double x;
        if (n < n_pr) {
          so_draw4(cfg->seed, (uint32_t)(j / 4), (uint32_t)p, SO_STREAM_PRIOR, cyc, cfg->run_id, u);
          x = so_clip(st->priorT[j] + (2.0 * u[j % 4] - 1.0) * cfg->pi_h, 0.0, ext);
        } else if (n < n_pr + n_pi) {
          so_draw4(cfg->seed, (uint32_t)(j / 4), (uint32_t)p, SO_STREAM_PI, cyc, cfg->run_id, u);
          x = so_clip(st->prevT[j] + (2.0 * u[j % 4] - 1.0) * cfg->pi_h, 0.0, ext);
        } else {
          so_draw4(cfg->seed, (uint32_t)(j / 4), (uint32_t)p, SO_STREAM_INIT_X, cyc, cfg->run_id, u);
          x = so_lo(cfg) + u[j % 4] * ext;
        }
        so_draw4(cfg->seed, (uint32_t)(j / 4), (uint32_t)p, SO_STREAM_INIT_V, cyc, cfg->run_id, u);
        const double vmax = vlim * ext; /* V_range = V_limit * X_range */
        st->X[(int64_t)p * D + j] = x;
        st->V[(int64_t)p * D + j] = (2.0 * u[j % 4] - 1.0) * vmax;
        st->P[(int64_t)p * D + j] = x;
      }
      st->Pfit[p] = INFINITY;
      st->PQ[p] = 0;
    }
    st->Gfit[g] = INFINITY;
    st->GQ[g] = 0;
    for (int32_t j = 0; j < D; ++j) st->Gb[g * D + j] = 0.0;
  }
  for (int32_t j = 0; j < D; ++j) st->Tb[j] = 0.0;
  *st->Tfit = INFINITY;
  *st->TQ = 0;
  *st->k = 0;
}

/* ------------------------------------------------------------------------- */
/* Auto Truncation, Sec. 3.3.4.                                              */
/* ------------------------------------------------------------------------- */

/* Population standard deviation of the n most recent window entries, oldest first. */
double so_window_std(const double* win, int32_t tw, int32_t n, int32_t head) {
  double sum = 0.0;
  for (int32_t i = 0; i < n; ++i) sum += win[(head - n + i + 2 * tw) % tw];
  const double mean = sum / (double)n;
  double ss = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    const double d = win[(head - n + i + 2 * tw) % tw] - mean;
    ss += d * d;
  }
  return sqrt(ss / (double)n);
}

/* Record this iteration's LFV and decide whether to truncate. */
int32_t so_at_update(const so_config* cfg, so_state* st) {
  const double lfv = *st->Tfit;
  if (cfg->at_mode == 1) {
    st->win[*st->win_head] = lfv;
    *st->win_head = (*st->win_head + 1) % cfg->tw;
    if (*st->win_n < cfg->tw) *st->win_n += 1;
    if (*st->win_n >= 2) {
      const double sd = so_window_std(st->win, cfg->tw, *st->win_n, *st->win_head);
      if (sd < cfg->delta && *st->TQ == 0) return 1;
    }
    return 0;
  }
  if (cfg->at_mode == 2) {
    if (lfv < *st->prev_lfv - cfg->stall_tol) *st->stall = 0;
    else *st->stall += 1;
    *st->prev_lfv = lfv;
    return (*st->stall >= cfg->stall_iters && *st->TQ == 0) ? 1 : 0;
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* One iteration of Algorithm 1.                                             */
/* ------------------------------------------------------------------------- */

/* check_stop = 0: always do the full body (no AT, no cap).
 * check_stop = 1: planning mode; returns 1 (and skips the omega/V/X update)
 *                 when AT fires or k reaches the cap.                       */
int32_t so_iteration(const so_config* cfg, const so_scene* sc, const double* hyper, so_state* st,
                     int32_t check_stop) {
  const int32_t G = cfg->G, N = cfg->N, D = so_dim(cfg), M = G * N;
  double* F = (double*)malloc(sizeof(double) * (size_t)M);
  int32_t* Q = (int32_t*)malloc(sizeof(int32_t) * (size_t)M);

  /* k <- k + 1 */
  *st->k += 1;
  const int32_t k = *st->k;

  /* Fitness = F(X^k) */
  so_evaluate(cfg, sc, M, st->X, F, Q, NULL);

  /* Update P_g (strictly better only) */
  for (int32_t p = 0; p < M; ++p) {
    if (F[p] < st->Pfit[p]) {
      st->Pfit[p] = F[p];
      st->PQ[p] = Q[p];
      memcpy(st->P + (int64_t)p * D, st->X + (int64_t)p * D, sizeof(double) * (size_t)D);
    }
  }
  /* Update G_g: lowest-index argmin of the group's Pbest fitness */
  for (int32_t g = 0; g < G; ++g) {
    double best = INFINITY;
    int32_t bi = -1;
    for (int32_t n = 0; n < N; ++n) {
      if (st->Pfit[g * N + n] < best) {
        best = st->Pfit[g * N + n];
        bi = n;
      }
    }
    if (bi >= 0 && best < st->Gfit[g]) {
      st->Gfit[g] = best;
      st->GQ[g] = st->PQ[g * N + bi];
      memcpy(st->Gb + (int64_t)g * D, st->P + (int64_t)(g * N + bi) * D, sizeof(double) * (size_t)D);
    }
  }
  /* Update T: lowest-index argmin over the groups */
  {
    double best = INFINITY;
    int32_t bg = -1;
    for (int32_t g = 0; g < G; ++g) {
      if (st->Gfit[g] < best) {
        best = st->Gfit[g];
        bg = g;
      }
    }
    if (bg >= 0 && best < *st->Tfit) {
      *st->Tfit = best;
      *st->TQ = st->GQ[bg];
      memcpy(st->Tb, st->Gb + (int64_t)bg * D, sizeof(double) * (size_t)D);
    }
  }
  free(F);
  free(Q);

  if (check_stop) {
    const int32_t stop = so_at_update(cfg, st);
    if (stop || k >= cfg->max_iters) return 1;
  }

  /* Eq. TOF_omega, then Eq. TOF_V (= Eq. DPPSO_V per group) with clipping,
   * then Eq. TOF_X with clipping (Algorithm 1). */
  for (int32_t g = 0; g < G; ++g) {
    const double* h = hyper + 6 * g;
    const double c1 = h[0], c2 = h[1], c3 = h[2], w_init = h[3], w_end = h[4], vlim = h[5];
    const double w = w_init - (w_init - w_end) / (double)cfg->max_iters * (double)k;
    for (int32_t n = 0; n < N; ++n) {
      const int32_t p = g * N + n;
      double r[4];
      so_draw4(cfg->seed, (uint32_t)k, (uint32_t)p, SO_STREAM_VEL, (uint32_t)*st->cycle, cfg->run_id, r);
      const double r1 = r[0], r2 = r[1], r3 = r[2];
      for (int32_t j = 0; j < D; ++j) {
        const int64_t i = (int64_t)p * D + j;
        const double ext = so_extent(cfg, j);
        const double vmax = vlim * ext;
        const double x = st->X[i];
        double v = w * st->V[i] + c1 * r1 * (st->P[i] - x) + c2 * r2 * (st->Gb[g * D + j] - x) +
                   c3 * r3 * (st->Tb[j] - x);
        v = so_clip(v, -vmax, vmax);
        st->V[i] = v;
        st->X[i] = so_clip(x + v, so_lo(cfg), so_hi(cfg, j));
      }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* A planning cycle (application phase) and a plain continuation.            */
/* ------------------------------------------------------------------------- */

/* result: D waypoints, then cost, length, Q, iterations. */
void so_plan(const so_config* cfg, const so_scene* sc, const double* hyper, so_state* st, double* result) {
  const int32_t D = so_dim(cfg);
  if (*st->cycle == 0) {
    *st->win_n = 0;
    *st->win_head = 0;
  }
  *st->stall = 0;
  *st->prev_lfv = INFINITY;
  so_init_swarm(cfg, hyper, st);
  while (!so_iteration(cfg, sc, hyper, st, 1)) {
  }
  for (int32_t j = 0; j < D; ++j) result[j] = st->Tb[j];
  result[D + 0] = *st->Tfit;
  result[D + 1] = so_path_length(cfg, sc, st->Tb);
  result[D + 2] = (double)*st->TQ;
  result[D + 3] = (double)*st->k;
  for (int32_t j = 0; j < D; ++j) st->prevT[j] = st->Tb[j];
  *st->has_prev = 1;
  *st->cycle += 1;
}

void so_step(const so_config* cfg, const so_scene* sc, const double* hyper, so_state* st, int32_t iters) {
  for (int32_t i = 0; i < iters; ++i) so_iteration(cfg, sc, hyper, st, 0);
}

/* ------------------------------------------------------------------------- */
/* Dynamic environment step (Fig. PP caption; Sec. 4.3).                     */
/* Circles move by their velocity; a velocity component flips when the disk */
/* crosses the border it is moving towards.  Start and target move the same */
/* way with zero radius.                                                     */
/* ------------------------------------------------------------------------- */
static void so_move(double* c, double* v, double r, double lo, double hi) {
  *c += *v;
  if (*c - r < lo && *v < 0.0) *v = -*v;
  if (*c + r > hi && *v > 0.0) *v = -*v;
}

void so_advance_scene(double W, double H, int32_t O, double* circ, double* cvel, double* start,
                      double* svel, double* target, double* tvel) {
  for (int32_t o = 0; o < O; ++o) {
    so_move(&circ[3 * o + 0], &cvel[2 * o + 0], circ[3 * o + 2], 0.0, W);
    so_move(&circ[3 * o + 1], &cvel[2 * o + 1], circ[3 * o + 2], 0.0, H);
  }
  so_move(&start[0], &svel[0], 0.0, 0.0, W);
  so_move(&start[1], &svel[1], 0.0, 0.0, H);
  so_move(&target[0], &tvel[0], 0.0, 0.0, W);
  so_move(&target[1], &tvel[1], 0.0, 0.0, H);
}

/* Moving polygon obstacles (Sec. 3.3.1's bounding boxes, moved as the Fig. PP
 * caption moves the obstacles): polygon p, the edges off[p] .. off[p+1]-1
 * (E x 4: x0, y0, x1, y1), is translated by its velocity (pvel[2p], pvel[2p+1]);
 * then a velocity component flips when the polygon's bounding box lies past the
 * border it is moving towards -- the circles' rule with the box's extent in place
 * of centre -/+ radius.  Start and target move as in so_advance_scene. */
void so_advance_polygons(double W, double H, int32_t P, const int32_t* off, double* edges, double* pvel,
                         double* start, double* svel, double* target, double* tvel) {
  for (int32_t p = 0; p < P; ++p) {
    const double vx = pvel[2 * p], vy = pvel[2 * p + 1];
    double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
    for (int32_t e = off[p]; e < off[p + 1]; ++e) {
      double* d = edges + 4 * e;
      d[0] += vx;
      d[1] += vy;
      d[2] += vx;
      d[3] += vy;
      xmin = fmin(xmin, fmin(d[0], d[2]));
      xmax = fmax(xmax, fmax(d[0], d[2]));
      ymin = fmin(ymin, fmin(d[1], d[3]));
      ymax = fmax(ymax, fmax(d[1], d[3]));
    }
    if (off[p + 1] > off[p]) {
      if (xmin < 0.0 && vx < 0.0) pvel[2 * p] = -vx;
      if (xmax > W && vx > 0.0) pvel[2 * p] = -vx;
      if (ymin < 0.0 && vy < 0.0) pvel[2 * p + 1] = -vy;
      if (ymax > H && vy > 0.0) pvel[2 * p + 1] = -vy;
    }
  }
  so_move(&start[0], &svel[0], 0.0, 0.0, W);
  so_move(&start[1], &svel[1], 0.0, 0.0, H);
  so_move(&target[0], &tvel[0], 0.0, 0.0, W);
  so_move(&target[1], &tvel[1], 0.0, 0.0, H);
}

/* ------------------------------------------------------------------------- */
/* HSEF, Sec. 3.2.1.  The H-swarm is DTPSO over hyper-parameter vectors;     */
/* each H-particle's fitness is the LFV (Eq. fit_h) of an L-run of          */
/* lcfg->max_iters iterations with that particle's hyper-parameters.         */
/* H-position layout: [w_1..w_G, C1_1..C1_G, C2_1..C2_G]; the L-run uses    */
/* C3 = 0, w_init = w_end = w and V_limit = l_vlimit.  All H-particles of   */
/* one evolution share the L-run's random streams (run id lcfg->run_id,     */
/* cycle field = evolution index - 1).                                       */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t HG, HN;          /* H-swarm groups and particles per group          */
  int32_t E;               /* evolutions (H iterations); also T of TOF_omega */
  const double* hhyper;    /* HG x 6, Table hyper8 layout                     */
  double lo[3], hi[3];     /* box of (w, C1, C2)                              */
  double l_vlimit;         /* V_limit of the L-runs                           */
  uint64_t hseed;          /* Philox key of the H-swarm                       */
} so_hsef_cfg;

/* The final H-swarm state (after the last H update), for the pins: HM x DH
 * positions, velocities and personal bests, HG x DH group bests, DH global best;
 * any pointer may be NULL. */
typedef struct {
  double *hx, *hv, *hp, *hgb, *htb;
} so_hsef_out;

static void hsef_run(const so_config* lcfg, const so_scene* sc, const so_hsef_cfg* hc, double* best_pos,
                     double* best_fit, double* history, const so_hsef_out* out);

void so_hsef(const so_config* lcfg, const so_scene* sc, const so_hsef_cfg* hc, double* best_pos,
             double* best_fit, double* history) {
  hsef_run(lcfg, sc, hc, best_pos, best_fit, history, NULL);
}

void so_hsef_state(const so_config* lcfg, const so_scene* sc, const so_hsef_cfg* hc, double* best_pos,
                   double* best_fit, double* history, double* hx, double* hv, double* hp, double* hgb,
                   double* htb) {
  const so_hsef_out out = {hx, hv, hp, hgb, htb};
  hsef_run(lcfg, sc, hc, best_pos, best_fit, history, &out);
}

static void hsef_run(const so_config* lcfg, const so_scene* sc, const so_hsef_cfg* hc, double* best_pos,
                     double* best_fit, double* history, const so_hsef_out* out) {
  const int32_t G = lcfg->G, DH = 3 * G, HM = hc->HG * hc->HN;
  const int32_t T = lcfg->T, D = 2 * T, M = lcfg->G * lcfg->N;
  double* HX = (double*)calloc((size_t)HM * DH, sizeof(double));
  double* HV = (double*)calloc((size_t)HM * DH, sizeof(double));
  double* HP = (double*)calloc((size_t)HM * DH, sizeof(double));
  double* HPfit = (double*)calloc((size_t)HM, sizeof(double));
  double* HGb = (double*)calloc((size_t)hc->HG * DH, sizeof(double));
  double* HGfit = (double*)calloc((size_t)hc->HG, sizeof(double));
  double HTb[3 * 64];
  double HTfit = INFINITY;
  double* HF = (double*)calloc((size_t)HM, sizeof(double));
  double* lhyper = (double*)calloc((size_t)G * 6, sizeof(double));
  /* L-run scratch state */
  double* X = (double*)calloc((size_t)M * D, sizeof(double));
  double* V = (double*)calloc((size_t)M * D, sizeof(double));
  double* P = (double*)calloc((size_t)M * D, sizeof(double));
  double* Pfit = (double*)calloc((size_t)M, sizeof(double));
  int32_t* PQ = (int32_t*)calloc((size_t)M, sizeof(int32_t));
  double* Gb = (double*)calloc((size_t)G * D, sizeof(double));
  double* Gfit = (double*)calloc((size_t)G, sizeof(double));
  int32_t* GQ = (int32_t*)calloc((size_t)G, sizeof(int32_t));
  double* Tb = (double*)calloc((size_t)D, sizeof(double));
  double* prevT = (double*)calloc((size_t)D, sizeof(double));
  double* win = (double*)calloc((size_t)(lcfg->tw > 0 ? lcfg->tw : 1), sizeof(double));
  double* res = (double*)calloc((size_t)D + 4, sizeof(double));
  double Tfit = INFINITY, prev_lfv = INFINITY;
  int32_t TQ = 0, k = 0, cycle = 0, has_prev = 0, win_n = 0, win_head = 0, stall = 0;
  so_state st = {X, V, P, Pfit, PQ, Gb, Gfit, GQ, Tb, &Tfit, &TQ, &k, &cycle, &has_prev, prevT,
                 win, &win_n, &win_head, &stall, &prev_lfv};

  /* H-swarm initialisation (Algorithm 1, first line) */
  for (int32_t h = 0; h < HM; ++h) {
    const int32_t hg = h / hc->HN;
    for (int32_t j = 0; j < DH; ++j) {
      const int32_t kind = j / G; /* 0 = w, 1 = C1, 2 = C2 */
      const double lo = hc->lo[kind], hi = hc->hi[kind];
      double u[4];
      so_draw4(hc->hseed, (uint32_t)(j / 4), (uint32_t)h, SO_STREAM_H_INIT_X, 0u, 0u, u);
      const double x = lo + u[j % 4] * (hi - lo);
      so_draw4(hc->hseed, (uint32_t)(j / 4), (uint32_t)h, SO_STREAM_H_INIT_V, 0u, 0u, u);
      const double vmax = hc->hhyper[6 * hg + 5] * (hi - lo);
      HX[h * DH + j] = x;
      HV[h * DH + j] = (2.0 * u[j % 4] - 1.0) * vmax;
      HP[h * DH + j] = x;
    }
    HPfit[h] = INFINITY;
  }
  for (int32_t g = 0; g < hc->HG; ++g) HGfit[g] = INFINITY;
  for (int32_t j = 0; j < DH; ++j) HTb[j] = 0.0;

  for (int32_t e = 1; e <= hc->E; ++e) {
    /* H-fitness: LFV of one L-run per H-particle (Eq. fit_h) */
    for (int32_t h = 0; h < HM; ++h) {
      for (int32_t g = 0; g < G; ++g) {
        lhyper[6 * g + 0] = HX[h * DH + G + g];
        lhyper[6 * g + 1] = HX[h * DH + 2 * G + g];
        lhyper[6 * g + 2] = 0.0;
        lhyper[6 * g + 3] = HX[h * DH + g];
        lhyper[6 * g + 4] = HX[h * DH + g];
        lhyper[6 * g + 5] = hc->l_vlimit;
      }
      cycle = e - 1;
      has_prev = 0;
      so_plan(lcfg, sc, lhyper, &st, res);
      HF[h] = res[D + 0];
    }
    /* H bests */
    for (int32_t h = 0; h < HM; ++h) {
      if (HF[h] < HPfit[h]) {
        HPfit[h] = HF[h];
        memcpy(HP + h * DH, HX + h * DH, sizeof(double) * (size_t)DH);
      }
    }
    for (int32_t g = 0; g < hc->HG; ++g) {
      double best = INFINITY;
      int32_t bi = -1;
      for (int32_t n = 0; n < hc->HN; ++n) {
        if (HPfit[g * hc->HN + n] < best) {
          best = HPfit[g * hc->HN + n];
          bi = n;
        }
      }
      if (bi >= 0 && best < HGfit[g]) {
        HGfit[g] = best;
        memcpy(HGb + g * DH, HP + (g * hc->HN + bi) * DH, sizeof(double) * (size_t)DH);
      }
    }
    {
      double best = INFINITY;
      int32_t bg = -1;
      for (int32_t g = 0; g < hc->HG; ++g) {
        if (HGfit[g] < best) {
          best = HGfit[g];
          bg = g;
        }
      }
      if (bg >= 0 && best < HTfit) {
        HTfit = best;
        memcpy(HTb, HGb + bg * DH, sizeof(double) * (size_t)DH);
      }
    }
    history[e - 1] = HTfit;
    /* H update: Eqs. TOF_omega, TOF_V, TOF_X with Table hyper8 per H-group */
    for (int32_t g = 0; g < hc->HG; ++g) {
      const double* hh = hc->hhyper + 6 * g;
      const double w = hh[3] - (hh[3] - hh[4]) / (double)hc->E * (double)e;
      for (int32_t n = 0; n < hc->HN; ++n) {
        const int32_t h = g * hc->HN + n;
        double r[4];
        so_draw4(hc->hseed, (uint32_t)e, (uint32_t)h, SO_STREAM_H_VEL, 0u, 0u, r);
        for (int32_t j = 0; j < DH; ++j) {
          const int32_t kind = j / G;
          const double lo = hc->lo[kind], hi = hc->hi[kind];
          const double vmax = hh[5] * (hi - lo);
          const double x = HX[h * DH + j];
          double v = w * HV[h * DH + j] + hh[0] * r[0] * (HP[h * DH + j] - x) +
                     hh[1] * r[1] * (HGb[g * DH + j] - x) + hh[2] * r[2] * (HTb[j] - x);
          v = so_clip(v, -vmax, vmax);
          HV[h * DH + j] = v;
          HX[h * DH + j] = so_clip(x + v, lo, hi);
        }
      }
    }
  }
  for (int32_t j = 0; j < DH; ++j) best_pos[j] = HTb[j];
  *best_fit = HTfit;
  if (out) {
    if (out->hx) memcpy(out->hx, HX, sizeof(double) * (size_t)HM * DH);
    if (out->hv) memcpy(out->hv, HV, sizeof(double) * (size_t)HM * DH);
    if (out->hp) memcpy(out->hp, HP, sizeof(double) * (size_t)HM * DH);
    if (out->hgb) memcpy(out->hgb, HGb, sizeof(double) * (size_t)hc->HG * DH);
    if (out->htb) memcpy(out->htb, HTb, sizeof(double) * (size_t)DH);
  }
  free(HX); free(HV); free(HP); free(HPfit); free(HGb); free(HGfit); free(HF); free(lhyper);
  free(X); free(V); free(P); free(Pfit); free(PQ); free(Gb); free(Gfit); free(GQ); free(Tb);
  free(prevT); free(win); free(res);
}
