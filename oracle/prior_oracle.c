/*
 * prior_oracle.c -- plain FP64 CPU oracle of the learned prior: a small MLP over an
 * occupancy raster of the scene plus its start and target that proposes the initial
 * waypoints of a planning cycle, beside Priori Initialization (Sec. 3.3.3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load this library.  The product path (the CUDA
 * library under paper_2308_10169_gb300/) never calls it and shares no code,
 * header, table or constant generator with it.
 *
 * The paper has no learned component.  PI (Sec. 3.3.3) seeds part of each group
 * around the previous cycle's best path; the network's proposal is a second seed
 * of the same kind.  What is defined here, written out without blocking or fusion:
 *   - occupancy raster: cell (i, j) of a g x g grid over [0, W] x [0, H] is occupied
 *     when its centre ((j + 1/2) W / g, (i + 1/2) H / g) lies in a closed disk of
 *     the scene.  The cell/disk decision is taken in FP32, the precision of the
 *     CUDA kernel, so that both sides decide each cell the same way.
 *   - features: the g*g raster values, then start and target divided by the map
 *     extent (x / W, y / H), then zeros up to K.
 *   - labels: a path of T waypoints (x_0..x_{T-1}, y_0..y_{T-1}) is encoded as its
 *     offset from the straight start-target line (point k at fraction
 *     (k + 1) / (T + 1)), divided by the map extent; decoding inverts that and
 *     clips to the map (the box of Eq. TOF_X's clip).
 *   - network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3.
 *   - loss: (1 / (2B)) * sum over the B rows and the 2T outputs of (y - t)^2.
 *   - gradients: the chain rule of that loss, layer by layer.
 *   - Adam (Kingma and Ba, ICLR 2015, Algorithm 1): exponential moving averages
 *     of g and g^2 with bias correction, step lr * m_hat / (sqrt(v_hat) + eps).
 *
 * Parameter layout (one flat vector): W1 (H1 x K, row-major), b1 (H1),
 * W2 (H2 x H1), b2 (H2), W3 (O x H2), b3 (O).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t K, H1, H2, O;
} so_mlp_dims;

long so_mlp_num_params(const so_mlp_dims* d) {
  return (long)d->H1 * d->K + d->H1 + (long)d->H2 * d->H1 + d->H2 + (long)d->O * d->H2 + d->O;
}

/* Offsets of the six tensors in the flat parameter vector. */
static void offsets(const so_mlp_dims* d, long off[6]) {
  off[0] = 0;
  off[1] = off[0] + (long)d->H1 * d->K;
  off[2] = off[1] + d->H1;
  off[3] = off[2] + (long)d->H2 * d->H1;
  off[4] = off[3] + d->H2;
  off[5] = off[4] + (long)d->O * d->H2;
}

/* ------------------------------------------------------------------------- */
/* Occupancy raster and features                                              */
/* ------------------------------------------------------------------------- */
void so_raster(int32_t grid, double W, double H, int32_t O, const double* circ, double sx, double sy,
               double tx, double ty, int32_t K, double* feat) {
  const float cw = (float)W / (float)grid;
  const float chh = (float)H / (float)grid;
  for (int i = 0; i < grid; ++i) {
    const float y = ((float)i + 0.5f) * chh;
    for (int j = 0; j < grid; ++j) {
      const float x = ((float)j + 0.5f) * cw;
      int occ = 0;
      for (int o = 0; o < O; ++o) {
        const float dx = x - (float)circ[3 * o];
        const float dy = y - (float)circ[3 * o + 1];
        const float r = (float)circ[3 * o + 2];
        const float d2 = dx * dx + dy * dy;
        if (d2 <= r * r) occ = 1;
      }
      feat[i * grid + j] = (double)occ;
    }
  }
  const int g2 = grid * grid;
  feat[g2 + 0] = sx / W;
  feat[g2 + 1] = sy / H;
  feat[g2 + 2] = tx / W;
  feat[g2 + 3] = ty / H;
  for (int k = g2 + 4; k < K; ++k) feat[k] = 0.0;
}

/* ------------------------------------------------------------------------- */
/* Label encoding: offset from the straight line, over the map extent          */
/* ------------------------------------------------------------------------- */
void so_prior_encode(int32_t T, double W, double H, double sx, double sy, double tx, double ty,
                     const double* wp, double* y) {
  for (int k = 0; k < T; ++k) {
    const double f = (double)(k + 1) / (double)(T + 1);
    y[k] = (wp[k] - (sx + f * (tx - sx))) / W;
    y[T + k] = (wp[T + k] - (sy + f * (ty - sy))) / H;
  }
}

void so_prior_decode(int32_t T, double W, double H, double sx, double sy, double tx, double ty,
                     const double* y, double* wp) {
  for (int k = 0; k < T; ++k) {
    const double f = (double)(k + 1) / (double)(T + 1);
    const double x = sx + f * (tx - sx) + y[k] * W;
    const double v = sy + f * (ty - sy) + y[T + k] * H;
    wp[k] = x < 0.0 ? 0.0 : (x > W ? W : x);
    wp[T + k] = v < 0.0 ? 0.0 : (v > H ? H : v);
  }
}

/* ------------------------------------------------------------------------- */
/* Network                                                                    */
/* ------------------------------------------------------------------------- */
static double relu(double v) { return v > 0.0 ? v : 0.0; }

/* out[b][i] = act(sum_k Wt[i][k] * in[b][k] + bias[i]) */
static void dense(int B, int nin, int nout, const double* Wt, const double* bias, const double* in, double* out,
                  int use_relu) {
  for (int b = 0; b < B; ++b)
    for (int i = 0; i < nout; ++i) {
      double s = bias[i];
      for (int k = 0; k < nin; ++k) s += Wt[(long)i * nin + k] * in[(long)b * nin + k];
      out[(long)b * nout + i] = use_relu ? relu(s) : s;
    }
}

void so_mlp_forward(const so_mlp_dims* d, const double* prm, int32_t B, const double* X, double* H1, double* H2,
                    double* Y) {
  long off[6];
  offsets(d, off);
  dense(B, d->K, d->H1, prm + off[0], prm + off[1], X, H1, 1);
  dense(B, d->H1, d->H2, prm + off[2], prm + off[3], H1, H2, 1);
  dense(B, d->H2, d->O, prm + off[4], prm + off[5], H2, Y, 0);
}

/* Loss of B rows against targets Tg (B x O) and its gradient (flat, same layout as
 * the parameters).  Returns the loss. */
double so_mlp_loss_grad(const so_mlp_dims* d, const double* prm, int32_t B, const double* X, const double* Tg,
                        double* grad) {
  long off[6];
  offsets(d, off);
  const int K = d->K, n1 = d->H1, n2 = d->H2, no = d->O;
  double* H1 = (double*)calloc((size_t)B * n1, sizeof(double));
  double* H2 = (double*)calloc((size_t)B * n2, sizeof(double));
  double* Y = (double*)calloc((size_t)B * no, sizeof(double));
  double* dY = (double*)calloc((size_t)B * no, sizeof(double));
  double* dH2 = (double*)calloc((size_t)B * n2, sizeof(double));
  double* dH1 = (double*)calloc((size_t)B * n1, sizeof(double));
  so_mlp_forward(d, prm, B, X, H1, H2, Y);
  double loss = 0.0;
  for (int b = 0; b < B; ++b)
    for (int i = 0; i < no; ++i) {
      const double e = Y[(long)b * no + i] - Tg[(long)b * no + i];
      loss += 0.5 * e * e / B;
      dY[(long)b * no + i] = e / B;
    }
  memset(grad, 0, sizeof(double) * (size_t)so_mlp_num_params(d));
  double *gW1 = grad + off[0], *gb1 = grad + off[1], *gW2 = grad + off[2], *gb2 = grad + off[3];
  double *gW3 = grad + off[4], *gb3 = grad + off[5];
  const double *W2 = prm + off[2], *W3 = prm + off[4];
  /* output layer */
  for (int b = 0; b < B; ++b)
    for (int i = 0; i < no; ++i) {
      const double g = dY[(long)b * no + i];
      gb3[i] += g;
      for (int k = 0; k < n2; ++k) gW3[(long)i * n2 + k] += g * H2[(long)b * n2 + k];
    }
  /* back through W3 and the second ReLU (derivative 1 where h2 > 0) */
  for (int b = 0; b < B; ++b)
    for (int k = 0; k < n2; ++k) {
      double s = 0.0;
      for (int i = 0; i < no; ++i) s += dY[(long)b * no + i] * W3[(long)i * n2 + k];
      dH2[(long)b * n2 + k] = H2[(long)b * n2 + k] > 0.0 ? s : 0.0;
    }
  for (int b = 0; b < B; ++b)
    for (int i = 0; i < n2; ++i) {
      const double g = dH2[(long)b * n2 + i];
      gb2[i] += g;
      for (int k = 0; k < n1; ++k) gW2[(long)i * n1 + k] += g * H1[(long)b * n1 + k];
    }
  /* back through W2 and the first ReLU */
  for (int b = 0; b < B; ++b)
    for (int k = 0; k < n1; ++k) {
      double s = 0.0;
      for (int i = 0; i < n2; ++i) s += dH2[(long)b * n2 + i] * W2[(long)i * n1 + k];
      dH1[(long)b * n1 + k] = H1[(long)b * n1 + k] > 0.0 ? s : 0.0;
    }
  for (int b = 0; b < B; ++b)
    for (int i = 0; i < n1; ++i) {
      const double g = dH1[(long)b * n1 + i];
      gb1[i] += g;
      for (int k = 0; k < K; ++k) gW1[(long)i * K + k] += g * X[(long)b * K + k];
    }
  free(H1);
  free(H2);
  free(Y);
  free(dY);
  free(dH2);
  free(dH1);
  return loss;
}

/* One Adam step t (1-based) over n parameters. */
void so_adam(long n, double* w, double* m, double* v, const double* g, double lr, double b1, double b2, double eps,
             int32_t t) {
  const double c1 = 1.0 - pow(b1, (double)t);
  const double c2 = 1.0 - pow(b2, (double)t);
  for (long i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    const double mh = m[i] / c1, vh = v[i] / c2;
    w[i] -= lr * mh / (sqrt(vh) + eps);
  }
}
