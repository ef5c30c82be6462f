/*
 * mlp.c -- FP64 reference of the learned control proposal's network.
 *
 * TEST INFRASTRUCTURE ONLY (see kpo.h).  The network is not part of the
 * paper; it is the learned proposal added on top of Algorithm 2's uniform
 * control draw: a multilayer perceptron mapping 24 node features (padded to
 * 32 inputs) through two ReLU layers of 256 units to 8 outputs, the mean
 * (tanh-squashed) and log standard deviation (clamped) of a Gaussian over 4
 * normalised quantities (3 controls and the duration).  Trained by
 * minimising the Gaussian negative log-likelihood of harvested targets.
 *
 * Parameter vector (float32 in, promoted), row-major:
 *   W1 [256][32], b1 [256], W2 [256][256], b2 [256], W3 [8][256], b3 [8]
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "kpo.h"

#define IN 32
#define H 256
#define OUT 8
#define NQ 4
#define LOGSTD_MIN -4.0
#define LOGSTD_MAX 1.0

int32_t kpo_mlp_num_params(void) { return H * IN + H + H * H + H + OUT * H + OUT; }

typedef struct {
  const double *W1, *b1, *W2, *b2, *W3, *b3;
} params;

static params split(const double *p) {
  params q;
  q.W1 = p;
  q.b1 = q.W1 + H * IN;
  q.W2 = q.b1 + H;
  q.b2 = q.W2 + H * H;
  q.W3 = q.b2 + H;
  q.b3 = q.W3 + OUT * H;
  return q;
}

/* y[n] = b[n] + sum_k W[n][k] x[k] */
static void dense(const double *W, const double *b, const double *x, int n_out, int n_in,
                  double *y) {
  for (int n = 0; n < n_out; ++n) {
    double s = b[n];
    for (int k = 0; k < n_in; ++k) s += W[n * n_in + k] * x[k];
    y[n] = s;
  }
}

/* Heads: mean = tanh(raw), log_std = clamp(raw, LOGSTD_MIN, LOGSTD_MAX). */
static void heads(const double *raw, double *mean, double *log_std) {
  for (int i = 0; i < NQ; ++i) {
    mean[i] = tanh(raw[i]);
    double l = raw[NQ + i];
    log_std[i] = l < LOGSTD_MIN ? LOGSTD_MIN : (l > LOGSTD_MAX ? LOGSTD_MAX : l);
  }
}

void kpo_mlp_forward(const double *p, const double *x, int32_t M, double *out) {
  params q = split(p);
  double h1[H], h2[H], raw[OUT];
  for (int m = 0; m < M; ++m) {
    dense(q.W1, q.b1, x + (size_t)m * IN, H, IN, h1);
    for (int i = 0; i < H; ++i) h1[i] = h1[i] > 0.0 ? h1[i] : 0.0;
    dense(q.W2, q.b2, h1, H, H, h2);
    for (int i = 0; i < H; ++i) h2[i] = h2[i] > 0.0 ? h2[i] : 0.0;
    dense(q.W3, q.b3, h2, OUT, H, raw);
    double mean[NQ], ls[NQ];
    heads(raw, mean, ls);
    for (int i = 0; i < NQ; ++i) {
      out[(size_t)m * OUT + i] = mean[i];
      out[(size_t)m * OUT + NQ + i] = ls[i];
    }
  }
}

/* Mean over the batch of sum_i [log_std_i + 0.5 ((t_i - mean_i) / std_i)^2]
 * and its gradient with respect to every parameter (backpropagation). */
double kpo_mlp_loss_grad(const double *p, const double *x, const double *t, int32_t M,
                         double *grad) {
  params q = split(p);
  const int np = kpo_mlp_num_params();
  if (grad) memset(grad, 0, sizeof(double) * (size_t)np);
  double *gW1 = grad, *gb1 = grad ? grad + H * IN : NULL;
  double *gW2 = grad ? gb1 + H : NULL, *gb2 = grad ? gW2 + H * H : NULL;
  double *gW3 = grad ? gb2 + H : NULL, *gb3 = grad ? gW3 + OUT * H : NULL;
  double loss = 0.0;
  double a1[H], h1[H], a2[H], h2[H], raw[OUT], draw[OUT], dh2[H], dh1[H];
  for (int m = 0; m < M; ++m) {
    const double *xm = x + (size_t)m * IN, *tm = t + (size_t)m * NQ;
    dense(q.W1, q.b1, xm, H, IN, a1);
    for (int i = 0; i < H; ++i) h1[i] = a1[i] > 0.0 ? a1[i] : 0.0;
    dense(q.W2, q.b2, h1, H, H, a2);
    for (int i = 0; i < H; ++i) h2[i] = a2[i] > 0.0 ? a2[i] : 0.0;
    dense(q.W3, q.b3, h2, OUT, H, raw);
    for (int i = 0; i < NQ; ++i) {
      const double mu = tanh(raw[i]);
      const double l = raw[NQ + i];
      const int clamped = l < LOGSTD_MIN || l > LOGSTD_MAX;
      const double ls = l < LOGSTD_MIN ? LOGSTD_MIN : (l > LOGSTD_MAX ? LOGSTD_MAX : l);
      const double z = (tm[i] - mu) * exp(-ls);
      loss += ls + 0.5 * z * z;
      /* d/d mu = -(t - mu) / std^2 = -z exp(-ls); d mu / d raw = 1 - mu^2 */
      draw[i] = -z * exp(-ls) * (1.0 - mu * mu) / (double)M;
      /* d/d ls = 1 - z^2 (zero where the clamp is active) */
      draw[NQ + i] = clamped ? 0.0 : (1.0 - z * z) / (double)M;
    }
    if (!grad) continue;
    for (int n = 0; n < OUT; ++n) {
      gb3[n] += draw[n];
      for (int k = 0; k < H; ++k) gW3[n * H + k] += draw[n] * h2[k];
    }
    for (int k = 0; k < H; ++k) {
      double s = 0.0;
      for (int n = 0; n < OUT; ++n) s += draw[n] * q.W3[n * H + k];
      dh2[k] = a2[k] > 0.0 ? s : 0.0;
    }
    for (int n = 0; n < H; ++n) {
      gb2[n] += dh2[n];
      for (int k = 0; k < H; ++k) gW2[n * H + k] += dh2[n] * h1[k];
    }
    for (int k = 0; k < H; ++k) {
      double s = 0.0;
      for (int n = 0; n < H; ++n) s += dh2[n] * q.W2[n * H + k];
      dh1[k] = a1[k] > 0.0 ? s : 0.0;
    }
    for (int n = 0; n < H; ++n) {
      gb1[n] += dh1[n];
      for (int k = 0; k < IN; ++k) gW1[n * IN + k] += dh1[n] * xm[k];
    }
  }
  return loss / (double)M;
}

/* Adam (Kingma & Ba 2015) on a flat vector: step t >= 1. */
void kpo_adam(double *p, const double *g, double *m, double *v, int32_t n, double lr,
              double beta1, double beta2, double eps, int32_t t) {
  const double c1 = 1.0 - pow(beta1, t), c2 = 1.0 - pow(beta2, t);
  for (int i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
    const double mh = m[i] / c1, vh = v[i] / c2;
    p[i] -= lr * mh / (sqrt(vh) + eps);
  }
}
