/*
 * Oracle (test infrastructure only): FP64 reference of the warm-start
 * multilayer perceptron (no counterpart in the paper; it maps droplet
 * parameters to an initial interface profile that seeds the solver).
 *
 * Network: sizes[0] inputs -> hidden layers of GELU units -> sizes[nlayers]
 * linear outputs.  GELU(x) = x/2 (1 + erf(x / sqrt 2)).  Parameters are packed
 * layer by layer: W_l (sizes[l+1] rows x sizes[l] columns, row-major) followed
 * by b_l (sizes[l+1]).  Loss = mean over batch and outputs of (y - target)^2.
 * Gradients by the chain rule, plain loops.  Adam: Kingma and Ba (2015),
 * bias-corrected first and second moments.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static double gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }
static double gelu_d(double x) {
  const double inv_sqrt_2pi = 0.39894228040143267794;
  return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * inv_sqrt_2pi * exp(-0.5 * x * x);
}

static long param_count(const int* sizes, int nl) {
  long n = 0;
  for (int l = 0; l < nl; ++l) n += (long)sizes[l + 1] * sizes[l] + sizes[l + 1];
  return n;
}

/* forward for one sample; z[l] pre-activations, h[l] activations (h[0] = x) */
static void forward_one(const int* sizes, int nl, const double* params, const double* x, double** z,
                        double** h) {
  memcpy(h[0], x, sizeof(double) * sizes[0]);
  const double* p = params;
  for (int l = 0; l < nl; ++l) {
    int in = sizes[l], out = sizes[l + 1];
    const double* W = p;
    const double* b = p + (long)out * in;
    for (int o = 0; o < out; ++o) {
      double acc = b[o];
      for (int i = 0; i < in; ++i) acc += W[(long)o * in + i] * h[l][i];
      z[l][o] = acc;
      h[l + 1][o] = (l < nl - 1) ? gelu(acc) : acc;
    }
    p += (long)out * in + out;
  }
}

static int alloc_layers(const int* sizes, int nl, double*** z, double*** h) {
  *z = (double**)calloc(nl, sizeof(double*));
  *h = (double**)calloc(nl + 1, sizeof(double*));
  if (!*z || !*h) return OR_ENOMEM;
  for (int l = 0; l <= nl; ++l) (*h)[l] = (double*)calloc(sizes[l], sizeof(double));
  for (int l = 0; l < nl; ++l) (*z)[l] = (double*)calloc(sizes[l + 1], sizeof(double));
  return OR_OK;
}

static void free_layers(int nl, double** z, double** h) {
  for (int l = 0; l <= nl; ++l) free(h[l]);
  for (int l = 0; l < nl; ++l) free(z[l]);
  free(z);
  free(h);
}

int or_mlp_forward(const int* sizes, int nl, const double* params, const double* x, int batch, double* y,
                   double* acts) {
  (void)acts;
  if (nl < 1 || batch < 0) return OR_EINVAL;
  double **z, **h;
  if (alloc_layers(sizes, nl, &z, &h) != OR_OK) return OR_ENOMEM;
  for (int s = 0; s < batch; ++s) {
    forward_one(sizes, nl, params, x + (long)s * sizes[0], z, h);
    memcpy(y + (long)s * sizes[nl], h[nl], sizeof(double) * sizes[nl]);
  }
  free_layers(nl, z, h);
  return OR_OK;
}

int or_mlp_loss_grad(const int* sizes, int nl, const double* params, const double* x, const double* target,
                     int batch, double* loss, double* grad) {
  if (nl < 1 || batch < 1) return OR_EINVAL;
  long np = param_count(sizes, nl);
  memset(grad, 0, sizeof(double) * np);
  double **z, **h;
  if (alloc_layers(sizes, nl, &z, &h) != OR_OK) return OR_ENOMEM;
  int maxw = 0;
  for (int l = 0; l <= nl; ++l) if (sizes[l] > maxw) maxw = sizes[l];
  double* delta = (double*)calloc(maxw, sizeof(double));
  double* prev = (double*)calloc(maxw, sizeof(double));
  int nout = sizes[nl];
  double scale = 1.0 / ((double)batch * nout);
  double total = 0;
  /* offsets of each layer's parameters */
  long* off = (long*)calloc(nl, sizeof(long));
  for (int l = 1; l < nl; ++l) off[l] = off[l - 1] + (long)sizes[l] * sizes[l - 1] + sizes[l];
  for (int s = 0; s < batch; ++s) {
    forward_one(sizes, nl, params, x + (long)s * sizes[0], z, h);
    const double* t = target + (long)s * nout;
    for (int o = 0; o < nout; ++o) {
      double d = h[nl][o] - t[o];
      total += d * d;
      delta[o] = 2.0 * d * scale; /* dL/dz of the linear output layer */
    }
    for (int l = nl - 1; l >= 0; --l) {
      int in = sizes[l], out = sizes[l + 1];
      double* gW = grad + off[l];
      double* gb = gW + (long)out * in;
      const double* W = params + off[l];
      for (int o = 0; o < out; ++o) {
        gb[o] += delta[o];
        for (int i = 0; i < in; ++i) gW[(long)o * in + i] += delta[o] * h[l][i];
      }
      if (l > 0) {
        for (int i = 0; i < in; ++i) {
          double acc = 0;
          for (int o = 0; o < out; ++o) acc += W[(long)o * in + i] * delta[o];
          prev[i] = acc * gelu_d(z[l - 1][i]);
        }
        memcpy(delta, prev, sizeof(double) * in);
      }
    }
  }
  *loss = total * scale;
  free(off);
  free(delta);
  free(prev);
  free_layers(nl, z, h);
  return OR_OK;
}

int or_adam_step(int n, double* params, double* m, double* v, const double* grad, double lr, double beta1,
                 double beta2, double eps, int t) {
  if (n < 0 || t < 1) return OR_EINVAL;
  double c1 = 1.0 - pow(beta1, t), c2 = 1.0 - pow(beta2, t);
  for (int i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
    double mh = m[i] / c1, vh = v[i] / c2;
    params[i] -= lr * mh / (sqrt(vh) + eps);
  }
  return OR_OK;
}
