/*
 * mlp.c -- FP64 reference of the small regime-classifier network used by the
 * learned path: 10 inputs -> 64 tanh -> 64 tanh -> 1 linear output, trained
 * with the mean squared error.  The paper has no network; this is the plain
 * definition (matrix products, tanh, chain rule) that the GPU training and
 * inference kernels are checked against.  TEST INFRASTRUCTURE ONLY.
 *
 * Packed parameter vector, row-major:
 *   W1[64][10], b1[64], W2[64][64], b2[64], W3[64], b3
 */
#include <math.h>
#include <stdlib.h>

#define NIN 10
#define NH 64

static void unpack(const double* P, const double** W1, const double** b1,
                   const double** W2, const double** b2, const double** W3,
                   const double** b3) {
  *W1 = P;
  *b1 = *W1 + NH * NIN;
  *W2 = *b1 + NH;
  *b2 = *W2 + NH * NH;
  *W3 = *b2 + NH;
  *b3 = *W3 + NH;
}

/* h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = W3 h2 + b3 */
static double forward_one(const double* P, const double* x, double* h1,
                          double* h2) {
  const double *W1, *b1, *W2, *b2, *W3, *b3;
  unpack(P, &W1, &b1, &W2, &b2, &W3, &b3);
  for (int j = 0; j < NH; ++j) {
    double s = b1[j];
    for (int i = 0; i < NIN; ++i) s += W1[j * NIN + i] * x[i];
    h1[j] = tanh(s);
  }
  for (int j = 0; j < NH; ++j) {
    double s = b2[j];
    for (int i = 0; i < NH; ++i) s += W2[j * NH + i] * h1[i];
    h2[j] = tanh(s);
  }
  double y = b3[0];
  for (int i = 0; i < NH; ++i) y += W3[i] * h2[i];
  return y;
}

void orc_mlp_forward(int n, const double* P, const double* X, double* y) {
  double h1[NH], h2[NH];
  for (int s = 0; s < n; ++s) y[s] = forward_one(P, X + (long)s * NIN, h1, h2);
}

/* L = (1/n) sum_s (y_s - t_s)^2 and dL/dP by the chain rule. */
double orc_mlp_loss_grad(int n, const double* P, const double* X,
                         const double* t, double* G) {
  const double *W1, *b1, *W2, *b2, *W3, *b3;
  unpack(P, &W1, &b1, &W2, &b2, &W3, &b3);
  double* gW1 = G;
  double* gb1 = gW1 + NH * NIN;
  double* gW2 = gb1 + NH;
  double* gb2 = gW2 + NH * NH;
  double* gW3 = gb2 + NH;
  double* gb3 = gW3 + NH;
  const long np = (long)NH * NIN + NH + NH * NH + NH + NH + 1;
  for (long i = 0; i < np; ++i) G[i] = 0.0;
  double loss = 0.0;
  double h1[NH], h2[NH], d2[NH], d1[NH];
  for (int s = 0; s < n; ++s) {
    const double* x = X + (long)s * NIN;
    const double y = forward_one(P, x, h1, h2);
    const double e = y - t[s];
    loss += e * e;
    const double dy = 2.0 * e / n;
    gb3[0] += dy;
    for (int i = 0; i < NH; ++i) {
      gW3[i] += dy * h2[i];
      d2[i] = dy * W3[i] * (1.0 - h2[i] * h2[i]);
    }
    for (int j = 0; j < NH; ++j) {
      gb2[j] += d2[j];
      for (int i = 0; i < NH; ++i) gW2[j * NH + i] += d2[j] * h1[i];
    }
    for (int i = 0; i < NH; ++i) {
      double s2 = 0.0;
      for (int j = 0; j < NH; ++j) s2 += W2[j * NH + i] * d2[j];
      d1[i] = s2 * (1.0 - h1[i] * h1[i]);
    }
    for (int j = 0; j < NH; ++j) {
      gb1[j] += d1[j];
      for (int i = 0; i < NIN; ++i) gW1[j * NIN + i] += d1[j] * x[i];
    }
  }
  return loss / n;
}
