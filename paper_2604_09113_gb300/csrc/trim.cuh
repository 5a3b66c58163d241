// The trimmed cell as the trainers integrate it (Sec. 2.2.3, height-function
// form): the solid intervals of xi2 at a given xi1 for the bilinear threshold
// of Sec. 2.1.2 (closed-form roots), and the Legendre polynomials and their
// antiderivatives with which the moments of the solid part are integrated
// exactly along xi2.  Shared by the host trainer and the GPU trainer.
#pragma once

#include <math.h>

#ifndef ROMB_HD
#define ROMB_HD __host__ __device__
#endif

// Legendre P_0..P_n at t in [-1, 1]
ROMB_HD inline void legendre(int n, double t, double* P) {
  P[0] = 1.0;
  if (n >= 1) P[1] = t;
  for (int k = 2; k <= n; ++k) P[k] = ((2 * k - 1) * t * P[k - 1] - (k - 1) * P[k - 2]) / k;
}

// int_0^y P_b(2s - 1) ds for b = 0..n  (needs P up to n+1)
ROMB_HD inline void legendre_antideriv(int n, double y, double* out) {
  double P[64];
  const double t = 2.0 * y - 1.0;
  legendre(n + 1, t, P);
  out[0] = y;
  for (int b = 1; b <= n; ++b) out[b] = 0.5 * (P[b + 1] - P[b - 1]) / (2 * b + 1);
}

// solid intervals of [0,1] in xi2 at xi1 = x (bilinear threshold)
ROMB_HD inline int solid_y(int family, const double* mu, double x, double* lo, double* hi) {
  const double a = mu[0] * (1.0 - x) + mu[1] * x;
  const double b = (mu[2] - mu[0]) * (1.0 - x) + (mu[3] - mu[1]) * x;
  int n = 0;
  if (family == 0) {
    const double A = 1.0 - b * b, B = -1.0 - 2.0 * a * b, C = (x - 0.5) * (x - 0.5) + 0.25 - a * a;
    const double disc = B * B - 4.0 * A * C;
    if (disc <= 0.0) {
      lo[0] = 0.0;
      hi[0] = 1.0;
      return 1;
    }
    const double s = sqrt(disc), r1 = (-B - s) / (2.0 * A), r2 = (-B + s) / (2.0 * A);
    if (r1 > 0.0 && fmin(r1, 1.0) > 0.0) {
      lo[n] = 0.0;
      hi[n++] = fmin(r1, 1.0);
    }
    if (r2 < 1.0 && fmax(r2, 0.0) < 1.0) {
      lo[n] = fmax(r2, 0.0);
      hi[n++] = 1.0;
    }
    return n;
  }
  double L[2], H[2];
  int m = 0;
  const double t = fabs(x - 0.5) - a;
  double l1 = 0, h1 = 0;
  bool has1 = true;
  if (b > 0.0) {
    l1 = t / b;
    h1 = 2.0;
  } else if (b < 0.0) {
    l1 = -1.0;
    h1 = t / b;
  } else if (t < 0.0) {
    l1 = -1.0;
    h1 = 2.0;
  } else {
    has1 = false;
  }
  if (has1 && fmin(h1, 1.0) > fmax(l1, 0.0)) {
    L[m] = fmax(l1, 0.0);
    H[m++] = fmin(h1, 1.0);
  }
  const double l2 = (0.5 - a) / (1.0 + b), h2 = (0.5 + a) / (1.0 - b);
  if (fmin(h2, 1.0) > fmax(l2, 0.0)) {
    L[m] = fmax(l2, 0.0);
    H[m++] = fmin(h2, 1.0);
  }
  if (m == 2 && L[1] < L[0]) {
    const double tl = L[0], th = H[0];
    L[0] = L[1];
    H[0] = H[1];
    L[1] = tl;
    H[1] = th;
  }
  for (int i = 0; i < m; ++i) {
    if (n > 0 && L[i] <= hi[n - 1]) hi[n - 1] = fmax(hi[n - 1], H[i]);
    else {
      lo[n] = L[i];
      hi[n++] = H[i];
    }
  }
  return n;
}

