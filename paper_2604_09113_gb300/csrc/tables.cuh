// Small host-side tables shared by the romb kernels: GLL nodes, local slot
// orderings and the hi/lo rounding used for the split-precision operands.
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#include "romb_internal.cuh"

// Degree-n Gauss-Lobatto-Legendre nodes on [0,1]: the end points and the roots
// of P_n'(2x-1), by Newton iteration from Chebyshev-Gauss-Lobatto guesses.
static inline void gll_nodes01(int n, double* x) {
  x[0] = 0.0;
  x[n] = 1.0;
  for (int i = 1; i < n; ++i) {
    double t = -cos(M_PI * i / n);
    for (int it = 0; it < 100; ++it) {
      // P_n, P_n', P_n'' by the three-term recurrence
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      // p1 = P_n(t), p0 = P_{n-1}(t)
      const double dp = n * (t * p1 - p0) / (t * t - 1.0);
      const double d2p = (2.0 * t * dp - n * (n + 1) * p1) / (1.0 - t * t);
      const double dt = dp / d2p;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    x[i] = 0.5 * (t + 1.0);
  }
  // sort ascending (Newton keeps the ordering of the guesses)
}

// Gauss-Legendre nodes/weights on [0,1] (Newton on P_n).
static inline void gauss01(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double t = -cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      dp = n * (t * p1 - p0) / (t * t - 1.0);
      const double dt = p1 / dp;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      dp = n * (t * p1 - p0) / (t * t - 1.0);
    }
    x[i] = 0.5 * (t + 1.0);
    w[i] = 1.0 / ((1.0 - t * t) * dp * dp);   // 2/((1-t^2)P'^2) scaled by 1/2
  }
}

// Round a float to TF32 (10 explicit mantissa bits, nearest, ties away).
static inline float tf32_round(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return f;
  u += 0x1000u;
  u &= 0xffffe000u;
  float r;
  memcpy(&r, &u, 4);
  return r;
}

// Local slot orderings of a degree-p cell: interior DoFs (nodes with
// 0 < a, b < p) and skeleton DoFs (boundary nodes), each in increasing local
// DoF index 2k + i.
struct LocalTables {
  int islot[2 * (ROMB_MAX_P - 1) * (ROMB_MAX_P - 1)];
  int uslot[8 * ROMB_MAX_P];
  int uslot_of_node[(ROMB_MAX_P + 1) * (ROMB_MAX_P + 1)];   // skeleton rank of a boundary node (-1 interior)
};

static inline LocalTables make_local_tables(int p) {
  LocalTables T;
  int ni = 0, nu = 0;
  for (int k = 0; k < (p + 1) * (p + 1); ++k) {
    const int a = k % (p + 1), b = k / (p + 1);
    const bool bnd = a == 0 || a == p || b == 0 || b == p;
    T.uslot_of_node[k] = bnd ? nu / 2 : -1;
    for (int i = 0; i < 2; ++i) {
      if (bnd) T.uslot[nu++] = 2 * k + i;
      else T.islot[ni++] = 2 * k + i;
    }
  }
  return T;
}
