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

#ifndef ROMB_MAX_IV
#define ROMB_MAX_IV 4   // solid intervals of one line, at most
#endif

// The TPMS level sets of Table GEO tpms (families 2..5: Schwarz Diamond,
// Schwarz Primitive, Schoen FRD with the sign flipped, Schoen IWP) on the line
// xi1 = x: phi0 = al cos(2 pi y) + be cos(4 pi y) + ga.
ROMB_HD inline void tpms_line(int family, double x, double* al, double* be, double* ga) {
  const double c1 = cos(2.0 * M_PI * x), d1 = cos(4.0 * M_PI * x);
  if (family == 2) {
    *al = c1; *be = 0.0; *ga = 0.0;
  } else if (family == 3) {
    *al = 1.0; *be = 0.0; *ga = c1 - 1.0;
  } else if (family == 4) {
    *al = 4.0 * c1; *be = -(d1 + 1.0); *ga = -d1;
  } else {
    *al = 2.0 * (c1 + 1.0); *be = -1.0; *ga = 2.0 * c1 - d1 - 1.0;
  }
}

// Solid intervals {y in [0,1] : phi0(x, y) < a + b y} of a TPMS line.  The
// sign changes of g = phi0 - a - b y are isolated with the bound
// M2 = (2 pi)^2 |al| + (4 pi)^2 |be| on |g''|: an interval of length h with
// equal end signs and min |g| > M2 h^2 / 8 holds no root, one with a sign
// change and |g'| > M2 h at an end holds exactly one, others are halved down
// to TPMS_HMIN (there: one root if the end signs differ, none otherwise);
// each root is found to machine precision by Newton steps kept inside its
// bracket (a step that leaves the bracket or shrinks it by less than half
// is replaced by bisection), and pairs closer than TPMS_HMIN cancel (a
// tangential touch, where rounding makes the sign noisy).
#define TPMS_HMIN 1e-10
ROMB_HD inline int tpms_solid_y(int family, double a, double b, double x, double* lo, double* hi) {
  double al, be, ga;
  tpms_line(family, x, &al, &be, &ga);
  const double w = 2.0 * M_PI;
  auto g = [&](double y) { return al * cos(w * y) + be * cos(2.0 * w * y) + ga - a - b * y; };
  auto dg = [&](double y) { return -w * al * sin(w * y) - 2.0 * w * be * sin(2.0 * w * y) - b; };
  const double M2 = w * w * fabs(al) + 4.0 * w * w * fabs(be);
  double roots[16];
  int nr = 0;
  const bool solid0 = g(0.0) < 0.0;
  if (M2 == 0.0) {
    if (b != 0.0) {
      const double y0 = (ga - a) / b;
      if (y0 > 0.0 && y0 < 1.0) roots[nr++] = y0;
    }
  } else {
    const int NG = 32;
    double gl = g(0.0);
    for (int i = 0; i < NG; ++i) {
      const double u0 = (double)i / NG, v0 = (double)(i + 1) / NG, gr = g(v0);
      // depth-first halving of [u0, v0]; at most 29 levels down to TPMS_HMIN
      double su[40], sv[40], sgu[40], sgv[40];
      int sp = 0;
      su[0] = u0; sv[0] = v0; sgu[0] = gl; sgv[0] = gr;
      sp = 1;
      while (sp > 0) {
        --sp;
        const double u = su[sp], v = sv[sp], gu = sgu[sp], gv = sgv[sp], h = v - u;
        if ((gu < 0.0) != (gv < 0.0)) {
          if (fabs(dg(u)) > M2 * h || fabs(dg(v)) > M2 * h || h < TPMS_HMIN) {
            double l = u, r = v;
            const bool neg = gu < 0.0;
            double y = 0.5 * (l + r);
            for (int it = 0; it < 200; ++it) {
              const double gy = g(y);
              if (gy == 0.0) {
                l = r = y;
                break;
              }
              if ((gy < 0.0) == neg) l = y;
              else r = y;
              const double w0 = r - l, d = dg(y);
              double yn = d != 0.0 ? y - gy / d : 0.5 * (l + r);
              if (!(yn > l && yn < r) || (it > 0 && fabs(yn - y) > 0.5 * w0)) yn = 0.5 * (l + r);
              if (yn <= l || yn >= r || yn == y) break;
              y = yn;
            }
            if (nr > 0 && y - roots[nr - 1] < TPMS_HMIN) --nr;
            else if (nr < 16) roots[nr++] = y;
            continue;
          }
        } else if (fmin(fabs(gu), fabs(gv)) > M2 * h * h / 8.0 || h < TPMS_HMIN) {
          continue;
        }
        if (sp + 2 > 40) continue;   // unreachable: the depth stays below 30
        const double m = 0.5 * (u + v), gm = g(m);
        su[sp] = m; sv[sp] = v; sgu[sp] = gm; sgv[sp] = gv; ++sp;
        su[sp] = u; sv[sp] = m; sgu[sp] = gu; sgv[sp] = gm; ++sp;
      }
      gl = gr;
    }
  }
  int n = 0;
  bool solid = solid0;
  double start = 0.0;
  for (int k = 0; k <= nr; ++k) {
    const double end = k < nr ? roots[k] : 1.0;
    if (solid && end > start && n < ROMB_MAX_IV) {
      lo[n] = start;
      hi[n++] = end;
    }
    start = end;
    solid = !solid;
  }
  return n;
}

// solid intervals of [0,1] in xi2 at xi1 = x (bilinear threshold); at most
// ROMB_MAX_IV
ROMB_HD inline int solid_y(int family, const double* mu, double x, double* lo, double* hi) {
  const double a = mu[0] * (1.0 - x) + mu[1] * x;
  const double b = (mu[2] - mu[0]) * (1.0 - x) + (mu[3] - mu[1]) * x;
  if (family >= 2) return tpms_solid_y(family, a, b, x, lo, hi);
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

