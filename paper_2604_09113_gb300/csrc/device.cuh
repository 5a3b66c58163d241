// Device-side helpers of romb: 1D bases, cell maps and the per-launch
// parameter block (passed by value to every per-cell kernel).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "romb_internal.cuh"
#include "trim.cuh"

#define ROMB_NQ 24   // Gauss points per edge for the coarse functionals

struct CellParams {
  int p, m, basis, nB, nI, nU, nx, ny, ncells, q, nL;
  unsigned dmask;
  // layouts with absent cells or clamped cell edges (null for the full rectangle)
  const int* cell_grid;         // [ncells] grid index c = cx + nx cy of each cell
  const int* grid_cell;         // [nx*ny] cell of each grid position, -1 absent
  const uint8_t* node_fixed;    // [skeleton nodes] clamped, or of no present cell
  double E, nu, rho, lam, mu;   // plane-stress Lame parameters
  double gll[ROMB_MAX_P + 1];   // degree-p GLL nodes of the cell basis
  double bw[ROMB_MAX_P + 1];    // their barycentric weights 1 / prod_{j != i} (gll_i - gll_j)
  double mw[5];                 // the same for the equispaced map nodes a/m
  double gq_x[ROMB_NQ], gq_w[ROMB_NQ];
  double bq[ROMB_NQ][ROMB_MAX_P + 1];        // cell basis (1D) at the Gauss points
  int uslot[8 * ROMB_MAX_P];
  int islot[2 * (ROMB_MAX_P - 1) * (ROMB_MAX_P - 1)];
  int uslot_of_node[(ROMB_MAX_P + 1) * (ROMB_MAX_P + 1)];
  // 1D map basis (order m, equispaced nodes) and its derivative at the edge
  // Gauss points gq_x[q], q < ROMB_NQ, and at the midpoint (q = ROMB_NQ)
  double mq[ROMB_NQ + 1][5], dmq[ROMB_NQ + 1][5];
};

// Values and derivatives of the n+1 Lagrange polynomials on `nodes` at t.
__host__ __device__ inline void lagrange1d(int n, const double* nodes, double t, double* v, double* d) {
  for (int i = 0; i <= n; ++i) {
    double den = 1.0, val = 1.0, der = 0.0;
    for (int j = 0; j <= n; ++j) {
      if (j == i) continue;
      den *= nodes[i] - nodes[j];
      der = der * (t - nodes[j]) + val;
      val *= t - nodes[j];
    }
    v[i] = val / den;
    if (d) d[i] = der / den;
  }
}

// Degree-p Bernstein polynomials and derivatives at t.
__host__ __device__ inline void bernstein1d(int p, double t, double* v, double* d) {
  double binom = 1.0;
  for (int i = 0; i <= p; ++i) {
    if (i > 0) binom = binom * (p - i + 1) / i;
    double ti = 1.0, si = 1.0;
    for (int k = 0; k < i; ++k) ti *= t;
    for (int k = 0; k < p - i; ++k) si *= 1.0 - t;
    v[i] = binom * ti * si;
    if (d) {
      double dv = 0.0;
      if (i > 0) {
        double a = 1.0;
        for (int k = 0; k < i - 1; ++k) a *= t;
        dv += binom * i * a * si;
      }
      if (i < p) {
        double b = 1.0;
        for (int k = 0; k < p - i - 1; ++k) b *= 1.0 - t;
        dv -= binom * (p - i) * ti * b;
      }
      d[i] = dv;
    }
  }
}

__host__ __device__ inline void cell_basis1d(const CellParams& P, double t, double* v, double* d) {
  if (P.basis == 0) lagrange1d(P.p, P.gll, t, v, d);
  else bernstein1d(P.p, t, v, d);
}

// The order-m Lagrange basis on the equispaced map nodes a/m, values and
// derivatives at t (the arithmetic of lagrange1d with the nodes formed in
// place, no local node table).
__host__ __device__ inline void map_basis1d(int m, double t, double* v, double* d) {
  for (int i = 0; i <= m; ++i) {
    const double ni = (double)i / m;
    double den = 1.0, val = 1.0, der = 0.0;
    for (int j = 0; j <= m; ++j) {
      if (j == i) continue;
      const double nj = (double)j / m;
      den *= ni - nj;
      der = der * (t - nj) + val;
      val *= t - nj;
    }
    v[i] = val / den;
    if (d) d[i] = der / den;
  }
}

// Map control point (a, b) of cell (cx, cy) from the shared grid.
__device__ inline const double* ctrl_pt(const double* ctrl, int nx, int m, int cx, int cy, int a, int b) {
  return ctrl + 2 * ((long long)(m * cy + b) * (m * nx + 1) + (m * cx + a));
}

// Physical point and Jacobian J[r][s] = dx_r/dxi_s of the cell map at xi.
__device__ inline void map_eval(const double* ctrl, int nx, int m, int cx, int cy, double x1, double x2, double* x,
                                double J[2][2]) {
  double v1[5], d1[5], v2[5], d2[5];
  map_basis1d(m, x1, v1, d1);
  map_basis1d(m, x2, v2, d2);
  x[0] = x[1] = 0.0;
  J[0][0] = J[0][1] = J[1][0] = J[1][1] = 0.0;
  for (int b = 0; b <= m; ++b)
    for (int a = 0; a <= m; ++a) {
      const double* X = ctrl_pt(ctrl, nx, m, cx, cy, a, b);
      const double w = v1[a] * v2[b], w1 = d1[a] * v2[b], w2 = v1[a] * d2[b];
      for (int r = 0; r < 2; ++r) {
        x[r] += w * X[r];
        J[r][0] += w1 * X[r];
        J[r][1] += w2 * X[r];
      }
    }
}

// Physical point and tangent dx/dt of the cell map on lattice-cell edge e
// (0 left, 1 right, 2 bottom, 3 top; t runs along the free coordinate) at the
// tabulated edge point q: on an edge one 1D factor of the tensor map basis is a
// Kronecker delta, so only the m+1 control points of that edge contribute.
__device__ inline void edge_map_point(const CellParams& P, const double* ctrl, int cx, int cy, int e, int q,
                                      double* x, double* tan) {
  const int m = P.m;
  x[0] = x[1] = tan[0] = tan[1] = 0.0;
  for (int s = 0; s <= m; ++s) {
    const int a = e == 0 ? 0 : e == 1 ? m : s;
    const int b = e == 2 ? 0 : e == 3 ? m : s;
    const double* X = ctrl_pt(ctrl, P.nx, m, cx, cy, a, b);
    const double w = P.mq[q][s], dw = P.dmq[q][s];
    x[0] = fma(w, X[0], x[0]);
    x[1] = fma(w, X[1], x[1]);
    tan[0] = fma(dw, X[0], tan[0]);
    tan[1] = fma(dw, X[1], tan[1]);
  }
}

// Grid position of cell `cell` (the cells are the present ones of the grid).
__device__ inline void cell_xy(const CellParams& P, long long cell, int* cx, int* cy) {
  const long long g = P.cell_grid ? P.cell_grid[cell] : cell;
  *cx = (int)(g % P.nx);
  *cy = (int)(g / P.nx);
}

// Cell at grid position (cx, cy): -1 outside the grid or absent.
__device__ inline long long cell_at(const CellParams& P, int cx, int cy) {
  if (cx < 0 || cy < 0 || cx >= P.nx || cy >= P.ny) return -1;
  const long long g = cx + (long long)P.nx * cy;
  return P.grid_cell ? P.grid_cell[g] : g;
}

__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Solid sub-intervals [lo, hi] of cell edge e (0 left, 1 right, 2 bottom, 3 top)
// in the edge parameter: the trimmed line of a vertical edge is the line
// xi1 = 0 or 1; a horizontal edge is the same line of the cell with xi1 and
// xi2 exchanged, i.e. with mu_2 and mu_3 exchanged (every family is symmetric
// under the exchange).  Returns the number of intervals (<= ROMB_MAX_IV).
__device__ inline int edge_solid_dev(int family, const double* mu4, int e, double* lo, double* hi) {
  const double c0 = (e == 1 || e == 3) ? 1.0 : 0.0;
  double m[4] = {mu4[0], mu4[1], mu4[2], mu4[3]};
  if (e >= 2) {
    m[1] = mu4[2];
    m[2] = mu4[1];
  }
  return solid_y(family, m, c0, lo, hi);
}

// Host helper: fill a CellParams from the context.
void fill_cell_params(const romb_ctx* c, CellParams* P);
