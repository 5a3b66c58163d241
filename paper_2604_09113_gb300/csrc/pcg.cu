// PCG on the interface Schur system S u = f (Eq. BDDC system) with the BDDC
// preconditioner (Eq. BDDC preconditioner, Algorithm 1), then the interior
// recovery u_I = K_II^-1 (f_I - K_IU u^(i)) (Sec. 3.2).
//
// Vectors live on the skeleton: DoF 2*id + comp of skeleton node id (nodes on
// horizontal grid lines first, then the remaining nodes of vertical lines).
// R^(i) (gather) and R^(i)T (sum over the sharing cells) are index maps; the
// sums are gathers in a fixed cell order, so every result is deterministic.
// Per iteration and cell: q = S p (matvec), z = D F D r + D Psi S_C^-1 Psi^T D r.
#include <math.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "bulk.cuh"
#include "device.cuh"
#include "tables.cuh"

#define RED_BLOCKS 256

// skeleton node id -> grid node (gx, gy)
__device__ inline void skel_node_xy(long long id, int p, int nx, long long NH, int* gx, int* gy) {
  if (id < NH) {
    *gy = p * (int)(id / (p * nx + 1));
    *gx = (int)(id % (p * nx + 1));
  } else {
    long long t = id - NH;
    const int b = (int)(t % (p - 1)) + 1;
    t /= (p - 1);
    *gx = p * (int)(t % (nx + 1));
    *gy = p * (int)(t / (nx + 1)) + b;
  }
}

// skeleton node `id` at grid node (gx, gy) carries no unknown: clamped (or,
// in layouts with absent cells, clamped or of no present cell)
__device__ inline bool dir_node(const CellParams& P, long long id, int gx, int gy) {
  if (P.node_fixed) return P.node_fixed[id] != 0;
  return ((P.dmask & 1) && gx == 0) || ((P.dmask & 2) && gx == P.p * P.nx) || ((P.dmask & 4) && gy == 0) ||
         ((P.dmask & 8) && gy == P.p * P.ny);
}

// out[dof] = sum over cells sharing the node of loc[cell][slot]  (R^T of a cell-local field)
__global__ void skel_gather_kernel(CellParams P, const double* __restrict__ loc, long long nnodes,
                                   double* __restrict__ out) {
  const int p = P.p, nx = P.nx, ny = P.ny, NU = P.nU;
  const long long NH = (long long)(ny + 1) * (p * nx + 1);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < nnodes;
       id += (long long)gridDim.x * blockDim.x) {
    int gx, gy;
    skel_node_xy(id, p, nx, NH, &gx, &gy);
    double s0 = 0.0, s1 = 0.0;
    if (!dir_node(P, id, gx, gy)) {
      const int cx1 = gx / p, cy1 = gy / p;
      for (int dy = (gy % p == 0) ? -1 : 0; dy <= 0; ++dy)
        for (int dx = (gx % p == 0) ? -1 : 0; dx <= 0; ++dx) {
          const int cx = cx1 + dx, cy = cy1 + dy;
          const long long cell = cell_at(P, cx, cy);
          if (cell < 0) continue;
          const int k = (gx - p * cx) + (p + 1) * (gy - p * cy);
          const int u = 2 * P.uslot_of_node[k];
          const double* l = loc + cell * NU;
          s0 += l[u];
          s1 += l[u + 1];
        }
    }
    out[2 * id] = s0;
    out[2 * id + 1] = s1;
  }
}

// y_loc = M_c v_loc for every cell (M_c a dense symmetric nU x nU cell matrix:
// S, or D F D), or c_loc = Phi_c^T v_loc (COARSE).  Persistent CTAs
// take the cells blockIdx.x, blockIdx.x + gridDim.x, ...; each streams its
// cells' M_c (and Phi_c) and index rows through a CA_STAGES-deep shared ring
// filled by bulk copies, so the HBM stream overlaps the FP64 work.  Row r of
// y is summed by two lanes (r, half of k) of one warp, one shuffle apart: every
// FP64 instruction has all its lanes busy.  One barrier per cell releases the
// stage and publishes the next cell's gathered v.
#define CA_STAGES 3
// modes: y = M v (the operators S and D F D); c = Phi^T v (coarse restriction)
#define CA_MATVEC 0
#define CA_RESTRICT 2
// The element type T of M and Phi: double, or float for the preconditioner's
// operators (D F D and Phi) of the split-precision forms; v, y and c stay
// double in memory, the products and sums run in T.
template <int P>
struct CellApplyShape {
  static constexpr int NU = 8 * P, WARPS = (NU + 15) / 16, THREADS = 32 * WARPS;
  static constexpr int stage_bytes(int mode, int esize) {
    return (mode != CA_RESTRICT ? NU * NU * esize : 0) + (mode != CA_MATVEC ? NU * 20 * esize : 0) + NU * 4;
  }
};

template <int P, int MODE, typename T>
__global__ void __launch_bounds__(CellApplyShape<P>::THREADS) cell_apply_kernel(
    int ncells, const T* __restrict__ M, const int* __restrict__ umap, const double* __restrict__ v,
    double* __restrict__ yloc, const T* __restrict__ Phi, double* __restrict__ cloc, int* __restrict__ err) {
  using Sh = CellApplyShape<P>;
  constexpr bool HAS_M = MODE != CA_RESTRICT, COARSE = MODE != CA_MATVEC;
  constexpr int NU = Sh::NU, H = NU / 2, NT = Sh::THREADS, ES = (int)sizeof(T);
  constexpr int MB = HAS_M ? NU * NU * ES : 0, PB = COARSE ? NU * 20 * ES : 0, SB = MB + PB + NU * 4;
  extern __shared__ __align__(16) unsigned char ring[];
  __shared__ uint64_t full[CA_STAGES];
  __shared__ T sv[2][NU];
  __shared__ T cpart[2][4][20];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nmine = blockIdx.x < ncells ? (ncells - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  auto cell_of = [&](int j) { return (long long)blockIdx.x + (long long)j * gridDim.x; };
  auto issue = [&](int j) {
    const long long cell = cell_of(j);
    unsigned char* st = ring + (size_t)(j % CA_STAGES) * SB;
    uint64_t* bar = &full[j % CA_STAGES];
    mbar_expect_tx(bar, SB);
    if (HAS_M) bulk_g2s(st, M + cell * NU * NU, MB, bar);
    if (COARSE) bulk_g2s(st + MB, Phi + cell * NU * 20, PB, bar);
    static_assert(MB % 16 == 0 && PB % 16 == 0 && (NU * 4) % 16 == 0, "bulk copies of whole 16-byte units");
    bulk_g2s(st + MB + PB, umap + cell * NU, NU * 4, bar);
  };
  if (tid == 0) {
    for (int s = 0; s < CA_STAGES; ++s) mbar_init(&full[s], 1);
    mbar_init_fence();
    for (int j = 0; j < CA_STAGES && j < nmine; ++j) issue(j);
  }
  __syncthreads();
  // v at the first cell's skeleton slots
  bool ok = true;
  if (nmine > 0) {
    ok = mbar_wait(&full[0], 0);
    if (ok) {
      const int* us = reinterpret_cast<const int*>(ring + MB + PB);
      for (int u = tid; u < NU; u += NT) sv[0][u] = us[u] >= 0 ? (T)v[us[u]] : (T)0;
    }
  }
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicExch(err, 1);
    return;
  }
  const int r = 16 * warp + (lane & 15), q = lane >> 4;
  for (int j = 0; j < nmine; ++j) {
    const long long cell = cell_of(j);
    const unsigned char* st = ring + (size_t)(j % CA_STAGES) * SB;
    const T* Ms = reinterpret_cast<const T*>(st);
    const T* x = sv[j & 1];
    // y = M_c v: lane (r, q) sums k in [q H, q H + H) of M[k][r] v[k] (M symmetric)
    if (HAS_M) {
      T acc = 0;
      if (r < NU) {
        const T* mk = Ms + q * H * NU + r;
#pragma unroll 8
        for (int k = 0; k < H; ++k) acc = fma(mk[k * NU], x[q * H + k], acc);
      }
      acc += __shfl_xor_sync(0xffffffffu, acc, 16);
      if (q == 0 && r < NU) yloc[cell * NU + r] = (double)acc;
    }
    if (COARSE) {
      // c = Phi^T v: thread (j, part) sums a quarter of the slots
      const T* Ps = reinterpret_cast<const T*>(st + MB);
      for (int t = tid; t < 80; t += NT) {
        const int jj = t % 20, part = t / 20;
        T a = 0;
        for (int u = part * (NU / 4); u < (part + 1) * (NU / 4); ++u) a = fma(Ps[u * 20 + jj], x[u], a);
        cpart[j & 1][part][jj] = a;
      }
    }
    // next cell's v (its stage was issued CA_STAGES - 1 cells ago)
    if (j + 1 < nmine) {
      ok = mbar_wait(&full[(j + 1) % CA_STAGES], (uint32_t)(((j + 1) / CA_STAGES) & 1));
      if (ok) {
        const int* us = reinterpret_cast<const int*>(ring + (size_t)((j + 1) % CA_STAGES) * SB + MB + PB);
        for (int u = tid; u < NU; u += NT) sv[(j + 1) & 1][u] = us[u] >= 0 ? (T)v[us[u]] : (T)0;
      }
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(err, 1);
      return;
    }
    if (COARSE && tid < 20)
      cloc[cell * 20 + tid] =
          (double)((cpart[j & 1][0][tid] + cpart[j & 1][1][tid]) + (cpart[j & 1][2][tid] + cpart[j & 1][3][tid]));
    if (tid == 0 && j + CA_STAGES < nmine) issue(j + CA_STAGES);   // stage j % CA_STAGES is free
  }
}

// y_loc += Phi g_loc  (coarse prolongation, Algorithm 1); half-warp per cell.
// T = float (the split-precision forms): Phi g summed in FP32, then added.
template <typename T>
__global__ void __launch_bounds__(256) cell_prolong_kernel(int ncells, int NU, const T* __restrict__ Phi,
                                                            const int* __restrict__ cmap, const double* __restrict__ g,
                                                            double* __restrict__ yloc) {
  __shared__ T sg[16][20];
  const int hl = threadIdx.x & 15, slot = threadIdx.x >> 4;
  const long long cell0 = (long long)blockIdx.x * 16 + slot;
  const bool active = cell0 < ncells;
  const long long cell = active ? cell0 : 0;
  for (int j = hl; j < 20; j += 16) {
    const int k = active ? cmap[cell * 20 + j] : -1;
    sg[slot][j] = k >= 0 ? (T)g[k] : (T)0;
  }
  __syncwarp();
  if (!active) return;
  const T* Pc = Phi + cell * NU * 20;
  for (int u = hl; u < NU; u += 16) {
    if constexpr (sizeof(T) == 8) {
      double acc = yloc[cell * NU + u];
#pragma unroll
      for (int j = 0; j < 20; ++j) acc = fma(Pc[u * 20 + j], sg[slot][j], acc);
      yloc[cell * NU + u] = acc;
    } else {
      T acc = 0;
#pragma unroll
      for (int j = 0; j < 20; ++j) acc = fma(Pc[u * 20 + j], sg[slot][j], acc);
      yloc[cell * NU + u] += (double)acc;
    }
  }
}

// z[k] = sum over the cells owning coarse DoF k of c_loc[cell][slot] (fixed order)
__global__ void coarse_gather_kernel(const int* __restrict__ owners, long long ncoarse, const double* __restrict__ cloc,
                                     double* __restrict__ z) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < ncoarse;
       k += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < 4; ++t) {
      const int o = owners[4 * k + t];
      if (o >= 0) s += cloc[o];
    }
    z[k] = s;
  }
}

// deterministic dot products: fixed-size grid of partial sums, then one block
__global__ void dot_partial_kernel(const double* __restrict__ a, const double* __restrict__ b, long long n,
                                   double* __restrict__ part) {
  __shared__ double sw[8];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sw[w];
    part[blockIdx.x] = t;
  }
}

__global__ void dot_final_kernel(const double* __restrict__ part, int np, double* __restrict__ out) {
  __shared__ double sw[8];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sw[w];
    *out = t;
  }
}

// scalars: [0] rz, [1] pq, [2] rz_new, [3] rr
__global__ void pcg_update_x_r(long long n, const double* __restrict__ sc, double* __restrict__ x,
                               double* __restrict__ r, const double* __restrict__ p, const double* __restrict__ q) {
  const double alpha = sc[0] / sc[1];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, q[i], r[i]);
  }
}

__global__ void pcg_update_p(long long n, double* __restrict__ sc, double* __restrict__ p,
                             const double* __restrict__ z) {
  const double beta = sc[2] / sc[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

__global__ void pcg_shift_scalars(double* sc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) sc[0] = sc[2];
}

// Traction loads on the solid part of the loaded lattice edges (Eq. ELA
// constitutive: that = j t): per (cell, edge), f_s = t int b_s j dt over the
// edge's solid intervals by the ROMB_NQ-point Gauss rule, lanes over the
// Gauss points; j from the edge's own m+1 control points (the other factor of
// the tensor map basis is a Kronecker delta on the edge), b_s in barycentric
// form.  One warp per (cell, edge).
#define LQ_WARPS 4
__global__ void __launch_bounds__(32 * LQ_WARPS) loads_kernel(CellParams P, const double* __restrict__ ctrl,
                                                               const double* __restrict__ mu,
                                                               const int32_t* __restrict__ family,
                                                               const double* __restrict__ trac,
                                                               double* __restrict__ fU) {
  const int lane = threadIdx.x & 31;
  long long t = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int ncell_e[4] = {P.ny, P.ny, P.nx, P.nx};
  int e = 0;
  while (e < 4 && t >= ncell_e[e]) {
    t -= ncell_e[e];
    ++e;
  }
  if (e >= 4) return;
  const double t0 = trac[2 * e], t1 = trac[2 * e + 1];
  if (t0 == 0.0 && t1 == 0.0) return;
  const int p = P.p, nx = P.nx, ny = P.ny, m = P.m;
  const int j = (int)t;
  const int cx = e == 0 ? 0 : e == 1 ? nx - 1 : j;
  const int cy = e == 2 ? 0 : e == 3 ? ny - 1 : j;
  const long long cell = cell_at(P, cx, cy);
  if (cell < 0) return;   // absent cell: no edge here
  double lo[ROMB_MAX_IV], hi[ROMB_MAX_IV];
  const int nint = edge_solid_dev(family[cell], mu + 4 * cell, e, lo, hi);
  double Xe[5][2];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    if (q > m) break;
    const int a = e == 0 ? 0 : e == 1 ? m : q;
    const int b = e == 2 ? 0 : e == 3 ? m : q;
    const double* X = ctrl_pt(ctrl, nx, m, cx, cy, a, b);
    Xe[q][0] = X[0];
    Xe[q][1] = X[1];
  }
  double acc[ROMB_MAX_P + 1];
#pragma unroll
  for (int s_ = 0; s_ <= ROMB_MAX_P; ++s_) acc[s_] = 0.0;
  for (int k = lane; k < nint * ROMB_NQ; k += 32) {
    const int iv = k / ROMB_NQ, qq = k % ROMB_NQ;
    const double len = hi[iv] - lo[iv], tt = lo[iv] + len * P.gq_x[qq];
    double tg0 = 0.0, tg1 = 0.0;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      if (q > m) break;
      double val = 1.0, der = 0.0;
#pragma unroll
      for (int jn = 0; jn < 5; ++jn) {
        if (jn > m) break;
        if (jn == q) continue;
        const double dt = tt - (double)jn / m;
        der = der * dt + val;
        val *= dt;
      }
      der *= P.mw[q];
      tg0 = fma(der, Xe[q][0], tg0);
      tg1 = fma(der, Xe[q][1], tg1);
    }
    const double wj = len * P.gq_w[qq] * hypot(tg0, tg1);
    if (P.basis == 0) {
#pragma unroll
      for (int s_ = 0; s_ <= ROMB_MAX_P; ++s_) {
        if (s_ > p) break;
        double val = P.bw[s_];
#pragma unroll
        for (int jn = 0; jn <= ROMB_MAX_P; ++jn) {
          if (jn > p) break;
          if (jn != s_) val *= tt - P.gll[jn];
        }
        acc[s_] = fma(wj, val, acc[s_]);
      }
    } else {
      double bv[ROMB_MAX_P + 1];
      bernstein1d(p, tt, bv, nullptr);
#pragma unroll
      for (int s_ = 0; s_ <= ROMB_MAX_P; ++s_)
        if (s_ <= p) acc[s_] = fma(wj, bv[s_], acc[s_]);
    }
  }
#pragma unroll
  for (int s_ = 0; s_ <= ROMB_MAX_P; ++s_) {
    if (s_ > p) break;
    const double v = warp_sum(acc[s_]);
    if (lane == 0) {
      const int k = e == 0 ? (p + 1) * s_ : e == 1 ? p + (p + 1) * s_ : e == 2 ? s_ : s_ + (p + 1) * p;
      const int u = 2 * P.uslot_of_node[k];
      atomicAdd(&fU[cell * P.nU + u], v * t0);
      atomicAdd(&fU[cell * P.nU + u + 1], v * t1);
    }
  }
}

// Traction loads through the reduced model of the force integrals (Eq. SPEED
// L ext with the ROM of Sec. 4.2): per loaded boundary edge of a cell,
// theta_f by tensor Lagrange interpolation of the grid coefficients at the
// cell's thresholds (Algorithm 5), J_e = U_f theta_f, and the load of edge
// node s, f_s = t sum_k J_e[s][k] j(t_k), with j the edge Jacobian at the
// q+1 GLL nodes t_k of the edge (t_hat = j t interpolated there).  One warp
// per (cell, edge).
struct ForceRomDev {
  const double* U;    // [r_f][n_f]
  const double* At;   // [(r+1)^4][r_f]
  int rf, nf, r;
  double lo4[4], hi4[4];   // the model's (cluster's) box per threshold
  double g01[12];     // degree-r GLL nodes of [0, 1]
};
struct QNodes {
  double n[8];        // GLL nodes of degree q on [0, 1]
};
#define LR_WARPS 4
__global__ void __launch_bounds__(32 * LR_WARPS) loads_rom_kernel(CellParams P, QNodes QN,
                                                                   const ForceRomDev* __restrict__ tab,
                                                                   const int32_t* __restrict__ slot,
                                                                   const double* __restrict__ ctrl,
                                                                   const double* __restrict__ mu,
                                                                   const double* __restrict__ trac,
                                                                   double* __restrict__ fU) {
  // the edge nodes are copied to shared memory with static indices; the
  // model descriptors are read from the table in global memory by slot
  __shared__ double sq[8];
  __shared__ double wts[LR_WARPS][4][12];
  __shared__ double th[LR_WARPS][128];
  __shared__ double Jv[LR_WARPS][(ROMB_MAX_P + 1) * 8];
  __shared__ double jk[LR_WARPS][8];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 8; ++k) sq[k] = QN.n[k];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long t = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int ncell_e[4] = {P.ny, P.ny, P.nx, P.nx};
  int e = 0;
  while (e < 4 && t >= ncell_e[e]) {
    t -= ncell_e[e];
    ++e;
  }
  if (e >= 4) return;
  const double t0 = trac[2 * e], t1 = trac[2 * e + 1];
  if (t0 == 0.0 && t1 == 0.0) return;
  const int p = P.p, q = P.q, nx = P.nx, ny = P.ny, m = P.m;
  const int j = (int)t;
  const int cx = e == 0 ? 0 : e == 1 ? nx - 1 : j;
  const int cy = e == 2 ? 0 : e == 3 ? ny - 1 : j;
  const long long cell = cell_at(P, cx, cy);
  if (cell < 0) return;   // absent cell: no edge here
  const ForceRomDev& F = tab[slot[cell]];
  const int r = F.r, n1 = r + 1, rf = F.rf;
  if (lane < 4) {
    double nodes[12];
    for (int i = 0; i < n1; ++i) nodes[i] = F.lo4[lane] + (F.hi4[lane] - F.lo4[lane]) * F.g01[i];
    lagrange1d(r, nodes, mu[4 * cell + lane], wts[warp][lane], nullptr);
  }
  __syncwarp();
  // theta_f = A_f w(mu), the grid node g = g1 + n1 (g2 + n1 (g3 + n1 g4))
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int ng = n1 * n1 * n1 * n1;
  for (int g = 0; g < ng; ++g) {
    const int g1 = g % n1, g2 = (g / n1) % n1, g3 = (g / (n1 * n1)) % n1, g4 = g / (n1 * n1 * n1);
    const double w = wts[warp][0][g1] * wts[warp][1][g2] * wts[warp][2][g3] * wts[warp][3][g4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int jj = lane + 32 * u;
      if (jj < rf) acc[u] = fma(w, F.At[(long long)g * rf + jj], acc[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
    if (lane + 32 * u < rf) th[warp][lane + 32 * u] = acc[u];
  // edge Jacobian j = |dx/dt| at the q+1 interpolation nodes of the edge: on
  // an edge one factor of the tensor map basis is a Kronecker delta, so the
  // tangent is the derivative of the 1D map basis against the m+1 control
  // points of that edge
  if (lane <= q) {
    double v[5], d[5];
    map_basis1d(m, sq[lane], v, d);
    double tx = 0.0, ty = 0.0;
    for (int s = 0; s <= m; ++s) {
      const int a = e == 0 ? 0 : e == 1 ? m : s;
      const int b = e == 2 ? 0 : e == 3 ? m : s;
      const double* X = ctrl_pt(ctrl, nx, m, cx, cy, a, b);
      tx = fma(d[s], X[0], tx);
      ty = fma(d[s], X[1], ty);
    }
    jk[warp][lane] = hypot(tx, ty);
  }
  __syncwarp();
  // J_e[s][k] = sum_t U_f[t][(e (p+1) + s)(q+1) + k] theta_f[t]
  const int ne = (p + 1) * (q + 1);
  for (int i = lane; i < ne; i += 32) {
    const int col = e * ne + i;
    double sum = 0.0;
    for (int tt = 0; tt < rf; ++tt) sum = fma(F.U[(long long)tt * F.nf + col], th[warp][tt], sum);
    Jv[warp][i] = sum;
  }
  __syncwarp();
  if (lane <= p) {
    const int s_ = lane;
    double gsum = 0.0;
    for (int k = 0; k <= q; ++k) gsum = fma(Jv[warp][s_ * (q + 1) + k], jk[warp][k], gsum);
    const int k_ = e == 0 ? (p + 1) * s_ : e == 1 ? p + (p + 1) * s_ : e == 2 ? s_ : s_ + (p + 1) * p;
    const int u = 2 * P.uslot_of_node[k_];
    atomicAdd(&fU[cell * P.nU + u], gsum * t0);
    atomicAdd(&fU[cell * P.nU + u + 1], gsum * t1);
  }
}

// Body-force loads through the reduced model of the external-force
// integrals (volume term of Eq. SPEED L ext): per cell, theta_f at the cell's
// thresholds, V[k][k3] = (U_f theta_f) over the volume rows, b_hat = det J b
// at the (q+1)^2 interpolation nodes (Eq. FAST b interpolation), and the load
// of node k, g_k b with g_k = sum_k3 V[k][k3] det J(xi_k3).  Boundary nodes
// add to the skeleton loads fU; interior nodes write f_I.  One warp per cell.
#define BL_WARPS 4
__global__ void __launch_bounds__(32 * BL_WARPS) body_loads_kernel(CellParams P, QNodes QN,
                                                                    const ForceRomDev* __restrict__ tab,
                                                                    const int32_t* __restrict__ slot,
                                                                    const double* __restrict__ ctrl,
                                                                    const double* __restrict__ mu, double bx,
                                                                    double by, double* __restrict__ fU,
                                                                    double* __restrict__ fI) {
  __shared__ double sq[8];
  __shared__ double wts[BL_WARPS][4][12];
  __shared__ double th[BL_WARPS][128];
  __shared__ double dj[BL_WARPS][64];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 8; ++k) sq[k] = QN.n[k];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long cell = (long long)blockIdx.x * BL_WARPS + warp;
  if (cell >= P.ncells) return;
  const int p = P.p, q = P.q, nx = P.nx, m = P.m, nq = q + 1, nL = nq * nq, nB = (p + 1) * (p + 1);
  int cx, cy;
  cell_xy(P, cell, &cx, &cy);
  const ForceRomDev& F = tab[slot[cell]];
  const int r = F.r, n1 = r + 1, rf = F.rf, ne = 4 * (p + 1) * nq;
  if (lane < 4) {
    double nodes[12];
    for (int i = 0; i < n1; ++i) nodes[i] = F.lo4[lane] + (F.hi4[lane] - F.lo4[lane]) * F.g01[i];
    lagrange1d(r, nodes, mu[4 * cell + lane], wts[warp][lane], nullptr);
  }
  // det J at the interpolation nodes (coordinates read from shared memory)
  for (int k3 = lane; k3 < nL; k3 += 32) {
    double x[2], J[2][2];
    map_eval(ctrl, nx, m, cx, cy, sq[k3 % nq], sq[k3 / nq], x, J);
    dj[warp][k3] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  }
  __syncwarp();
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int ng = n1 * n1 * n1 * n1;
  for (int g = 0; g < ng; ++g) {
    const int g1 = g % n1, g2 = (g / n1) % n1, g3 = (g / (n1 * n1)) % n1, g4 = g / (n1 * n1 * n1);
    const double w = wts[warp][0][g1] * wts[warp][1][g2] * wts[warp][2][g3] * wts[warp][3][g4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int jj = lane + 32 * u;
      if (jj < rf) acc[u] = fma(w, F.At[(long long)g * rf + jj], acc[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
    if (lane + 32 * u < rf) th[warp][lane + 32 * u] = acc[u];
  __syncwarp();
  for (int k = lane; k < nB; k += 32) {
    double gk = 0.0;
    for (int k3 = 0; k3 < nL; ++k3) {
      const long long col = ne + (long long)k * nL + k3;
      double v = 0.0;
      for (int t = 0; t < rf; ++t) v = fma(F.U[(long long)t * F.nf + col], th[warp][t], v);
      gk = fma(v, dj[warp][k3], gk);
    }
    const int us = P.uslot_of_node[k];
    if (us >= 0) {
      atomicAdd(&fU[cell * P.nU + 2 * us], gk * bx);
      atomicAdd(&fU[cell * P.nU + 2 * us + 1], gk * by);
    }
  }
  // interior DoFs in islot order
  for (int i = lane; i < P.nI; i += 32) {
    const int dof = P.islot[i], k = dof / 2, comp = dof % 2;
    double gk = 0.0;
    for (int k3 = 0; k3 < nL; ++k3) {
      const long long col = ne + (long long)k * nL + k3;
      double v = 0.0;
      for (int t = 0; t < rf; ++t) v = fma(F.U[(long long)t * F.nf + col], th[warp][t], v);
      gk = fma(v, dj[warp][k3], gk);
    }
    fI[cell * P.nI + i] = gk * (comp == 0 ? bx : by);
  }
}

// Static condensation of the interior loads (Sec. 3.2): y = L^-1 f_I (kept in
// fI for the recovery) and f_U -= W^T y, W = L^-1 K_IU.  One warp per cell.
__global__ void condense_kernel(CellParams P, const double* __restrict__ LII, const double* __restrict__ W,
                                double* __restrict__ fI, double* __restrict__ fU) {
  __shared__ double sy[4][128];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long cell = (long long)blockIdx.x * 4 + warp;
  if (cell >= P.ncells) return;
  const int NI = P.nI, NU = P.nU;
  for (int i = lane; i < NI; i += 32) sy[warp][i] = fI[cell * NI + i];
  __syncwarp();
  const double* L = LII + cell * (NI * (NI + 1) / 2);
  // forward substitution L y = f_I, one row at a time, dot over lanes
  for (int i = 0; i < NI; ++i) {
    double s = 0.0;
    for (int k = lane; k < i; k += 32) s += L[(long long)i * (i + 1) / 2 + k] * sy[warp][k];
    s = warp_sum(s);
    if (lane == 0) sy[warp][i] = (sy[warp][i] - s) / L[(long long)i * (i + 1) / 2 + i];
    __syncwarp();
  }
  for (int i = lane; i < NI; i += 32) fI[cell * NI + i] = sy[warp][i];
  const double* Wc = W + cell * NI * NU;
  for (int u = lane; u < NU; u += 32) {
    double acc = 0.0;
    for (int i = 0; i < NI; ++i) acc = fma(Wc[i * NU + u], sy[warp][i], acc);
    fU[cell * NU + u] -= acc;
  }
}

// Interior recovery and nodal output: u_I = -L^-T W u_loc (f_I = 0: no body force),
// one warp per cell.
__global__ void recover_kernel(CellParams P, const double* __restrict__ LII, const double* __restrict__ W,
                               const int* __restrict__ umap, const double* __restrict__ x,
                               const double* __restrict__ yI, double* __restrict__ u) {
  __shared__ double sv[4][64];
  __shared__ double sy[4][128];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long cell = (long long)blockIdx.x * 4 + warp;
  if (cell >= P.ncells) return;
  const int NI = P.nI, NU = P.nU, p = P.p;
  for (int t = lane; t < NU; t += 32) {
    const int g = umap[cell * NU + t];
    sv[warp][t] = g >= 0 ? x[g] : 0.0;
  }
  __syncwarp();
  const double* Wc = W + cell * NI * NU;
  for (int i = lane; i < NI; i += 32) {
    double acc = 0.0;
    for (int t = 0; t < NU; ++t) acc = fma(Wc[i * NU + t], sv[warp][t], acc);
    sy[warp][i] = (yI ? yI[cell * NI + i] : 0.0) - acc;   // L^-1 f_I - W u (f_I = 0 without body forces)
  }
  __syncwarp();
  const double* L = LII + cell * (NI * (NI + 1) / 2);
  // backward substitution L^T z = y, one lane at a time per row, dot over lanes
  for (int i = NI - 1; i >= 0; --i) {
    double s = 0.0;
    for (int k = i + 1 + lane; k < NI; k += 32) s += L[(long long)k * (k + 1) / 2 + i] * sy[warp][k];
    s = warp_sum(s);
    if (lane == 0) sy[warp][i] = (sy[warp][i] - s) / L[(long long)i * (i + 1) / 2 + i];
    __syncwarp();
  }
  int cx, cy;
  cell_xy(P, cell, &cx, &cy);
  const long long gnx = (long long)p * P.nx + 1;
  for (int i = lane; i < NI; i += 32) {
    const int dof = P.islot[i], k = dof / 2, comp = dof % 2;
    const int a = k % (p + 1), b = k / (p + 1);
    u[2 * ((long long)(p * cy + b) * gnx + (p * cx + a)) + comp] = sy[warp][i];
  }
}

// skeleton nodes of the nodal output (Dirichlet nodes get 0)
__global__ void skel_to_nodes_kernel(CellParams P, long long nnodes, const double* __restrict__ x,
                                     double* __restrict__ u) {
  const int p = P.p, nx = P.nx, ny = P.ny;
  const long long NH = (long long)(ny + 1) * (p * nx + 1);
  const long long gnx = (long long)p * nx + 1;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < nnodes;
       id += (long long)gridDim.x * blockDim.x) {
    int gx, gy;
    skel_node_xy(id, p, nx, NH, &gx, &gy);
    const bool d = dir_node(P, id, gx, gy);
    u[2 * (gy * gnx + gx)] = d ? 0.0 : x[2 * id];
    u[2 * (gy * gnx + gx) + 1] = d ? 0.0 : x[2 * id + 1];
  }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
static romb_status dot_on(romb_ctx* c, cudaStream_t st, double* red, const double* a, const double* b, long long n,
                          double* out) {
  double* part = red + 64;
  dot_partial_kernel<<<RED_BLOCKS, 256, 0, st>>>(a, b, n, part); ++c->launches;
  dot_final_kernel<<<1, 256, 0, st>>>(part, RED_BLOCKS, out); ++c->launches;
  ROMB_CUDA(cudaGetLastError());
  return ROMB_OK;
}
// context-level dot product (the compliance), on the context's stream
romb_status romb_dot(romb_ctx* c, const double* a, const double* b, long long n, double* out) {
  return dot_on(c, c->stream, c->d_red, a, b, n, out);
}
static romb_status dot(romb_ctx* c, PcgLane& L, const double* a, const double* b, long long n, double* out) {
  return dot_on(c, L.stream, L.d_red, a, b, n, out);
}

static int grid_for(const romb_ctx* c, long long n) {
  long long g = (n + 255) / 256;
  const long long cap = 8LL * c->sms;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

// z = S_BDDC^-1 r  (Algorithm 1)
// prepare = true (outside stream capture): set the shared-memory limit and size
// the persistent grid (resident CTAs per SM x SMs); prepare = false: launch.
template <int P, int MODE, typename T>
static romb_status cell_apply_p(romb_ctx* c, cudaStream_t st, bool prepare, const T* M, const double* v,
                                double* yloc, double* cloc, int grid_override, const T* Phi) {
  using Sh = CellApplyShape<P>;
  const size_t smem = (size_t)CA_STAGES * Sh::stage_bytes(MODE, (int)sizeof(T));
  const int gi = MODE + (sizeof(T) == 4 ? 1 : 0);   // persistent grid per mode and element type
  if (prepare) {
    ROMB_CUDA(cudaFuncSetAttribute(cell_apply_kernel<P, MODE, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
    int per_sm = 0;
    ROMB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cell_apply_kernel<P, MODE, T>, Sh::THREADS,
                                                            smem));
    c->ca_grid[gi] = std::max(1, std::min(c->ncells, std::max(1, per_sm) * c->sms));
    return ROMB_OK;
  }
  const int grid = grid_override > 0 ? std::min(grid_override, c->ca_grid[gi]) : c->ca_grid[gi];
  cell_apply_kernel<P, MODE, T><<<grid, Sh::THREADS, smem, st>>>(c->ncells, M, c->d_ucell_map, v, yloc, Phi, cloc,
                                                                 c->d_pcg_err);
  ++c->launches;
  ROMB_CUDA(cudaGetLastError());
  return ROMB_OK;
}

template <int MODE, typename T = double>
static romb_status cell_apply(romb_ctx* c, cudaStream_t st, bool prepare, const T* M, const double* v,
                              double* yloc, double* cloc, int grid_override = 0, const T* Phi = nullptr) {
  switch (c->p) {
    case 3: return cell_apply_p<3, MODE, T>(c, st, prepare, M, v, yloc, cloc, grid_override, Phi);
    case 4: return cell_apply_p<4, MODE, T>(c, st, prepare, M, v, yloc, cloc, grid_override, Phi);
    case 5: return cell_apply_p<5, MODE, T>(c, st, prepare, M, v, yloc, cloc, grid_override, Phi);
    case 6: return cell_apply_p<6, MODE, T>(c, st, prepare, M, v, yloc, cloc, grid_override, Phi);
    case 7: return cell_apply_p<7, MODE, T>(c, st, prepare, M, v, yloc, cloc, grid_override, Phi);
    case 8: return cell_apply_p<8, MODE, T>(c, st, prepare, M, v, yloc, cloc, grid_override, Phi);
  }
  return ROMB_E_ARG;
}

static romb_status precondition(romb_ctx* c, PcgLane& L, const CellParams& P, const double* r, double* z) {
  // restriction c = Phi^T r, then the coarse correction on the side stream
  // while the fine part y = D F D r runs here; join before the prolongation
  romb_status s = c->pre32 ? cell_apply<CA_RESTRICT, float>(c, L.stream, false, nullptr, r, nullptr, L.d_cloc, 0,
                                                             c->d_Phi32)
                           : cell_apply<CA_RESTRICT, double>(c, L.stream, false, nullptr, r, nullptr, L.d_cloc, 0, c->d_Phi);
  if (s != ROMB_OK) return s;
  double* zc = L.d_coarse;
  double* gc = L.d_coarse + c->ncoarse_all;
  ROMB_CUDA(cudaEventRecord(L.evfork, L.stream));
  ROMB_CUDA(cudaStreamWaitEvent(L.side, L.evfork, 0));
  coarse_gather_kernel<<<grid_for(c, c->ncoarse_all), 256, 0, L.side>>>(c->d_cowner, c->ncoarse_all, L.d_cloc, zc);
  ++c->launches;
  ROMB_CUDA(cudaGetLastError());
  if ((s = coarse_solve(c, zc, gc, L.side, L.nd_ybuf, L.nd_sbuf)) != ROMB_OK) return s;
  ROMB_CUDA(cudaEventRecord(L.evjoin, L.side));
  // one CTA per SM: the rest of each SM stays free for the coarse chain
  s = c->pre32 ? cell_apply<CA_MATVEC, float>(c, L.stream, false, c->d_G32, r, L.d_yloc, nullptr, c->sms)
               : cell_apply<CA_MATVEC, double>(c, L.stream, false, c->d_G, r, L.d_yloc, nullptr, c->sms);
  if (s != ROMB_OK) return s;
  ROMB_CUDA(cudaStreamWaitEvent(L.stream, L.evjoin, 0));
  const int cb = (c->ncells + 15) / 16;
  if (c->pre32)
    cell_prolong_kernel<float><<<cb, 256, 0, L.stream>>>(c->ncells, c->nU, c->d_Phi32, c->d_cmap, gc, L.d_yloc);
  else
    cell_prolong_kernel<double><<<cb, 256, 0, L.stream>>>(c->ncells, c->nU, c->d_Phi, c->d_cmap, gc, L.d_yloc);
  ++c->launches;
  skel_gather_kernel<<<grid_for(c, c->nskel_nodes), 256, 0, L.stream>>>(P, L.d_yloc, c->nskel_nodes, z); ++c->launches;
  ROMB_CUDA(cudaGetLastError());
  return ROMB_OK;
}

static romb_status apply_S(romb_ctx* c, PcgLane& L, const CellParams& P, const double* v, double* out) {
  romb_status s0 = cell_apply<CA_MATVEC, double>(c, L.stream, false, c->d_S, v, L.d_yloc, nullptr);
  if (s0 != ROMB_OK) return s0;
  skel_gather_kernel<<<grid_for(c, c->nskel_nodes), 256, 0, L.stream>>>(P, L.d_yloc, c->nskel_nodes, out); ++c->launches;
  ROMB_CUDA(cudaGetLastError());
  return ROMB_OK;
}

// One PCG iteration (Algorithm 1 inside CG), a fixed sequence of launches:
//   z = M r; rz' = r.z; p = z + (rz'/rz) p; rz = rz'; q = S p; pq = p.q;
//   x += (rz/pq) p; r -= (rz/pq) q; rr = r.r -> pinned host word.
// With p = 0 and rz = 1 on entry the first iteration is the same body.
static romb_status pcg_body(romb_ctx* c, PcgLane& L, const CellParams& P, bool host_copy) {
  romb_status s;
  const long long n = c->nskel;
  const int g = grid_for(c, n);
  double* sc = L.d_red;
  if ((s = precondition(c, L, P, L.d_r, L.d_z)) != ROMB_OK) return s;
  if ((s = dot(c, L, L.d_r, L.d_z, n, sc + 2)) != ROMB_OK) return s;
  pcg_update_p<<<g, 256, 0, L.stream>>>(n, sc, L.d_pv, L.d_z); ++c->launches;
  pcg_shift_scalars<<<1, 32, 0, L.stream>>>(sc); ++c->launches;
  if ((s = apply_S(c, L, P, L.d_pv, L.d_q)) != ROMB_OK) return s;
  if ((s = dot(c, L, L.d_pv, L.d_q, n, sc + 1)) != ROMB_OK) return s;
  pcg_update_x_r<<<g, 256, 0, L.stream>>>(n, sc, L.d_x, L.d_r, L.d_pv, L.d_q); ++c->launches;
  if ((s = dot(c, L, L.d_r, L.d_r, n, sc + 3)) != ROMB_OK) return s;
  if (host_copy) ROMB_CUDA(cudaMemcpyAsync(L.h_red, sc + 3, 8, cudaMemcpyDeviceToHost, L.stream));
  ROMB_CUDA(cudaGetLastError());
  return ROMB_OK;
}

// Loop control of the device-side PCG loop: sc[16] = (rtol |f|)^2, sc[17] =
// maxit, sc[18] = iterations done.  Continues while |r|^2 > sc[16], |r| is
// finite and fewer than maxit iterations have run.
__global__ void pcg_loop_init(double* sc, double thr2, int maxit) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    sc[0] = 1.0;
    sc[16] = thr2;
    sc[17] = (double)maxit;
    sc[18] = 0.0;
  }
}

__global__ void pcg_loop_check(cudaGraphConditionalHandle h, double* sc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double it = sc[18] + 1.0;
    sc[18] = it;
    const double rr = sc[3];
    cudaGraphSetConditional(h, (rr == rr && rr > sc[16] && it < sc[17]) ? 1u : 0u);
  }
}

// The whole PCG loop as one graph: a conditional while node whose body is the
// captured iteration followed by pcg_loop_check.  Returns false (with the
// stream out of capture and no error pending) if the CUDA driver refuses any step.
static bool build_device_loop(romb_ctx* c, PcgLane& L, const CellParams& P) {
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return (void)cudaGetLastError(), false;
  bool ok = false;
  cudaGraphConditionalHandle h;
  cudaGraphNodeParams np = {};
  cudaGraphNode_t node;
  if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess &&
        cudaStreamBeginCaptureToGraph(L.stream, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const long long l0 = c->launches;
      romb_status s = pcg_body(c, L, P, false);
      pcg_loop_check<<<1, 32, 0, L.stream>>>(h, L.d_red);
      ++c->launches;
      cudaGraph_t body = nullptr;
      const cudaError_t e = cudaStreamEndCapture(L.stream, &body);
      if (s == ROMB_OK && e == cudaSuccess && cudaGraphInstantiate(&L.graph, g, 0) == cudaSuccess) {
        L.graph_launches = c->launches - l0;
        ok = true;
      }
      c->launches = l0;
    }
  }
  cudaGraphDestroy(g);
  if (!ok) {
    (void)cudaGetLastError();
    if (L.graph) cudaGraphExecDestroy(L.graph);
    L.graph = nullptr;
  }
  return ok;
}

__global__ void pcg_init_scalars(double* sc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) sc[0] = 1.0;
}

// Streams and events of a lane (created once, kept across lattices).
romb_status pcg_lane_streams(romb_ctx* c, PcgLane& L, bool main_is_context_stream) {
  if (L.have_streams) return ROMB_OK;
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (main_is_context_stream) {
    L.stream = c->stream;
    L.own_stream = false;
  } else {
    ROMB_CUDA(cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking));
    L.own_stream = true;
  }
  ROMB_CUDA(cudaStreamCreateWithPriority(&L.side, cudaStreamNonBlocking, hi));
  ROMB_CUDA(cudaEventCreateWithFlags(&L.evfork, cudaEventDisableTiming));
  ROMB_CUDA(cudaEventCreateWithFlags(&L.evjoin, cudaEventDisableTiming));
  ROMB_CUDA(cudaEventCreate(&L.ev0));
  ROMB_CUDA(cudaEventCreate(&L.ev1));
  if (cudaMallocHost(&L.h_red, 64 * sizeof(double)) != cudaSuccess) return ROMB_E_OOM;
  L.have_streams = true;
  return ROMB_OK;
}

void pcg_lane_destroy(PcgLane& L) {
  if (L.graph) cudaGraphExecDestroy(L.graph);
  L.graph = nullptr;
  if (!L.have_streams) return;
  if (L.own_stream && L.stream) cudaStreamDestroy(L.stream);
  if (L.side) cudaStreamDestroy(L.side);
  for (cudaEvent_t e : {L.evfork, L.evjoin, L.ev0, L.ev1})
    if (e) cudaEventDestroy(e);
  if (L.h_red) cudaFreeHost(L.h_red);
  L = PcgLane();
}

// Loads -> f and ||f||^2 into L.h_red[1] (read after synchronising L.stream).
romb_status pcg_begin(romb_ctx* c, PcgLane& L, const double* tr, bool tr_on_device) {
  CellParams P;
  fill_cell_params(c, &P);
  ROMB_CUDA(cudaMemcpyAsync(L.d_traction, tr, 64, tr_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            L.stream));
  ROMB_CUDA(cudaMemsetAsync(L.d_fU, 0, 8 * (size_t)c->ncells * c->nU, L.stream));
  if (c->load_form == ROMB_LOADS_REDUCED) {
    QNodes QN;
    memset(&QN, 0, sizeof(QN));
    gll_nodes01(c->q, QN.n);
    std::vector<ForceRomDev> tab(ROMB_MAX_MODELS);
    memset(tab.data(), 0, sizeof(ForceRomDev) * tab.size());
    for (int f = 0; f < ROMB_MAX_MODELS; ++f) {
      if (c->famcount[f] == 0) continue;
      const RombRom& R = c->roms[f];
      if (!R.force_U) {
        romb_set_error("reduced loads: the reduced model of a family in use has no force model");
        return ROMB_E_STATE;
      }
      ForceRomDev& D = tab[f];
      D.U = R.force_U;
      D.At = R.force_At;
      D.rf = R.force_rf;
      D.nf = R.force_nf;
      D.r = R.r;
      for (int d = 0; d < 4; ++d) {
        D.lo4[d] = R.lo4[d];
        D.hi4[d] = R.hi4[d];
      }
      gll_nodes01(R.r, D.g01);
      if (D.rf > 128) return ROMB_E_ARG;
    }
    if (!L.d_forcetab) {
      romb_status s = romb_alloc_t(c, &L.d_forcetab, sizeof(ForceRomDev) * ROMB_MAX_MODELS);
      if (s != ROMB_OK) return s;
    }
    // pageable source: the call returns once the table has been staged
    ROMB_CUDA(cudaMemcpyAsync(L.d_forcetab, tab.data(), sizeof(ForceRomDev) * ROMB_MAX_MODELS,
                              cudaMemcpyHostToDevice, L.stream));
    const long long nwarps = 2LL * c->ny + 2LL * c->nx;
    loads_rom_kernel<<<(int)((nwarps + LR_WARPS - 1) / LR_WARPS), 32 * LR_WARPS, 0, L.stream>>>(
        P, QN, reinterpret_cast<const ForceRomDev*>(L.d_forcetab), c->d_slot, c->d_ctrl, c->d_mu, L.d_traction,
        L.d_fU); ++c->launches;
    ROMB_CUDA(cudaGetLastError());
  } else {
    const long long nwarps = 2LL * c->ny + 2LL * c->nx;
    loads_kernel<<<(int)((nwarps + LQ_WARPS - 1) / LQ_WARPS), 32 * LQ_WARPS, 0, L.stream>>>(
        P, c->d_ctrl, c->d_mu, c->d_family, L.d_traction, L.d_fU); ++c->launches;
    ROMB_CUDA(cudaGetLastError());
  }
  L.body_on = c->body[0] != 0.0 || c->body[1] != 0.0;
  if (L.body_on) {   // the reduced form's table was filled above (the solve checked the form)
    QNodes QN;
    memset(&QN, 0, sizeof(QN));
    gll_nodes01(c->q, QN.n);
    body_loads_kernel<<<(c->ncells + BL_WARPS - 1) / BL_WARPS, 32 * BL_WARPS, 0, L.stream>>>(
        P, QN, reinterpret_cast<const ForceRomDev*>(L.d_forcetab), c->d_slot, c->d_ctrl, c->d_mu, c->body[0],
        c->body[1], L.d_fU, L.d_fI); ++c->launches;
    condense_kernel<<<(c->ncells + 3) / 4, 128, 0, L.stream>>>(P, c->d_LII, c->d_W, L.d_fI, L.d_fU); ++c->launches;
    ROMB_CUDA(cudaGetLastError());
  }
  skel_gather_kernel<<<grid_for(c, c->nskel_nodes), 256, 0, L.stream>>>(P, L.d_fU, c->nskel_nodes, L.d_f); ++c->launches;
  if (romb_status s = dot(c, L, L.d_f, L.d_f, c->nskel, L.d_red + 4); s != ROMB_OK) return s;
  ROMB_CUDA(cudaMemcpyAsync(L.h_red + 1, L.d_red + 4, 8, cudaMemcpyDeviceToHost, L.stream));
  return ROMB_OK;
}

// The PCG loop (x0 = 0) and the recovery into L.d_u; the caller has read
// ||f|| into L.nf.  With the device-side loop nothing here waits for the GPU.
romb_status pcg_finish(romb_ctx* c, PcgLane& L, double rtol, int maxit) {
  CellParams P;
  fill_cell_params(c, &P);
  romb_status s;
  const long long n = c->nskel;
  double* sc = L.d_red;   // scalars: [0] rz, [1] pq, [2] rz_new, [3] rr, [4] ff
  ROMB_CUDA(cudaMemsetAsync(L.d_x, 0, 8 * n, L.stream));
  L.h_red[0] = 0.0;
  L.h_red[3] = 0.0;
  if (L.nf > 0.0) {
    ROMB_CUDA(cudaMemcpyAsync(L.d_r, L.d_f, 8 * n, cudaMemcpyDeviceToDevice, L.stream));
    ROMB_CUDA(cudaMemsetAsync(L.d_pv, 0, 8 * n, L.stream));
    // the loop (or, where the CUDA driver cannot build it, one iteration) is captured
    // once per factorisation and lane and replayed
    if (!L.graph) {
      if ((s = cell_apply<CA_MATVEC, double>(c, L.stream, true, nullptr, nullptr, nullptr, nullptr)) != ROMB_OK) return s;
      if ((s = cell_apply<CA_RESTRICT, double>(c, L.stream, true, nullptr, nullptr, nullptr, nullptr)) != ROMB_OK) return s;
      if (c->pre32) {
        if ((s = cell_apply<CA_MATVEC, float>(c, L.stream, true, nullptr, nullptr, nullptr, nullptr)) != ROMB_OK)
          return s;
        if ((s = cell_apply<CA_RESTRICT, float>(c, L.stream, true, nullptr, nullptr, nullptr, nullptr)) != ROMB_OK)
          return s;
      }
      // ROMB_PCG_HOST_LOOP=1 keeps the loop on the host (one graph launch per
      // iteration): profilers cannot replay kernels inside conditional nodes.
      const char* hl = getenv("ROMB_PCG_HOST_LOOP");
      L.device_loop = !(hl && hl[0] == '1') && build_device_loop(c, L, P);
      if (!L.device_loop) {
        const long long l0 = c->launches;
        ROMB_CUDA(cudaStreamBeginCapture(L.stream, cudaStreamCaptureModeThreadLocal));
        s = pcg_body(c, L, P, true);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(L.stream, &graph);
        if (s != ROMB_OK) return s;
        ROMB_CUDA(e);
        ROMB_CUDA(cudaGraphInstantiate(&L.graph, graph, 0));
        cudaGraphDestroy(graph);
        L.graph_launches = c->launches - l0;
        c->launches = l0;
      }
    }
    if (L.device_loop) {   // the while body runs at least once
      const double thr = rtol * L.nf;
      pcg_loop_init<<<1, 32, 0, L.stream>>>(sc, thr * thr, maxit); ++c->launches;
      ROMB_CUDA(cudaGraphLaunch(L.graph, L.stream));
      ROMB_CUDA(cudaMemcpyAsync(L.h_red, sc + 3, 8, cudaMemcpyDeviceToHost, L.stream));
      ROMB_CUDA(cudaMemcpyAsync(L.h_red + 3, sc + 18, 8, cudaMemcpyDeviceToHost, L.stream));
    } else {
      // host-driven loop: one graph launch and one synchronisation per iteration
      pcg_init_scalars<<<1, 32, 0, L.stream>>>(sc); ++c->launches;
      int it = 0;
      while (it < maxit) {
        ROMB_CUDA(cudaGraphLaunch(L.graph, L.stream));
        c->launches += L.graph_launches;
        ROMB_CUDA(cudaStreamSynchronize(L.stream));
        ++it;
        const double rel = sqrt(L.h_red[0]) / L.nf;
        if (!(rel == rel) || rel <= rtol) break;
      }
      L.h_red[3] = (double)it;
    }
  }
  // recovery + nodal output
  cudaEventRecord(L.ev0, L.stream);
  if (c->layout)   // nodes of no present cell are written by no kernel below
    ROMB_CUDA(cudaMemsetAsync(L.d_u, 0, 16LL * (c->p * c->nx + 1) * (c->p * c->ny + 1), L.stream));
  recover_kernel<<<(c->ncells + 3) / 4, 128, 0, L.stream>>>(P, c->d_LII, c->d_W, c->d_ucell_map, L.d_x,
                                                            L.body_on ? L.d_fI : nullptr, L.d_u);
  ++c->launches;
  skel_to_nodes_kernel<<<grid_for(c, c->nskel_nodes), 256, 0, L.stream>>>(P, c->nskel_nodes, L.d_x, L.d_u);
  ++c->launches;
  ROMB_CUDA(cudaGetLastError());
  cudaEventRecord(L.ev1, L.stream);
  return ROMB_OK;
}

// Iterations and relative residual of the lane's last solve (its stream has
// been synchronised); device-side error reports of the solve kernels.
romb_status pcg_result(romb_ctx* c, PcgLane& L, double rtol, int maxit, int* iters, double* relres) {
  romb_status result = ROMB_OK;
  int it = 0;
  double rel = 0.0;
  if (L.nf > 0.0) {
    it = (int)L.h_red[3];
    rel = sqrt(L.h_red[0]) / L.nf;
    if (L.device_loop) c->launches += (long long)it * L.graph_launches;
    if (!(rel == rel)) result = ROMB_E_NAN;
    else if (rel > rtol) result = ROMB_E_NOT_CONVERGED;
  }
  (void)maxit;
  *iters = it;
  *relres = rel;
  romb_status s;
  if ((s = coarse_solve_check(c)) != ROMB_OK) return s;
  int e = 0;
  ROMB_CUDA(cudaMemcpy(&e, c->d_pcg_err, 4, cudaMemcpyDeviceToHost));
  if (e) {
    ROMB_CUDA(cudaMemset(c->d_pcg_err, 0, 4));
    romb_set_error("PCG: a cell-operator staging copy did not complete in time");
    return ROMB_E_CUDA;
  }
  return result;
}
