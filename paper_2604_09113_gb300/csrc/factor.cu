// BDDC local set-up, one CTA per cell, everything in shared memory, FP64.
//
//  (Sec. 3.2)   K_II = L L^T,  W = L^-1 K_IU,  S = K_UU - W^T W
//  (Sec. 3.3.3) D_jj = K_jj / K^tot_j  (stiffness-weighted partition of unity)
//  (Sec. 3.3.1) coarse functionals: corner values, per edge int u_1, int u_2 and
//               int f.u over the edge of the trimmed domain, f = (x2 - xbar2,
//               xbar1 - x1) (edge_functional_kernel)
//  (Alg. 2)     cross-point DoFs removed: Shat = S minus corners, Chat = edge rows,
//               That = Chat Shat^-1 Chat^T
//  (Eq. BDDC local basis) Psi column per local coarse DoF, corner values moved
//               to the right-hand side
//  local coarse matrix Psi^T S Psi, and the explicit fine operator
//  F = Shat^-1 - Shat^-1 Chat^T That^-1 Chat Shat^-1 (the top-left block of the
//  saddle-point inverse), stored as D F D for the preconditioner.
//
// Skeleton (U) slots follow increasing local DoF 2k+i over the boundary nodes;
// Dirichlet slots are kept as identity rows of S and have D = 0.
#include <stdio.h>

#include "device.cuh"
#include "tables.cuh"

#include "dense.cuh"

__device__ inline long long packed_idx(long long r, long long q, long long nd) {
  if (r > q) {
    const long long t = r;
    r = q;
    q = t;
  }
  return r * nd - r * (r - 1) / 2 + (q - r);
}

template <int P>
struct FactorDims {
  static constexpr int NB = (P + 1) * (P + 1), ND = 2 * NB, NI = 2 * (P - 1) * (P - 1), NU = 8 * P, NK = NU - 8;
  // phase 1 (doubles)
  static constexpr int oAII = 0, oAIU = oAII + NI * NI, oAUU = oAIU + NI * NU, oCr = oAUU + NU * NU,
                       oKd = oCr + 20 * NU, oDv = oKd + NU, oEnd1 = oDv + NU;
  // phase 2 reuses [oAII, oAUU) when it fits there (S stays in place), else
  // it goes after the phase-1 arrays
  static constexpr int size2 = NK * NK + NK * 12 + 144 + NK * 20 + NU * 20 + NK * 20;
  static constexpr int base2 = size2 <= oAUU ? 0 : oEnd1;
  static constexpr int oSh = base2, oY = oSh + NK * NK, oT = oY + NK * 12, oZ = oT + 144, oPsi = oZ + NK * 20,
                       oQ = oPsi + NU * 20, oEnd2 = oQ + NK * 20;
  static constexpr int total = oEnd2 > oEnd1 ? oEnd2 : oEnd1;
};

// The edge functionals of Sec. 3.3.1 on the skeleton nodes of every cell
// edge: a_s = int b_s j dt, m1_s = int b_s (x2 - xbar2) j dt and
// m2_s = int b_s (xbar1 - x1) j dt (j = |dx/dt|, xbar the image of the edge
// midpoint) over the edge of the trimmed domain: where both cells sharing the
// edge are solid (the skeleton of Omega), the cell's own solid part on the
// lattice boundary, the whole edge where that part is shorter than
// ROMB_EDGE_MIN_SOLID; each interval by the ROMB_NQ-point Gauss rule.  One
// warp per (cell, edge); out[cell][e][s][3].
#define ROMB_EDGE_MIN_SOLID 1e-3
#define ROMB_EIV (1 + 2 * ROMB_MAX_IV)   // per (cell, edge): count, then lo/hi pairs

// The solid intervals of every cell edge (edge_solid_dev), one thread each.
__global__ void edge_interval_kernel(int ncells, const double* __restrict__ mu, const int32_t* __restrict__ family,
                                     double* __restrict__ eiv) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= 4LL * ncells) return;
  const long long cell = t >> 2;
  double lo[ROMB_MAX_IV], hi[ROMB_MAX_IV];
  const int n = edge_solid_dev(family[cell], mu + 4 * cell, (int)(t & 3), lo, hi);
  double* o = eiv + t * ROMB_EIV;
  o[0] = n;
  for (int i = 0; i < n; ++i) {
    o[1 + 2 * i] = lo[i];
    o[2 + 2 * i] = hi[i];
  }
}

template <int PD>
__global__ void __launch_bounds__(128) edge_functional_kernel(CellParams P, const double* __restrict__ ctrl,
                                                              const double* __restrict__ eiv,
                                                              double* __restrict__ out) {
  // one warp per lattice edge: vertical edges (vx, cy) first, then horizontal
  // (cx, vy); the edge is computed from one of its present cells (edge e) and
  // written for both (the other sees it as edge e ^ 1, same parameter and nodes)
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, m = P.m, nx = P.nx, ny = P.ny;
  const long long nV = (long long)(nx + 1) * ny, nH = (long long)nx * (ny + 1);
  if (w >= nV + nH) return;
  int cx, cy, e, cx2, cy2;
  if (w < nV) {
    const int vx = (int)(w % (nx + 1));
    cy = cy2 = (int)(w / (nx + 1));
    cx = vx;         // the cell right of the edge sees it as its left edge
    cx2 = vx - 1;    // the cell left of it, as its right edge
    e = 0;
  } else {
    const long long wh = w - nV;
    const int vy = (int)(wh / nx);
    cx = cx2 = (int)(wh % nx);
    cy = vy;         // the cell above, bottom edge
    cy2 = vy - 1;    // the cell below, top edge
    e = 2;
  }
  long long cell = cell_at(P, cx, cy), cell2 = cell_at(P, cx2, cy2);
  if (cell < 0) {   // computed from the other cell
    cell = cell2;
    cell2 = -1;
    cx = cx2;
    cy = cy2;
    e ^= 1;
  }
  if (cell < 0) return;   // no present cell on this edge
  // intervals: where this cell and its neighbour across the edge are both
  // solid (the cell's own solid part on the boundary of the domain)
  double lo[ROMB_MAX_IV * ROMB_MAX_IV], hi[ROMB_MAX_IV * ROMB_MAX_IV];
  const double* own = eiv + (cell * 4 + e) * ROMB_EIV;
  int nm = (int)own[0];
  for (int i = 0; i < nm; ++i) {
    lo[i] = own[1 + 2 * i];
    hi[i] = own[2 + 2 * i];
  }
  if (cell2 >= 0) {
    const double* nbv = eiv + (cell2 * 4 + (e ^ 1)) * ROMB_EIV;
    const int n1 = nm, n2 = (int)nbv[0];
    nm = 0;
    for (int i = 0; i < n1; ++i)    // both lists are sorted and disjoint: so is the result
      for (int k = 0; k < n2; ++k) {
        const double u = fmax(own[1 + 2 * i], nbv[1 + 2 * k]), v = fmin(own[2 + 2 * i], nbv[2 + 2 * k]);
        if (v > u) {
          lo[nm] = u;
          hi[nm++] = v;
        }
      }
  }
  double len = 0.0;
  for (int i = 0; i < nm; ++i) len += hi[i] - lo[i];
  if (len < ROMB_EDGE_MIN_SOLID) {
    nm = 1;
    lo[0] = 0.0;
    hi[0] = 1.0;
  }
  // the edge's m+1 map control points (a Kronecker delta in the other
  // direction); the map basis and its derivative in barycentric form with the
  // weights of the equispaced nodes (P.mw), no division
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
  auto edge_pt = [&](double t, double* x, double* tg) {
    x[0] = x[1] = tg[0] = tg[1] = 0.0;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      if (q > m) break;
      double val = 1.0, der = 0.0;
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        if (j > m) break;
        if (j == q) continue;
        const double dt = t - (double)j / m;
        der = der * dt + val;
        val *= dt;
      }
      val *= P.mw[q];
      der *= P.mw[q];
      x[0] = fma(val, Xe[q][0], x[0]);
      x[1] = fma(val, Xe[q][1], x[1]);
      tg[0] = fma(der, Xe[q][0], tg[0]);
      tg[1] = fma(der, Xe[q][1], tg[1]);
    }
  };
  double xb[2], tb[2];
  edge_pt(0.5, xb, tb);
  double acc[3 * (PD + 1)];
#pragma unroll
  for (int i = 0; i < 3 * (PD + 1); ++i) acc[i] = 0.0;
  for (int t = lane; t < nm * ROMB_NQ; t += 32) {
    const int iv = t / ROMB_NQ, qq = t % ROMB_NQ;
    const double L = hi[iv] - lo[iv], tt = lo[iv] + L * P.gq_x[qq];
    double x[2], tg[2], bv[PD + 1];
    edge_pt(tt, x, tg);
    if (P.basis == 0) {   // GLL Lagrange: barycentric weights P.bw
#pragma unroll
      for (int s_ = 0; s_ <= PD; ++s_) {
        double val = P.bw[s_];
#pragma unroll
        for (int j = 0; j <= PD; ++j)
          if (j != s_) val *= tt - P.gll[j];
        bv[s_] = val;
      }
    } else {
      bernstein1d(PD, tt, bv, nullptr);
    }
    const double wj = L * P.gq_w[qq] * hypot(tg[0], tg[1]);
#pragma unroll
    for (int s_ = 0; s_ <= PD; ++s_) {
      const double wb = wj * bv[s_];
      acc[3 * s_] += wb;
      acc[3 * s_ + 1] += wb * (x[1] - xb[1]);
      acc[3 * s_ + 2] += wb * (xb[0] - x[0]);
    }
  }
  double* o = out + (cell * 4 + e) * (PD + 1) * 3;
  double* o2 = cell2 >= 0 ? out + (cell2 * 4 + (e ^ 1)) * (PD + 1) * 3 : nullptr;
#pragma unroll
  for (int i = 0; i < 3 * (PD + 1); ++i) {
    const double v = warp_sum(acc[i]);
    if (lane == 0) {
      o[i] = v;
      if (o2) o2[i] = v;
    }
  }
}

// Threads per cell: at p = 8 one cell's working set (167 KB) allows one CTA
// per SM, which 256 threads leave short of warps to hide the FP64 latency.
template <int P>
struct FactorThreads {
  static constexpr int value = P >= 8 ? 512 : 256;
};

template <int P>
__global__ void __launch_bounds__(FactorThreads<P>::value) factor_kernel(CellParams Pm, const double* __restrict__ Kp,
                                                      const double* __restrict__ efun, const int* __restrict__ umap,
                                                      const int* __restrict__ cmap, const double* __restrict__ ktot,
                                                      double* __restrict__ LII_out, double* __restrict__ W_out,
                                                      double* __restrict__ S_out, double* __restrict__ G_out,
                                                      double* __restrict__ Phi_out, double* __restrict__ Psi_out,
                                                      double* __restrict__ SCl_out, double* __restrict__ D_out,
                                                      int32_t* __restrict__ flags, int rowsum_fix) {
  using Dm = FactorDims<P>;
  constexpr int ND = Dm::ND, NI = Dm::NI, NU = Dm::NU, NK = Dm::NK;
  extern __shared__ double sm[];
  double* AII = sm + Dm::oAII;
  double* AIU = sm + Dm::oAIU;
  double* S = sm + Dm::oAUU;
  double* Cr = sm + Dm::oCr;
  double* kd = sm + Dm::oKd;
  double* Dv = sm + Dm::oDv;
  __shared__ int s_umap[NU], s_cmap[20], s_keep[NK], s_cu[8], s_islot[NI], s_uslot[NU], s_bad;
  __shared__ double s_rs[ND][2];   // row sums over each displacement component (translation test)
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long cell = blockIdx.x;
  const int cx = (int)(cell % Pm.nx), cy = (int)(cell / Pm.nx);
  for (int i = tid; i < NU; i += nt) {
    s_umap[i] = umap[cell * NU + i];
    s_uslot[i] = Pm.uslot[i];
  }
  for (int i = tid; i < NI; i += nt) s_islot[i] = Pm.islot[i];
  if (tid < 20) s_cmap[tid] = cmap[cell * 20 + tid];
  if (tid == 0) {
    s_bad = 0;
    const int kc[4] = {0, P, (P + 1) * P, (P + 1) * P + P};
    for (int v = 0; v < 4; ++v)
      for (int cc = 0; cc < 2; ++cc) s_cu[2 * v + cc] = 2 * Pm.uslot_of_node[kc[v]] + cc;
    int n = 0;
    for (int u = 0; u < NU; ++u) {
      bool corner = false;
      for (int t = 0; t < 8; ++t) corner |= (s_cu[t] == u);
      if (!corner) s_keep[n++] = u;
    }
  }
  __syncthreads();
  // ---- load K in (I, U) order; Dirichlet skeleton slots become identity ----
  const double* Kc = Kp + cell * ((long long)ND * (ND + 1) / 2);
  // Split-precision matrices: restore the exact null space of rigid translations
  // (sum_k2 K[(k1 i1), (k2 i2)] = 0, since the basis derivatives sum to zero) by
  // moving each row sum onto the node's own 2x2 diagonal block, symmetrised.
  for (int t = tid; t < 2 * ND; t += nt) {
    const int r = t >> 1, i2 = t & 1;
    double acc = 0.0;
    if (rowsum_fix)
      for (int k2 = 0; k2 < ND / 2; ++k2) acc += Kc[packed_idx(r, 2 * k2 + i2, ND)];
    s_rs[r][i2] = acc;
  }
  __syncthreads();
  auto kval = [&](int r, int q) -> double {
    double v = Kc[packed_idx(r, q, ND)];
    if ((r >> 1) == (q >> 1)) v -= 0.5 * (s_rs[r][q & 1] + s_rs[q][r & 1]);
    return v;
  };
  for (int t = tid; t < NI * NI; t += nt) {
    const int i = t / NI, j = t % NI;
    AII[t] = kval(s_islot[i], s_islot[j]);
  }
  for (int t = tid; t < NI * NU; t += nt) {
    const int i = t / NU, u = t % NU;
    AIU[t] = s_umap[u] < 0 ? 0.0 : Kc[packed_idx(s_islot[i], s_uslot[u], ND)];
  }
  for (int t = tid; t < NU * NU; t += nt) {
    const int u = t / NU, v = t % NU;
    double val = kval(s_uslot[u], s_uslot[v]);
    if (u == v) kd[u] = val;
    if (s_umap[u] < 0 || s_umap[v] < 0) val = (u == v) ? 1.0 : 0.0;
    S[t] = val;
  }
  for (int t = tid; t < 20 * NU; t += nt) Cr[t] = 0.0;
  __syncthreads();
  // ---- coarse functionals ----
  if (tid < 8) {
    if (s_cmap[tid] >= 0) Cr[tid * NU + s_cu[tid]] = 1.0;
  }
  for (int t = tid; t < 4 * (P + 1); t += nt) {
    const int e = t / (P + 1), s = t % (P + 1);
    const int k = e == 0 ? (P + 1) * s : e == 1 ? P + (P + 1) * s : e == 2 ? s : s + (P + 1) * P;
    const int u0 = 2 * Pm.uslot_of_node[k];
    const double* ef = efun + ((cell * 4 + e) * (P + 1) + s) * 3;
    const double a = ef[0], m1 = ef[1], m2 = ef[2];
    const int r = 8 + 3 * e;
    if (s_cmap[r] >= 0) {
      if (s_umap[u0] >= 0) {
        Cr[r * NU + u0] = a;
        Cr[(r + 2) * NU + u0] = m1;
      }
      if (s_umap[u0 + 1] >= 0) {
        Cr[(r + 1) * NU + u0 + 1] = a;
        Cr[(r + 2) * NU + u0 + 1] = m2;
      }
    }
  }
  // ---- K_II = L L^T ----
  __shared__ double s_inv[NI > NK ? NI : NK];
  __shared__ double s_invT[12];
  chol_smem(AII, NI, NI, s_inv, &s_bad);
  // ---- W = L^-1 K_IU ----
  trsm_lower(AII, NI, NI, s_inv, AIU, NU, NU);
  // ---- S = K_UU - W^T W (lower triangle, mirrored) ----
  for (int t = tid; t < NU * (NU + 1) / 2; t += nt) {
    int u, v;
    tri_ij(t, u, v);
    double acc = 0.0;
#pragma unroll 5
    for (int k = 0; k < NI; ++k) acc = fma(AIU[k * NU + u], AIU[k * NU + v], acc);
    const double val = S[u * NU + v] - acc;
    S[u * NU + v] = val;
    S[v * NU + u] = val;
  }
  // write L (packed lower) and W for the interior recovery
  for (int t = tid; t < NI * (NI + 1) / 2; t += nt) {
    int i, j;
    tri_ij(t, i, j);
    LII_out[cell * (NI * (NI + 1) / 2) + t] = AII[i * NI + j];
  }
  for (int t = tid; t < NI * NU; t += nt) W_out[cell * NI * NU + t] = AIU[t];
  for (int u = tid; u < NU; u += nt) {
    const int g = s_umap[u];
    Dv[u] = g >= 0 ? kd[u] / ktot[g] : 0.0;
  }
  __syncthreads();
  // ---- phase 2 (AII / AIU region reused; S is written out and its area
  //      becomes M = Lhat^-1 once Shat, Chat^T and the right-hand sides are built) ----
  double* Sh = sm + Dm::oSh;
  double* Y = sm + Dm::oY;
  double* T = sm + Dm::oT;
  double* Z = sm + Dm::oZ;
  double* Psi = sm + Dm::oPsi;
  double* Q = sm + Dm::oQ;
  double* M = S;
  double* Sg = S_out + cell * NU * NU;
  for (int t = tid; t < NU * NU; t += nt) Sg[t] = S[t];
  for (int t = tid; t < NK * NK; t += nt) Sh[t] = S[s_keep[t / NK] * NU + s_keep[t % NK]];
  // right-hand sides of Eq. (BDDC local basis) after removing the corners:
  // fhat = -S[keep, corner_j] for vertex slots (into Q, then Z = Shat^-1 fhat)
  for (int t = tid; t < NK * 20; t += nt) {
    const int i = t / 20, j = t % 20;
    Q[t] = (j < 8 && s_cmap[j] >= 0) ? -S[s_keep[i] * NU + s_cu[j]] : 0.0;
  }
  __syncthreads();
  chol_smem(Sh, NK, NK, s_inv, &s_bad);
  tri_inverse(Sh, NK, NK, s_inv, M, NK);
  // Y = M Chat^T (M lower triangular)
  for (int t = tid; t < NK * 12; t += nt) {
    const int i = t / 12, e = t % 12;
    const double* Ce = Cr + (8 + e) * NU;
    double acc = 0.0;
    for (int k = 0; k <= i; ++k) acc = fma(M[i * NK + k], Ce[s_keep[k]], acc);
    Y[t] = acc;
  }
  // Z1 = M fhat
  for (int t = tid; t < NK * 20; t += nt) {
    const int i = t / 20, j = t % 20;
    double acc = 0.0;
    for (int k = 0; k <= i; ++k) acc = fma(M[i * NK + k], Q[k * 20 + j], acc);
    Z[t] = acc;
  }
  __syncthreads();
  // That = Y^T Y
  for (int t = tid; t < 144; t += nt) {
    const int a = t / 12, b = t % 12;
    double acc = 0.0;
    for (int i = 0; i < NK; ++i) acc = fma(Y[i * 12 + a], Y[i * 12 + b], acc);
    if (s_cmap[8 + a] < 0 || s_cmap[8 + b] < 0) acc = (a == b) ? 1.0 : 0.0;
    T[t] = acc;
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    // 12 x 12 Cholesky of That on one warp (lane = row, right-looking),
    // while the other warps form Z
    for (int k = 0; k < 12; ++k) {
      if (lane == k) {
        double d = T[k * 12 + k];
        if (!(d > 0.0)) {
          s_bad = 1;
          d = 1.0;
        }
        const double y = pivot_rsqrt(d);
        T[k * 12 + k] = d * y;
        s_invT[k] = y;
      }
      __syncwarp();
      if (lane > k && lane < 12) T[lane * 12 + k] *= s_invT[k];
      __syncwarp();
      if (lane > k && lane < 12)
        for (int j = k + 1; j <= lane; ++j) T[lane * 12 + j] = fma(-T[lane * 12 + k], T[j * 12 + k], T[lane * 12 + j]);
      __syncwarp();
    }
  } else {
    // Z = M^T Z1 = Shat^-1 fhat
    for (int t = tid - 32; t < NK * 20; t += nt - 32) {
      const int i = t / 20, j = t % 20;
      double acc = 0.0;
      for (int k = i; k < NK; ++k) acc = fma(M[k * NK + i], Z[k * 20 + j], acc);
      Q[t] = acc;
    }
  }
  __syncthreads();
  for (int t = tid; t < NK * 20; t += nt) Z[t] = Q[t];
  __syncthreads();
  // R = Chat Z - ghat ; ghat = -C[edge, corner_j] (vertex slots) or e_{j-8} (edge slots)
  double* R = Q;   // [12][20]
  for (int t = tid; t < 240; t += nt) {
    const int e = t / 20, j = t % 20;
    double acc = 0.0;
    for (int i = 0; i < NK; ++i) acc = fma(Cr[(8 + e) * NU + s_keep[i]], Z[i * 20 + j], acc);
    double g = 0.0;
    if (s_cmap[j] >= 0) g = (j < 8) ? -Cr[(8 + e) * NU + s_cu[j]] : ((j - 8 == e) ? 1.0 : 0.0);
    R[t] = (s_cmap[8 + e] >= 0) ? acc - g : 0.0;
  }
  __syncthreads();
  // Lambda = That^-1 R (one thread per column, 12 x 12 triangles)
  for (int j = tid; j < 20; j += nt) {
    for (int i = 0; i < 12; ++i) {
      double s = R[i * 20 + j];
      for (int k = 0; k < i; ++k) s -= T[i * 12 + k] * R[k * 20 + j];
      R[i * 20 + j] = s * s_invT[i];
    }
    for (int i = 11; i >= 0; --i) {
      double s = R[i * 20 + j];
      for (int k = i + 1; k < 12; ++k) s -= T[k * 12 + i] * R[k * 20 + j];
      R[i * 20 + j] = s * s_invT[i];
    }
  }
  __syncthreads();
  // Xhat = Z - Lhat^-T (Y Lambda) = Z - M^T (Y Lambda)
  double* Q2 = Psi;   // temporary [NK][20] in the Psi area (NU*20 >= NK*20)
  for (int t = tid; t < NK * 20; t += nt) {
    const int i = t / 20, j = t % 20;
    double acc = 0.0;
    for (int e = 0; e < 12; ++e) acc = fma(Y[i * 12 + e], R[e * 20 + j], acc);
    Q2[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < NK * 20; t += nt) {
    const int i = t / 20, j = t % 20;
    double acc = 0.0;
    for (int k = i; k < NK; ++k) acc = fma(M[k * NK + i], Q2[k * 20 + j], acc);
    Z[t] -= acc;
  }
  __syncthreads();
  for (int t = tid; t < NU * 20; t += nt) Psi[t] = 0.0;
  __syncthreads();
  for (int t = tid; t < NK * 20; t += nt) {
    const int i = t / 20, j = t % 20;
    Psi[s_keep[i] * 20 + j] = (s_cmap[j] >= 0) ? Z[t] : 0.0;
  }
  if (tid < 8 && s_cmap[tid] >= 0) Psi[s_cu[tid] * 20 + tid] = 1.0;
  __syncthreads();
  // S Psi, with S read back from its copy in global memory (written above by this CTA)
  double* SP = Cr;   // constraints no longer needed: [NU][20] fits in 20*NU
  for (int t = tid; t < NU * 20; t += nt) {
    const int u = t / 20, j = t % 20;
    const double* Su = Sg + u * NU;
    double acc = 0.0;
#pragma unroll 4
    for (int v = 0; v < NU; ++v) acc = fma(Su[v], Psi[v * 20 + j], acc);
    SP[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < 400; t += nt) {
    const int a = t / 20, b = t % 20;
    double acc = 0.0;
    for (int u = 0; u < NU; ++u) acc = fma(Psi[u * 20 + a], SP[u * 20 + b], acc);
    SCl_out[cell * 400 + t] = acc;
  }
  for (int t = tid; t < NU * 20; t += nt) {
    Psi_out[cell * NU * 20 + t] = Psi[t];
    Phi_out[cell * NU * 20 + t] = Dv[t / 20] * Psi[t];
  }
  for (int u = tid; u < NU; u += nt) D_out[cell * NU + u] = Dv[u];
  // ---- explicit fine operator F = M^T M - N^T N with N = L_T^-1 Y^T M ----
  // V = L_T^-1 Y^T  (12 x NK), stored transposed in Y: column i of Y^T = row i of Y
  for (int i = tid; i < NK; i += nt) {
    double v[12];
    for (int e = 0; e < 12; ++e) {
      double s = Y[i * 12 + e];
      for (int k = 0; k < e; ++k) s -= T[e * 12 + k] * v[k];
      v[e] = s * s_invT[e];
    }
    for (int e = 0; e < 12; ++e) Y[i * 12 + e] = v[e];
  }
  __syncthreads();
  double* N = Q;   // [12][NK] (Q area holds NK*20 >= 12*NK)
  for (int t = tid; t < 12 * NK; t += nt) {
    const int e = t / NK, j = t % NK;
    double acc = 0.0;
    for (int i = j; i < NK; ++i) acc = fma(Y[i * 12 + e], M[i * NK + j], acc);
    N[t] = acc;
  }
  __syncthreads();
  double* Gc = G_out + cell * NU * NU;
  for (int t = tid; t < NU * NU; t += nt) Gc[t] = 0.0;
  __syncthreads();
  for (int t = tid; t < NK * (NK + 1) / 2; t += nt) {
    int a, b;
    tri_ij(t, a, b);
    double acc = 0.0;
    for (int i = a; i < NK; ++i) acc = fma(M[i * NK + a], M[i * NK + b], acc);
    for (int e = 0; e < 12; ++e) acc = fma(-N[e * NK + a], N[e * NK + b], acc);
    const int ua = s_keep[a], ub = s_keep[b];
    const double v = Dv[ua] * acc * Dv[ub];
    Gc[ua * NU + ub] = v;
    Gc[ub * NU + ua] = v;
  }
  if (tid == 0 && s_bad) atomicOr(&flags[cell], ROMB_FLAG_NOT_SPD);
}

// K^tot per skeleton DoF: sum of the diagonal entries of every cell sharing the
// node (Sec. 3.3.3), gathered in a fixed order.
__global__ void ktot_kernel(CellParams P, const double* __restrict__ Kp, long long nskel_nodes,
                            double* __restrict__ ktot) {
  const int p = P.p, nx = P.nx, ny = P.ny;
  const long long NH = (long long)(ny + 1) * (p * nx + 1);
  const int ND = 2 * P.nB;
  const long long kp = (long long)ND * (ND + 1) / 2;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < nskel_nodes;
       id += (long long)gridDim.x * blockDim.x) {
    int gx, gy;
    if (id < NH) {
      gy = p * (int)(id / (p * nx + 1));
      gx = (int)(id % (p * nx + 1));
    } else {
      long long t = id - NH;
      const int b = (int)(t % (p - 1)) + 1;
      t /= (p - 1);
      gx = p * (int)(t % (nx + 1));
      gy = p * (int)(t / (nx + 1)) + b;
    }
    double s0 = 0.0, s1 = 0.0;
    const int cx1 = gx / p, cy1 = gy / p;
    for (int dy = (gy % p == 0) ? -1 : 0; dy <= 0; ++dy)
      for (int dx = (gx % p == 0) ? -1 : 0; dx <= 0; ++dx) {
        const int cx = cx1 + dx, cy = cy1 + dy;
        const long long cell = cell_at(P, cx, cy);
        if (cell < 0) continue;
        const int k = (gx - p * cx) + (p + 1) * (gy - p * cy);
        const double* Kc = Kp + cell * kp;
        const long long r0 = 2 * k, r1 = 2 * k + 1;
        s0 += Kc[r0 * ND - r0 * (r0 - 1) / 2];
        s1 += Kc[r1 * ND - r1 * (r1 - 1) / 2];
      }
    ktot[2 * id] = s0;
    ktot[2 * id + 1] = s1;
  }
}

romb_status launch_ktot(romb_ctx* c) {
  CellParams P;
  fill_cell_params(c, &P);
  ktot_kernel<<<4 * c->sms, 256, 0, c->stream>>>(P, c->d_K, c->nskel_nodes, c->d_ktot); ++c->launches;
  ROMB_CUDA(cudaGetLastError());
  return ROMB_OK;
}

template <int P>
static romb_status launch_factor_p(romb_ctx* c, const CellParams& Pm) {
  const size_t smem = sizeof(double) * FactorDims<P>::total;
  ROMB_CUDA(cudaFuncSetAttribute(factor_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  factor_kernel<P><<<c->ncells, FactorThreads<P>::value, smem, c->stream>>>(Pm, c->d_K, c->d_efun, c->d_ucell_map, c->d_cmap, c->d_ktot,
                                                        c->d_LII, c->d_W, c->d_S, c->d_G, c->d_Phi, c->d_Psi,
                                                        c->d_SCl, c->d_D, c->d_flags,
                                                        c->assembled_split ? 1 : 0); ++c->launches;
  ROMB_CUDA(cudaGetLastError());
  return ROMB_OK;
}

romb_status launch_edge_functionals(romb_ctx* c) {
  CellParams Pm;
  fill_cell_params(c, &Pm);
  const long long nw = 4LL * c->ncells;   // cell edges (interval kernel)
  const long long ne = (long long)(c->nx + 1) * c->ny + (long long)c->nx * (c->ny + 1);   // lattice edges
  const int nb = (int)((ne + 3) / 4);
  auto k = c->p == 3 ? edge_functional_kernel<3> : c->p == 4 ? edge_functional_kernel<4>
           : c->p == 5 ? edge_functional_kernel<5> : c->p == 6 ? edge_functional_kernel<6>
           : c->p == 7 ? edge_functional_kernel<7> : edge_functional_kernel<8>;
  edge_interval_kernel<<<(int)((nw + 255) / 256), 256, 0, c->stream>>>(c->ncells, c->d_mu, c->d_family, c->d_eiv);
  ++c->launches;
  k<<<nb, 128, 0, c->stream>>>(Pm, c->d_ctrl, c->d_eiv, c->d_efun); ++c->launches;
  ROMB_CUDA(cudaGetLastError());
  c->efun_ready = true;
  return ROMB_OK;
}

romb_status launch_factor(romb_ctx* c) {
  CellParams Pm;
  fill_cell_params(c, &Pm);
  if (!c->efun_ready) {   // cell matrices given by the caller: no assembly computed them
    romb_status s = launch_edge_functionals(c);
    if (s != ROMB_OK) return s;
  }
  switch (c->p) {
    case 3: return launch_factor_p<3>(c, Pm);
    case 4: return launch_factor_p<4>(c, Pm);
    case 5: return launch_factor_p<5>(c, Pm);
    case 6: return launch_factor_p<6>(c, Pm);
    case 7: return launch_factor_p<7>(c, Pm);
    case 8: return launch_factor_p<8>(c, Pm);
  }
  return ROMB_E_ARG;
}
