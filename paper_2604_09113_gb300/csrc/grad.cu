// Compliance and its gradient (discrete adjoint of the assembled model).
//
// c = f^T u with K u = f; K symmetric, so dc = 2 u^T df - sum_i u_i^T dK_i u_i.
// Cell matrices of Algorithm 4: K_i = sum_e I'_i[e] Chat_i[e] with
// I'_i = U'^T theta_i, theta_i = (rho, (1 - rho) I_r(mu_i)), so
//   u_i^T (dK_i/dx) u_i  = sum_e W_i[e] . dChat_i[e]/dx,
//   W_i[k3][i1 j1 i2 j2] = sum_{k1 k2} u[k1 i1] I'_i[k1 k2 k3 j1 j2] u[k2 i2],
//   u_i^T (dK_i/dtheta_t) u_i = Q_i[t] = sum_{k1 k2 e} U'_t[k1 k2 e] (u u Chat)[k1 k2 e],
//   dc/dmu_d = -(1 - rho) sum_t dI_r,t/dmu_d Q_i[t+1].
// W and Q are formed in FP64 by one pass over U' (CTAs of 8 cells share each
// U' tile); dChat/dJ is analytic; the traction term uses dj/dx of the loaded
// edges.  Control-point gradients are gathered over the sharing cells in a
// fixed order.
#include <math.h>
#include <stdio.h>

#include "device.cuh"
#include "tables.cuh"

#define GW_CELLS 8
#define GW_PAIRS 4

__global__ void __launch_bounds__(512) grad_wq_kernel(CellParams P, const double* __restrict__ U, long long n_half,
                                                       int K, const int* __restrict__ list, int count,
                                                       const int2* __restrict__ pairs, int npairs,
                                                       const double* __restrict__ theta, const double* __restrict__ chat,
                                                       const double* __restrict__ unodal, double* __restrict__ Wout,
                                                       double* __restrict__ Qout) {
  extern __shared__ double sm[];
  double* Ut = sm;                                   // [K][GW_PAIRS*36]
  double* su = Ut + (size_t)K * GW_PAIRS * 36;       // [8][2 nB]
  double* sth = su + GW_CELLS * 2 * P.nB;            // [8][K]
  double* sC = sth + GW_CELLS * K;                   // [8][144]
  double* Ib = sC + GW_CELLS * 144;                  // [8][36]
  double* Yb = Ib + GW_CELLS * 36;                   // [8][36]
  const int tid = threadIdx.x, g = tid >> 6, lt = tid & 63;
  const int ci = blockIdx.x * GW_CELLS + g;
  const bool valid = ci < count;
  const long long cell = valid ? list[ci] : 0;
  const int p = P.p, nB = P.nB;
  const int cx = (int)(cell % P.nx), cy = (int)(cell / P.nx);
  const long long gnx = (long long)p * P.nx + 1;
  for (int d = lt; d < 2 * nB; d += 64) {
    const int k = d >> 1, comp = d & 1, a = k % (p + 1), b = k / (p + 1);
    su[g * 2 * nB + d] = valid ? unodal[2 * ((long long)(p * cy + b) * gnx + (p * cx + a)) + comp] : 0.0;
  }
  for (int t = lt; t < K; t += 64) sth[g * K + t] = valid ? theta[cell * 128 + t] : 0.0;
  for (int e = lt; e < 144; e += 64) sC[g * 144 + e] = valid ? chat[cell * 144 + e] : 0.0;
  double w[2][2] = {{0.0, 0.0}, {0.0, 0.0}};   // thread e < 36: W[k3][i1 j1 i2 j2] for its (k3, j1, j2)
  double q = 0.0;                              // thread t < K: Q[t]
  const int e = lt, k3 = e >> 2, j1 = (e >> 1) & 1, j2 = e & 1, es = k3 * 4 + 2 * j2 + j1;
  const double* u = su + g * 2 * nB;
  const double* C = sC + g * 144;
  const int ntiles = (npairs + GW_PAIRS - 1) / GW_PAIRS;
  for (int tile = 0; tile < ntiles; ++tile) {
    __syncthreads();
    const int p0 = tile * GW_PAIRS, npl = min(GW_PAIRS, npairs - p0);
    for (int i = tid; i < K * GW_PAIRS * 36; i += blockDim.x) {
      const int t = i / (GW_PAIRS * 36), col = i % (GW_PAIRS * 36);
      Ut[i] = col < npl * 36 ? U[(long long)t * n_half + (long long)p0 * 36 + col] : 0.0;
    }
    __syncthreads();
    for (int pl = 0; pl < npl; ++pl) {
      const int2 kk = pairs[p0 + pl];
      if (lt < 36) {
        double s = 0.0;
        for (int t = 0; t < K; ++t) s = fma(sth[g * K + t], Ut[t * GW_PAIRS * 36 + pl * 36 + lt], s);
        Ib[g * 36 + lt] = s;
      }
      __syncthreads();
      if (lt < 36) {
        const bool diag = kk.x == kk.y;
        const double Ie = Ib[g * 36 + e], Is = Ib[g * 36 + es];
        double y = 0.0;
#pragma unroll
        for (int i1 = 0; i1 < 2; ++i1)
#pragma unroll
          for (int i2 = 0; i2 < 2; ++i2) {
            const double a = u[2 * kk.x + i1] * u[2 * kk.y + i2];
            const double b = diag ? 0.0 : u[2 * kk.y + i1] * u[2 * kk.x + i2];
            w[i1][i2] = fma(a, Ie, fma(b, Is, w[i1][i2]));
            y = fma(a, C[16 * k3 + ((i1 * 2 + j1) * 2 + i2) * 2 + j2],
                    fma(b, C[16 * k3 + ((i1 * 2 + j2) * 2 + i2) * 2 + j1], y));
          }
        Yb[g * 36 + e] = y;
      }
      __syncthreads();
      if (lt < K) {
        double s = 0.0;
#pragma unroll 4
        for (int ee = 0; ee < 36; ++ee) s = fma(Ut[lt * GW_PAIRS * 36 + pl * 36 + ee], Yb[g * 36 + ee], s);
        q += s;
      }
    }
  }
  if (!valid) return;
  if (lt < 36) {
    double* Wc = Wout + cell * 144;
#pragma unroll
    for (int i1 = 0; i1 < 2; ++i1)
#pragma unroll
      for (int i2 = 0; i2 < 2; ++i2) Wc[16 * k3 + ((i1 * 2 + j1) * 2 + i2) * 2 + j2] = w[i1][i2];
  }
  if (lt < K) Qout[cell * 128 + lt] = q;
}

// Per cell: -sum_e W[e] dChat[e]/dx for each local control point, plus the
// traction term 2 u . df/dx on loaded lattice edges.  One thread per cell.
__global__ void grad_chain_kernel(CellParams P, const double* __restrict__ ctrl, const double* __restrict__ mu,
                                  const int32_t* __restrict__ family, const double* __restrict__ W,
                                  const double* __restrict__ unodal, const double* __restrict__ trac,
                                  double* __restrict__ gloc) {
  const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (cell >= P.ncells) return;
  const int m = P.m, p = P.p, nx = P.nx;
  const int cx = (int)(cell % nx), cy = (int)(cell / nx);
  const int ncp = (m + 1) * (m + 1);
  double* out = gloc + cell * ncp * 2;
  for (int i = 0; i < 2 * ncp; ++i) out[i] = 0.0;
  const double qn[3] = {0.0, 0.5, 1.0};
  const double* Wc = W + cell * 144;
  for (int k3 = 0; k3 < 9; ++k3) {
    const double x1 = qn[k3 % 3], x2 = qn[k3 / 3];
    double x[2], J[2][2];
    map_eval(ctrl, nx, m, cx, cy, x1, x2, x, J);
    const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double G[2][2] = {{J[1][1] / det, -J[0][1] / det}, {-J[1][0] / det, J[0][0] / det}};
    double v1[5], d1[5], v2[5], d2[5];
    map_basis1d(m, x1, v1, d1);
    map_basis1d(m, x2, v2, d2);
    // Chat at this node (needed for the det J term)
    double Ch[16];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 2; ++k)
          for (int l = 0; l < 2; ++l) {
            const double GGt = G[j][0] * G[l][0] + G[j][1] * G[l][1];
            const double v = P.lam * (G[j][i] * G[l][k]) + P.mu * ((i == k ? GGt : 0.0) + G[j][k] * G[l][i]);
            Ch[((i * 2 + j) * 2 + k) * 2 + l] = det * v;
          }
    for (int b = 0; b <= m; ++b)
      for (int a = 0; a <= m; ++a) {
        const double dN[2] = {d1[a] * v2[b], v1[a] * d2[b]};
        for (int comp = 0; comp < 2; ++comp) {
          // dJ[r][s] = delta(r, comp) dN[s];  H = G dJ G, tr(G dJ) = sum_s G[s][comp] dN[s]
          const double tr = G[0][comp] * dN[0] + G[1][comp] * dN[1];
          double H[2][2];
          for (int r = 0; r < 2; ++r)
            for (int s = 0; s < 2; ++s) H[r][s] = G[r][comp] * (dN[0] * G[0][s] + dN[1] * G[1][s]);
          double acc = 0.0;
          for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
              for (int k = 0; k < 2; ++k)
                for (int l = 0; l < 2; ++l) {
                  // d(G_jm C_imkn G_ln) with dG = -H
                  const double dGGt = H[j][0] * G[l][0] + H[j][1] * G[l][1] + G[j][0] * H[l][0] + G[j][1] * H[l][1];
                  const double dv = P.lam * (H[j][i] * G[l][k] + G[j][i] * H[l][k]) +
                                    P.mu * ((i == k ? dGGt : 0.0) + H[j][k] * G[l][i] + G[j][k] * H[l][i]);
                  const int idx = ((i * 2 + j) * 2 + k) * 2 + l;
                  acc += Wc[16 * k3 + idx] * (tr * Ch[idx] - det * dv);
                }
          out[2 * (b * (m + 1) + a) + comp] -= acc;
        }
      }
  }
  // traction term: f[2k+i] = int b_k(t) t_i j(t) dt over the solid part of loaded edges
  const long long gnx = (long long)p * nx + 1;
  for (int e = 0; e < 4; ++e) {
    const bool on = (e == 0 && cx == 0) || (e == 1 && cx == nx - 1) || (e == 2 && cy == 0) || (e == 3 && cy == P.ny - 1);
    const double t0 = trac[2 * e], t1 = trac[2 * e + 1];
    if (!on || (t0 == 0.0 && t1 == 0.0)) continue;
    double lo[ROMB_MAX_IV], hi[ROMB_MAX_IV];
    const int nint = edge_solid_dev(family[cell], mu + 4 * cell, e, lo, hi);
    for (int iv = 0; iv < nint; ++iv) {
      const double len = hi[iv] - lo[iv];
      for (int qq = 0; qq < ROMB_NQ; ++qq) {
        const double t = lo[iv] + len * P.gq_x[qq];
        // the edge tangent dx/dt: on the edge one factor of the tensor map basis
        // is a Kronecker delta, so only the edge's m+1 control points vary
        double vs[5], ds[5];
        map_basis1d(m, t, vs, ds);
        double tg[2] = {0.0, 0.0};
        for (int s2 = 0; s2 <= m; ++s2) {
          const int ea = e == 0 ? 0 : e == 1 ? m : s2, eb = e == 2 ? 0 : e == 3 ? m : s2;
          const double* X = ctrl_pt(ctrl, nx, m, cx, cy, ea, eb);
          tg[0] = fma(ds[s2], X[0], tg[0]);
          tg[1] = fma(ds[s2], X[1], tg[1]);
        }
        const double jj = hypot(tg[0], tg[1]);
        double bv[ROMB_MAX_P + 1];
        cell_basis1d(P, t, bv, nullptr);
        // u . (b t) along the edge
        double ub = 0.0;
        for (int s = 0; s <= p; ++s) {
          const int k = e == 0 ? (p + 1) * s : e == 1 ? p + (p + 1) * s : e == 2 ? s : s + (p + 1) * p;
          const int a = k % (p + 1), bb = k / (p + 1);
          const long long node = (long long)(p * cy + bb) * gnx + (p * cx + a);
          ub += bv[s] * (unodal[2 * node] * t0 + unodal[2 * node + 1] * t1);
        }
        const double wq = len * P.gq_w[qq];
        for (int s2 = 0; s2 <= m; ++s2) {   // d N / dt along the edge: ds for the edge's control points
          const int ea = e == 0 ? 0 : e == 1 ? m : s2, eb = e == 2 ? 0 : e == 3 ? m : s2;
          for (int comp = 0; comp < 2; ++comp)
            out[2 * (eb * (m + 1) + ea) + comp] += 2.0 * wq * ub * tg[comp] * ds[s2] / jj;
        }
      }
    }
  }
}

// dc/dmu_d = -(1 - rho) sum_t dI_r,t/dmu_d Q[t+1]: one warp per cell, lanes over the grid.
struct GradNodes {
  double nd[4][12];   // the GLL nodes of each threshold's interval of the model's box
};
__global__ void grad_mu_kernel(CellParams P, const double* __restrict__ A, int n_r, int r, GradNodes N,
                               const int* __restrict__ list, int count, const double* __restrict__ mu,
                               const double* __restrict__ Q, double* __restrict__ dmu) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ci = blockIdx.x * (blockDim.x >> 5) + warp;
  if (ci >= count) return;
  const long long cell = list[ci];
  const int n1 = r + 1;
  double nodes[12], v[4][12], d[4][12];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    for (int i = 0; i < n1; ++i) nodes[i] = N.nd[k][i];
    lagrange1d(r, nodes, mu[4 * cell + k], v[k], d[k]);
  }
  const double* Qc = Q + cell * 128 + 1;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  const int ng = n1 * n1 * n1 * n1;
  for (int gg = lane; gg < ng; gg += 32) {
    double z = 0.0;
    for (int t = 0; t < n_r; ++t) z = fma(A[(long long)t * ng + gg], Qc[t], z);
    const int g1 = gg % n1, g2 = (gg / n1) % n1, g3 = (gg / (n1 * n1)) % n1, g4 = gg / (n1 * n1 * n1);
    s[0] = fma(z, d[0][g1] * v[1][g2] * v[2][g3] * v[3][g4], s[0]);
    s[1] = fma(z, v[0][g1] * d[1][g2] * v[2][g3] * v[3][g4], s[1]);
    s[2] = fma(z, v[0][g1] * v[1][g2] * d[2][g3] * v[3][g4], s[2]);
    s[3] = fma(z, v[0][g1] * v[1][g2] * v[2][g3] * d[3][g4], s[3]);
  }
  for (int k = 0; k < 4; ++k) {
    const double t = warp_sum(s[k]);
    if (lane == 0) dmu[4 * cell + k] = -(1.0 - P.rho) * t;
  }
}

// global control point gradient: sum over the cells sharing the point
__global__ void grad_gather_kernel(CellParams P, const double* __restrict__ gloc, double* __restrict__ out) {
  const int m = P.m, nx = P.nx, ny = P.ny;
  const long long gnx = (long long)m * nx + 1, n = gnx * ((long long)m * ny + 1);
  const int ncp = (m + 1) * (m + 1);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x) {
    const int gx = (int)(id % gnx), gy = (int)(id / gnx);
    double s0 = 0.0, s1 = 0.0;
    for (int dy = (gy % m == 0) ? -1 : 0; dy <= 0; ++dy)
      for (int dx = (gx % m == 0) ? -1 : 0; dx <= 0; ++dx) {
        const int cx = gx / m + dx, cy = gy / m + dy;
        if (cx < 0 || cy < 0 || cx >= nx || cy >= ny) continue;
        const int a = gx - m * cx, b = gy - m * cy;
        const double* l = gloc + ((long long)cy * nx + cx) * ncp * 2 + 2 * (b * (m + 1) + a);
        s0 += l[0];
        s1 += l[1];
      }
    out[2 * id] = s0;
    out[2 * id + 1] = s1;
  }
}

// The per-threshold GLL nodes of a model's box (as the theta kernel forms them).
static GradNodes grad_nodes(const RombRom& R) {
  GradNodes N;
  memset(&N, 0, sizeof(N));
  double g1[12];
  gll_nodes01(R.r, g1);
  for (int k = 0; k < 4; ++k)
    for (int i = 0; i <= R.r; ++i) N.nd[k][i] = R.lo4[k] + (R.hi4[k] - R.lo4[k]) * g1[i];
  return N;
}

romb_status launch_grad(romb_ctx* c, double* d_dctrl, double* d_dmu) {
  CellParams P;
  fill_cell_params(c, &P);
  romb_status s;
  if (!c->d_gW) {
    if ((s = romb_alloc_t(c, &c->d_gW, (size_t)c->ncells * 144)) != ROMB_OK) return s;
    if ((s = romb_alloc_t(c, &c->d_gQ, (size_t)c->ncells * 128)) != ROMB_OK) return s;
    const int ncp = (c->m + 1) * (c->m + 1);
    if ((s = romb_alloc_t(c, &c->d_gloc, (size_t)c->ncells * ncp * 2)) != ROMB_OK) return s;
  }
  const int npairs = c->nB * (c->nB + 1) / 2;
  for (int f = 0; f < ROMB_MAX_MODELS; ++f) {
    if (c->famcount[f] == 0) continue;
    const RombRom& R = c->roms[f];
    const int K = R.n_r + 1;
    const size_t smem = 8 * ((size_t)K * GW_PAIRS * 36 + GW_CELLS * 2 * c->nB + GW_CELLS * K + GW_CELLS * 144 +
                             2 * GW_CELLS * 36);
    ROMB_CUDA(cudaFuncSetAttribute(grad_wq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    grad_wq_kernel<<<(c->famcount[f] + GW_CELLS - 1) / GW_CELLS, 512, smem, c->stream>>>(
        P, R.U64, R.n_half, K, c->d_famlist + c->famstart[f], c->famcount[f], c->d_pairs, npairs, c->d_theta,
        c->d_chat, c->lane[0].d_u, c->d_gW, c->d_gQ); ++c->launches;
    ROMB_CUDA(cudaGetLastError());
    if (d_dmu) {
      grad_mu_kernel<<<(c->famcount[f] + 7) / 8, 256, 0, c->stream>>>(
          P, R.A, R.n_r, R.r, grad_nodes(R), c->d_famlist + c->famstart[f], c->famcount[f], c->d_mu, c->d_gQ,
          d_dmu); ++c->launches;
      ROMB_CUDA(cudaGetLastError());
    }
  }
  grad_chain_kernel<<<(c->ncells + 127) / 128, 128, 0, c->stream>>>(P, c->d_ctrl, c->d_mu, c->d_family, c->d_gW,
                                                                     c->lane[0].d_u, c->lane[0].d_traction, c->d_gloc); ++c->launches;
  grad_gather_kernel<<<4 * c->sms, 256, 0, c->stream>>>(P, c->d_gloc, d_dctrl); ++c->launches;
  ROMB_CUDA(cudaGetLastError());
  return ROMB_OK;
}

// The launches of launch_grad with caller-supplied intermediate arrays: W
// [cells][144], Q [cells][128], gloc [cells][2 (m+1)^2] and one 16-double
// node table per family (nodes_dev + 16 f), so that families need no stream
// synchronisation between them.  Used by the no-allocation gradient.
romb_status launch_grad_scratch(romb_ctx* c, double* W, double* Q, double* gloc, double* d_dctrl, double* d_dmu) {
  CellParams P;
  fill_cell_params(c, &P);
  const int npairs = c->nB * (c->nB + 1) / 2;
  for (int f = 0; f < ROMB_MAX_MODELS; ++f) {
    if (c->famcount[f] == 0) continue;
    const RombRom& R = c->roms[f];
    const int K = R.n_r + 1;
    const size_t smem = 8 * ((size_t)K * GW_PAIRS * 36 + GW_CELLS * 2 * c->nB + GW_CELLS * K + GW_CELLS * 144 +
                             2 * GW_CELLS * 36);
    ROMB_CUDA(cudaFuncSetAttribute(grad_wq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    grad_wq_kernel<<<(c->famcount[f] + GW_CELLS - 1) / GW_CELLS, 512, smem, c->stream>>>(
        P, R.U64, R.n_half, K, c->d_famlist + c->famstart[f], c->famcount[f], c->d_pairs, npairs, c->d_theta,
        c->d_chat, c->lane[0].d_u, W, Q); ++c->launches;
    ROMB_CUDA(cudaGetLastError());
    grad_mu_kernel<<<(c->famcount[f] + 7) / 8, 256, 0, c->stream>>>(
        P, R.A, R.n_r, R.r, grad_nodes(R), c->d_famlist + c->famstart[f], c->famcount[f], c->d_mu, Q, d_dmu);
    ++c->launches;
    ROMB_CUDA(cudaGetLastError());
  }
  grad_chain_kernel<<<(c->ncells + 127) / 128, 128, 0, c->stream>>>(P, c->d_ctrl, c->d_mu, c->d_family, W, c->lane[0].d_u,
                                                                     c->lane[0].d_traction, gloc); ++c->launches;
  grad_gather_kernel<<<4 * c->sms, 256, 0, c->stream>>>(P, gloc, d_dctrl); ++c->launches;
  ROMB_CUDA(cudaGetLastError());
  return ROMB_OK;
}
