// Online assembly of the cell stiffness matrices (Sec. 4.1, Algorithms 4-5).
//
//  theta kernel (one warp per 4 cells of one family):
//    I_r(mu)  = sum_g A[g] prod_d l_{g_d}(mu_d)       (tensor GLL interpolation, Sec. 4.2.3)
//    theta    = (rho, (1 - rho) I_r)                  (Algorithm 4: I + rho (I_Pi - I))
//    Chat_k   = det J J^-1 C J^-T at the (q+1)^2 GLL interpolation nodes
//               (Eq. ELA constitutive, Eq. FAST interpolation)
//  contraction (FP64 form): I_c = theta_c U' per (k1 <= k2) pair, then
//    K[(k1 i1),(k2 i2)] = sum_{j1 j2 k3} I_c[k1 k2 k3 j1 j2] Chat_c[k3][i1 j1 i2 j2]
//  (Eq. SPEED L int), written as the packed upper triangle of each cell matrix.
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "device.cuh"
#include "tables.cuh"

struct RomDev {
  const double* U64;     // [K][n_half]
  const double* At;      // [ngrid][n_r]  (transposed interpolation samples)
  const float2* At2;     // the same as (hi, lo) FP32 pairs
  int n_r, r;
  double lo4[4], hi4[4]; // the cluster's box per threshold
  long long n_half;
  double g01[12];        // degree-r GLL nodes of [0, 1]; node i of threshold d is lo4 + (hi4 - lo4) g01[i]
};

// the models of one theta launch: model k owns CTAs [cta0[k], cta0[k+1])
struct ThetaFams {
  RomDev rom[ROMB_MAX_MODELS];
  const int* list[ROMB_MAX_MODELS];
  int count[ROMB_MAX_MODELS], cta0[ROMB_MAX_MODELS];
  int nfam;
};

// FindCluster (Algorithm 5, Sec. 4.2.1): the model slot of each cell, from its
// family's cluster table: k_d = floor((mu_d - lo) / h) capped at n_k - 1
// (an interior subinterval boundary belongs to the upper cluster).  Cells
// outside their family's box are flagged and kept in the nearest cluster;
// cells of a family without models get slot -1.
struct FamTab {
  int n_k[ROMB_MAX_FAMILIES], slot0[ROMB_MAX_FAMILIES];
  double lo[ROMB_MAX_FAMILIES], hi[ROMB_MAX_FAMILIES];
};
__global__ void cell_model_kernel(FamTab T, const int32_t* __restrict__ family, const double* __restrict__ mu,
                                  int ncells, int32_t* __restrict__ slot, int32_t* __restrict__ flags) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  const int f = family[c];
  int nk = 0, s0 = -1;
  double lo = 0.0, hi = 0.0;
#pragma unroll
  for (int k = 0; k < ROMB_MAX_FAMILIES; ++k)
    if (k == f) {
      nk = T.n_k[k];
      s0 = T.slot0[k];
      lo = T.lo[k];
      hi = T.hi[k];
    }
  if (nk == 0) {
    slot[c] = -1;
    return;
  }
  const double h = (hi - lo) / nk;
  int k = 0, stride = 1;
  for (int d = 0; d < 4; ++d) {
    const double m = mu[4 * c + d];
    if (!(m >= lo && m <= hi)) atomicOr(&flags[c], ROMB_FLAG_OUT_OF_BOX);
    int kd = (int)floor((m - lo) / h);
    kd = kd < 0 ? 0 : kd > nk - 1 ? nk - 1 : kd;
    k += kd * stride;
    stride *= nk;
  }
  slot[c] = s0 + k;
}

void fill_cell_params(const romb_ctx* c, CellParams* P) {
  memset(P, 0, sizeof(*P));
  P->p = c->p;
  P->m = c->m;
  P->basis = c->basis;
  P->nB = c->nB;
  P->nI = c->nI;
  P->nU = c->nU;
  P->nx = c->nx;
  P->ny = c->ny;
  P->ncells = c->ncells;
  if (c->layout) {
    P->cell_grid = c->d_cell_grid;
    P->grid_cell = c->d_grid_cell;
    P->node_fixed = c->d_node_fixed;
  }
  P->q = c->q;
  P->nL = c->nL;
  P->dmask = c->dmask;
  P->E = c->E;
  P->nu = c->nu;
  P->rho = c->rho;
  P->lam = c->E * c->nu / (1.0 - c->nu * c->nu);
  P->mu = c->E / (2.0 * (1.0 + c->nu));
  gll_nodes01(c->p, P->gll);
  for (int i = 0; i <= c->p; ++i) {
    double den = 1.0;
    for (int j = 0; j <= c->p; ++j)
      if (j != i) den *= P->gll[i] - P->gll[j];
    P->bw[i] = 1.0 / den;
  }
  for (int i = 0; i <= c->m; ++i) {
    double den = 1.0;
    for (int j = 0; j <= c->m; ++j)
      if (j != i) den *= (double)i / c->m - (double)j / c->m;
    P->mw[i] = 1.0 / den;
  }
  gauss01(ROMB_NQ, P->gq_x, P->gq_w);
  for (int i = 0; i < ROMB_NQ; ++i) cell_basis1d(*P, P->gq_x[i], P->bq[i], nullptr);
  for (int i = 0; i <= ROMB_NQ; ++i) map_basis1d(c->m, i < ROMB_NQ ? P->gq_x[i] : 0.5, P->mq[i], P->dmq[i]);
  LocalTables T = make_local_tables(c->p);
  memcpy(P->uslot, T.uslot, sizeof(P->uslot));
  memcpy(P->islot, T.islot, sizeof(P->islot));
  memcpy(P->uslot_of_node, T.uslot_of_node, sizeof(P->uslot_of_node));
}

// ---------------------------------------------------------------------------
// family lists: cells grouped by family, in increasing cell index (one CTA)
// ---------------------------------------------------------------------------
__global__ void family_list_kernel(const int32_t* __restrict__ family, int ncells, int nfam, int* __restrict__ list,
                                   int* __restrict__ counts, int32_t* __restrict__ flags) {
  __shared__ int warp_tot[32];
  __shared__ int base;
  const int tid = threadIdx.x, nt = blockDim.x;
  int out = 0;
  for (int f = 0; f < nfam; ++f) {
    if (tid == 0) base = out;
    __syncthreads();
    for (int c0 = 0; c0 < ncells; c0 += nt) {
      const int c = c0 + tid;
      const int fam = c < ncells ? family[c] : -1;
      const int mine = fam == f;
      // block exclusive scan of `mine`
      const unsigned bal = __ballot_sync(0xffffffffu, mine);
      const int lane = tid & 31, w = tid >> 5;
      const int pre = __popc(bal & ((1u << lane) - 1u));
      if (lane == 0) warp_tot[w] = __popc(bal);
      __syncthreads();
      int wpre = 0, tot = 0;
      for (int i = 0; i < nt / 32; ++i) {
        if (i < w) wpre += warp_tot[i];
        tot += warp_tot[i];
      }
      if (mine) list[base + wpre + pre] = c;
      __syncthreads();
      if (tid == 0) base += tot;
      __syncthreads();
    }
    if (tid == 0) counts[f] = base - out;
    out = base;
    __syncthreads();
  }
  // cells whose family has no loaded model
  for (int c = tid; c < ncells; c += nt)
    if (family[c] < 0 || family[c] >= nfam) flags[c] |= ROMB_FLAG_OUT_OF_BOX;
}

// ---------------------------------------------------------------------------
// theta kernel
// ---------------------------------------------------------------------------
#define TH_CELLS 8
__device__ inline float tf32_round_dev(float f) {
  uint32_t u = __float_as_uint(f);
  if ((u & 0x7f800000u) == 0x7f800000u) return f;
  u = (u + 0x1000u) & 0xffffe000u;
  return __uint_as_float(u);
}

// ---- double-float theta for the split assembly forms ----
// The split forms consume theta rows 2.. as TF32 hi / lo pairs (~22 bits) and
// rows 0-1 in double-float, so theta needs no more than double-float
// precision (pairs of FP32, ~48-bit significands), which runs on the FP32
// pipe (GB300 issues FP32 ~64x faster than FP64).  Products are error-free
// (x.h y.h exactly as p + e via fmaf, plus the cross terms); sums are
// compensated (two-sum, errors collected in the low word), the dot-product
// scheme of Ogita, Rump and Oishi (2005).  __fmul_rn keeps the compiler from
// contracting a product into a following add, which would break the
// error-free transformations.
struct DfPair {
  float h, l;
};
__device__ __forceinline__ DfPair df_prod(float2 x, float2 y) {   // (x.x + x.y)(y.x + y.y), renormalised
  const float p = __fmul_rn(x.x, y.x);
  float e = fmaf(x.x, y.x, -p);
  e = fmaf(x.x, y.y, e);
  e = fmaf(x.y, y.x, e);
  const float s = __fadd_rn(p, e);
  return {s, __fsub_rn(e, __fsub_rn(s, p))};
}
// (h, l) += (a.x + a.y)(b.x + b.y), low word not renormalised
__device__ __forceinline__ void df_dot_step(float& h, float& l, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  const float s = __fadd_rn(h, p), bb = __fsub_rn(s, h);
  l = __fadd_rn(l, __fadd_rn(__fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb)), e));
  h = s;
}

// lambda_t of TH_CELLS cells (lanes over t), the loop of the FP64 kernel in
// double-float: inner sums over g1 per (g2, g3, g4), then the weighted outer sum.
// N1 > 0: n1 = r + 1 as a compile-time constant, so that the n1 sample loads
// of a (g2, g3, g4) step are all issued before its FP32 work.
template <int NS, int N1>
__device__ __forceinline__ void theta_contract_df(const float2* __restrict__ At2, const float2 (*wdf)[4][12],
                                                  int lane, int n1_rt, int nr, double (&lam)[NS][TH_CELLS]) {
  const int n1 = N1 > 0 ? N1 : n1_rt;
  float ah[NS][TH_CELLS], al[NS][TH_CELLS];
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int j = 0; j < TH_CELLS; ++j) ah[s][j] = al[s][j] = 0.f;
  const int n2 = n1 * n1;
  for (int g34 = 0; g34 < n2; ++g34) {
    const int g3 = g34 % n1, g4 = g34 / n1;
    float2 w34[TH_CELLS];
#pragma unroll
    for (int j = 0; j < TH_CELLS; ++j) {
      const DfPair q = df_prod(wdf[j][2][g3], wdf[j][3][g4]);
      w34[j] = make_float2(q.h, q.l);
    }
    for (int g2 = 0; g2 < n1; ++g2) {
      const int g234 = g34 * n1 + g2;
      float sh[NS][TH_CELLS], sc[NS][TH_CELLS];
#pragma unroll
      for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int j = 0; j < TH_CELLS; ++j) sh[s][j] = sc[s][j] = 0.f;
      if constexpr (N1 > 0) {
        float2 av[N1][NS];
#pragma unroll
        for (int g1 = 0; g1 < N1; ++g1)
#pragma unroll
          for (int s = 0; s < NS; ++s) {
            const int t = lane + 32 * s;
            av[g1][s] = t < nr ? __ldg(At2 + (long long)(g234 * N1 + g1) * nr + t) : make_float2(0.f, 0.f);
          }
#pragma unroll
        for (int g1 = 0; g1 < N1; ++g1)
#pragma unroll
          for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int j = 0; j < TH_CELLS; ++j) df_dot_step(sh[s][j], sc[s][j], av[g1][s], wdf[j][0][g1]);
      } else {
        for (int g1 = 0; g1 < n1; ++g1) {
          const float2* Ag = At2 + (long long)(g234 * n1 + g1) * nr;
#pragma unroll
          for (int s = 0; s < NS; ++s) {
            const int t = lane + 32 * s;
            const float2 a = t < nr ? __ldg(Ag + t) : make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < TH_CELLS; ++j) df_dot_step(sh[s][j], sc[s][j], a, wdf[j][0][g1]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < TH_CELLS; ++j) {
        const DfPair q = df_prod(wdf[j][1][g2], w34[j]);
        const float2 w234 = make_float2(q.h, q.l);
#pragma unroll
        for (int s = 0; s < NS; ++s) df_dot_step(ah[s][j], al[s][j], make_float2(sh[s][j], sc[s][j]), w234);
      }
    }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int j = 0; j < TH_CELLS; ++j) lam[s][j] = (double)ah[s][j] + (double)al[s][j];
}

// NS = ceil(n_r / 32) lane slots per reduced coefficient: FP64 instructions
// with every lane predicated off still occupy the FP64 pipe, so the slot
// count is a compile-time constant.
template <int NS, bool DF, int N1 = 0>
__global__ void __launch_bounds__(128) theta_kernel(CellParams P, ThetaFams F,
                                                     const double* __restrict__ ctrl, const double* __restrict__ mu,
                                                     double* __restrict__ theta, double* __restrict__ chat,
                                                     float* __restrict__ th_hi, float* __restrict__ th_lo,
                                                     float* __restrict__ chat32, int32_t* __restrict__ flags) {
  __shared__ double wts[4][TH_CELLS][4][12];   // [warp][cell][param][node]
  __shared__ float2 wdf[DF ? 4 : 1][TH_CELLS][4][12];   // the same as (hi, lo) FP32 pairs (DF only)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // the family of this CTA (families own consecutive CTA ranges)
  int fi = 0;
  for (int k = 1; k < F.nfam; ++k)
    if ((int)blockIdx.x >= F.cta0[k]) fi = k;
  const RomDev& R = F.rom[fi];
  const int* __restrict__ list = F.list[fi];
  const int count = F.count[fi];
  const int first = (((int)blockIdx.x - F.cta0[fi]) * 4 + warp) * TH_CELLS;
  const int r = R.r, n1 = r + 1;
  int cells[TH_CELLS];
  for (int j = 0; j < TH_CELLS; ++j) cells[j] = (first + j < count) ? list[first + j] : -1;
  // 1D interpolation weights: lane = (cell j, parameter d)
  for (int task = lane; task < 4 * TH_CELLS; task += 32) {
    const int j = task >> 2, d = task & 3;
    const int c = cells[j];
    double v[12];
    if (c >= 0) {
      const double m = mu[4 * (long long)c + d];
      if (!(m >= R.lo4[d] && m <= R.hi4[d])) atomicOr(&flags[c], ROMB_FLAG_OUT_OF_BOX);
      double nodes[12];
      for (int i = 0; i < n1; ++i) nodes[i] = R.lo4[d] + (R.hi4[d] - R.lo4[d]) * R.g01[i];
      lagrange1d(r, nodes, m, v, nullptr);
    } else {
      for (int i = 0; i < n1; ++i) v[i] = 0.0;
    }
    for (int i = 0; i < n1; ++i) wts[warp][j][d][i] = v[i];
    if constexpr (DF)
      for (int i = 0; i < n1; ++i) {
        const float h = (float)v[i];
        wdf[warp][j][d][i] = make_float2(h, (float)(v[i] - (double)h));
      }
  }
  __syncwarp();
  // lambda_t = sum_{g2 g3 g4} w2 w3 w4 (sum_{g1} w1[g1] At[g][t]): lanes over t
  const int nr = R.n_r;
  const int n2 = n1 * n1;
  double lam[NS][TH_CELLS];
  if constexpr (!DF) {
    double acc[NS][TH_CELLS];
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int j = 0; j < TH_CELLS; ++j) acc[s][j] = 0.0;
    for (int g34 = 0; g34 < n2; ++g34) {
      const int g3 = g34 % n1, g4 = g34 / n1;
      double w34[TH_CELLS];
#pragma unroll
      for (int j = 0; j < TH_CELLS; ++j) w34[j] = wts[warp][j][2][g3] * wts[warp][j][3][g4];
      for (int g2 = 0; g2 < n1; ++g2) {
        const int g234 = g34 * n1 + g2;
        double inner[NS][TH_CELLS];
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
          for (int j = 0; j < TH_CELLS; ++j) inner[s][j] = 0.0;
        for (int g1 = 0; g1 < n1; ++g1) {
          const double* Ag = R.At + (long long)(g234 * n1 + g1) * nr;
#pragma unroll
          for (int s = 0; s < NS; ++s) {
            const int t = lane + 32 * s;
            const double a = t < nr ? __ldg(Ag + t) : 0.0;
#pragma unroll
            for (int j = 0; j < TH_CELLS; ++j) inner[s][j] = fma(a, wts[warp][j][0][g1], inner[s][j]);
          }
        }
#pragma unroll
        for (int j = 0; j < TH_CELLS; ++j) {
          const double w234 = wts[warp][j][1][g2] * w34[j];
#pragma unroll
          for (int s = 0; s < NS; ++s) acc[s][j] = fma(w234, inner[s][j], acc[s][j]);
        }
      }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int j = 0; j < TH_CELLS; ++j) lam[s][j] = acc[s][j];
  } else {
    theta_contract_df<NS, N1>(R.At2, wdf[warp], lane, n1, nr, lam);
  }
  for (int j = 0; j < TH_CELLS; ++j) {
    const int c = cells[j];
    if (c < 0) continue;
    double* th = theta + 128 * (long long)c;
    float* hi = th_hi + 128 * (long long)c;
    float* lo = th_lo + 128 * (long long)c;
    if (lane == 0) th[0] = P.rho;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int t = lane + 32 * s;
      if (t < nr) th[1 + t] = (1.0 - P.rho) * lam[s][j];
    }
    __syncwarp();
    // TF32 hi / lo split of the tensor-core slots of theta (0 and 2..; slot 1
    // is applied in the epilogue), zero padded to 128 slots
    for (int t = lane; t < 128; t += 32) {
      const double v = (t == 0 || (t >= 2 && t <= nr)) ? th[t] : 0.0;
      const float h = tf32_round_dev((float)v);
      hi[t] = h;
      lo[t] = tf32_round_dev((float)(v - (double)h));
    }
  }
  // Chat at the 9 interpolation nodes: lane = (cell j, node k3)
  for (int task = lane; task < TH_CELLS * 9; task += 32) {
    const int j = task / 9, k3 = task % 9;
    const int c = cells[j];
    if (c < 0) continue;
    int cx, cy;
    cell_xy(P, c, &cx, &cy);
    const double qn[3] = {0.0, 0.5, 1.0};
    double x[2], J[2][2];
    map_eval(ctrl, P.nx, P.m, cx, cy, qn[k3 % 3], qn[k3 / 3], x, J);
    const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    if (!(det > 0.0)) atomicOr(&flags[c], ROMB_FLAG_BAD_MAP);
    // G = J^-1, G[j][m] = dxi_j / dx_m
    const double G[2][2] = {{J[1][1] / det, -J[0][1] / det}, {-J[1][0] / det, J[0][0] / det}};
    double* out = chat + (long long)c * 144 + 16 * k3;
    for (int i = 0; i < 2; ++i)
      for (int jj = 0; jj < 2; ++jj)
        for (int k = 0; k < 2; ++k)
          for (int l = 0; l < 2; ++l) {
            // Chat_ijkl = det [lam G_ji G_lk + mu (d_ik (G G^T)_jl + G_jk G_li)]
            const double GGt = G[jj][0] * G[l][0] + G[jj][1] * G[l][1];
            // products grouped so that Chat_ijkl and Chat_klij round identically
            const double v = P.lam * (G[jj][i] * G[l][k]) + P.mu * ((i == k ? GGt : 0.0) + G[jj][k] * G[l][i]);
            out[((i * 2 + jj) * 2 + k) * 2 + l] = det * v;
            chat32[(long long)c * 144 + 16 * k3 + ((i * 2 + jj) * 2 + k) * 2 + l] = (float)(det * v);
          }
  }
}

// ---------------------------------------------------------------------------
// FP64 contraction: 32 cells x 4 pairs per CTA
// ---------------------------------------------------------------------------
#define A64_CELLS 32
#define A64_PAIRS 4
__global__ void __launch_bounds__(128) assemble_fp64_kernel(const double* __restrict__ U, long long n_half, int K,
                                                             const int* __restrict__ list, int count,
                                                             const int2* __restrict__ pairs, int npairs, int ndof,
                                                             const double* __restrict__ theta,
                                                             const double* __restrict__ chat,
                                                             double* __restrict__ Kout) {
  extern __shared__ double sm[];
  const int KS = K | 1;                      // odd stride: no bank conflicts across cells
  double* sU = sm;                           // [K][A64_PAIRS*36]
  double* sT = sU + (size_t)K * A64_PAIRS * 36;   // [32][KS]
  double* sC = sT + A64_CELLS * KS;          // [32][145]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int pair0 = blockIdx.y * A64_PAIRS;
  const int c0 = blockIdx.x * A64_CELLS;
  const int npl = min(A64_PAIRS, npairs - pair0);
  for (int i = tid; i < K * A64_PAIRS * 36; i += blockDim.x) {
    const int t = i / (A64_PAIRS * 36), e = i % (A64_PAIRS * 36);
    sU[i] = (e < npl * 36) ? U[(long long)t * n_half + (long long)pair0 * 36 + e] : 0.0;
  }
  for (int i = tid; i < A64_CELLS * K; i += blockDim.x) {
    const int j = i / K, t = i % K;
    const int c = c0 + j < count ? list[c0 + j] : -1;
    sT[j * KS + t] = c >= 0 ? theta[128 * (long long)c + t] : 0.0;
  }
  for (int i = tid; i < A64_CELLS * 144; i += blockDim.x) {
    const int j = i / 144, e = i % 144;
    const int c = c0 + j < count ? list[c0 + j] : -1;
    sC[j * 145 + e] = c >= 0 ? chat[144 * (long long)c + e] : 0.0;
  }
  __syncthreads();
  const int pl = warp;
  if (pl >= npl) return;
  const int cl = lane;
  const int cell = c0 + cl < count ? list[c0 + cl] : -1;
  double acc[36];
#pragma unroll
  for (int e = 0; e < 36; ++e) acc[e] = 0.0;
  const double* u = sU + pl * 36;
  const double* th = sT + cl * KS;
  for (int t = 0; t < K; ++t) {
    const double a = th[t];
    const double* ut = u + t * A64_PAIRS * 36;
#pragma unroll
    for (int e = 0; e < 36; ++e) acc[e] = fma(a, ut[e], acc[e]);
  }
  if (cell < 0) return;
  const int2 kk = pairs[pair0 + pl];
  const double* C = sC + cl * 145;
  double* Kc = Kout + (long long)cell * ((long long)ndof * (ndof + 1) / 2);
#pragma unroll
  for (int i1 = 0; i1 < 2; ++i1)
#pragma unroll
    for (int i2 = 0; i2 < 2; ++i2) {
      if (kk.x == kk.y && i1 > i2) continue;
      double v = 0.0;
#pragma unroll
      for (int k3 = 0; k3 < 9; ++k3)
#pragma unroll
        for (int j1 = 0; j1 < 2; ++j1)
#pragma unroll
          for (int j2 = 0; j2 < 2; ++j2)
            v = fma(acc[k3 * 4 + 2 * j1 + j2], C[16 * k3 + ((i1 * 2 + j1) * 2 + i2) * 2 + j2], v);
      const long long r = 2 * kk.x + i1, q = 2 * kk.y + i2;
      Kc[r * ndof - r * (r - 1) / 2 + (q - r)] = v;
    }
}

// dense [cells][ndof][ndof] -> packed upper triangle
__global__ void pack_dense_kernel(const double* __restrict__ dense, int ndof, long long cells,
                                  double* __restrict__ Kout) {
  const long long kp = (long long)ndof * (ndof + 1) / 2;
  const long long total = cells * kp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long c = i / kp;
    long long t = i % kp;
    // row r: entries t in [r*ndof - r(r-1)/2, ...)
    int r = 0;
    long long rowlen = ndof;
    while (t >= rowlen) {
      t -= rowlen;
      ++r;
      --rowlen;
    }
    const int q = r + (int)t;
    Kout[i] = dense[(c * ndof + r) * ndof + q];
  }
}

__global__ void flag_or_kernel(const int32_t* __restrict__ flags, long long n, int* __restrict__ out) {
  int v = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v |= flags[i];
  for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicOr(out, v);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static romb_status ensure_pairs(romb_ctx* c) {
  if (c->d_pairs) return ROMB_OK;
  const int nB = c->nB;
  std::vector<int2> pr;
  for (int k1 = 0; k1 < nB; ++k1)
    for (int k2 = k1; k2 < nB; ++k2) pr.push_back(make_int2(k1, k2));
  romb_status s = romb_alloc_t(c, &c->d_pairs, pr.size());
  if (s != ROMB_OK) return s;
  ROMB_CUDA(cudaMemcpy(c->d_pairs, pr.data(), sizeof(int2) * pr.size(), cudaMemcpyHostToDevice));
  return ROMB_OK;
}

romb_status launch_theta(romb_ctx* c) {
  romb_status s;
  if ((s = ensure_pairs(c)) != ROMB_OK) return s;
  // the model slot of every cell, then the cells grouped by slot
  {
    FamTab T;
    for (int f = 0; f < ROMB_MAX_FAMILIES; ++f) {
      T.n_k[f] = c->fams[f].n_k;
      T.slot0[f] = c->fams[f].slot0;
      T.lo[f] = c->fams[f].lo;
      T.hi[f] = c->fams[f].hi;
    }
    cell_model_kernel<<<(c->ncells + 255) / 256, 256, 0, c->stream>>>(T, c->d_family, c->d_mu, c->ncells, c->d_slot,
                                                                      c->d_flags); ++c->launches;
    ROMB_CUDA(cudaGetLastError());
  }
  int* d_counts = (int*)(c->d_red + 64);
  family_list_kernel<<<1, 1024, 0, c->stream>>>(c->d_slot, c->ncells, c->nslots, c->d_famlist, d_counts,
                                                c->d_flags); ++c->launches;
  ROMB_CUDA(cudaGetLastError());
  int counts[ROMB_MAX_MODELS] = {0};
  if (c->nslots > 0)
    ROMB_CUDA(cudaMemcpyAsync(counts, d_counts, sizeof(int) * c->nslots, cudaMemcpyDeviceToHost, c->stream));
  ROMB_CUDA(cudaStreamSynchronize(c->stream));
  CellParams P;
  fill_cell_params(c, &P);
  int start = 0;
  for (int f = 0; f < ROMB_MAX_MODELS; ++f) {
    c->famstart[f] = start;
    c->famcount[f] = counts[f];
    start += counts[f];
  }
  // cells of a family without models (slot -1) fall in no group
  if (start != c->ncells) return ROMB_E_ARG;
  // one launch per group of families that share the kernel's template
  // arguments (lane slots per coefficient, compile-time r + 1)
  const bool df = c->prec != ROMB_FP64;   // split forms: theta in double-float
  bool done[ROMB_MAX_MODELS] = {false};
  for (int f0 = 0; f0 < ROMB_MAX_MODELS; ++f0) {
    if (done[f0] || counts[f0] == 0) continue;
    const int ns = (c->roms[f0].n_r + 31) / 32;
    const bool r6 = df && c->roms[f0].r == 6;
    ThetaFams F;
    memset(&F, 0, sizeof(F));
    int grid = 0;
    for (int f = f0; f < ROMB_MAX_MODELS; ++f) {
      const RombRom& Rr = c->roms[f];
      if (done[f] || counts[f] == 0 || (Rr.n_r + 31) / 32 != ns || (df && Rr.r == 6) != r6) continue;
      done[f] = true;
      RomDev& R = F.rom[F.nfam];
      memset(&R, 0, sizeof(R));
      R.U64 = Rr.U64;
      R.At = Rr.At;
      R.At2 = Rr.At2;
      R.n_r = Rr.n_r;
      R.r = Rr.r;
      for (int d = 0; d < 4; ++d) {
        R.lo4[d] = Rr.lo4[d];
        R.hi4[d] = Rr.hi4[d];
      }
      R.n_half = Rr.n_half;
      gll_nodes01(Rr.r, R.g01);
      F.list[F.nfam] = c->d_famlist + c->famstart[f];
      F.count[F.nfam] = counts[f];
      F.cta0[F.nfam] = grid;
      grid += (counts[f] + 4 * TH_CELLS - 1) / (4 * TH_CELLS);
      ++F.nfam;
    }
    auto k = !df ? (ns <= 1 ? theta_kernel<1, false> : ns == 2 ? theta_kernel<2, false>
                              : ns == 3 ? theta_kernel<3, false> : theta_kernel<4, false>)
             : r6 ? (ns <= 1 ? theta_kernel<1, true, 7> : ns == 2 ? theta_kernel<2, true, 7>
                     : ns == 3 ? theta_kernel<3, true, 7> : theta_kernel<4, true, 7>)
                  : (ns <= 1 ? theta_kernel<1, true> : ns == 2 ? theta_kernel<2, true>
                     : ns == 3 ? theta_kernel<3, true> : theta_kernel<4, true>);
    k<<<grid, 128, 0, c->stream>>>(P, F, c->d_ctrl, c->d_mu, c->d_theta, c->d_chat, c->d_theta_hi, c->d_theta_lo,
                                   c->d_chat32, c->d_flags);
    ++c->launches;
    ROMB_CUDA(cudaGetLastError());
  }
  return ROMB_OK;
}

romb_status launch_assemble_fp64(romb_ctx* c) {
  const int npairs = c->nB * (c->nB + 1) / 2;
  for (int f = 0; f < ROMB_MAX_MODELS; ++f) {
    if (c->famcount[f] == 0) continue;
    const RombRom& R = c->roms[f];
    const int K = R.n_r + 1;
    const size_t smem = 8 * ((size_t)K * A64_PAIRS * 36 + A64_CELLS * (K | 1) + A64_CELLS * 145);
    static bool attr_done = false;
    if (!attr_done) {
      ROMB_CUDA(cudaFuncSetAttribute(assemble_fp64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      attr_done = true;
    }
    dim3 grid((c->famcount[f] + A64_CELLS - 1) / A64_CELLS, (npairs + A64_PAIRS - 1) / A64_PAIRS);
    assemble_fp64_kernel<<<grid, 128, smem, c->stream>>>(R.U64, R.n_half, K, c->d_famlist + c->famstart[f],
                                                         c->famcount[f], c->d_pairs, npairs, c->ndof, c->d_theta,
                                                         c->d_chat, c->d_K); ++c->launches;
    ROMB_CUDA(cudaGetLastError());
  }
  return ROMB_OK;
}

// The FP64 contraction for a list of cells against a given U' (K rows, half
// layout) and the cells' own theta rows.
romb_status launch_assemble_cells_fp64(romb_ctx* c, const double* U, long long n_half, int K, const int* d_list,
                                       int count) {
  const int npairs = c->nB * (c->nB + 1) / 2;
  const size_t smem = 8 * ((size_t)K * A64_PAIRS * 36 + A64_CELLS * (K | 1) + A64_CELLS * 145);
  ROMB_CUDA(cudaFuncSetAttribute(assemble_fp64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  dim3 grid((count + A64_CELLS - 1) / A64_CELLS, (npairs + A64_PAIRS - 1) / A64_PAIRS);
  assemble_fp64_kernel<<<grid, 128, smem, c->stream>>>(U, n_half, K, d_list, count, c->d_pairs, npairs, c->ndof,
                                                       c->d_theta, c->d_chat, c->d_K);
  ++c->launches;
  ROMB_CUDA(cudaGetLastError());
  return ROMB_OK;
}

romb_status launch_pack_dense(romb_ctx* c, const double* d_dense) {
  pack_dense_kernel<<<4 * c->sms, 256, 0, c->stream>>>(d_dense, c->ndof, c->ncells, c->d_K); ++c->launches;
  ROMB_CUDA(cudaGetLastError());
  return ROMB_OK;
}

romb_status launch_flag_or(romb_ctx* c, int* d_any) {
  flag_or_kernel<<<c->sms, 256, 0, c->stream>>>(c->d_flags, c->ncells, d_any); ++c->launches;
  ROMB_CUDA(cudaGetLastError());
  return ROMB_OK;
}
