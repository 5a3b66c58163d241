// Offline ROM training on the GPU (Sec. 4.2 and the offline phase of
// Sec. 4.4): the algorithm of the host trainer (train.cu), with every pass
// over the snapshots on the device.
//
//   moments     M(mu) of the trimmed cell (Legendre moments, height-function
//               form): one CTA per parameter point runs the adaptive panel
//               bisection of the host trainer (20-point Gauss panels, halved
//               until a panel and its two halves agree to 1e-15, depth <= 50)
//               on a shared-memory stack of intervals;
//   snapshots   I(mu) = F^T M G (Eq. MDEIM I): one CTA per point forms
//               H = M F^T in shared memory, then one entry of I per thread;
//   basis       Gram matrix S S^T (tiled FP64 GEMM), its eigenvectors on the
//               host (cyclic Jacobi, n_s x n_s), U_r = the leading
//               combinations of snapshots, orthonormalised by two passes of
//               Cholesky QR (Gram matrix, host Cholesky, triangular product);
//   magic pts   Algorithm 3 with the interpolatory residual, one residual
//               and arg-max pass over the n_i entries per point on the device
//               (ties: lowest index), the small solves on the host;
//   samples     moments at the (r+1)^4 tensor GLL nodes of the box and the
//               entries of I at the magic points on the device; I_r from
//               U_r[magic, :] I_r = I[magic] by LU on the host.
// Output: the ROM file of romb.h.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "romb_internal.cuh"
#include "tables.cuh"
#include "trim.cuh"

#define TG_MAXN 19      // D + 1 = 2 p + q + 1 <= 19
#define TG_PANEL 20     // Gauss points per panel
#define TG_STACK 64     // depth-first bisection keeps at most depth + 2 intervals

namespace {

struct TgQuad {
  int family, n, nm, maxdepth;
  double tol;
  double gx[TG_PANEL], gw[TG_PANEL];
};

// Moments M[s][t] = int_Omega P_s(2 xi1 - 1) P_t(2 xi2 - 1) of the solid part,
// one CTA per parameter point.
__global__ void __launch_bounds__(256) tg_moments_kernel(TgQuad Q, const double* __restrict__ mus, int npts,
                                                          double* __restrict__ Mout) {
  const int pt = blockIdx.x;
  if (pt >= npts) return;
  __shared__ double mu[4];
  __shared__ double sa[TG_STACK], sb[TG_STACK];
  __shared__ int sd[TG_STACK];
  __shared__ int top, cur_d, accept;
  __shared__ double cur_a, cur_b;
  __shared__ double Pv[3 * TG_PANEL][TG_MAXN], Iv[3 * TG_PANEL][TG_MAXN], W[3 * TG_PANEL];
  __shared__ double Mp[3][TG_MAXN * TG_MAXN];
  __shared__ double Macc[TG_MAXN * TG_MAXN];
  __shared__ double red[256];
  const int tid = threadIdx.x, n = Q.n, nm = Q.nm;
  if (tid < 4) mu[tid] = mus[4 * (long long)pt + tid];
  for (int i = tid; i < nm; i += blockDim.x) Macc[i] = 0.0;
  if (tid == 0) {   // the host trainer's two first panels, popped last-in first
    sa[0] = 0.0;
    sb[0] = 0.5;
    sd[0] = 0;
    sa[1] = 0.5;
    sb[1] = 1.0;
    sd[1] = 0;
    top = 2;
  }
  __syncthreads();
  while (true) {
    if (tid == 0) {
      if (top > 0) {
        --top;
        cur_a = sa[top];
        cur_b = sb[top];
        cur_d = sd[top];
      } else {
        cur_d = -1;
      }
    }
    __syncthreads();
    if (cur_d < 0) break;
    const double a = cur_a, b = cur_b, m = 0.5 * (a + b);
    // the Gauss points of the panels [a, b], [a, m], [m, b]
    for (int g = tid; g < 3 * TG_PANEL; g += blockDim.x) {
      const int k = g / TG_PANEL, j = g % TG_PANEL;
      const double lo_ = k == 2 ? m : a, hi_ = k == 1 ? m : b;
      const double x = lo_ + (hi_ - lo_) * Q.gx[j];
      W[g] = (hi_ - lo_) * Q.gw[j];
      double lo[4], hi[4], Au[TG_MAXN + 1], Av[TG_MAXN + 1], P[TG_MAXN + 1];
      const int ni = solid_y(Q.family, mu, x, lo, hi);
      double inner[TG_MAXN];
      for (int t = 0; t < n; ++t) inner[t] = 0.0;
      for (int kk = 0; kk < ni; ++kk) {
        legendre_antideriv(n - 1, lo[kk], Au);
        legendre_antideriv(n - 1, hi[kk], Av);
        for (int t = 0; t < n; ++t) inner[t] += Av[t] - Au[t];
      }
      legendre(n - 1, 2.0 * x - 1.0, P);
      for (int t = 0; t < n; ++t) {
        Pv[g][t] = P[t];
        Iv[g][t] = inner[t];
      }
    }
    __syncthreads();
    for (int idx = tid; idx < 3 * nm; idx += blockDim.x) {
      const int k = idx / nm, st = idx % nm, s = st / n, t = st % n;
      double acc = 0.0;
      for (int j = 0; j < TG_PANEL; ++j) {
        const int g = k * TG_PANEL + j;
        acc = fma(W[g] * Pv[g][s], Iv[g][t], acc);
      }
      Mp[k][st] = acc;
    }
    __syncthreads();
    double e = 0.0;
    for (int i = tid; i < nm; i += blockDim.x) e = fmax(e, fabs(Mp[0][i] - Mp[1][i] - Mp[2][i]));
    red[tid] = e;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (tid < o) red[tid] = fmax(red[tid], red[tid + o]);
      __syncthreads();
    }
    if (tid == 0) {
      accept = red[0] <= Q.tol || cur_d >= Q.maxdepth || top + 2 > TG_STACK;
      if (!accept) {
        sa[top] = a;
        sb[top] = m;
        sd[top] = cur_d + 1;
        sa[top + 1] = m;
        sb[top + 1] = b;
        sd[top + 1] = cur_d + 1;
        top += 2;
      }
    }
    __syncthreads();
    if (accept)
      for (int i = tid; i < nm; i += blockDim.x) Macc[i] += Mp[1][i] + Mp[2][i];
    __syncthreads();
  }
  for (int i = tid; i < nm; i += blockDim.x) Mout[(long long)pt * nm + i] = Macc[i];
}

struct TgShape {
  int p, q, n, nF, nB, nL, n_i;
};

// factor indices (xi1 factor f, xi2 factor g) of entry e of I
__device__ __forceinline__ void tg_factors(const TgShape& S, int e, int* f, int* g) {
  const int j2 = e & 1, j1 = (e >> 1) & 1;
  int t = e >> 2;
  const int k3 = t % S.nL;
  t /= S.nL;
  const int k2 = t % S.nB, k1 = t / S.nB;
  const int a1 = k1 % (S.p + 1), b1 = k1 / (S.p + 1), a2 = k2 % (S.p + 1), b2 = k2 / (S.p + 1);
  const int c1 = k3 % (S.q + 1), c2 = k3 / (S.q + 1);
  *f = (((a1 * 2 + (j1 == 0)) * (S.p + 1) + a2) * 2 + (j2 == 0)) * (S.q + 1) + c1;
  *g = (((b1 * 2 + (j1 == 1)) * (S.p + 1) + b2) * 2 + (j2 == 1)) * (S.q + 1) + c2;
}

// I(mu) from the moments: H = M F^T in shared memory, then I[e] = F[f] . H[:, g].
__global__ void __launch_bounds__(256) tg_snapshot_kernel(TgShape S, const double* __restrict__ F,
                                                           const double* __restrict__ M, double* __restrict__ I) {
  extern __shared__ double sh[];
  const int n = S.n, nF = S.nF, nm = n * n;
  double* H = sh;              // [n][nF]
  double* Ms = sh + n * nF;    // [n][n]
  const long long pt = blockIdx.x;
  for (int i = threadIdx.x; i < nm; i += blockDim.x) Ms[i] = M[pt * nm + i];
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * nF; idx += blockDim.x) {
    const int a = idx / nF, g = idx % nF;
    double s = 0.0;
    for (int b = 0; b < n; ++b) s += Ms[a * n + b] * __ldg(F + (long long)g * n + b);
    H[idx] = s;
  }
  __syncthreads();
  double* out = I + pt * S.n_i;
  for (int e = threadIdx.x; e < S.n_i; e += blockDim.x) {
    int f, g;
    tg_factors(S, e, &f, &g);
    double s = 0.0;
    for (int a = 0; a < n; ++a) s += __ldg(F + (long long)f * n + a) * H[a * nF + g];
    out[e] = s;
  }
}

// selected entries: out[a][pt] = I(mu_pt)[idx[a]]
__global__ void tg_entries_kernel(TgShape S, const double* __restrict__ F, const double* __restrict__ M,
                                  const long long* __restrict__ idx, int nidx, int npts, double* __restrict__ out) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nidx * npts) return;
  const int a0 = (int)(t / npts), pt = (int)(t % npts);
  const int n = S.n;
  int f, g;
  tg_factors(S, (int)idx[a0], &f, &g);
  const double* Mp = M + (long long)pt * n * n;
  double s = 0.0;
  for (int a = 0; a < n; ++a) {
    double h = 0.0;
    for (int b = 0; b < n; ++b) h += Mp[a * n + b] * F[(long long)g * n + b];
    s += F[(long long)f * n + a] * h;
  }
  out[t] = s;
}

// C[i][j] = sum_k A(i, k) B(k, j) with strided operands (FP64, 64 x 64 tiles,
// 256 threads x 4 x 4 outputs); C row-major M x N.
#define TG_T 64
#define TG_K 16
__global__ void __launch_bounds__(256) tg_gemm_kernel(int Mr, int Nc, int K, const double* __restrict__ A,
                                                       long long lai, long long lak, const double* __restrict__ B,
                                                       long long lbk, long long lbj, double* __restrict__ C) {
  __shared__ double As[TG_K][TG_T + 1], Bs[TG_K][TG_T + 1];
  const int i0 = blockIdx.y * TG_T, j0 = blockIdx.x * TG_T;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += TG_K) {
    for (int l = threadIdx.x; l < TG_K * TG_T; l += blockDim.x) {
      // contiguous along k when the operand is stored that way
      int kk, ii;
      if (lak == 1) {
        kk = l % TG_K;
        ii = l / TG_K;
      } else {
        kk = l / TG_T;
        ii = l % TG_T;
      }
      const int gi = i0 + ii, gk = k0 + kk;
      As[kk][ii] = (gi < Mr && gk < K) ? A[gi * lai + gk * lak] : 0.0;
      int kb, jj;
      if (lbk == 1) {
        kb = l % TG_K;
        jj = l / TG_K;
      } else {
        kb = l / TG_T;
        jj = l % TG_T;
      }
      const int gj = j0 + jj, gkb = k0 + kb;
      Bs[kb][jj] = (gj < Nc && gkb < K) ? B[gkb * lbk + gj * lbj] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TG_K; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        av[u] = As[kk][ty + 16 * u];
        bv[u] = Bs[kk][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
      if (i < Mr && j < Nc) C[(long long)i * Nc + j] = acc[u][v];
    }
}

// rows of U scaled: U[k][:] *= s[k]
__global__ void tg_scale_rows_kernel(double* __restrict__ U, const double* __restrict__ s, int nr, long long ni) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nr * ni; t += (long long)gridDim.x * blockDim.x)
    U[t] *= s[t / ni];
}

// Algorithm 3 step j: residual r_e = U[j][e] - sum_b c[b] U[b][e] and its
// arg-max |r| (lowest index on ties), per block into (val, idx) partials.
__global__ void __launch_bounds__(256) tg_residual_argmax_kernel(const double* __restrict__ U, long long ni, int j,
                                                                  const double* __restrict__ c,
                                                                  double* __restrict__ pval, long long* __restrict__ pidx) {
  __shared__ double sv[256];
  __shared__ long long si[256];
  double best = -1.0;
  long long bi = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ni; e += (long long)gridDim.x * blockDim.x) {
    double s = U[(long long)j * ni + e];
    for (int b = 0; b < j; ++b) s -= U[(long long)b * ni + e] * c[b];
    const double v = fabs(s);
    if (v > best) {   // e increases within a thread: strict > keeps the lowest index
      best = v;
      bi = e;
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double v2 = sv[threadIdx.x + o];
      const long long i2 = si[threadIdx.x + o];
      if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
        sv[threadIdx.x] = v2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pval[blockIdx.x] = sv[0];
    pidx[blockIdx.x] = si[0];
  }
}

// gather U[:, col] (nr values)
__global__ void tg_column_kernel(const double* __restrict__ U, long long ni, int nr, long long col,
                                 double* __restrict__ out) {
  const int k = threadIdx.x;
  if (k < nr) out[k] = U[(long long)k * ni + col];
}

// Device buffers freed on every exit path.
struct DevBufs {
  std::vector<void*> ptrs;
  template <class T>
  cudaError_t get(T** p, size_t n) {
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, std::max<size_t>(1, n) * sizeof(T));
    if (e == cudaSuccess) ptrs.push_back(q);
    *p = static_cast<T*>(q);
    return e;
  }
  ~DevBufs() {
    for (void* q : ptrs) cudaFree(q);
  }
};

romb_status gemm(int Mr, int Nc, int K, const double* A, long long lai, long long lak, const double* B, long long lbk,
                 long long lbj, double* C) {
  const dim3 grid((Nc + TG_T - 1) / TG_T, (Mr + TG_T - 1) / TG_T);
  tg_gemm_kernel<<<grid, 256>>>(Mr, Nc, K, A, lai, lak, B, lbk, lbj, C);
  ROMB_CUDA(cudaGetLastError());
  return ROMB_OK;
}

// lower Cholesky of an n x n SPD matrix (row-major, in place); false if not SPD
bool host_cholesky(int n, std::vector<double>& A) {
  for (int j = 0; j < n; ++j) {
    double d = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
    if (!(d > 0.0)) return false;
    d = sqrt(d);
    A[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
      A[(size_t)i * n + j] = s / d;
    }
    for (int k = j + 1; k < n; ++k) A[(size_t)j * n + k] = 0.0;
  }
  return true;
}

// inverse of a lower-triangular n x n matrix (row-major)
std::vector<double> host_lower_inverse(int n, const std::vector<double>& L) {
  std::vector<double> X((size_t)n * n, 0.0);
  for (int c = 0; c < n; ++c) {
    for (int i = c; i < n; ++i) {
      double s = i == c ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) s -= L[(size_t)i * n + k] * X[(size_t)k * n + c];
      X[(size_t)i * n + c] = s / L[(size_t)i * n + i];
    }
  }
  return X;
}

// LU with partial pivoting, in place; solve for several right-hand sides
struct HostLU {
  int n = 0;
  std::vector<double> a;
  std::vector<int> piv;
  bool factor(int n_, const std::vector<double>& A) {
    n = n_;
    a = A;
    piv.assign(n, 0);
    for (int k = 0; k < n; ++k) {
      int m = k;
      for (int i = k + 1; i < n; ++i)
        if (fabs(a[(size_t)i * n + k]) > fabs(a[(size_t)m * n + k])) m = i;
      piv[k] = m;
      if (a[(size_t)m * n + k] == 0.0) return false;
      if (m != k)
        for (int j = 0; j < n; ++j) std::swap(a[(size_t)k * n + j], a[(size_t)m * n + j]);
      for (int i = k + 1; i < n; ++i) {
        a[(size_t)i * n + k] /= a[(size_t)k * n + k];
        for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= a[(size_t)i * n + k] * a[(size_t)k * n + j];
      }
    }
    return true;
  }
  void solve(double* b) const {
    for (int k = 0; k < n; ++k) std::swap(b[k], b[piv[k]]);
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < i; ++k) b[i] -= a[(size_t)i * n + k] * b[k];
    for (int i = n - 1; i >= 0; --i) {
      for (int k = i + 1; k < n; ++k) b[i] -= a[(size_t)i * n + k] * b[k];
      b[i] /= a[(size_t)i * n + i];
    }
  }
};

romb_status check_spec(const romb_train_spec* sp) {
  if (!sp || sp->p < 3 || sp->p > ROMB_MAX_P || sp->q != 2 || (sp->family < 0 || sp->family > 5) ||
      (sp->basis != 0 && sp->basis != 1))
    return ROMB_E_ARG;
  return ROMB_OK;
}

// shared set-up: tables on the host, their device copies, the moment quadrature
struct TgSetup {
  std::vector<double> F, gx, gw, Ipi;
  int D = 0, nF = 0;
  TgQuad Q;
  TgShape S;
  double* dF = nullptr;
  romb_status init(const romb_train_spec* sp, DevBufs& buf) {
    romb_status s = train_host_tables(sp, F, &D, &nF, gx, gw, Ipi);
    if (s != ROMB_OK) return s;
    Q.family = sp->family;
    Q.n = D + 1;
    Q.nm = Q.n * Q.n;
    Q.maxdepth = 50;
    Q.tol = 1e-15;
    for (int j = 0; j < TG_PANEL; ++j) {
      Q.gx[j] = gx[j];
      Q.gw[j] = gw[j];
    }
    S.p = sp->p;
    S.q = sp->q;
    S.n = D + 1;
    S.nF = nF;
    S.nB = (sp->p + 1) * (sp->p + 1);
    S.nL = (sp->q + 1) * (sp->q + 1);
    S.n_i = S.nB * S.nB * S.nL * 4;
    ROMB_CUDA(buf.get(&dF, F.size()));
    ROMB_CUDA(cudaMemcpy(dF, F.data(), 8 * F.size(), cudaMemcpyHostToDevice));
    const size_t smem = 8 * ((size_t)S.n * S.nF + (size_t)S.n * S.n);
    ROMB_CUDA(cudaFuncSetAttribute(tg_snapshot_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return ROMB_OK;
  }
  // moments of n points (device mus) into dM
  romb_status moments(const double* dmus, int npts, double* dM) const {
    tg_moments_kernel<<<npts, 256>>>(Q, dmus, npts, dM);
    ROMB_CUDA(cudaGetLastError());
    return ROMB_OK;
  }
  romb_status snapshots(const double* dM, int npts, double* dI) const {
    const size_t smem = 8 * ((size_t)S.n * S.nF + (size_t)S.n * S.n);
    tg_snapshot_kernel<<<npts, 256, smem>>>(S, dF, dM, dI);
    ROMB_CUDA(cudaGetLastError());
    return ROMB_OK;
  }
};

}  // namespace

extern "C" romb_status romb_train_snapshots_gpu(int device, const romb_train_spec* sp, const double* mus, int n,
                                                double* I_out) {
  romb_status s;
  if ((s = check_spec(sp)) != ROMB_OK) return s;
  if (!mus || !I_out || n < 1) return ROMB_E_ARG;
  ROMB_CUDA(cudaSetDevice(device));
  DevBufs buf;
  TgSetup T;
  if ((s = T.init(sp, buf)) != ROMB_OK) return s;
  double *dmu = nullptr, *dM = nullptr, *dI = nullptr;
  ROMB_CUDA(buf.get(&dmu, 4 * (size_t)n));
  ROMB_CUDA(buf.get(&dM, (size_t)n * T.Q.nm));
  ROMB_CUDA(buf.get(&dI, (size_t)n * T.S.n_i));
  ROMB_CUDA(cudaMemcpy(dmu, mus, 32 * (size_t)n, cudaMemcpyHostToDevice));
  if ((s = T.moments(dmu, n, dM)) != ROMB_OK) return s;
  if ((s = T.snapshots(dM, n, dI)) != ROMB_OK) return s;
  ROMB_CUDA(cudaMemcpy(I_out, dI, 8 * (size_t)n * T.S.n_i, cudaMemcpyDeviceToHost));
  return ROMB_OK;
}

namespace {
// One model (one cluster) on the box [lo4[d], hi4[d]]: U_r [n_r][n_i], A
// [n_r][(r+1)^4], the magic points and the force model, in host arrays.
struct TgModel {
  std::vector<double> U, A;
  std::vector<long long> magic;
  RombForceModel force;
};
romb_status tg_train_box(const romb_train_spec* sp, const TgSetup& T, const double* lo4, const double* hi4,
                         const double* samples, int n_s, TgModel* out) {
  romb_status s;
  DevBufs buf;   // this model's device buffers, freed on return
  const long long ni = T.S.n_i;
  const int nm = T.Q.nm, n_r = sp->n_r;
  // snapshots S [n_s][n_i]
  double *dmu = nullptr, *dM = nullptr, *dS = nullptr, *dG = nullptr;
  ROMB_CUDA(buf.get(&dmu, 4 * (size_t)n_s));
  ROMB_CUDA(buf.get(&dM, (size_t)n_s * nm));
  ROMB_CUDA(buf.get(&dS, (size_t)n_s * ni));
  ROMB_CUDA(buf.get(&dG, (size_t)n_s * n_s));
  ROMB_CUDA(cudaMemcpy(dmu, samples, 32 * (size_t)n_s, cudaMemcpyHostToDevice));
  if ((s = T.moments(dmu, n_s, dM)) != ROMB_OK) return s;
  if ((s = T.snapshots(dM, n_s, dS)) != ROMB_OK) return s;
  // Gram matrix G = S S^T and its eigen-decomposition (host)
  if ((s = gemm(n_s, n_s, (int)ni, dS, ni, 1, dS, 1, ni, dG)) != ROMB_OK) return s;
  std::vector<double> G((size_t)n_s * n_s), w, V;
  ROMB_CUDA(cudaMemcpy(G.data(), dG, 8 * G.size(), cudaMemcpyDeviceToHost));
  for (int i = 0; i < n_s; ++i)   // symmetric to rounding: use the mean of both triangles
    for (int j = 0; j < i; ++j) G[(size_t)i * n_s + j] = G[(size_t)j * n_s + i] = 0.5 * (G[(size_t)i * n_s + j] + G[(size_t)j * n_s + i]);
  train_jacobi_eig(n_s, G, w, V);
  std::vector<int> order(n_s);
  for (int i = 0; i < n_s; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return w[a] > w[b]; });
  // U_r = rows V_sel^T S, scaled by 1 / sqrt(eigenvalue), then Cholesky QR twice
  std::vector<double> Vsel((size_t)n_s * n_r), scale(n_r);
  for (int k = 0; k < n_r; ++k) {
    if (!(w[order[k]] > 0.0)) return ROMB_E_NAN;
    scale[k] = 1.0 / sqrt(w[order[k]]);
    for (int si = 0; si < n_s; ++si) Vsel[(size_t)si * n_r + k] = V[(size_t)si * n_s + order[k]];
  }
  double *dV = nullptr, *dU = nullptr, *dU2 = nullptr, *dsc = nullptr, *dC = nullptr, *dL = nullptr;
  ROMB_CUDA(buf.get(&dV, Vsel.size()));
  ROMB_CUDA(buf.get(&dU, (size_t)n_r * ni));
  ROMB_CUDA(buf.get(&dU2, (size_t)n_r * ni));
  ROMB_CUDA(buf.get(&dsc, (size_t)n_r));
  ROMB_CUDA(buf.get(&dC, (size_t)n_r * n_r));
  ROMB_CUDA(buf.get(&dL, (size_t)n_r * n_r));
  ROMB_CUDA(cudaMemcpy(dV, Vsel.data(), 8 * Vsel.size(), cudaMemcpyHostToDevice));
  ROMB_CUDA(cudaMemcpy(dsc, scale.data(), 8 * (size_t)n_r, cudaMemcpyHostToDevice));
  if ((s = gemm(n_r, (int)ni, n_s, dV, 1, n_r, dS, ni, 1, dU)) != ROMB_OK) return s;
  tg_scale_rows_kernel<<<1024, 256>>>(dU, dsc, n_r, ni);
  ROMB_CUDA(cudaGetLastError());
  for (int pass = 0; pass < 2; ++pass) {
    if ((s = gemm(n_r, n_r, (int)ni, dU, ni, 1, dU, 1, ni, dC)) != ROMB_OK) return s;
    std::vector<double> C((size_t)n_r * n_r);
    ROMB_CUDA(cudaMemcpy(C.data(), dC, 8 * C.size(), cudaMemcpyDeviceToHost));
    for (int i = 0; i < n_r; ++i)
      for (int j = 0; j < i; ++j) C[(size_t)i * n_r + j] = C[(size_t)j * n_r + i];
    if (!host_cholesky(n_r, C)) return ROMB_E_NAN;
    const std::vector<double> Li = host_lower_inverse(n_r, C);
    ROMB_CUDA(cudaMemcpy(dL, Li.data(), 8 * Li.size(), cudaMemcpyHostToDevice));
    if ((s = gemm(n_r, (int)ni, n_r, dL, n_r, 1, dU, ni, 1, dU2)) != ROMB_OK) return s;
    std::swap(dU, dU2);
  }
  // magic points (Algorithm 3, interpolatory residual)
  const int nblk = 1024;
  double *dpv = nullptr, *dc = nullptr, *dcol = nullptr;
  long long *dpi = nullptr, *dmagic = nullptr;
  ROMB_CUDA(buf.get(&dpv, (size_t)nblk));
  ROMB_CUDA(buf.get(&dpi, (size_t)nblk));
  ROMB_CUDA(buf.get(&dc, (size_t)n_r));
  ROMB_CUDA(buf.get(&dcol, (size_t)n_r));
  ROMB_CUDA(buf.get(&dmagic, (size_t)n_r));
  std::vector<long long>& magic = out->magic;
  magic.assign(n_r, 0);
  std::vector<double> Um((size_t)n_r * n_r);   // Um[a][b] = U[b][magic[a]]
  std::vector<double> pv(nblk), col(n_r);
  std::vector<long long> pi(nblk);
  for (int j = 0; j < n_r; ++j) {
    std::vector<double> cvec(std::max(1, j));
    if (j > 0) {
      std::vector<double> A((size_t)j * j);
      for (int a = 0; a < j; ++a) {
        for (int b = 0; b < j; ++b) A[(size_t)a * j + b] = Um[(size_t)a * n_r + b];
        cvec[a] = Um[(size_t)a * n_r + j];
      }
      HostLU lu;
      if (!lu.factor(j, A)) return ROMB_E_NAN;
      lu.solve(cvec.data());
      ROMB_CUDA(cudaMemcpy(dc, cvec.data(), 8 * (size_t)j, cudaMemcpyHostToDevice));
    }
    tg_residual_argmax_kernel<<<nblk, 256>>>(dU, ni, j, dc, dpv, dpi);
    ROMB_CUDA(cudaGetLastError());
    ROMB_CUDA(cudaMemcpy(pv.data(), dpv, 8 * (size_t)nblk, cudaMemcpyDeviceToHost));
    ROMB_CUDA(cudaMemcpy(pi.data(), dpi, 8 * (size_t)nblk, cudaMemcpyDeviceToHost));
    int best = 0;
    for (int b = 1; b < nblk; ++b)
      if (pv[b] > pv[best] || (pv[b] == pv[best] && pi[b] < pi[best])) best = b;
    magic[j] = pi[best];
    tg_column_kernel<<<1, 128>>>(dU, ni, n_r, magic[j], dcol);
    ROMB_CUDA(cudaGetLastError());
    ROMB_CUDA(cudaMemcpy(col.data(), dcol, 8 * (size_t)n_r, cudaMemcpyDeviceToHost));
    for (int b = 0; b < n_r; ++b) Um[(size_t)j * n_r + b] = col[b];
  }
  // interpolation samples on the tensor GLL grid of the box
  const int n1 = sp->r + 1;
  const int ng = n1 * n1 * n1 * n1;
  double g1d[12];
  gll_nodes01(sp->r, g1d);
  std::vector<double> gmu(4 * (size_t)ng);
  for (int g = 0; g < ng; ++g) {
    const int i1 = g % n1, i2 = (g / n1) % n1, i3 = (g / (n1 * n1)) % n1, i4 = g / (n1 * n1 * n1);
    const int ii[4] = {i1, i2, i3, i4};
    for (int d = 0; d < 4; ++d) gmu[4 * (size_t)g + d] = lo4[d] + (hi4[d] - lo4[d]) * g1d[ii[d]];
  }
  double *dgmu = nullptr, *dgM = nullptr, *dB = nullptr;
  ROMB_CUDA(buf.get(&dgmu, gmu.size()));
  ROMB_CUDA(buf.get(&dgM, (size_t)ng * nm));
  ROMB_CUDA(buf.get(&dB, (size_t)n_r * ng));
  ROMB_CUDA(cudaMemcpy(dgmu, gmu.data(), 8 * gmu.size(), cudaMemcpyHostToDevice));
  ROMB_CUDA(cudaMemcpy(dmagic, magic.data(), 8 * (size_t)n_r, cudaMemcpyHostToDevice));
  if ((s = T.moments(dgmu, ng, dgM)) != ROMB_OK) return s;
  {
    const long long tot = (long long)n_r * ng;
    tg_entries_kernel<<<(int)((tot + 255) / 256), 256>>>(T.S, T.dF, dgM, dmagic, n_r, ng, dB);
    ROMB_CUDA(cudaGetLastError());
  }
  std::vector<double> Bm((size_t)n_r * ng);
  std::vector<double>& U = out->U;
  U.resize((size_t)n_r * ni);
  ROMB_CUDA(cudaMemcpy(Bm.data(), dB, 8 * Bm.size(), cudaMemcpyDeviceToHost));
  ROMB_CUDA(cudaMemcpy(U.data(), dU, 8 * U.size(), cudaMemcpyDeviceToHost));
  HostLU lu;
  if (!lu.factor(n_r, Um)) return ROMB_E_NAN;
  std::vector<double>& A = out->A;
  A.resize((size_t)n_r * ng);
  std::vector<double> b(n_r);
  for (int g = 0; g < ng; ++g) {
    for (int a = 0; a < n_r; ++a) b[a] = Bm[(size_t)a * ng + g];
    lu.solve(b.data());
    for (int a = 0; a < n_r; ++a) A[(size_t)a * ng + g] = b[a];
  }
  // J(mu) is small (n_f = 4 (p+1) (q+1)): trained on the host
  return train_force_model_box(sp, lo4, hi4, samples, n_s, &out->force);
}

bool tg_write_header(FILE* f, const romb_train_spec* sp, int n_k, long long ni, const std::vector<double>& Ipi) {
  unsigned char hdr[128];
  memset(hdr, 0, sizeof(hdr));
  memcpy(hdr, "ROMBDDC1", 8);
  const int32_t iv[8] = {2, sp->family, sp->basis, sp->p, sp->q, sp->r, sp->n_r, n_k};
  memcpy(hdr + 8, iv, 32);
  const double lohi[2] = {sp->lo, sp->hi};
  memcpy(hdr + 40, lohi, 16);
  const int64_t ni64 = ni;
  memcpy(hdr + 56, &ni64, 8);
  bool ok = fwrite(hdr, 1, 128, f) == 128;
  return ok && fwrite(Ipi.data(), 8, (size_t)ni, f) == (size_t)ni;
}

bool tg_write_model(FILE* f, const TgModel& M) {
  bool ok = fwrite(M.U.data(), 8, M.U.size(), f) == M.U.size();
  ok = ok && fwrite(M.A.data(), 8, M.A.size(), f) == M.A.size();
  ok = ok && fwrite(M.magic.data(), 8, M.magic.size(), f) == M.magic.size();
  return ok && write_force_section(f, M.force);
}
}  // namespace

extern "C" romb_status romb_train_gpu(int device, const romb_train_spec* sp, const double* samples, int n_s,
                                      const char* path) {
  return romb_train_gpu_clustered(device, sp, 1, samples, n_s, path);
}

extern "C" romb_status romb_train_gpu_clustered(int device, const romb_train_spec* sp, int n_k, const double* samples,
                                                int n_s, const char* path) {
  romb_status s;
  if ((s = check_spec(sp)) != ROMB_OK) return s;
  if (!samples || !path || n_s < 1 || n_k < 1 || n_k > 2 || sp->r < 1 || sp->r > 10 || sp->n_r < 1 ||
      sp->n_r > 127 || sp->n_r > n_s || !(sp->hi > sp->lo))
    return ROMB_E_ARG;
  ROMB_CUDA(cudaSetDevice(device));
  DevBufs buf;
  TgSetup T;
  if ((s = T.init(sp, buf)) != ROMB_OK) return s;
  FILE* f = fopen(path, "wb");
  if (!f) return ROMB_E_ARG;
  bool ok = tg_write_header(f, sp, n_k, T.S.n_i, T.Ipi);
  const int nK = n_k * n_k * n_k * n_k;
  const double h = (sp->hi - sp->lo) / n_k;
  for (int k = 0; k < nK && ok; ++k) {
    double lo4[4], hi4[4];
    for (int d = 0, kk = k; d < 4; ++d, kk /= n_k) {
      lo4[d] = sp->lo + h * (kk % n_k);
      hi4[d] = sp->lo + h * (kk % n_k + 1);
    }
    TgModel M;
    if ((s = tg_train_box(sp, T, lo4, hi4, samples + 4 * (size_t)n_s * k, n_s, &M)) != ROMB_OK) {
      fclose(f);
      return s;
    }
    ok = tg_write_model(f, M);
  }
  fclose(f);
  return ok ? ROMB_OK : ROMB_E_ARG;
}
