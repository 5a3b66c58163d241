// Dense FP64 factorisations in shared memory by one CTA (all threads take
// part): Cholesky, triangular solve and triangular inverse, used by the local
// BDDC set-up of every cell and by the diagonal blocks of the coarse fronts.
#pragma once

// GB300 issues an FP64 warp instruction every 16 SM cycles, so every dense
// step below maps threads onto exactly the entries that do work (lower
// triangles through tri_ij, trailing blocks row-major) and multiplies by
// reciprocal pivots instead of dividing.

// Lower-triangle position (i, j), j <= i, of the row-major linear index t.
__device__ __forceinline__ void tri_ij(int t, int& i, int& j) {
  int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  if ((r + 1) * (r + 2) / 2 <= t) ++r;
  else if (r * (r + 1) / 2 > t) --r;
  i = r;
  j = t - r * (r + 1) / 2;
}

// 1 / sqrt(d) for a pivot d > 0 by Newton's iteration for the reciprocal
// square root, y <- y + y (1/2 - (d/2) y^2), started from the FP32 estimate
// (relative error below 2^-22): the error squares with each step, so two
// steps leave only FP64 rounding (a few ulp).  Pivots outside the FP32 range
// use the FP64 square root and division.
__device__ __forceinline__ double pivot_rsqrt(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  const double h = 0.5 * d;
  double y = (double)rsqrtf((float)d);
  y = fma(y, fma(-h, y * y, 0.5), y);
  y = fma(y, fma(-h, y * y, 0.5), y);
  return y;
}

// In-place Cholesky (lower) of the n x n row-major A (stride lda); invd[k] =
// 1 / L_kk.  Right-looking in blocks of CB columns, three barriers per block:
// thread 0 factors the CB x CB diagonal block, every row below solves its CB
// entries against it, then a rank-CB update of the trailing lower triangle
// (CB = 2 measured fastest: larger blocks lengthen thread 0's serial part).
// Each entry receives the same FMAs in the same order as the column-by-column
// algorithm.
static __device__ void chol_smem(double* A, int n, int lda, double* invd, int* bad) {
  const int tid = threadIdx.x, nt = blockDim.x;
  constexpr int CB = 2;   // columns per block
  for (int k0 = 0; k0 < n; k0 += CB) {
    const int kb = min(CB, n - k0);
    if (tid == 0) {
      for (int a = 0; a < kb; ++a) {
        const int k = k0 + a;
        double d = A[k * lda + k];
        for (int b = 0; b < a; ++b) d = fma(-A[k * lda + k0 + b], A[k * lda + k0 + b], d);
        if (!(d > 0.0)) {
          *bad = 1;
          d = 1.0;
        }
        const double y = pivot_rsqrt(d);
        A[k * lda + k] = d * y;
        invd[k] = y;
        for (int r = a + 1; r < kb; ++r) {
          double v = A[(k0 + r) * lda + k];
          for (int b = 0; b < a; ++b) v = fma(-A[(k0 + r) * lda + k0 + b], A[k * lda + k0 + b], v);
          A[(k0 + r) * lda + k] = v * y;
        }
      }
    }
    __syncthreads();
    // panel: L[r][k0 + a] for rows r below the block (forward substitution)
    for (int r = k0 + kb + tid; r < n; r += nt) {
      double l[CB];
#pragma unroll
      for (int a = 0; a < CB; ++a) {
        if (a < kb) {
          double v = A[r * lda + k0 + a];
#pragma unroll
          for (int b = 0; b < a; ++b) v = fma(-l[b], A[(k0 + a) * lda + k0 + b], v);
          l[a] = v * invd[k0 + a];
          A[r * lda + k0 + a] = l[a];
        }
      }
    }
    __syncthreads();
    const int m = n - k0 - kb, np = m * (m + 1) / 2;
    for (int t = tid; t < np; t += nt) {
      int a, b;
      tri_ij(t, a, b);
      const int i = k0 + kb + a, j = k0 + kb + b;
      double v = A[i * lda + j];
#pragma unroll
      for (int c = 0; c < CB; ++c)
        if (c < kb) v = fma(-A[i * lda + k0 + c], A[j * lda + k0 + c], v);
      A[i * lda + j] = v;
    }
    __syncthreads();
  }
}

// B <- L^-1 B (n x ncols, stride ldb), in blocks of 4 rows, two barriers per
// block: each column solves the block's rows (forward substitution with the
// 4 x 4 diagonal block), then a rank-4 update of the rows below.  Each entry
// receives the same FMAs in the same order as the row-by-row algorithm.
static __device__ void trsm_lower(const double* L, int n, int ldl, const double* invd, double* B, int ldb, int ncols) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i0 = 0; i0 < n; i0 += 4) {
    const int ib = min(4, n - i0);
    for (int c = tid; c < ncols; c += nt) {
      double x[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        if (a < ib) {
          double v = B[(i0 + a) * ldb + c];
#pragma unroll
          for (int b = 0; b < a; ++b) v = fma(-L[(i0 + a) * ldl + i0 + b], x[b], v);
          x[a] = v * invd[i0 + a];
          B[(i0 + a) * ldb + c] = x[a];
        }
      }
    }
    __syncthreads();
    const int tot = (n - i0 - ib) * ncols;
    for (int t = tid; t < tot; t += nt) {
      const int r = i0 + ib + t / ncols, c = t % ncols;
      double v = B[r * ldb + c];
#pragma unroll
      for (int a = 0; a < 4; ++a)
        if (a < ib) v = fma(-L[r * ldl + i0 + a], B[(i0 + a) * ldb + c], v);
      B[r * ldb + c] = v;
    }
    __syncthreads();
  }
}

// M <- L^-1: M (n x n, stride ldm) is written whole (zero above the
// diagonal).  Blocks of 4 rows, two barriers per block: each column c solves
// the block's rows (M[r][c], c < r, from the rows above, then scaled by
// 1 / L_rr; M[r][r] = 1 / L_rr), then a rank-4 update of the rows below in
// the columns left of the block's end.  Same FMAs in the same order as the
// row-by-row algorithm.
static __device__ void tri_inverse(const double* L, int n, int ldl, const double* invd, double* M, int ldm) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int t = tid; t < n * n; t += nt) {
    const int r = t / n, c = t % n;
    M[r * ldm + c] = (r == c) ? invd[r] : 0.0;
  }
  __syncthreads();
  for (int i0 = 0; i0 < n; i0 += 4) {
    const int ib = min(4, n - i0), w = i0 + ib;
    for (int c = tid; c < w; c += nt) {
      double x[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        if (a < ib) {
          const int r = i0 + a;
          double v = M[r * ldm + c];
#pragma unroll
          for (int b = 0; b < a; ++b) v = fma(-L[r * ldl + i0 + b], x[b], v);
          if (c < r) v *= invd[r];
          x[a] = v;
          M[r * ldm + c] = v;
        }
      }
    }
    __syncthreads();
    const int tot = (n - w) * w;
    for (int t = tid; t < tot; t += nt) {
      const int r = w + t / w, c = t % w;
      double v = M[r * ldm + c];
#pragma unroll
      for (int a = 0; a < 4; ++a)
        if (a < ib) v = fma(-L[r * ldl + i0 + a], M[(i0 + a) * ldm + c], v);
      M[r * ldm + c] = v;
    }
    __syncthreads();
  }
}
