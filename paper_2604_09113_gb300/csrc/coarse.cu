// Coarse problem of BDDC (Sec. 3.3.4): S_C = sum_i R_C^(i)T Psi^(i)T S^(i) Psi^(i) R_C^(i),
// assembled and factorised by a sparse Cholesky.  The coarse unknowns live on
// the lattice vertices (2 DoFs) and edges (3 DoFs), so a geometric nested
// dissection of the cell rectangle by grid lines gives the elimination tree:
// every front holds its separator DoFs (eliminated) and the DoFs on the
// internal sides of its rectangle (updated), as dense lower triangles.
//
// Numeric factorisation, level by level from the leaves:
//   assemble   leaves: the cells' 20 x 20 coarse matrices; inner fronts: the
//              children's update matrices (extend-add), in a fixed order;
//   partial Cholesky of every front of the level, blocked by 32 columns:
//              diagonal block (one CTA per front), panel solve, trailing update.
//   The rows appended below each front (an identity block) take part in the
//   elimination and end as B = [L11^-T | -(L21 L11^-1)^T].
// Solve: forward (leaves -> root) and backward (root -> leaves) substitution,
// one GEMV with B per front and sweep, one launch per level and sweep.
#include <stdio.h>

#include <algorithm>
#include <map>
#include <unordered_map>
#include <vector>

#include "bulk.cuh"
#include "dense.cuh"
#include "device.cuh"
#include "tables.cuh"

#define ND_NB 32
#define ND_SMALL_N 256       // levels whose fronts all have n <= this use one warp per front,
#define ND_SMALL_SMEM 6144   // ... if B and one vector of the largest fit in this many doubles

namespace {

struct Group {
  int px, py;      // doubled coordinates
  int ndof;        // 2 (vertex) or 3 (edge)
  int base;        // first global coarse DoF
};

struct Builder {
  int nx, ny;
  unsigned dmask;
  long long NCV, NCH;
  // layouts with absent cells or clamped cell edges (empty for the full
  // rectangle): the coarse DoFs some present cell holds, and the cell number
  // of every grid position (-1 absent)
  std::vector<char> used;
  std::vector<int> grid_cell;
  std::vector<NdFront>* fronts;
  std::vector<std::vector<int>> rows;        // per front: global coarse DoFs (sep first)
  std::vector<std::vector<int>> leaf_cells;  // per front (leaves only)
  std::vector<int> depth;

  bool vertex_dir(int vx, int vy) const {
    return ((dmask & 1) && vx == 0) || ((dmask & 2) && vx == nx) || ((dmask & 4) && vy == 0) ||
           ((dmask & 8) && vy == ny);
  }
  // all non-Dirichlet groups in the closed doubled rectangle
  void groups_in(int x0, int x1, int y0, int y1, std::vector<Group>& out) const {
    for (int py = 2 * y0; py <= 2 * y1; ++py)
      for (int px = 2 * x0; px <= 2 * x1; ++px) {
        const bool ex = (px & 1) == 0, ey = (py & 1) == 0;
        if (!ex && !ey) continue;   // cell centre
        Group g;
        if (ex && ey) {
          const int vx = px / 2, vy = py / 2;
          if (vertex_dir(vx, vy)) continue;
          g = {px, py, 2, (int)(2LL * ((long long)vy * (nx + 1) + vx))};
        } else if (ey) {   // horizontal edge (cx, vy)
          const int cx = px / 2, vy = py / 2;
          if ((vy == 0 && (dmask & 4)) || (vy == ny && (dmask & 8))) continue;
          g = {px, py, 3, (int)(NCV + 3LL * ((long long)vy * nx + cx))};
        } else {           // vertical edge (vx, cy)
          const int vx = px / 2, cy = py / 2;
          if ((vx == 0 && (dmask & 1)) || (vx == nx && (dmask & 2))) continue;
          g = {px, py, 3, (int)(NCV + NCH + 3LL * ((long long)cy * (nx + 1) + vx))};
        }
        if (!used.empty() && !used[g.base]) continue;
        out.push_back(g);
      }
  }
  bool internal_side(const Group& g, int x0, int x1, int y0, int y1) const {
    return (g.px == 2 * x0 && x0 > 0) || (g.px == 2 * x1 && x1 < nx) || (g.py == 2 * y0 && y0 > 0) ||
           (g.py == 2 * y1 && y1 < ny);
  }
  int build(int x0, int x1, int y0, int y1) {
    const int w = x1 - x0, h = y1 - y0;
    std::vector<Group> gs;
    groups_in(x0, x1, y0, y1, gs);
    NdFront F;
    std::vector<int> elim, bnd;
    std::vector<int> kids;
    auto push = [](std::vector<int>& v, const Group& g) {
      for (int t = 0; t < g.ndof; ++t) v.push_back(g.base + t);
    };
    const bool leaf = w <= 2 && h <= 2;
    int xm = -1, ym = -1;
    if (!leaf) {
      if (w >= h) xm = x0 + w / 2;
      else ym = y0 + h / 2;
    }
    for (const Group& g : gs) {
      if (internal_side(g, x0, x1, y0, y1)) push(bnd, g);
      else if (leaf || (xm >= 0 && g.px == 2 * xm) || (ym >= 0 && g.py == 2 * ym)) push(elim, g);
    }
    if (!leaf) {
      if (xm >= 0) {
        kids.push_back(build(x0, xm, y0, y1));
        kids.push_back(build(xm, x1, y0, y1));
      } else {
        kids.push_back(build(x0, x1, y0, ym));
        kids.push_back(build(x0, x1, ym, y1));
      }
    }
    F.ns = (int)elim.size();
    F.nb = (int)bnd.size();
    F.children = kids;
    const int id = (int)fronts->size();
    fronts->push_back(F);
    std::vector<int> r = elim;
    r.insert(r.end(), bnd.begin(), bnd.end());
    rows.push_back(r);
    std::vector<int> cells;
    if (leaf)
      for (int cy = y0; cy < y1; ++cy)
        for (int cx = x0; cx < x1; ++cx) {
          const int g = cx + nx * cy;
          const int cell = grid_cell.empty() ? g : grid_cell[g];
          if (cell >= 0) cells.push_back(cell);
        }
    leaf_cells.push_back(cells);
    int d = 0;
    for (int k : kids) {
      (*fronts)[k].parent = id;
      d = std::max(d, depth[k] + 1);
    }
    depth.push_back(d);
    return id;
  }
};

struct FrontDev {
  int ns, nb;
  long long off;     // dense front (n x n)
  int idx_off;       // global coarse index of each row
  int child_off, nchild;
  int cell_off, ncell;
  int emap_off;      // extend-add positions of this front's update rows in its parent
  int ybuf_off;      // forward-solve update vector (nb)
  int wbuf_off;      // extend-add sources of each of the n rows (gsrc)
  int sbuf_off;      // forward result y_s = L11^-1 w_s (ns)
  long long bt_off;  // B^T (n x ns, row-major) of fronts on the row-kernel levels, -1 elsewhere
  long long bf_off;  // B (ns x n) in the FP32 copy of the split-precision forms
};

// The front's B = [L11^-T | -(L21 L11^-1)^T] (ns x n, row-major): the rows
// below the front in the FP64 pool, or its FP32 copy.
__device__ __forceinline__ const double* front_B(const FrontDev& f, const double* F) {
  const long long n = f.ns + f.nb;
  return F + f.off + n * n;
}
__device__ __forceinline__ const float* front_B(const FrontDev& f, const float* BF) { return BF + f.bf_off; }

}  // namespace

// ---------------------------------------------------------------------------
// device kernels
// ---------------------------------------------------------------------------
// Leaf fronts (level 0): zero the front, put the identity below it and add the
// cells' 20 x 20 coarse matrices (cells in a fixed order).  One CTA per front.
__global__ void nd_assemble_kernel(const FrontDev* __restrict__ fr, const int* __restrict__ level, double* __restrict__ F,
                                   const int* __restrict__ children, const int* __restrict__ emap,
                                   const int* __restrict__ cells, const int* __restrict__ cell_pos,
                                   const double* __restrict__ SCl) {
  const FrontDev f = fr[level[blockIdx.x]];
  const int n = f.ns + f.nb;
  double* A = F + f.off;
  for (long long t = threadIdx.x; t < (long long)(n + f.ns) * n; t += blockDim.x) A[t] = 0.0;
  __syncthreads();
  // identity below the front: the elimination turns it into L11^-T
  for (int e = threadIdx.x; e < f.ns; e += blockDim.x) A[(long long)(n + e) * n + e] = 1.0;
  for (int k = 0; k < f.ncell; ++k) {
    const int cell = cells[f.cell_off + k];
    const int* pos = cell_pos + 20 * (long long)cell;
    const double* s = SCl + 400 * (long long)cell;
    for (int t = threadIdx.x; t < 400; t += blockDim.x) {
      const int a = t / 20, b = t % 20;
      const int pa = pos[a], pb = pos[b];
      if (pa >= 0 && pb >= 0 && pa >= pb) A[(long long)pa * n + pb] += s[t];
    }
    __syncthreads();
  }
  for (int k = 0; k < f.nchild; ++k) {
    const FrontDev ch = fr[children[f.child_off + k]];
    const int cn = ch.ns + ch.nb;
    const double* C = F + ch.off;
    const int* em = emap + ch.emap_off;
    for (long long t = threadIdx.x; t < (long long)ch.nb * ch.nb; t += blockDim.x) {
      const int a = (int)(t / ch.nb), b = (int)(t % ch.nb);
      if (b > a) continue;
      int pa = em[a], pb = em[b];
      if (pa < pb) {
        const int tmp = pa;
        pa = pb;
        pb = tmp;
      }
      A[(long long)pa * n + pb] += C[(long long)(ch.ns + a) * cn + (ch.ns + b)];
    }
    __syncthreads();
  }
}

// Inner fronts: every entry of the lower triangle and of the identity rows
// below the front is written once, as the sum of the (at most two) children's
// update-matrix entries that land on it (asrc: per front row, the child front
// and the child's update row of each source, -1 if none).  The upper triangle
// is never read and is not written.  CTA = 8 rows of one front, warp per row.
__global__ void __launch_bounds__(256) nd_assemble_inner_kernel(const FrontDev* __restrict__ fr,
                                                                 const int* __restrict__ level, double* __restrict__ F,
                                                                 const int4* __restrict__ asrc) {
  const FrontDev f = fr[level[blockIdx.y]];
  const int ns = f.ns, n = ns + f.nb;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * 8 + warp;
  if (i >= n + ns) return;
  double* A = F + f.off + (long long)i * n;
  if (i >= n) {   // identity rows: the elimination turns them into [L11^-T | -M^T]
    for (int j = lane; j < n; j += 32) A[j] = (j == i - n) ? 1.0 : 0.0;
    return;
  }
  const int4* src = asrc + f.wbuf_off;
  const int4 si = src[i];
  for (int j = lane; j <= i; j += 32) {
    const int4 sj = src[j];
    double v = 0.0;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int chi = a == 0 ? si.x : si.z, ri = a == 0 ? si.y : si.w;
      if (chi < 0) continue;
      int rj = -1;
      if (sj.x == chi) rj = sj.y;
      else if (sj.z == chi) rj = sj.w;
      if (rj < 0) continue;
      const FrontDev ch = fr[chi];
      const int cn = ch.ns + ch.nb, hi = max(ri, rj), lo = min(ri, rj);
      v += F[ch.off + (long long)(ch.ns + hi) * cn + (ch.ns + lo)];
    }
    A[j] = v;
  }
}

// In-place Cholesky of the nbk x nbk block D (lower part used, zero padded to
// ND_NB) and M = L^-1 (zero padded), by the whole CTA with the blocked
// shared-memory routines (Newton pivots, same FMA order as column by column).
__device__ void nd_chol_inv_block(double (*D)[ND_NB + 1], double (*M)[ND_NB + 1], double* invd, int nbk,
                                  int32_t* bad) {
  chol_smem(&D[0][0], nbk, ND_NB + 1, invd, bad);
  tri_inverse(&D[0][0], nbk, ND_NB + 1, invd, &M[0][0], ND_NB + 1);
  for (int t = threadIdx.x; t < ND_NB * ND_NB; t += blockDim.x) {
    const int i = t / ND_NB, j = t % ND_NB;
    if (i >= nbk || j >= nbk) M[i][j] = 0.0;
  }
  __syncthreads();
}

// Factor the diagonal block [k0, k0 + nbk) of front f in place and store
// Linv = L_kk^-1 (ND_NB x ND_NB, zero padded) in slot `slot`.
__device__ void nd_factor_diag(const FrontDev& f, double* __restrict__ F, int k0, int32_t* bad,
                               double* __restrict__ Linv, int slot) {
  __shared__ double D[ND_NB][ND_NB + 1];
  __shared__ double M[ND_NB][ND_NB + 1];
  __shared__ double invd[ND_NB];
  const int n = f.ns + f.nb, nbk = min(ND_NB, f.ns - k0);
  double* A = F + f.off;
  for (int t = threadIdx.x; t < ND_NB * ND_NB; t += blockDim.x) {
    const int i = t / ND_NB, j = t % ND_NB;
    D[i][j] = (i < nbk && j <= i) ? A[(long long)(k0 + i) * n + (k0 + j)] : 0.0;
  }
  __syncthreads();
  nd_chol_inv_block(D, M, invd, nbk, bad);
  double* Li = Linv + (size_t)slot * ND_NB * ND_NB;
  for (int t = threadIdx.x; t < ND_NB * ND_NB; t += blockDim.x) {
    const int i = t / ND_NB, j = t % ND_NB;
    Li[t] = M[i][j];
    if (i < nbk && j <= i) A[(long long)(k0 + i) * n + (k0 + j)] = D[i][j];
  }
}

// First diagonal block of every front of a level (one CTA per front); the
// later blocks are factored by the trailing update that completes them.
__global__ void nd_potrf_kernel(const FrontDev* __restrict__ fr, const int* __restrict__ level, double* __restrict__ F,
                                int k0, int32_t* __restrict__ bad, double* __restrict__ Linv) {
  const FrontDev f = fr[level[blockIdx.x]];
  if (k0 >= f.ns) return;
  nd_factor_diag(f, F, k0, bad, Linv, blockIdx.x);
}

// Panel: rows r >= k1 of columns [k0, k1): A[r, :] <- A[r, :] L_kk^-T, as the
// product with Linv^T.  CTA = 32 rows of one front; thread = row x 4 columns
// (j = g, g+8, g+16, g+24: equal work per thread).
__global__ void __launch_bounds__(256) nd_trsm_kernel(const FrontDev* __restrict__ fr, const int* __restrict__ level,
                                                       double* __restrict__ F, int k0, const double* __restrict__ Linv) {
  const FrontDev f = fr[level[blockIdx.y]];
  if (k0 >= f.ns) return;
  const int n = f.ns + f.nb;
  const int nbk = min(ND_NB, f.ns - k0);
  const int k1 = k0 + nbk;
  const int r0 = k1 + blockIdx.x * 32;
  // rows below the front: identity row n + e is still e_e until the panel
  // holding column e, so rows n + e with e >= k1 are zero here: no work
  const int rend = n + k1;
  if (r0 >= rend) return;
  __shared__ double Li[ND_NB][ND_NB + 1];
  __shared__ double Ap[32][ND_NB + 1];
  double* A = F + f.off;
  const double* Lg = Linv + (size_t)blockIdx.y * ND_NB * ND_NB;
  for (int t = threadIdx.x; t < ND_NB * ND_NB; t += blockDim.x) {
    const int i = t / ND_NB, j = t % ND_NB;
    Li[i][j] = Lg[t];
    const int r = r0 + i;
    Ap[i][j] = (r < rend && j < nbk) ? A[(long long)r * n + k0 + j] : 0.0;
  }
  __syncthreads();
  const int rr = threadIdx.x >> 3, g = threadIdx.x & 7;
  const int r = r0 + rr;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = g + 8 * q;
    if (j >= nbk) continue;   // padding columns of a narrow last block: no work
    double x = 0.0;
    for (int tt = 0; tt <= j; ++tt) x = fma(Ap[rr][tt], Li[j][tt], x);
    if (r < rend) A[(long long)r * n + k0 + j] = x;
  }
}

// Trailing update: A[i][j] -= sum_{t in [k0,k1)} A[i][t] A[j][t] for rows i >= k1,
// columns k1 <= j < n with j <= i for front rows and every j < n for the rows
// below the front, which end as B = [L11^-T | -(L21 L11^-1)^T].
// 32 x 32 tiles, 256 threads (4 outputs each).  The CTA of the first tile
// (the next diagonal block, complete after this update) then factors that
// block and its inverse while the other tiles are still being updated.
__global__ void __launch_bounds__(256) nd_syrk_kernel(const FrontDev* __restrict__ fr, const int* __restrict__ level,
                                                       double* __restrict__ F, int k0, int32_t* __restrict__ bad,
                                                       double* __restrict__ Linv) {
  const FrontDev f = fr[level[blockIdx.y]];
  if (k0 >= f.ns) return;
  const int n = f.ns + f.nb;
  const int nbk = min(ND_NB, f.ns - k0);
  const int k1 = k0 + nbk;
  const int ntr = (n + f.ns - k1 + 31) / 32, ntc = (n - k1 + 31) / 32;
  const int tix = blockIdx.x;
  if (tix >= ntr * ntc) return;
  const int ti = tix / ntc, tj = tix % ntc;
  const int r0 = k1 + ti * 32, c0 = k1 + tj * 32;
  // rows n + e with e >= k1 below the front are still e_e, zero in this panel:
  // their update is exactly zero (the first tile, which carries the
  // lookahead, starts at row k1 and is never skipped)
  const int rend = n + k1;
  if (r0 >= rend) return;
  // skip tiles with no valid output
  if (r0 < n && c0 > r0 + 31) return;
  __shared__ double Pi[32][ND_NB + 1], Pj[32][ND_NB + 1];
  double* A = F + f.off;
  for (int t = threadIdx.x; t < 32 * ND_NB; t += blockDim.x) {
    const int rr = t / ND_NB, kk = t % ND_NB;
    const int ri = r0 + rr, rj = c0 + rr;
    Pi[rr][kk] = (ri < rend && kk < nbk) ? A[(long long)ri * n + k0 + kk] : 0.0;
    Pj[rr][kk] = (rj < n && kk < nbk) ? A[(long long)rj * n + k0 + kk] : 0.0;
  }
  __syncthreads();
  const int lr = threadIdx.x / 8, lc0 = (threadIdx.x % 8) * 4;
  const int gi = r0 + lr;
  if (gi < rend) {
    double acc[4] = {0, 0, 0, 0};
    for (int kk = 0; kk < nbk; ++kk) {
      const double a = Pi[lr][kk];
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[c] = fma(a, Pj[lc0 + c][kk], acc[c]);
    }
    const int jmax = gi < n ? gi : n - 1;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gj = c0 + lc0 + c;
      if (gj < n && gj <= jmax) A[(long long)gi * n + gj] -= acc[c];
    }
  }
  if (tix == 0 && k1 < f.ns) {   // lookahead: the next diagonal block is final now
    __syncthreads();
    nd_factor_diag(f, F, k1, bad, Linv, blockIdx.y);
  }
}

// ---- solves: one GEMV per front and sweep over B = [L11^-T | -M^T] ----
//
// With M = L21 L11^-1 (= A21 A11^-1) the forward step of a front,
//   y_s = L11^-1 w_s,   u_b = w_b - M w_s,
// is z = B^T w_s (y_s = z[0, ns), u_b = w_b + z[ns, n)), and the backward step,
//   x_s = L11^-T (y_s - L21^T x_b) = L11^-T y_s - M^T x_b,
// is x_s = B [y_s; x_b].  Both read the ns x n rows below the front once.
// w is gathered from the right-hand side and the children's update vectors
// through gsrc (up to two sources per row, in a fixed order).
struct NdRows {
  int front, row0;
};

__device__ inline double nd_gather_row(const int2 s, const double* __restrict__ ybuf) {
  double v = 0.0;
  if (s.x >= 0) v += ybuf[s.x];
  if (s.y >= 0) v += ybuf[s.y];
  return v;
}

// Every solve kernel first stages its part of B (static between solves) into
// shared memory with bulk copies, then waits for the previous kernel
// (programmatic dependent launch: the copies and the launch overlap the
// previous level's tail), gathers what that level produced and finally waits
// (bounded) for its copies.  GB300 issues an FP64 warp instruction every 16 SM
// cycles, so the loops have exact, warp-uniform trip counts.  A copy that does
// not arrive in time sets *err and the CTA skips its work.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

#define ND_WPC 4     // warps (fronts) per CTA in the small-front kernels

// Small fronts: one warp per front.  Shared memory per warp: `stride`
// doubles = the B block (ns x n, contiguous in the front, staged by one bulk
// copy) at offset 0 and a vector of n at offset `voff`.
template <typename T, typename S>
__device__ __forceinline__ bool nd_stage_block(const FrontDev& f, const S* __restrict__ Bsrc, T* region,
                                               uint64_t* bar, int lane, int* first) {
  const int n = f.ns + f.nb;
  const Span16 sp = span16t(front_B(f, Bsrc), (long long)f.ns * n);
  *first = sp.first;
  if (lane == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
    mbar_expect_tx(bar, sp.bytes);
    if (sp.bytes) bulk_g2s(region, sp.start, sp.bytes, bar);
  }
  return true;
}

// T = double: B from the FP64 pool (Bsrc = F); T = float: from its FP32 copy.
template <typename T>
__global__ void __launch_bounds__(32 * ND_WPC) nd_fwd_small_kernel(
    const FrontDev* __restrict__ fr, const int* __restrict__ level, int nfronts, const T* __restrict__ Bsrc,
    const int* __restrict__ idx, const int2* __restrict__ gsrc, const double* __restrict__ rhs,
    double* __restrict__ ybuf, double* __restrict__ sbuf, int stride, int voff, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char sh_raw[];
  T* sh = reinterpret_cast<T*>(sh_raw);
  __shared__ uint64_t bar[ND_WPC];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int fi = blockIdx.x * ND_WPC + warp;
  const bool has = fi < nfronts;
  const FrontDev f = fr[level[has ? fi : 0]];
  const int ns = f.ns, n = ns + f.nb;
  T* region = sh + (size_t)warp * stride;
  T* w = region + voff;
  int first = 0;
  if (has) nd_stage_block(f, Bsrc, region, &bar[warp], lane, &first);
  __syncwarp();   // the barrier is initialised before any lane waits on it
  // static gather indices before the wait: afterwards only the data loads remain
  int pid[ND_SMALL_N / 32];
  int2 pgs[ND_SMALL_N / 32];
#pragma unroll
  for (int k = 0; k < ND_SMALL_N / 32; ++k) {
    const int t = lane + 32 * k;
    pid[k] = (has && t < ns) ? idx[f.idx_off + t] : -1;
    pgs[k] = (has && t < n) ? gsrc[f.wbuf_off + t] : make_int2(-1, -1);
  }
  pdl_trigger();
  pdl_wait();
  if (!has) return;
#pragma unroll
  for (int k = 0; k < ND_SMALL_N / 32; ++k) {
    const int t = lane + 32 * k;
    if (t < n) w[t] = (T)((pid[k] >= 0 ? rhs[pid[k]] : 0.0) + nd_gather_row(pgs[k], ybuf));
  }
  const bool ok = mbar_wait(&bar[warp], 0);
  if (!__all_sync(0xffffffffu, ok)) {
    if (lane == 0) atomicExch(err, 1);
    return;
  }
  __syncwarp();
  const T* Bs = region + first;
  for (int c0 = 0; c0 < n; c0 += 32) {
    const int c = c0 + lane;
    const int emax = min(ns, c0 + 32);   // rows e > c of L11^-T are zero
    if (c < n) {
      T z0 = 0, z1 = 0;
      int e = 0;
      for (; e + 1 < emax; e += 2) {
        z0 = fma(Bs[e * n + c], w[e], z0);
        z1 = fma(Bs[(e + 1) * n + c], w[e + 1], z1);
      }
      if (e < emax) z0 = fma(Bs[e * n + c], w[e], z0);
      const double z = (double)(z0 + z1);
      if (c < ns) sbuf[f.sbuf_off + c] = z;
      else ybuf[f.ybuf_off + c - ns] = (double)w[c] + z;
    }
  }
}

// x_s = B [y_s; x_b]: lanes = (row r, column phase h) with R rows x P phases,
// R the smallest power of two >= min(ns, 32); phases combined by shuffles.
template <typename T>
__global__ void __launch_bounds__(32 * ND_WPC) nd_bwd_small_kernel(
    const FrontDev* __restrict__ fr, const int* __restrict__ level, int nfronts, const T* __restrict__ Bsrc,
    const int* __restrict__ idx, const double* __restrict__ sbuf, double* __restrict__ x, int stride, int voff,
    int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char sh_raw[];
  T* sh = reinterpret_cast<T*>(sh_raw);
  __shared__ uint64_t bar[ND_WPC];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int fi = blockIdx.x * ND_WPC + warp;
  const bool has = fi < nfronts;
  const FrontDev f = fr[level[has ? fi : 0]];
  const int ns = f.ns, n = ns + f.nb;
  T* region = sh + (size_t)warp * stride;
  T* v = region + voff;
  int first = 0;
  if (has) nd_stage_block(f, Bsrc, region, &bar[warp], lane, &first);
  __syncwarp();   // the barrier is initialised before any lane waits on it
  int pid[ND_SMALL_N / 32];
#pragma unroll
  for (int k = 0; k < ND_SMALL_N / 32; ++k) {
    const int c = lane + 32 * k;
    pid[k] = (has && c < n) ? idx[f.idx_off + c] : 0;
  }
  pdl_trigger();
  pdl_wait();
  if (!has) return;
  const int* id = idx + f.idx_off;
#pragma unroll
  for (int k = 0; k < ND_SMALL_N / 32; ++k) {
    const int c = lane + 32 * k;
    if (c < n) v[c] = (T)(c < ns ? sbuf[f.sbuf_off + c] : x[pid[k]]);
  }
  const bool ok = mbar_wait(&bar[warp], 0);
  if (!__all_sync(0xffffffffu, ok)) {
    if (lane == 0) atomicExch(err, 1);
    return;
  }
  __syncwarp();
  const T* Bs = region + first;
  int R = 1;
  while (R < ns && R < 32) R <<= 1;
  const int P = 32 / R, r = lane & (R - 1), h = lane / R;
  for (int e0 = 0; e0 < ns; e0 += R) {
    const int e = e0 + r;
    T s = 0;
    if (e < ns) {
      const T* row = Bs + e * n;
      for (int c = (e0 / P) * P + h; c < n; c += P) s = fma(row[c], v[c], s);
    }
    for (int o = R; o < 32; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (h == 0 && e < ns) x[id[e]] = (double)s;
  }
}

// ---- levels of wide fronts: row kernels over contiguous rows ----
// Forward z = B^T w_s runs over the rows of B^T (n x ns, stored after the
// factorisation), backward x_s = B [y_s; x_b] over the rows of B: a CTA owns
// `rb` consecutive rows, staged by one bulk copy, and its 8 warps take R rows
// each with P = 32 / R lanes per row (lane = row x column phase, phases summed
// by shuffles), P chosen per level so that every lane has ~16 FMAs.
struct NdRowShape {
  int P, rb, ld;   // lanes per row, rows per CTA, shared row stride (doubles, even)
};

// B^T of the fronts on the row-kernel levels (T = float: the FP32 copy).
template <typename T>
__global__ void nd_transpose_kernel(const FrontDev* __restrict__ fr, const int* __restrict__ level,
                                    const double* __restrict__ F, T* __restrict__ BT) {
  __shared__ double tile[32][33];
  const FrontDev f = fr[level[blockIdx.z]];
  const int ns = f.ns, n = ns + f.nb;
  const int e0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  if (e0 >= ns || c0 >= n) return;
  const double* B = F + f.off + (long long)n * n;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int e = e0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (e < ns && c < n) ? B[(long long)e * n + c] : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, e = e0 + threadIdx.x;
    if (c < n && e < ns) BT[f.bt_off + (long long)c * ns + e] = (T)tile[threadIdx.x][i];
  }
}

// The FP32 copy of every front's B (one CTA per front).
__global__ void nd_copy_b32_kernel(const FrontDev* __restrict__ fr, int nfronts, const double* __restrict__ F,
                                   float* __restrict__ BF) {
  for (int fi = blockIdx.x; fi < nfronts; fi += gridDim.x) {
    const FrontDev f = fr[fi];
    const long long len = (long long)f.ns * (f.ns + f.nb);
    const double* src = front_B(f, F);
    for (long long t = threadIdx.x; t < len; t += blockDim.x) BF[f.bf_off + t] = (float)src[t];
  }
}

template <typename T>
__device__ __forceinline__ void nd_stage_rows(const T* src, long long len, T* dst, uint64_t* bar, int* first) {
  const Span16 sp = span16t(src, len);
  *first = sp.first;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
    mbar_expect_tx(bar, sp.bytes);
    if (sp.bytes) bulk_g2s(dst, sp.start, sp.bytes, bar);
  }
}

// Offset of the vector behind the staged rows: len elements and the span's
// slack, rounded up to a 16-byte boundary.
template <typename T>
__device__ __forceinline__ long long nd_vec_offset(long long len) {
  constexpr long long g = 16 / sizeof(T);
  return (len + 2 * (g - 1) + (g - 1)) & ~(g - 1);
}

template <typename T>
__global__ void __launch_bounds__(256) nd_fwd_rows_kernel(const FrontDev* __restrict__ fr, const NdRows* __restrict__ items,
                                                           NdRowShape sh_, const T* __restrict__ BT,
                                                           const int* __restrict__ idx, const int2* __restrict__ gsrc,
                                                           const double* __restrict__ rhs, double* __restrict__ ybuf,
                                                           double* __restrict__ sbuf, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char sh_raw[];   // rows [rb][ns] (+slack), then w_s [ns]
  T* sh = reinterpret_cast<T*>(sh_raw);
  __shared__ uint64_t bar;
  __shared__ int first_s;
  const NdRows it = items[blockIdx.x];
  const FrontDev f = fr[it.front];
  const int ns = f.ns, n = ns + f.nb;
  const int nr = min(sh_.rb, n - it.row0);
  T* ws = sh + nd_vec_offset<T>((long long)nr * ns);
  int first = 0;
  nd_stage_rows(BT + f.bt_off + (long long)it.row0 * ns, (long long)nr * ns, sh, &bar, &first);
  if (threadIdx.x == 0) first_s = first;
  const int* id = idx + f.idx_off;
  const int2* gs = gsrc + f.wbuf_off;
  int pid[4];
  int2 pgs[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int e = threadIdx.x + 256 * k;
    pid[k] = e < ns ? id[e] : 0;
    pgs[k] = e < ns ? gs[e] : make_int2(-1, -1);
  }
  const int P = sh_.P, R = 32 / P;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = lane / P, h = lane % P;
  const int j = warp * R + r;       // row within the CTA
  const int c = it.row0 + j;        // row of B^T = column of B
  const int2 gsc = (j < nr && h == 0 && c >= ns) ? gs[c] : make_int2(-1, -1);
  pdl_trigger();
  pdl_wait();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int e = threadIdx.x + 256 * k;
    if (e < ns) ws[e] = (T)(rhs[pid[k]] + nd_gather_row(pgs[k], ybuf));
  }
  for (int e = threadIdx.x + 1024; e < ns; e += blockDim.x) ws[e] = (T)(rhs[id[e]] + nd_gather_row(gs[e], ybuf));
  const double wb = nd_gather_row(gsc, ybuf);
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }
  T z = 0;
  if (j < nr) {
    const T* row = sh + first_s + (long long)j * ns;
    const int emax = c < ns ? c : ns - 1;   // L11^-T is upper triangular: B^T row c < ns has e <= c
    T z1 = 0;
    int e = h;
    for (; e + P <= emax; e += 2 * P) {
      z = fma(row[e], ws[e], z);
      z1 = fma(row[e + P], ws[e + P], z1);
    }
    if (e <= emax) z = fma(row[e], ws[e], z);
    z += z1;
  }
  for (int o = 1; o < P; o <<= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
  if (j < nr && h == 0) {
    if (c < ns) sbuf[f.sbuf_off + c] = (double)z;
    else ybuf[f.ybuf_off + c - ns] = wb + (double)z;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) nd_bwd_rows_kernel(const FrontDev* __restrict__ fr, const NdRows* __restrict__ items,
                                                           NdRowShape sh_, const T* __restrict__ Bsrc,
                                                           const int* __restrict__ idx, const double* __restrict__ sbuf,
                                                           double* __restrict__ x, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char sh_raw[];   // rows [rb][n] (+slack), then v [n]
  T* sh = reinterpret_cast<T*>(sh_raw);
  __shared__ uint64_t bar;
  __shared__ int first_s;
  const NdRows it = items[blockIdx.x];
  const FrontDev f = fr[it.front];
  const int ns = f.ns, n = ns + f.nb;
  const int nr = min(sh_.rb, ns - it.row0);
  T* v = sh + nd_vec_offset<T>((long long)nr * n);
  int first = 0;
  nd_stage_rows(front_B(f, Bsrc) + (long long)it.row0 * n, (long long)nr * n, sh, &bar, &first);
  if (threadIdx.x == 0) first_s = first;
  const int* id = idx + f.idx_off;
  int pid[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int cc = threadIdx.x + 256 * k;
    pid[k] = (cc >= ns && cc < n) ? id[cc] : 0;
  }
  const int P = sh_.P, R = 32 / P;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = lane / P, h = lane % P;
  const int j = warp * R + r;
  const int e = it.row0 + j;
  pdl_trigger();
  pdl_wait();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int cc = threadIdx.x + 256 * k;
    if (cc < n) v[cc] = (T)(cc < ns ? sbuf[f.sbuf_off + cc] : x[pid[k]]);
  }
  for (int cc = threadIdx.x + 1024; cc < n; cc += blockDim.x)
    v[cc] = (T)(cc < ns ? sbuf[f.sbuf_off + cc] : x[id[cc]]);
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }
  T s = 0;
  if (j < nr) {
    const T* row = sh + first_s + (long long)j * n;
    T s1 = 0;
    int cc = (e / P) * P + h;   // columns left of row e are zero in L11^-T
    for (; cc + P < n; cc += 2 * P) {
      s = fma(row[cc], v[cc], s);
      s1 = fma(row[cc + P], v[cc + P], s1);
    }
    if (cc < n) s = fma(row[cc], v[cc], s);
    s += s1;
  }
  for (int o = 1; o < P; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (j < nr && h == 0) x[id[e]] = (double)s;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct NdDevice {
  FrontDev* fr = nullptr;
  int2* gsrc = nullptr;
  int4* asrc = nullptr;
  double* sbuf = nullptr;
  double* BT = nullptr;       // B^T of the fronts on row-kernel levels
  float* BF = nullptr;        // FP32 copies of every front's B and of B^T (split-precision
  float* BTF = nullptr;       // forms, allocated on their first factorisation)
  long long bf_n = 0, bt_n = 0;
  int nfronts = 0;
  std::vector<NdRows*> fwd_rows, bwd_rows;
  std::vector<int> fwd_n, bwd_n, level_small, level_maxb;
  std::vector<NdRowShape> fwd_shape, bwd_shape;
  std::vector<size_t> fwd_smem, bwd_smem;
  int* idx = nullptr;
  int* children = nullptr;
  int* emap = nullptr;
  int* cells = nullptr;
  int* cell_pos = nullptr;
  double* F = nullptr;
  double* ybuf = nullptr;
  std::vector<int*> level_ids;
  std::vector<int> level_count, level_maxns, level_maxn, level_maxtiles_trsm, level_maxtiles_syrk;
  int32_t* bad = nullptr;
  int* err = nullptr;   // set by a solve kernel whose staging copy timed out
  double* linv = nullptr;   // [fronts of the widest level][32 x 32] inverses of the diagonal blocks
  int ybuf_n = 0, sbuf_n = 0;   // sizes of the per-solve buffers (one pair per PCG lane)
};

static std::unordered_map<const romb_ctx*, NdDevice> g_nd;

romb_status coarse_build(romb_ctx* c) {
  NdPlan& plan = c->nd;
  plan = NdPlan();
  Builder B;
  B.nx = c->nx;
  B.ny = c->ny;
  B.dmask = c->dmask;
  B.NCV = 2LL * (c->nx + 1) * (c->ny + 1);
  B.NCH = 3LL * c->nx * (c->ny + 1);
  B.fronts = &plan.fronts;
  std::vector<int> cmap((size_t)c->ncells * 20);
  ROMB_CUDA(cudaMemcpy(cmap.data(), c->d_cmap, 4 * cmap.size(), cudaMemcpyDeviceToHost));
  if (c->layout) {
    B.used.assign((size_t)c->ncoarse_all, 0);
    for (int g : cmap)
      if (g >= 0) B.used[g] = 1;
    B.grid_cell.assign((size_t)c->nx * c->ny, -1);
    for (int i = 0; i < c->ncells; ++i) B.grid_cell[c->h_cell_grid[i]] = i;
  }
  const int root = B.build(0, c->nx, 0, c->ny);
  (void)root;
  const int nf = (int)plan.fronts.size();
  int maxd = 0;
  for (int d : B.depth) maxd = std::max(maxd, d);
  plan.levels.assign(maxd + 1, {});
  for (int i = 0; i < nf; ++i) {
    plan.fronts[i].level = B.depth[i];
    plan.levels[B.depth[i]].push_back(i);
  }
  // host arrays
  std::vector<FrontDev> fd(nf);
  std::vector<int> idx, children, emap, cells, cell_pos((size_t)c->ncells * 20, -1);
  long long off = 0, bttot = 0, bftot = 0;
  int ybuf = 0, wbuf_tot = 0, sbuf_tot = 0;
  for (int i = 0; i < nf; ++i) {
    const NdFront& F = plan.fronts[i];
    FrontDev& d = fd[i];
    d.ns = F.ns;
    d.nb = F.nb;
    const long long n = F.ns + F.nb;
    d.off = off;
    off += (n + F.ns) * n;   // rows n.. hold L11^-T after the factorisation
    d.idx_off = (int)idx.size();
    idx.insert(idx.end(), B.rows[i].begin(), B.rows[i].end());
    d.child_off = (int)children.size();
    d.nchild = (int)F.children.size();
    children.insert(children.end(), F.children.begin(), F.children.end());
    d.cell_off = (int)cells.size();
    d.ncell = (int)B.leaf_cells[i].size();
    cells.insert(cells.end(), B.leaf_cells[i].begin(), B.leaf_cells[i].end());
    d.ybuf_off = ybuf;
    ybuf += F.nb;
    d.wbuf_off = wbuf_tot;
    wbuf_tot += (int)n;
    d.sbuf_off = sbuf_tot;
    sbuf_tot += F.ns;
    d.emap_off = -1;
    d.bt_off = -1;
    d.bf_off = bftot;
    bftot += (long long)F.ns * n;
  }
  // extend-add positions of each front's update rows in its parent
  for (int i = 0; i < nf; ++i) {
    const NdFront& F = plan.fronts[i];
    if (F.parent < 0) continue;
    std::unordered_map<int, int> pos;
    const std::vector<int>& pr = B.rows[F.parent];
    for (int t = 0; t < (int)pr.size(); ++t) pos[pr[t]] = t;
    fd[i].emap_off = (int)emap.size();
    for (int t = F.ns; t < F.ns + F.nb; ++t) {
      auto it = pos.find(B.rows[i][t]);
      if (it == pos.end()) {
        romb_set_error("nested dissection: update row missing from parent front");
        return ROMB_E_CUDA;
      }
      emap.push_back(it->second);
    }
  }
  // extend-add sources of every front row: the children's update-vector entries
  // (gsrc, for the solves) and the child front / update row (asrc, for the assembly)
  std::vector<int4> asrc((size_t)std::max(1, wbuf_tot), make_int4(-1, -1, -1, -1));
  std::vector<int2> gsrc((size_t)std::max(1, wbuf_tot), make_int2(-1, -1));
  for (int i = 0; i < nf; ++i) {
    const NdFront& F = plan.fronts[i];
    if (F.parent < 0) continue;
    const FrontDev& pd = fd[F.parent];
    for (int a = 0; a < F.nb; ++a) {
      int2& s = gsrc[(size_t)pd.wbuf_off + emap[fd[i].emap_off + a]];
      int4& q = asrc[(size_t)pd.wbuf_off + emap[fd[i].emap_off + a]];
      const int src = fd[i].ybuf_off + a;
      if (s.x < 0) {
        s.x = src;
        q.x = i;
        q.y = a;
      } else if (s.y < 0) {
        s.y = src;
        q.z = i;
        q.w = a;
      } else {
        romb_set_error("nested dissection: more than two update sources for a front row");
        return ROMB_E_CUDA;
      }
    }
  }
  // cell -> leaf-front row of each local coarse slot
  for (int i = 0; i < nf; ++i) {
    if (B.leaf_cells[i].empty()) continue;
    std::unordered_map<int, int> pos;
    for (int t = 0; t < (int)B.rows[i].size(); ++t) pos[B.rows[i][t]] = t;
    for (int cell : B.leaf_cells[i])
      for (int s = 0; s < 20; ++s) {
        const int g = cmap[(size_t)cell * 20 + s];
        if (g < 0) continue;
        auto it = pos.find(g);
        if (it == pos.end()) {
          romb_set_error("nested dissection: cell coarse DoF missing from its leaf front");
          return ROMB_E_CUDA;
        }
        cell_pos[(size_t)cell * 20 + s] = it->second;
      }
  }
  plan.n = 0;
  for (int i = 0; i < nf; ++i) plan.n += plan.fronts[i].ns;
  plan.pool = off;
  // device
  NdDevice& D = g_nd[c];
  D = NdDevice();
  romb_status s;
  if ((s = romb_alloc(c, (void**)&D.fr, sizeof(FrontDev) * nf)) != ROMB_OK) return s;
  if ((s = romb_alloc_t(c, &D.idx, std::max<size_t>(1, idx.size()))) != ROMB_OK) return s;
  if ((s = romb_alloc_t(c, &D.children, std::max<size_t>(1, children.size()))) != ROMB_OK) return s;
  if ((s = romb_alloc_t(c, &D.emap, std::max<size_t>(1, emap.size()))) != ROMB_OK) return s;
  if ((s = romb_alloc_t(c, &D.cells, std::max<size_t>(1, cells.size()))) != ROMB_OK) return s;
  if ((s = romb_alloc_t(c, &D.cell_pos, cell_pos.size())) != ROMB_OK) return s;
  // +2 doubles: bulk copies read 16-byte aligned spans that may pass the end
  if ((s = romb_alloc_t(c, &D.F, (size_t)off + 2)) != ROMB_OK) return s;
  if ((s = romb_alloc_t(c, &D.ybuf, std::max(1, ybuf))) != ROMB_OK) return s;
  if ((s = romb_alloc_t(c, &D.gsrc, gsrc.size())) != ROMB_OK) return s;
  if ((s = romb_alloc_t(c, &D.asrc, asrc.size())) != ROMB_OK) return s;
  if ((s = romb_alloc_t(c, &D.sbuf, std::max(1, sbuf_tot))) != ROMB_OK) return s;
  D.ybuf_n = std::max(1, ybuf);
  D.sbuf_n = std::max(1, sbuf_tot);
  c->lane[0].nd_ybuf = D.ybuf;
  c->lane[0].nd_sbuf = D.sbuf;

  if ((s = romb_alloc_t(c, &D.bad, 1)) != ROMB_OK) return s;
  if ((s = romb_alloc_t(c, &D.err, 1)) != ROMB_OK) return s;
  {
    size_t widest = 1;
    for (const auto& lv : plan.levels) widest = std::max(widest, lv.size());
    if ((s = romb_alloc_t(c, &D.linv, widest * ND_NB * ND_NB)) != ROMB_OK) return s;
  }
  ROMB_CUDA(cudaMemset(D.err, 0, 4));
  D.nfronts = nf;
  ROMB_CUDA(cudaMemcpy(D.gsrc, gsrc.data(), sizeof(int2) * gsrc.size(), cudaMemcpyHostToDevice));
  ROMB_CUDA(cudaMemcpy(D.asrc, asrc.data(), sizeof(int4) * asrc.size(), cudaMemcpyHostToDevice));
  ROMB_CUDA(cudaMemcpy(D.idx, idx.data(), 4 * idx.size(), cudaMemcpyHostToDevice));
  if (!children.empty())
    ROMB_CUDA(cudaMemcpy(D.children, children.data(), 4 * children.size(), cudaMemcpyHostToDevice));
  if (!emap.empty()) ROMB_CUDA(cudaMemcpy(D.emap, emap.data(), 4 * emap.size(), cudaMemcpyHostToDevice));
  ROMB_CUDA(cudaMemcpy(D.cells, cells.data(), 4 * cells.size(), cudaMemcpyHostToDevice));
  ROMB_CUDA(cudaMemcpy(D.cell_pos, cell_pos.data(), 4 * cell_pos.size(), cudaMemcpyHostToDevice));
  for (const auto& lv : plan.levels) {
    int* d;
    if ((s = romb_alloc_t(c, &d, lv.size())) != ROMB_OK) return s;
    ROMB_CUDA(cudaMemcpy(d, lv.data(), 4 * lv.size(), cudaMemcpyHostToDevice));
    D.level_ids.push_back(d);
    D.level_count.push_back((int)lv.size());
    int mns = 0, mn = 0;
    for (int f : lv) {
      mns = std::max(mns, plan.fronts[f].ns);
      mn = std::max(mn, plan.fronts[f].ns + plan.fronts[f].nb);
    }
    D.level_maxns.push_back(mns);
    D.level_maxn.push_back(mn);
    int mb = 0;
    for (int f : lv) mb = std::max(mb, plan.fronts[f].ns * (plan.fronts[f].ns + plan.fronts[f].nb));
    D.level_maxb.push_back(mb);
    D.level_small.push_back(mn <= ND_SMALL_N && mb + mn + 8 <= ND_SMALL_SMEM);
    // row-kernel shapes: P lanes per row with ~16 FMAs each, 8 warps x 32/P rows per CTA
    auto shape_for = [](int len, int width) {
      NdRowShape q;
      q.P = 1;
      while (q.P < 32 && q.P * 16 < len) q.P <<= 1;
      q.rb = 8 * (32 / q.P);
      while (q.rb > 8 && (size_t)q.rb * width * 8 > 96 * 1024) q.rb >>= 1;
      q.ld = width;
      return q;
    };
    const NdRowShape fs = shape_for(mns, mns), bs = shape_for(mn, mn);
    D.fwd_shape.push_back(fs);
    D.bwd_shape.push_back(bs);
    D.fwd_smem.push_back(8 * ((((size_t)fs.rb * mns + 2) + 1 & ~(size_t)1) + mns));
    D.bwd_smem.push_back(8 * ((((size_t)bs.rb * mn + 2) + 1 & ~(size_t)1) + mn));
    std::vector<NdRows> fr_items, br_items;
    if (!D.level_small.back()) {
      for (int f : lv) {
        const NdFront& Fr = plan.fronts[f];
        const int n = Fr.ns + Fr.nb;
        fd[f].bt_off = bttot;
        bttot += (long long)n * Fr.ns;
        for (int r0 = 0; r0 < n; r0 += fs.rb) fr_items.push_back({f, r0});
        for (int e0 = 0; e0 < Fr.ns; e0 += bs.rb) br_items.push_back({f, e0});
      }
    }
    for (auto* pr : {&fr_items, &br_items}) {
      NdRows* dptr = nullptr;
      if (!pr->empty()) {
        if ((s = romb_alloc_t(c, &dptr, pr->size())) != ROMB_OK) return s;
        ROMB_CUDA(cudaMemcpy(dptr, pr->data(), sizeof(NdRows) * pr->size(), cudaMemcpyHostToDevice));
      }
      if (pr == &fr_items) {
        D.fwd_rows.push_back(dptr);
        D.fwd_n.push_back((int)pr->size());
      } else {
        D.bwd_rows.push_back(dptr);
        D.bwd_n.push_back((int)pr->size());
      }
    }
  }
  // B^T storage (+2 doubles: bulk copies read 16-byte aligned spans)
  if ((s = romb_alloc_t(c, &D.BT, (size_t)bttot + 2)) != ROMB_OK) return s;
  D.bf_n = bftot;
  D.bt_n = bttot;
  // front descriptors last: they carry the tile counts
  ROMB_CUDA(cudaMemcpy(D.fr, fd.data(), sizeof(FrontDev) * nf, cudaMemcpyHostToDevice));
  const int small_smem = 8 * ND_WPC * ND_SMALL_SMEM;
  size_t fmax = 0, bmax = 0;
  for (size_t l = 0; l < D.level_small.size(); ++l)
    if (!D.level_small[l]) {
      fmax = std::max(fmax, D.fwd_smem[l]);
      bmax = std::max(bmax, D.bwd_smem[l]);
    }
  if (fmax > 227 * 1024 || bmax > 227 * 1024) {
    romb_set_error("nested dissection: a coarse front is too wide for the staged solve kernels");
    return ROMB_E_ARG;
  }
  ROMB_CUDA(cudaFuncSetAttribute(nd_fwd_rows_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)std::max<size_t>(fmax, 16)));
  ROMB_CUDA(cudaFuncSetAttribute(nd_bwd_rows_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)std::max<size_t>(bmax, 16)));
  ROMB_CUDA(cudaFuncSetAttribute(nd_fwd_rows_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)std::max<size_t>(fmax, 16)));
  ROMB_CUDA(cudaFuncSetAttribute(nd_bwd_rows_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)std::max<size_t>(bmax, 16)));
  ROMB_CUDA(cudaFuncSetAttribute(nd_fwd_small_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, small_smem));
  ROMB_CUDA(cudaFuncSetAttribute(nd_bwd_small_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, small_smem));
  ROMB_CUDA(cudaFuncSetAttribute(nd_fwd_small_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, small_smem));
  ROMB_CUDA(cudaFuncSetAttribute(nd_bwd_small_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, small_smem));
  return ROMB_OK;
}

romb_status coarse_factor(romb_ctx* c) {
  NdDevice& D = g_nd[c];
  if (c->pre32 && !D.BF) {   // +4 floats: bulk copies read 16-byte aligned spans
    romb_status s;
    if ((s = romb_alloc_t(c, &D.BF, (size_t)D.bf_n + 4)) != ROMB_OK) return s;
    if ((s = romb_alloc_t(c, &D.BTF, (size_t)D.bt_n + 4)) != ROMB_OK) return s;
  }
  ROMB_CUDA(cudaMemsetAsync(D.bad, 0, 4, c->stream));
  for (size_t l = 0; l < D.level_ids.size(); ++l) {
    const int nfl = D.level_count[l];
    if (l == 0) {
      nd_assemble_kernel<<<nfl, 256, 0, c->stream>>>(D.fr, D.level_ids[l], D.F, D.children, D.emap, D.cells,
                                                     D.cell_pos, c->d_SCl);
    } else {
      const dim3 ga((D.level_maxn[l] + D.level_maxns[l] + 7) / 8, nfl);
      if (ga.x == 0) continue;   // every front of the level empty (layouts with absent cells)
      nd_assemble_inner_kernel<<<ga, 256, 0, c->stream>>>(D.fr, D.level_ids[l], D.F, D.asrc);
    }
    ++c->launches;
    ROMB_CUDA(cudaGetLastError());
    const int mns = D.level_maxns[l], mn = D.level_maxn[l];
    if (mns > 0) {
      nd_potrf_kernel<<<nfl, 256, 0, c->stream>>>(D.fr, D.level_ids[l], D.F, 0, D.bad, D.linv); ++c->launches;
    }
    for (int k0 = 0; k0 < mns; k0 += ND_NB) {
      const int rows = mn + mns - k0, cols = mn - k0;
      if (rows > 0 && cols > 0) {
        dim3 g1((rows + 31) / 32, nfl);
        nd_trsm_kernel<<<g1, 256, 0, c->stream>>>(D.fr, D.level_ids[l], D.F, k0, D.linv); ++c->launches;
        const int ntr = (rows + 31) / 32, ntc = (cols + 31) / 32;
        dim3 g2(ntr * ntc, nfl);
        nd_syrk_kernel<<<g2, 256, 0, c->stream>>>(D.fr, D.level_ids[l], D.F, k0, D.bad, D.linv); ++c->launches;
      }
      ROMB_CUDA(cudaGetLastError());
    }
    if (!D.level_small[l] && mns > 0) {   // B^T for the forward row kernel
      const dim3 gt((mn + 31) / 32, (mns + 31) / 32, nfl);
      if (c->pre32)
        nd_transpose_kernel<float><<<gt, dim3(32, 8), 0, c->stream>>>(D.fr, D.level_ids[l], D.F, D.BTF);
      else
        nd_transpose_kernel<double><<<gt, dim3(32, 8), 0, c->stream>>>(D.fr, D.level_ids[l], D.F, D.BT);
      ++c->launches;
      ROMB_CUDA(cudaGetLastError());
    }
  }
  if (c->pre32) {   // the solves of the split-precision forms read B in FP32
    nd_copy_b32_kernel<<<std::min(D.nfronts, 8 * c->sms), 256, 0, c->stream>>>(D.fr, D.nfronts, D.F, D.BF);
    ++c->launches;
    ROMB_CUDA(cudaGetLastError());
  }
  int bad = 0;
  ROMB_CUDA(cudaMemcpyAsync(&bad, D.bad, 4, cudaMemcpyDeviceToHost, c->stream));
  ROMB_CUDA(cudaStreamSynchronize(c->stream));
  if (bad) return ROMB_E_NOT_SPD;
  return ROMB_OK;
}

// out = S_C^-1 in over the non-Dirichlet coarse DoFs (Dirichlet entries of out are 0).
// Levels whose fronts are all small use one warp per front; the few levels of
// large fronts spread each GEMV over many CTAs.
// Launch with programmatic stream serialisation: the kernel may start while
// the previous one drains; it waits (griddepcontrol.wait) before reading what
// that kernel wrote.
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Per-solve buffers of the coarse solve for an additional PCG lane.
romb_status coarse_lane_buffers(romb_ctx* c, double** ybuf, double** sbuf) {
  NdDevice& D = g_nd[c];
  romb_status s;
  if ((s = romb_alloc_t(c, ybuf, (size_t)D.ybuf_n)) != ROMB_OK) return s;
  return romb_alloc_t(c, sbuf, (size_t)D.sbuf_n);
}

template <typename T>
static romb_status coarse_solve_t(romb_ctx* c, const double* d_in, double* d_out, cudaStream_t st, double* ybuf,
                                  double* sbuf, const T* Bsrc, const T* BTsrc) {
  NdDevice& D = g_nd[c];
  ROMB_CUDA(cudaMemsetAsync(d_out, 0, 8 * c->ncoarse_all, st));
  const int L = (int)D.level_ids.size();
  constexpr int g = 16 / (int)sizeof(T);   // elements per 16 bytes
  auto small_shape = [&](int l, int* stride, int* voff) {
    *voff = (D.level_maxb[l] + 2 * (g - 1) + (g - 1)) & ~(g - 1);   // B block + span slack, 16-byte aligned
    *stride = (*voff + D.level_maxn[l] + (g - 1)) & ~(g - 1);       // + one vector (16-byte regions)
  };
  for (int l = 0; l < L; ++l) {
    if (D.level_small[l]) {
      int stride, voff;
      small_shape(l, &stride, &voff);
      ROMB_CUDA(launch_pdl(nd_fwd_small_kernel<T>, (D.level_count[l] + ND_WPC - 1) / ND_WPC, 32 * ND_WPC,
                           sizeof(T) * ND_WPC * (size_t)stride, st, (const FrontDev*)D.fr,
                           (const int*)D.level_ids[l], D.level_count[l], Bsrc, (const int*)D.idx,
                           (const int2*)D.gsrc, d_in, ybuf, sbuf, stride, voff, D.err));
      ++c->launches;
    } else if (D.fwd_n[l]) {
      ROMB_CUDA(launch_pdl(nd_fwd_rows_kernel<T>, D.fwd_n[l], 256, D.fwd_smem[l], st, (const FrontDev*)D.fr,
                           (const NdRows*)D.fwd_rows[l], D.fwd_shape[l], BTsrc, (const int*)D.idx,
                           (const int2*)D.gsrc, d_in, ybuf, sbuf, D.err));
      ++c->launches;
    }
  }
  for (int l = L - 1; l >= 0; --l) {
    if (D.level_small[l]) {
      int stride, voff;
      small_shape(l, &stride, &voff);
      ROMB_CUDA(launch_pdl(nd_bwd_small_kernel<T>, (D.level_count[l] + ND_WPC - 1) / ND_WPC, 32 * ND_WPC,
                           sizeof(T) * ND_WPC * (size_t)stride, st, (const FrontDev*)D.fr,
                           (const int*)D.level_ids[l], D.level_count[l], Bsrc, (const int*)D.idx,
                           (const double*)sbuf, d_out, stride, voff, D.err));
      ++c->launches;
    } else if (D.bwd_n[l]) {
      ROMB_CUDA(launch_pdl(nd_bwd_rows_kernel<T>, D.bwd_n[l], 256, D.bwd_smem[l], st, (const FrontDev*)D.fr,
                           (const NdRows*)D.bwd_rows[l], D.bwd_shape[l], Bsrc, (const int*)D.idx,
                           (const double*)sbuf, d_out, D.err));
      ++c->launches;
    }
  }
  ROMB_CUDA(cudaGetLastError());
  return ROMB_OK;
}

// out = S_C^-1 in over the coarse DoFs that exist (the others of out are 0);
// the split-precision forms run the substitutions in FP32.
romb_status coarse_solve(romb_ctx* c, const double* d_in, double* d_out, cudaStream_t st, double* ybuf,
                         double* sbuf) {
  NdDevice& D = g_nd[c];
  if (c->pre32) return coarse_solve_t<float>(c, d_in, d_out, st, ybuf, sbuf, (const float*)D.BF, (const float*)D.BTF);
  return coarse_solve_t<double>(c, d_in, d_out, st, ybuf, sbuf, (const double*)D.F, (const double*)D.BT);
}

// Reports (and clears) a staging timeout of the solve kernels since the last call.
romb_status coarse_solve_check(romb_ctx* c) {
  NdDevice& D = g_nd[c];
  int e = 0;
  ROMB_CUDA(cudaMemcpy(&e, D.err, 4, cudaMemcpyDeviceToHost));
  if (e) {
    ROMB_CUDA(cudaMemset(D.err, 0, 4));
    romb_set_error("coarse solve: a shared-memory staging copy did not complete in time");
    return ROMB_E_CUDA;
  }
  return ROMB_OK;
}
