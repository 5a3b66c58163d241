// Tensor-core form of the assembly contraction (Sec. 4.1, Algorithm 4) on the
// 5th-generation tensor cores (tcgen05, kind::tf32), FP32 split precision.
//
//   I_c = theta_c U'          [128 cells x K] x [K x 144]  per N-tile (4 pairs k1 <= k2)
//   K_c[(k1 i1),(k2 i2)] = sum_{j1 j2 k3} I_c[k1 k2 k3 j1 j2] Chat_c[k3][i1 j1 i2 j2]
//
// The two dominant rows of U' (rho I_Pi and the first reduced basis vector) are
// applied exactly in FP64 in the epilogue; the remaining rows run on the tensor
// cores with the FP64 operands split x = hi + lo into TF32 values, accumulated
// in FP32 as hi*hi + hi*lo + lo*hi.  The epilogue forms I in FP64 and contracts
// it with Chat in FP64 (Chat rounded to FP32, exactly symmetric, held in
// registers).  The factor kernel then restores the exact null space of rigid
// translations (zero row sums) that the rounding perturbs.  The theta tile (A) stays in shared memory for the
// whole CTA; the U' tiles (B, hi and lo, pre-arranged at ROM load time in the
// canonical no-swizzle K-major layout) stream through a two-stage ring filled
// by bulk copies (cp.async.bulk + mbarrier transaction counts).  Accumulators
// live in tensor memory, double buffered, so the epilogue (tcgen05.ld, the
// Chat contraction in FP32 registers, packed FP64 stores) overlaps the MMAs of
// the next tile.  Every wait is bounded: on timeout the kernel records an error
// and all roles leave their loops; tensor memory is freed before exit.
//
// The BF16 form (kind::f16 with BF16 A and B, K = 16 per instruction) uses the
// same pipeline and epilogue on BF16 hi / lo splits (~16-bit products).
//
// Roles (256 threads): warp 0 allocates tensor memory and issues the copies,
// warp 1 issues the MMAs (one thread), warps 4-7 run the epilogue (TMEM lanes
// 0-127 = the 128 cells of the tile).
#include <stdint.h>
#include <stdio.h>

#include <vector>

#include <string.h>

#include <string>

#include "bulk.cuh"
#include "device.cuh"
#include "tables.cuh"

#define TC_M 128
#define TC_N 144
#define TC_PAIRS 4
#define TC_THREADS 384

struct TcFamily {
  const float* Utiles;     // per tile: hi, lo [TC_N x KT] (canonical layout), then rows 0, 1 as float pairs [2][TC_N][2]
  const int* list;         // cells of this family
  int count, mtile0;       // cells, first M-tile index of this family in the grid
};

struct TcParams {
  TcFamily fam[ROMB_MAX_FAMILIES];
  int nfam;
  const double* theta;     // [cells][128] f64 (slots 0, 1 applied exactly in the epilogue)
  int ntiles, KT;
  const float* th_hi;      // [cells][128]
  const float* th_lo;
  const float* chat32;     // [cells][144]
  double* Kout;            // [cells][ndof(ndof+1)/2]
  int ndof;
  const int2* pairs;
  int npairs;
  int stages;
  int* err;
};

// Shared-memory matrix descriptor: no swizzle, K-major canonical layout of
// 8-row x 16-byte core matrices; LBO = core-matrix stride along K, SBO = stride
// between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of the 5th-generation tensor cores
  return d;                 // base offset 0, swizzle mode 0 (none)
}

// Instruction descriptor of kind::tf32: D = F32, A = B = TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// BF16 bits of f, round to nearest even (finite inputs)
__host__ __device__ inline uint16_t bf16_bits(float f) {
  uint32_t u;
#ifdef __CUDA_ARCH__
  u = __float_as_uint(f);
#else
  memcpy(&u, &f, 4);
#endif
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
__host__ __device__ inline float bf16_value(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float* v) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ---- double-float (pair of FP32) arithmetic for the epilogue: ~48-bit
// significands on the FP32 pipe, which GB300 runs ~64x faster than FP64 ----
struct dfl {
  float hi, lo;
};
// Compensated accumulation (h, l) += x * y: the product is error-free
// (p + e via fmaf, plus the cross terms), the sum a two-sum whose error goes to
// the low word, which is not renormalised until the end (the dot-product
// scheme of Ogita, Rump and Oishi, 2005).  __fmul_rn keeps the compiler from
// contracting the product into the following add.
__device__ __forceinline__ void df_acc(float& h, float& l, dfl x, float2 y) {
  const float p = __fmul_rn(x.hi, y.x);
  float e = fmaf(x.hi, y.x, -p);
  e = fmaf(x.hi, y.y, e);
  e = fmaf(x.lo, y.x, e);
  const float s = __fadd_rn(h, p), bb = __fsub_rn(s, h);
  l = __fadd_rn(l, __fadd_rn(__fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb)), e));
  h = s;
}
__device__ __forceinline__ void df_acc_f(float& h, float& l, float xh, float xl, float c) {
  const float p = __fmul_rn(xh, c);
  float e = fmaf(xh, c, -p);
  e = fmaf(xl, c, e);
  const float s = __fadd_rn(h, p), bb = __fsub_rn(s, h);
  l = __fadd_rn(l, __fadd_rn(__fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb)), e));
  h = s;
}
__device__ __forceinline__ dfl df_from_double(double d) {
  const float h = (float)d;
  return {h, (float)(d - (double)h)};
}

// byte offset of element (row, k) in a canonical tile with SBO = KT * 32
__host__ __device__ inline uint32_t canon_off(int row, int k, int KT) {
  return (uint32_t)((row >> 3) * (KT * 32) + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}
// the same for 16-bit elements: core matrices of 8 rows x 8 elements, SBO = KT * 16
__host__ __device__ inline uint32_t canon_off16(int row, int k, int KT) {
  return (uint32_t)((row >> 3) * (KT * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

template <bool BF>
__global__ void __launch_bounds__(TC_THREADS, 1) assemble_tc_kernel(TcParams P) {
  constexpr uint32_t ES = BF ? 2 : 4;   // operand element size
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[2], bar_empty[2], bar_accfull[2], bar_accempty[2], bar_done;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int KT = P.KT;
  const uint32_t a_bytes = TC_M * KT * ES, b_bytes = TC_N * KT * ES;
  const uint32_t stage_bytes = 2 * b_bytes + 2 * TC_N * 8;
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* A_hi = base;
  unsigned char* A_lo = base + a_bytes;
  unsigned char* Bst = base + 2 * a_bytes;   // stage s at Bst + s * 2 * b_bytes (hi, lo)
  const int S = P.stages;
  const int T = P.ntiles;
  int fi = 0;
  while (fi + 1 < P.nfam && (int)blockIdx.x >= P.fam[fi + 1].mtile0) ++fi;
  const TcFamily F = P.fam[fi];
  const int m0 = ((int)blockIdx.x - F.mtile0) * TC_M;

  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < 2; ++s) {
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_empty[s], 1 + 8);   // MMA commit + one arrival per epilogue warp
      mbar_init(&bar_accfull[s], 1);
      mbar_init(&bar_accempty[s], 256);
    }
    mbar_init(&bar_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    // 512 columns: two 144-column accumulators
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base_s))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // A tile: theta hi / lo of the 128 cells, canonical layout
  for (int i = tid; i < TC_M * KT; i += TC_THREADS) {
    const int row = i / KT, k = i % KT;
    const int ci = m0 + row;
    float h = 0.f, l = 0.f;
    if (ci < F.count) {
      const long long cell = F.list[ci];
      h = P.th_hi[cell * 128 + k];
      l = P.th_lo[cell * 128 + k];
    }
    if (BF) {
      const float x = h + l;   // theta in TF32 hi + lo (zero padded), re-split into BF16
      const uint16_t bh = bf16_bits(x), bl = bf16_bits(x - bf16_value(bh));
      const uint32_t off = canon_off16(row, k, KT);
      *(uint16_t*)(A_hi + off) = bh;
      *(uint16_t*)(A_lo + off) = bl;
    } else {
      const uint32_t off = canon_off(row, k, KT);
      *(float*)(A_hi + off) = h;
      *(float*)(A_lo + off) = l;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  if (warp == 0) {
    if (lane == 0) {
      // producer: U' tiles into the ring
      int armed_last[2] = {-1, -1};
      for (int t = 0; t < T && !s_abort; ++t) {
        const int s = t % S;
        if (t >= S && !mbar_wait(&bar_empty[s], (uint32_t)(((t / S) - 1) & 1), &s_abort)) {
          s_abort = 1;
          atomicOr(P.err, 1);
          break;
        }
        unsigned char* dst = Bst + (size_t)s * stage_bytes;
        mbar_expect_tx(&bar_full[s], stage_bytes);
        bulk_g2s(dst, (const unsigned char*)F.Utiles + (size_t)t * stage_bytes, stage_bytes, &bar_full[s]);
        armed_last[s] = t;
      }
      // drain: every armed copy must land before the CTA exits
      for (int s = 0; s < 2; ++s)
        if (armed_last[s] >= 0) mbar_wait(&bar_full[s], (uint32_t)((armed_last[s] / S) & 1), nullptr);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = BF ? idesc_bf16(TC_M, TC_N) : idesc_tf32(TC_M, TC_N);
      const uint32_t sbo = (uint32_t)KT * 8 * ES, lbo = 128;
      const uint32_t a_hi = smem_u32(A_hi), a_lo = smem_u32(A_lo);
      for (int t = 0; t < T && !s_abort; ++t) {
        const int s = t % S, b = t & 1;
        if (!mbar_wait(&bar_full[s], (uint32_t)((t / S) & 1), &s_abort)) {
          s_abort = 1;
          atomicOr(P.err, 2);
          break;
        }
        if (t >= 2 && !mbar_wait(&bar_accempty[b], (uint32_t)(((t >> 1) - 1) & 1), &s_abort)) {
          s_abort = 1;
          atomicOr(P.err, 4);
          break;
        }
        tc_fence_after();
        const uint32_t b_hi = smem_u32(Bst + (size_t)s * stage_bytes), b_lo = b_hi + b_bytes;
        const uint32_t d = tmem + (uint32_t)(b * TC_N);
        // one instruction covers two core matrices along K (32 bytes): 8 TF32 or 16 BF16
        for (int kk = 0; kk < KT / (32 / (int)ES); ++kk) {
          const uint32_t ko = (uint32_t)kk * 256;
          if (BF) {
            mma_bf16(d, smem_desc(a_hi + ko, lbo, sbo), smem_desc(b_hi + ko, lbo, sbo), idesc, kk > 0);
            mma_bf16(d, smem_desc(a_hi + ko, lbo, sbo), smem_desc(b_lo + ko, lbo, sbo), idesc, 1);
            mma_bf16(d, smem_desc(a_lo + ko, lbo, sbo), smem_desc(b_hi + ko, lbo, sbo), idesc, 1);
          } else {
            mma_tf32(d, smem_desc(a_hi + ko, lbo, sbo), smem_desc(b_hi + ko, lbo, sbo), idesc, kk > 0);
            mma_tf32(d, smem_desc(a_hi + ko, lbo, sbo), smem_desc(b_lo + ko, lbo, sbo), idesc, 1);
            mma_tf32(d, smem_desc(a_lo + ko, lbo, sbo), smem_desc(b_hi + ko, lbo, sbo), idesc, 1);
          }
        }
        mma_commit(&bar_empty[s]);
        mma_commit(&bar_accfull[b]);
      }
      // all issued MMAs complete before tensor memory is released
      mma_commit(&bar_done);
      mbar_wait(&bar_done, 0, nullptr);
    }
  } else if (warp >= 4) {
    // two epilogue warpgroups read the same 128 TMEM lanes (cells); warpgroup g
    // produces the rows i1 = g of every 2x2 block
    const int g = (warp - 4) >> 2;
    const int row = ((warp & 3) << 5) + lane;
    const int ci = m0 + row;
    const bool valid = ci < F.count;
    const long long cell = valid ? F.list[ci] : 0;
    float C[72];   // Chat[k3][g][j1][i2][j2]
#pragma unroll
    for (int k3 = 0; k3 < 9; ++k3)
#pragma unroll
      for (int e = 0; e < 8; ++e) C[8 * k3 + e] = valid ? P.chat32[cell * 144 + 16 * k3 + 8 * g + e] : 0.f;
    const dfl th0 = df_from_double(valid ? P.theta[cell * 128 + 0] : 0.0);
    const dfl th1 = df_from_double(valid ? P.theta[cell * 128 + 1] : 0.0);
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const long long kp = (long long)P.ndof * (P.ndof + 1) / 2;
    double* Kc = P.Kout + cell * kp;
    for (int t = 0; t < T && !s_abort; ++t) {
      const int b = t & 1, s = t % S;
      if (!mbar_wait(&bar_accfull[b], (uint32_t)((t >> 1) & 1), &s_abort)) {
        s_abort = 1;
        atomicOr(P.err, 8);
        break;
      }
      tc_fence_after();
      const float2* U01 = (const float2*)(Bst + (size_t)s * stage_bytes + 2 * b_bytes);   // [2][TC_N] (hi, lo)
#pragma unroll 1
      for (int pl = 0; pl < TC_PAIRS; ++pl) {
        float acc[36];
        const uint32_t col = tmem + lane_base + (uint32_t)(b * TC_N + 36 * pl);
        tmem_ld16(col, acc);
        tmem_ld16(col + 16, acc + 16);
        tmem_ld4(col + 32, acc + 32);
        tmem_wait_ld();
        const int pr = t * TC_PAIRS + pl;
        if (!valid || pr >= P.npairs) continue;
        const int2 kk = P.pairs[pr];
        float v0h = 0.f, v0l = 0.f, v1h = 0.f, v1l = 0.f;
#pragma unroll
        for (int k3 = 0; k3 < 9; ++k3)
#pragma unroll
          for (int j1 = 0; j1 < 2; ++j1)
#pragma unroll
            for (int j2 = 0; j2 < 2; ++j2) {
              const int e = k3 * 4 + 2 * j1 + j2;
              // I_e = theta_0 U'_0 + theta_1 U'_1 + (tensor-core rows 2..)
              float ih = acc[e], il = 0.f;
              df_acc(ih, il, th0, U01[36 * pl + e]);
              df_acc(ih, il, th1, U01[TC_N + 36 * pl + e]);
              df_acc_f(v0h, v0l, ih, il, C[8 * k3 + 4 * j1 + j2]);       // i2 = 0
              df_acc_f(v1h, v1l, ih, il, C[8 * k3 + 4 * j1 + 2 + j2]);   // i2 = 1
            }
        const long long r = 2 * kk.x + g, q0 = 2 * kk.y;
        double* Kr = Kc + r * P.ndof - r * (r - 1) / 2 - r;
        if (!(kk.x == kk.y && g == 1)) Kr[q0] = (double)v0h + (double)v0l;
        Kr[q0 + 1] = (double)v1h + (double)v1l;
      }
      tc_fence_before();
      mbar_arrive(&bar_accempty[b]);
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_empty[s]);   // this warp is done with U'0, U'1 of the stage
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// Re-arrange U' (hi / lo, [kpad][n_half] row-major over K) into N-tiles of 144
// columns in the canonical K-major layout, hi then lo per tile.
// Tiles of 144 columns: TF32 hi and lo of rows 2.. of U' in the canonical
// K-major layout (rows 0 and 1 zero there), then rows 0 and 1 in FP64.
void tc_tile_rom(const std::vector<double>& U, long long n_half, int K, int kpad, std::vector<float>& tiles,
                 int* ntiles) {
  const int ncol_tile = TC_N;
  const long long T = (n_half + ncol_tile - 1) / ncol_tile;
  *ntiles = (int)T;
  const size_t tile_floats = (size_t)ncol_tile * kpad;
  const size_t stage_floats = 2 * tile_floats + 2 * ncol_tile * 2;   // + 2 rows of doubles
  tiles.assign((size_t)T * stage_floats, 0.f);
  for (long long t = 0; t < T; ++t) {
    float* base = tiles.data() + (size_t)t * stage_floats;
    float* rows01 = base + 2 * tile_floats;   // [2][TC_N][hi, lo]
    for (int n = 0; n < ncol_tile; ++n) {
      const long long col = t * ncol_tile + n;
      if (col >= n_half) continue;
      for (int rr = 0; rr < 2; ++rr) {
        const double x = rr < K ? U[(size_t)rr * n_half + col] : 0.0;
        const float h = (float)x;
        rows01[2 * (rr * ncol_tile + n)] = h;
        rows01[2 * (rr * ncol_tile + n) + 1] = (float)(x - (double)h);
      }
      for (int k = 2; k < K; ++k) {
        const double x = U[(size_t)k * n_half + col];
        const float h = tf32_round((float)x);
        const size_t off = canon_off(n, k, kpad) / 4;
        base[off] = h;
        base[tile_floats + off] = tf32_round((float)(x - (double)h));
      }
    }
  }
}

// The same tiles with BF16 hi / lo of rows 2.. (16-bit canonical layout) and
// rows 0 and 1 as float pairs; same byte layout per stage otherwise.
void tc_tile_rom_bf16(const std::vector<double>& U, long long n_half, int K, int kpad, std::vector<uint16_t>& tiles) {
  const int ncol_tile = TC_N;
  const long long T = (n_half + ncol_tile - 1) / ncol_tile;
  const size_t tile_elems = (size_t)ncol_tile * kpad;               // one BF16 tile
  const size_t stage_elems = 2 * tile_elems + 2 * ncol_tile * 4;    // + 2 rows of float pairs (4 halves each)
  tiles.assign((size_t)T * stage_elems, 0);
  for (long long t = 0; t < T; ++t) {
    uint16_t* base = tiles.data() + (size_t)t * stage_elems;
    float* rows01 = (float*)(base + 2 * tile_elems);   // [2][TC_N][hi, lo]
    for (int n = 0; n < ncol_tile; ++n) {
      const long long col = t * ncol_tile + n;
      if (col >= n_half) continue;
      for (int rr = 0; rr < 2; ++rr) {
        const double x = rr < K ? U[(size_t)rr * n_half + col] : 0.0;
        const float h = (float)x;
        rows01[2 * (rr * ncol_tile + n)] = h;
        rows01[2 * (rr * ncol_tile + n) + 1] = (float)(x - (double)h);
      }
      for (int k = 2; k < K; ++k) {
        const double x = U[(size_t)k * n_half + col];
        const uint16_t h = bf16_bits((float)x);
        const size_t off = canon_off16(n, k, kpad) / 2;
        base[off] = h;
        base[tile_elems + off] = bf16_bits((float)(x - (double)bf16_value(h)));
      }
    }
  }
}

romb_status launch_assemble_tc(romb_ctx* c) {
  const bool bf = c->prec == ROMB_BF16_SPLIT;
  if (c->prec != ROMB_FP32_SPLIT && !bf) {
    romb_set_error("tensor-core assembly: unknown split form");
    return ROMB_E_ARG;
  }
  int* d_err = (int*)c->d_red + 32;
  ROMB_CUDA(cudaMemsetAsync(d_err, 0, 4, c->stream));
  TcParams P;
  memset(&P, 0, sizeof(P));
  int KT = -1, T = -1, grid = 0;
  for (int f = 0; f < ROMB_MAX_FAMILIES; ++f) {
    if (c->famcount[f] == 0) continue;
    const RombRom& R = c->roms[f];
    const int kp = bf ? R.kpad16 : R.kpad;
    if (KT < 0) {
      KT = kp;
      T = R.ntiles;
    } else if (KT != kp || T != R.ntiles) {
      romb_set_error("tensor-core assembly: all reduced models of one lattice must share n_r");
      return ROMB_E_ARG;
    }
    TcFamily& F = P.fam[P.nfam++];
    F.Utiles = bf ? (const float*)R.Utiles16 : R.Utiles;
    F.list = c->d_famlist + c->famstart[f];
    F.count = c->famcount[f];
    F.mtile0 = grid;
    grid += (F.count + TC_M - 1) / TC_M;
  }
  if (grid == 0) return ROMB_OK;
  P.theta = c->d_theta;
  P.ntiles = T;
  P.KT = KT;
  P.th_hi = c->d_theta_hi;
  P.th_lo = c->d_theta_lo;
  P.chat32 = c->d_chat32;
  P.Kout = c->d_K;
  P.ndof = c->ndof;
  P.pairs = c->d_pairs;
  P.npairs = c->nB * (c->nB + 1) / 2;
  P.err = d_err;
  const size_t es = bf ? 2 : 4;
  const size_t a_bytes = (size_t)TC_M * KT * es, b_bytes = (size_t)TC_N * KT * es;
  const size_t stage_bytes = 2 * b_bytes + 2 * TC_N * 8;
  const size_t limit = 227 * 1024 - 1024 - 256;
  int stages = 2;
  if (2 * a_bytes + 2 * stage_bytes > limit) stages = 1;
  if (2 * a_bytes + stage_bytes > limit) {
    romb_set_error("tensor-core assembly: reduced basis too large for shared memory");
    return ROMB_E_ARG;
  }
  P.stages = stages;
  const size_t smem = 1024 + 2 * a_bytes + (size_t)stages * stage_bytes;
  auto kern = bf ? assemble_tc_kernel<true> : assemble_tc_kernel<false>;
  ROMB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, TC_THREADS, smem, c->stream>>>(P); ++c->launches;
  ROMB_CUDA(cudaGetLastError());
  int h_err = 0;
  ROMB_CUDA(cudaMemcpyAsync(&h_err, d_err, 4, cudaMemcpyDeviceToHost, c->stream));
  ROMB_CUDA(cudaStreamSynchronize(c->stream));
  if (h_err) {
    romb_set_error("tensor-core assembly: a pipeline wait timed out (code " + std::to_string(h_err) + ")");
    return ROMB_E_CUDA;
  }
  return ROMB_OK;
}
