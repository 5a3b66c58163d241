// Tensor-core form of the assembly contraction (Sec. 4.1, Algorithm 4) on the
// 5th-generation tensor cores (tcgen05 kind::tf32 / kind::f16), split precision.
//
//   I_c = theta_c U'          [128 cells x K] x [K x 144]  per N-tile (4 pairs k1 <= k2)
//   K_c[(k1 i1),(k2 i2)] = sum_{j1 j2 k3} I_c[k1 k2 k3 j1 j2] Chat_c[k3][i1 j1 i2 j2]
//
// The dominant row of U' (the first reduced basis vector, ~90 % of K) is
// applied in the epilogue in double-float arithmetic; the other rows (rho I_Pi,
// ~5e-4 of K, and rows 2..) run on the tensor cores with the FP64 operands
// split x = hi + lo into TF32 values, accumulated in FP32 as
// hi*hi + hi*lo + lo*hi.  The epilogue forms I in double-float and contracts
// it with Chat in double-float (Chat rounded to FP32, exactly symmetric, held
// in registers).  The factor kernel then restores the exact null space of rigid
// translations (zero row sums) that the rounding perturbs.  The theta tile (A) stays in shared memory for the
// whole CTA; the U' tiles (B, hi and lo, pre-arranged at ROM load time in the
// canonical no-swizzle K-major layout) stream through a ring of one or two
// stages filled by bulk copies (cp.async.bulk + mbarrier transaction counts);
// row 1 of each tile goes to a separate double buffer for the epilogue, so a
// stage is refilled as soon as its MMAs complete.  Accumulators
// live in tensor memory, double buffered, so the epilogue (tcgen05.ld, the
// Chat contraction in FP32 registers, packed FP64 stores) overlaps the MMAs of
// the next tile.  Every wait is bounded: on timeout the kernel records an error
// and all roles leave their loops; tensor memory is freed before exit.
//
// The BF16 form (kind::f16 with BF16 A and B, K = 16 per instruction) uses the
// same pipeline and epilogue on four-part BF16 splits (x = b0 + b1 + b2 + b3,
// ~32 significant bits) with the ten products b_i b_j, i + j <= 3 (the
// dropped ones are below 2^-32 relative); BF16 MMAs run at twice the TF32 rate.
//
// Roles (384 threads): warp 0 allocates tensor memory and issues the copies,
// warp 1 issues the MMAs (one thread), warps 4-11 run the epilogue as two
// warpgroups over the same TMEM lanes 0-127 (the 128 cells of the tile).
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
  TcFamily fam[ROMB_MAX_MODELS];
  int nfam;
  const double* theta;     // [cells][128] f64 (slots 0, 1 applied exactly in the epilogue)
  int ntiles, KT;
  int nr;                  // reduced basis size: theta slots 0..nr are used
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

__device__ __forceinline__ void tmem_ld2(uint32_t taddr, float* v) {
  uint32_t r[2];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(taddr));
  v[0] = __uint_as_float(r[0]);
  v[1] = __uint_as_float(r[1]);
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

// Operand parts of the split forms: TF32 hi + lo (products lo hi, hi lo,
// hi hi), BF16 b0 + b1 + b2 + b3 (~32 significant bits; the ten products
// b_i b_j with i + j <= 3); both lists smallest first.
template <bool BF>
struct TcSplit {
  static constexpr int NPART = BF ? 4 : 2;
  static constexpr int NPROD = BF ? 10 : 3;
};
__constant__ int8_t c_tc_prod[2][10][2] = {
    {{1, 0}, {0, 1}, {0, 0}},
    {{3, 0}, {2, 1}, {1, 2}, {0, 3}, {2, 0}, {1, 1}, {0, 2}, {1, 0}, {0, 1}, {0, 0}}};

// BF16 parts of x: b0 = bf16(x), b1 = bf16(x - b0), ... (residuals exact in FP64)
__host__ __device__ inline void bf16_split4(double x, uint16_t* b) {
  for (int i = 0; i < 4; ++i) {
    b[i] = bf16_bits((float)x);
    x -= (double)bf16_value(b[i]);
  }
}

template <bool BF>
__global__ void __launch_bounds__(TC_THREADS, 1) assemble_tc_kernel(TcParams P) {
  using Sp = TcSplit<BF>;
  constexpr int NPART = Sp::NPART;
  constexpr uint32_t ES = BF ? 2 : 4;   // operand element size
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[2], bar_empty[2], bar_accfull[2], bar_accempty[2], bar_done;
  __shared__ __align__(8) uint64_t bar_u1full[2], bar_u1empty[2], bar_xch[2];
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int KT = P.KT;
  const uint32_t a_bytes = TC_M * KT * ES, b_bytes = TC_N * KT * ES;
  const uint32_t stage_bytes = NPART * b_bytes;            // B parts of one tile in shared memory
  const size_t gstage_bytes = (size_t)stage_bytes + 2 * TC_N * 8;   // per tile in global: + rows 0, 1 pairs
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* Ast = base;                                // A part i at Ast + i * a_bytes
  unsigned char* Bst = base + NPART * a_bytes;              // stage s at Bst + s * stage_bytes
  const int S = P.stages;
  const int T = P.ntiles;
  // row 1 of U' per tile (float pairs), double buffered apart from the ring so
  // that a stage is free as soon as its MMAs complete
  float2* u1buf = reinterpret_cast<float2*>(Bst + (size_t)S * stage_bytes);
  // partial sums exchanged by the epilogue warpgroups: [pair parity][writer g][i2][128 cells]
  float2* xch = u1buf + 2 * TC_N;
  int fi = 0;
  while (fi + 1 < P.nfam && (int)blockIdx.x >= P.fam[fi + 1].mtile0) ++fi;
  const TcFamily F = P.fam[fi];
  const int m0 = ((int)blockIdx.x - F.mtile0) * TC_M;

  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < 2; ++s) {
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_empty[s], 1);       // MMA commit
      mbar_init(&bar_accfull[s], 1);
      mbar_init(&bar_accempty[s], 256);
      mbar_init(&bar_u1full[s], 1);
      mbar_init(&bar_u1empty[s], 8);     // one arrival per epilogue warp
      mbar_init(&bar_xch[s], 256);       // both epilogue warpgroups, once per pair
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
  // A tile: the split parts of theta of the 128 cells (slot 1 zero: it is
  // applied in the epilogue), canonical layout
  for (int i = tid; i < TC_M * KT; i += TC_THREADS) {
    const int row = i / KT, k = i % KT;
    const int ci = m0 + row;
    if (BF) {
      double x = 0.0;
      if (ci < F.count && k != 1 && k <= P.nr) x = P.theta[(long long)F.list[ci] * 128 + k];
      uint16_t b[4];
      bf16_split4(x, b);
      const uint32_t off = canon_off16(row, k, KT);
#pragma unroll
      for (int q = 0; q < NPART; ++q) *(uint16_t*)(Ast + q * a_bytes + off) = b[q];
    } else {
      float h = 0.f, l = 0.f;
      if (ci < F.count) {
        const long long cell = F.list[ci];
        h = P.th_hi[cell * 128 + k];
        l = P.th_lo[cell * 128 + k];
      }
      const uint32_t off = canon_off(row, k, KT);
      *(float*)(Ast + off) = h;
      *(float*)(Ast + a_bytes + off) = l;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  if (warp == 0) {
    if (lane == 0) {
      // producer: the B parts of each tile into the ring, row 1 into its buffer
      int armed_last[2] = {-1, -1}, u1_last[2] = {-1, -1};
      for (int t = 0; t < T && !s_abort; ++t) {
        const int s = t % S, u = t & 1;
        if (t >= S && !mbar_wait(&bar_empty[s], (uint32_t)(((t / S) - 1) & 1), &s_abort)) {
          s_abort = 1;
          atomicOr(P.err, 1);
          break;
        }
        const unsigned char* src = (const unsigned char*)F.Utiles + (size_t)t * gstage_bytes;
        mbar_expect_tx(&bar_full[s], stage_bytes);
        bulk_g2s(Bst + (size_t)s * stage_bytes, src, stage_bytes, &bar_full[s]);
        armed_last[s] = t;
        if (t >= 2 && !mbar_wait(&bar_u1empty[u], (uint32_t)(((t >> 1) - 1) & 1), &s_abort)) {
          s_abort = 1;
          atomicOr(P.err, 32);
          break;
        }
        mbar_expect_tx(&bar_u1full[u], TC_N * 8);
        bulk_g2s(u1buf + u * TC_N, src + stage_bytes + TC_N * 8, TC_N * 8, &bar_u1full[u]);
        u1_last[u] = t;
      }
      // drain: every armed copy must land before the CTA exits
      for (int s = 0; s < 2; ++s) {
        if (armed_last[s] >= 0) mbar_wait(&bar_full[s], (uint32_t)((armed_last[s] / S) & 1), nullptr);
        if (u1_last[s] >= 0) mbar_wait(&bar_u1full[s], (uint32_t)((u1_last[s] >> 1) & 1), nullptr);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = BF ? idesc_bf16(TC_M, TC_N) : idesc_tf32(TC_M, TC_N);
      const uint32_t sbo = (uint32_t)KT * 8 * ES, lbo = 128;
      const uint32_t a0 = smem_u32(Ast);
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
        const uint32_t b0 = smem_u32(Bst + (size_t)s * stage_bytes);
        const uint32_t d = tmem + (uint32_t)(b * TC_N);
        // One instruction covers two core matrices along K (32 bytes): 8 TF32
        // or 16 BF16.  Every instruction rounds the FP32 accumulator, so the
        // small correction products go first, over all of K, while the
        // accumulator is still small; the leading products come last and
        // round the full-size sum only KT / 8 (TF32) or KT / 16 (BF16) times.
        const int nk = KT / (32 / (int)ES);
#pragma unroll 1
        for (int m = 0; m < Sp::NPROD; ++m) {
          const int ia = c_tc_prod[BF][m][0], ib = c_tc_prod[BF][m][1];
          for (int kk = 0; kk < nk; ++kk) {
            const uint32_t ko = (uint32_t)kk * 256;
            const uint64_t ad = smem_desc(a0 + ia * a_bytes + ko, lbo, sbo);
            const uint64_t bd = smem_desc(b0 + ib * b_bytes + ko, lbo, sbo);
            if (BF) mma_bf16(d, ad, bd, idesc, (kk > 0 || m > 0) ? 1u : 0u);
            else mma_tf32(d, ad, bd, idesc, (kk > 0 || m > 0) ? 1u : 0u);
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
    // Epilogue: the four outputs K[2 k1 + i1][2 k2 + i2] of a cell and pair
    // are sums over the 36 terms e = (k3, j1, j2) of I_e Chat[k3][i1 j1 i2 j2].
    // Both warpgroups read the same 128 TMEM lanes (cells); warpgroup g sums
    // the terms e in [18 g, 18 g + 18) for all four outputs, so each I_e is
    // formed once, and stores the row i1 = g after adding the other
    // warpgroup's partial sums of that row (exchanged through shared memory).
    const int g = (warp - 4) >> 2;
    const int row = ((warp & 3) << 5) + lane;
    const int ci = m0 + row;
    const bool valid = ci < F.count;
    const long long cell = valid ? F.list[ci] : 0;
    float C[72];   // C[4 el + 2 i1 + i2] = Chat[k3][i1][j1][i2][j2] of term e = 18 g + el
#pragma unroll
    for (int el = 0; el < 18; ++el) {
      const int e = 18 * g + el, k3 = e >> 2, j1 = (e >> 1) & 1, j2 = e & 1;
#pragma unroll
      for (int o = 0; o < 4; ++o)
        C[4 * el + o] = valid ? P.chat32[cell * 144 + 16 * k3 + 8 * (o >> 1) + 4 * j1 + 2 * (o & 1) + j2] : 0.f;
    }
    const dfl th1 = df_from_double(valid ? P.theta[cell * 128 + 1] : 0.0);
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const long long kp = (long long)P.ndof * (P.ndof + 1) / 2;
    double* Kc = P.Kout + cell * kp;
    for (int t = 0; t < T && !s_abort; ++t) {
      const int b = t & 1;
      if (!mbar_wait(&bar_accfull[b], (uint32_t)((t >> 1) & 1), &s_abort) ||
          !mbar_wait(&bar_u1full[b], (uint32_t)((t >> 1) & 1), &s_abort)) {
        s_abort = 1;
        atomicOr(P.err, 8);
        break;
      }
      tc_fence_after();
      const float2* U1 = u1buf + b * TC_N;   // row 1 of U' (hi, lo)
      bool ok = true;
#pragma unroll 1
      for (int pl = 0; pl < TC_PAIRS; ++pl) {
        float acc[18];
        const uint32_t col = tmem + lane_base + (uint32_t)(b * TC_N + 36 * pl + 18 * g);
        tmem_ld16(col, acc);
        tmem_ld2(col + 16, acc + 16);
        tmem_wait_ld();
        const int pr = t * TC_PAIRS + pl;
        const bool act = valid && pr < P.npairs;
        float vh[4] = {0.f, 0.f, 0.f, 0.f}, vl[4] = {0.f, 0.f, 0.f, 0.f};
        if (act) {
#pragma unroll
          for (int el = 0; el < 18; ++el) {
            // I_e = theta_1 U'_1 + (tensor-core rows 0, 2..), in double-float
            float ih = acc[el], il = 0.f;
            df_acc(ih, il, th1, U1[36 * pl + 18 * g + el]);
#pragma unroll
            for (int o = 0; o < 4; ++o) df_acc_f(vh[o], vl[o], ih, il, C[4 * el + o]);
          }
        }
        // the row i1 = 1 - g goes to the other warpgroup (g is warp-uniform:
        // selects, not indexing, keep vh / vl in registers)
        const float kh0 = g ? vh[2] : vh[0], kl0 = g ? vl[2] : vl[0];
        const float kh1 = g ? vh[3] : vh[1], kl1 = g ? vl[3] : vl[1];
        const int par = pr & 1;
        float2* mine = xch + (size_t)(2 * par + g) * 2 * TC_M;
        mine[row] = g ? make_float2(vh[0], vl[0]) : make_float2(vh[2], vl[2]);
        mine[TC_M + row] = g ? make_float2(vh[1], vl[1]) : make_float2(vh[3], vl[3]);
        mbar_arrive(&bar_xch[par]);
        if (!mbar_wait(&bar_xch[par], (uint32_t)((pr >> 1) & 1), &s_abort)) {
          s_abort = 1;
          atomicOr(P.err, 16);
          ok = false;
          break;
        }
        if (!act) continue;
        const float2* other = xch + (size_t)(2 * par + (1 - g)) * 2 * TC_M;
        const int2 kk = P.pairs[pr];
        const long long r = 2 * kk.x + g, q0 = 2 * kk.y;
        double* Kr = Kc + r * P.ndof - r * (r - 1) / 2 - r;
        // (h, l) + (w.x, w.y) in double-float (two-sum of the high words)
        auto combine = [](float h, float l, float2 w) {
          const float sh = __fadd_rn(h, w.x), bb = __fsub_rn(sh, h);
          const float er = __fadd_rn(__fsub_rn(h, __fsub_rn(sh, bb)), __fsub_rn(w.x, bb));
          const float sl = __fadd_rn(__fadd_rn(l, w.y), er);
          return (double)sh + (double)sl;
        };
        const double out0 = combine(kh0, kl0, other[row]);
        const double out1 = combine(kh1, kl1, other[TC_M + row]);
        if (!(kk.x == kk.y && g == 1)) Kr[q0] = out0;
        Kr[q0 + 1] = out1;
      }
      if (!ok) break;
      tc_fence_before();
      mbar_arrive(&bar_accempty[b]);
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_u1empty[b]);   // this warp is done with row 1 of the tile
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
// Tiles of 144 columns: TF32 hi and lo of rows 0, 2, 3, .. of U' in the
// canonical K-major layout (row 1 zero there), then rows 0 and 1 as float
// pairs (only row 1 is read, by the epilogue).
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
      for (int k = 0; k < K; ++k) {
        if (k == 1) continue;   // row 1 is applied in the epilogue
        const double x = U[(size_t)k * n_half + col];
        const float h = tf32_round((float)x);
        const size_t off = canon_off(n, k, kpad) / 4;
        base[off] = h;
        base[tile_floats + off] = tf32_round((float)(x - (double)h));
      }
    }
  }
}

// The same tiles with the four BF16 parts of rows 0, 2, 3, .. (16-bit
// canonical layout, part q at q * tile_elems) and rows 0 and 1 as float pairs.
void tc_tile_rom_bf16(const std::vector<double>& U, long long n_half, int K, int kpad, std::vector<uint16_t>& tiles) {
  const int ncol_tile = TC_N;
  const long long T = (n_half + ncol_tile - 1) / ncol_tile;
  const size_t tile_elems = (size_t)ncol_tile * kpad;               // one BF16 part
  const size_t stage_elems = 4 * tile_elems + 2 * ncol_tile * 4;    // + 2 rows of float pairs (4 halves each)
  tiles.assign((size_t)T * stage_elems, 0);
  for (long long t = 0; t < T; ++t) {
    uint16_t* base = tiles.data() + (size_t)t * stage_elems;
    float* rows01 = (float*)(base + 4 * tile_elems);   // [2][TC_N][hi, lo]
    for (int n = 0; n < ncol_tile; ++n) {
      const long long col = t * ncol_tile + n;
      if (col >= n_half) continue;
      for (int rr = 0; rr < 2; ++rr) {
        const double x = rr < K ? U[(size_t)rr * n_half + col] : 0.0;
        const float h = (float)x;
        rows01[2 * (rr * ncol_tile + n)] = h;
        rows01[2 * (rr * ncol_tile + n) + 1] = (float)(x - (double)h);
      }
      for (int k = 0; k < K; ++k) {
        if (k == 1) continue;   // row 1 is applied in the epilogue
        uint16_t b[4];
        bf16_split4(U[(size_t)k * n_half + col], b);
        const size_t off = canon_off16(n, k, kpad) / 2;
        for (int q = 0; q < 4; ++q) base[q * tile_elems + off] = b[q];
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
  for (int f = 0; f < ROMB_MAX_MODELS; ++f) {
    if (c->famcount[f] == 0) continue;
    const RombRom& R = c->roms[f];
    const int kp = bf ? R.kpad16 : R.kpad;
    if (KT < 0) {
      KT = kp;
      T = R.ntiles;
      P.nr = R.n_r;
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
  const size_t es = bf ? 2 : 4, npart = bf ? 4 : 2;
  const size_t a_bytes = (size_t)TC_M * KT * es, b_bytes = (size_t)TC_N * KT * es;
  const size_t stage_bytes = npart * b_bytes;
  // row-1 double buffer and the epilogue exchange buffer
  const size_t extra = (size_t)2 * TC_N * 8 + (size_t)2 * 2 * 2 * TC_M * 8;
  const size_t limit = 227 * 1024 - 1024 - 256 - extra;
  int stages = 2;
  if (npart * a_bytes + 2 * stage_bytes > limit) stages = 1;
  if (npart * a_bytes + stage_bytes > limit) {
    romb_set_error("tensor-core assembly: reduced basis too large for shared memory");
    return ROMB_E_ARG;
  }
  P.stages = stages;
  const size_t smem = 1024 + npart * a_bytes + (size_t)stages * stage_bytes + extra;
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
