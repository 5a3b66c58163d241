// Shared-memory staging helpers: mbarriers with bounded waits and 1D bulk
// copies (cp.async.bulk, tracked by mbarrier transaction counts).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

// Upper bound of every mbarrier wait, in SM clock cycles (~2 s at 2 GHz);
// a wait that runs out reports failure instead of spinning on.
#define ROMB_WAIT_CYCLES (4000000000LL)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes preceding mbarrier.init visible to the asynchronous (bulk-copy) proxy.
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bounded wait for the phase with the given parity; false on timeout (or when
// *abort_flag becomes non-zero).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag = nullptr) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (abort_flag && *abort_flag) return false;
    if (clock64() - t0 > ROMB_WAIT_CYCLES) return false;
  }
}

// dst (shared, 16-byte aligned) <- bytes at src (global, 16-byte aligned);
// bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// The 16-byte aligned span covering the doubles [src, src + len): its start,
// its size in bytes and the position (0 or 1) of src[0] in it.  The span may
// reach 8 bytes before src and after src + len.
struct Span16 {
  const void* start;
  uint32_t bytes;
  int first;
};
__device__ __forceinline__ Span16 span16(const double* src, long long len) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(src);
  const uintptr_t a0 = a & ~uintptr_t(15);
  const uintptr_t e = (a + 8u * (uintptr_t)len + 15u) & ~uintptr_t(15);
  Span16 s;
  s.start = reinterpret_cast<const void*>(a0);
  s.bytes = len > 0 ? (uint32_t)(e - a0) : 0u;
  s.first = (int)((a - a0) >> 3);
  return s;
}

// The same for an array of T (4 or 8 bytes): the span may reach 16 - sizeof(T)
// bytes before src and after src + len; first < 16 / sizeof(T).
template <typename T>
__device__ __forceinline__ Span16 span16t(const T* src, long long len) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(src);
  const uintptr_t a0 = a & ~uintptr_t(15);
  const uintptr_t e = (a + sizeof(T) * (uintptr_t)len + 15u) & ~uintptr_t(15);
  Span16 s;
  s.start = reinterpret_cast<const void*>(a0);
  s.bytes = len > 0 ? (uint32_t)(e - a0) : 0u;
  s.first = (int)((a - a0) / sizeof(T));
  return s;
}
