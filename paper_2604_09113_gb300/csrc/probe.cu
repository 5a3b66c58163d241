// romb_fma_probe: the FMA issue rate of this GPU's FP64 and FP32 pipes, the
// denominators of the FP64-bound rooflines (local factor, PCG, coarse solve)
// and of the FP32-bound tensor-core epilogue.  The paper has no counterpart;
// this is a measurement utility.
//
// Every thread runs NCHAIN independent dependent chains a <- a * b + c
// (NCHAIN in flight hide the pipe latency), fully unrolled, so the kernel
// issues nothing but FMAs in its loop; the chains' sum is written out so the
// compiler keeps them.
#include <cuda_runtime.h>

#include "romb_internal.cuh"

namespace {

constexpr int NCHAIN = 8;
constexpr int UNROLL = 16;

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, T b, T c, T* __restrict__ out) {
  T a[NCHAIN];
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
      for (int k = 0; k < NCHAIN; ++k) a[k] = fma(a[k], b, c);
    }
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" romb_status romb_fma_probe(int precision, int blocks, int threads, int iters, void* cuda_stream,
                                      void* out, double* flops) {
  if (blocks <= 0 || threads <= 0 || threads > 256 || (threads & 31) || iters <= 0 || !out || !flops)
    return ROMB_E_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // b slightly below 1 and c small keep every chain bounded and normal
  if (precision == 0)
    fma_probe_kernel<double><<<blocks, threads, 0, s>>>(iters, 0.999999, 1e-6, static_cast<double*>(out));
  else if (precision == 1)
    fma_probe_kernel<float><<<blocks, threads, 0, s>>>(iters, 0.999999f, 1e-6f, static_cast<float*>(out));
  else
    return ROMB_E_ARG;
  ROMB_CUDA(cudaGetLastError());
  *flops = 2.0 * NCHAIN * UNROLL * (double)iters * (double)blocks * (double)threads;
  return ROMB_OK;
}
