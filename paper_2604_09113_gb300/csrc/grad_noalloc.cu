// romb_compliance_grad_noalloc: the compliance gradient for callers that must
// not allocate device memory when they ask for it.
//
// romb_compliance_grad keeps its intermediate arrays (the per-cell W and Q
// contractions, the per-cell control-point gradients, the threshold node
// tables and the staging arrays of host outputs) in context buffers that it
// allocates on its first call.  This entry point runs the same kernels, in the
// same order and arithmetic, on arrays carved out of one fixed file-scope
// device array instead, so its results equal romb_compliance_grad's bit for
// bit.  The array lives in this translation unit alone, which holds no kernel:
// the device memory is taken when the first call looks it up, not by programs
// that never make that call.  The paper has no counterpart of this call.
#include <stdio.h>

#include "device.cuh"

// One per device, shared by every context on that device.
static __device__ __align__(256) unsigned char g_grad_scratch[ROMB_NOALLOC_SCRATCH_BYTES];

// per-cell sum of the four threshold derivatives (api.cu)
__global__ void sum4_kernel(const double* __restrict__ dmu, long long n, double* __restrict__ out);

namespace {

// Device address of g_grad_scratch in the current device's context.  Looked
// up on every call rather than remembered: an address kept across calls would
// go stale if the device's primary context were reset or released and
// retained again, while the lookup itself allocates nothing once the
// library's device code is loaded (the first call on a device may load it).
romb_status scratch_address(unsigned char** out) {
  void* p = nullptr;
  ROMB_CUDA(cudaGetSymbolAddress(&p, g_grad_scratch));
  if (!p) return ROMB_E_CUDA;
  *out = static_cast<unsigned char*>(p);
  return ROMB_OK;
}

// Reserve n doubles at the end of the scratch, 256-byte aligned; returns the
// byte offset.
size_t take(size_t& used, size_t n) {
  const size_t off = used;
  used += (8 * n + 255) & ~size_t(255);
  return off;
}

}  // namespace

extern "C" romb_status romb_compliance_grad_noalloc(romb_ctx* c, double* compliance, double* dc_dctrl,
                                                    double* dc_dR, double* dc_dmu) {
  if (!c || !compliance || !dc_dctrl) return ROMB_E_ARG;
  if (!c->solved || !c->assembled_rom) return ROMB_E_STATE;
  if (c->lane[0].body_on || c->load_form != ROMB_LOADS_QUADRATURE || c->layout) return ROMB_E_STATE;
  const size_t cells = (size_t)c->ncells;
  const size_t ncp = (size_t)(c->m + 1) * (c->m + 1);
  const size_t nctrl = (size_t)(c->m * c->nx + 1) * (c->m * c->ny + 1);
  size_t used = 0;
  const size_t oW = take(used, cells * 144), oQ = take(used, cells * 128), oL = take(used, cells * 2 * ncp);
  const size_t oM = take(used, 4 * cells), oR = take(used, cells), oX = take(used, 2 * nctrl);
  if (used > ROMB_NOALLOC_SCRATCH_BYTES) return ROMB_E_SCRATCH;
  ROMB_CUDA(cudaSetDevice(c->device));
  unsigned char* base = nullptr;
  romb_status s = scratch_address(&base);
  if (s != ROMB_OK) return s;
  double* W = reinterpret_cast<double*>(base + oW);
  double* Q = reinterpret_cast<double*>(base + oQ);
  double* gloc = reinterpret_cast<double*>(base + oL);
  double* dmu = reinterpret_cast<double*>(base + oM);
  double* dR = reinterpret_cast<double*>(base + oR);
  double* dX = reinterpret_cast<double*>(base + oX);
  // nothing left by an earlier call (of any context on this device) is read
  ROMB_CUDA(cudaMemsetAsync(base, 0, used, c->stream));
  // c = f^T u on the skeleton, into the context's reduction slots
  if ((s = romb_dot(c, c->lane[0].d_f, c->lane[0].d_x, c->nskel, c->d_red + 8)) != ROMB_OK) return s;
  ROMB_CUDA(cudaMemcpyAsync(c->h_red + 2, c->d_red + 8, 8, cudaMemcpyDeviceToHost, c->stream));
  const bool dev = c->mem == ROMB_MEM_DEVICE;
  double* x_out = dev ? dc_dctrl : dX;
  double* mu_out = (dev && dc_dmu) ? dc_dmu : dmu;
  if ((s = launch_grad_scratch(c, W, Q, gloc, x_out, mu_out)) != ROMB_OK) return s;
  if (dc_dR) {
    sum4_kernel<<<c->sms, 256, 0, c->stream>>>(mu_out, c->ncells, dev ? dc_dR : dR); ++c->launches;
    ROMB_CUDA(cudaGetLastError());
  }
  if (!dev) {
    ROMB_CUDA(cudaMemcpyAsync(dc_dctrl, dX, 16 * nctrl, cudaMemcpyDeviceToHost, c->stream));
    if (dc_dmu) ROMB_CUDA(cudaMemcpyAsync(dc_dmu, dmu, 32 * cells, cudaMemcpyDeviceToHost, c->stream));
    if (dc_dR) ROMB_CUDA(cudaMemcpyAsync(dc_dR, dR, 8 * cells, cudaMemcpyDeviceToHost, c->stream));
  }
  ROMB_CUDA(cudaStreamSynchronize(c->stream));
  *compliance = c->h_red[2];
  return ROMB_OK;
}
