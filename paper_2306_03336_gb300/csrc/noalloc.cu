// noalloc.cu -- the weight-gradient reduction for callers that cannot
// allocate device memory.
//
// The regular entry point (j2d5pt_weight_grad) keeps its per-block partial
// sums in a plan's workspace, and making a plan calls cudaMalloc.  Some
// callers cannot do that: code running while a stream is being captured into
// a CUDA graph (allocation calls are not allowed inside the capture), code
// whose device memory belongs to a framework's caching allocator (a foreign
// cudaMalloc/cudaFree synchronises the device and fragments the pool), and
// latency-bound loops that cannot absorb cudaFree's implicit device-wide
// synchronisation.  This file gives them the same reduction with its scratch
// in a fixed device array compiled into the library.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <mutex>

#include "internal.h"

namespace j2d {

// Partial sums of the weight-gradient reduction: 5 doubles per block of the
// partial kernel, at most kNoAllocMaxBlocks blocks (2.5 MiB).  Every GPU that
// loads the library holds this array until the process exits.
constexpr long kNoAllocMaxBlocks = 65536;
static __device__ __align__(256) double g_wgrad_scratch[5 * kNoAllocMaxBlocks];

// Device address of the array, looked up once per device and context: a
// context that was torn down and created again (cudaDeviceReset) loads the
// module afresh, possibly at another address, so the address is looked up
// again whenever the current context differs from the one it was taken in.
constexpr int kMaxDevices = 128;
static double *g_scratch_addr[kMaxDevices];
static CUcontext g_scratch_ctx[kMaxDevices];
static std::mutex g_scratch_mu;

// cuCtxGetCurrent through the runtime's driver entry point (no -lcuda).
static CUcontext current_context() {
  static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void *f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuCtxGetCurrent_v4000)f;
  }
  CUcontext c = nullptr;
  if (fn) fn(&c);
  return c;
}

}  // namespace j2d

using namespace j2d;

extern "C" j2d_status j2d5pt_weight_grad_noalloc(int nx, int ny, j2d_dtype dtype, const void *u_t,
                                                 const void *lam_t1, double *dw, void *stream) {
  if (nx < 1 || ny < 1) return record_error(J2D_ERR_ARG, "weight_grad_noalloc: nx=%d ny=%d (need >= 1)", nx, ny);
  if (dtype != J2D_F64 && dtype != J2D_F32) return record_error(J2D_ERR_ARG, "weight_grad_noalloc: unknown dtype %d", (int)dtype);
  if (!u_t || !lam_t1 || !dw) return record_error(J2D_ERR_ARG, "weight_grad_noalloc: null pointer");
  if (((uintptr_t)u_t & 15u) || ((uintptr_t)lam_t1 & 15u) || ((uintptr_t)dw & 7u))
    return record_error(J2D_ERR_ALIGN, "weight_grad_noalloc: u_t/lam_t1 must be 16-byte and dw 8-byte aligned");
  const GridDesc g = plan_layout(dtype, nx, ny);  // the layout j2d5pt_plan gives this grid
  const long nblocks = wgrad_partial_count(dtype, g);
  if (nblocks > kNoAllocMaxBlocks)
    return record_error(J2D_ERR_ARG,
                        "weight_grad_noalloc: grid %d x %d needs %ld partial-sum blocks; the fixed scratch holds "
                        "%ld (use j2d5pt_weight_grad with a plan)",
                        nx, ny, nblocks, kNoAllocMaxBlocks);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return record_error(J2D_ERR_DEVICE, "weight_grad_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return record_error(J2D_ERR_DEVICE, "weight_grad_noalloc: device %d out of range", dev);
  double *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    const CUcontext ctx = current_context();
    if (!g_scratch_addr[dev] || ctx != g_scratch_ctx[dev]) {
      // set-up, once per device (and again after its context was replaced),
      // with that device current: the host-side name of the array is not a
      // device address
      double *p = nullptr;
      e = cudaGetSymbolAddress((void **)&p, g_wgrad_scratch);
      if (e != cudaSuccess)
        return record_error(J2D_ERR_DEVICE, "weight_grad_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
      g_scratch_ctx[dev] = current_context();
    }
    scratch = g_scratch_addr[dev];
  }
  // every block of the partial kernel overwrites its own 5 slots, and the
  // final kernel reads only those: nothing in the array needs clearing
  e = launch_wgrad(dtype, u_t, lam_t1, dw, scratch, g, (cudaStream_t)stream);
  if (e != cudaSuccess) return record_error(J2D_ERR_DEVICE, "weight_grad_noalloc: launch: %s", cudaGetErrorString(e));
  return J2D_OK;
}
