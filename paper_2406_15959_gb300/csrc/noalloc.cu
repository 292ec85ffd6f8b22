// Triangular solves with a Cholesky factor, without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is being
// captured in global capture mode (where the allocation would invalidate the capture),
// hosts that hand out every byte of device memory through their own pool and forbid
// hidden allocations, and real-time loops that must not pay for an allocation.  For
// them, elm_ddm_chol_solve_noalloc solves L L^T u = b with the blocked forward and
// backward substitution kernels of the Schur solve, keeping its working vectors in a
// fixed file-scope device array instead of handle workspace.
#include "elm_ddm.h"
#include "common.cuh"

#include <mutex>

using namespace elmddm;

namespace {

constexpr int kMaxDevices = 64;

// Working right-hand sides r and intermediate y of L y = r, for every call on a device.
// It is part of the library image: each GPU that loads the library holds these
// 2 * ELM_DDM_NOALLOC_MAX_ELEMS doubles (2 MiB) until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[2 * ELM_DDM_NOALLOC_MAX_ELEMS];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device
// and kept for the life of the process (a device reset would invalidate it; the header
// says not to call the entry point after one).  In host code g_noalloc_scratch names a
// host-side stand-in, not device memory.
cudaError_t scratch_on_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int elm_ddm_chol_solve_noalloc(const double* L, int n, int ld, const double* b,
                                          int nrhs, double* u, void* stream) {
  // nrhs is the y dimension of the substitution kernels' grids (at most 65535)
  if (!L || !b || !u || n < 1 || nrhs < 1 || nrhs > 65535 || ld < n) return ELM_DDM_ERR_ARG;
  if ((long long)n * nrhs > ELM_DDM_NOALLOC_MAX_ELEMS) return ELM_DDM_ERR_CAPACITY;
  double* scratch = nullptr;
  if (scratch_on_current_device(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return ELM_DDM_ERR_CUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t elems = (size_t)n * nrhs;
  double* r = scratch;           // working copy of b, overwritten in full below
  double* y = scratch + elems;   // every block of y is written before it is read
  if (cudaMemcpyAsync(r, b, elems * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    return ELM_DDM_ERR_CUDA;
  }
  for (int k = 0; k < n; k += CHOL_NB) {
    const int nb = n - k < CHOL_NB ? n - k : CHOL_NB;
    if (launch_chol_fwd(L, ld, n, k, nb, r, y, nrhs, st) != cudaSuccess) return ELM_DDM_ERR_CUDA;
  }
  for (int k = ((n - 1) / CHOL_NB) * CHOL_NB; k >= 0; k -= CHOL_NB) {
    const int nb = n - k < CHOL_NB ? n - k : CHOL_NB;
    if (launch_chol_bwd(L, ld, n, k, nb, y, u, nrhs, st) != cudaSuccess) return ELM_DDM_ERR_CUDA;
  }
  return ELM_DDM_OK;
}
