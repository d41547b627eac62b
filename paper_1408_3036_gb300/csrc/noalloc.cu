// Allocation-free inverse of the tridiagonal Lanczos matrix.
//
// gw_epsinv_elements needs a context (gw_setup allocates device workspaces)
// and stages its pivots and multipliers in context-owned device memory.  Some
// callers cannot allocate at the point where they need T_K^-1: code whose
// device memory is entirely reserved by another allocator (a framework's
// caching allocator holding the whole GPU), code that must not introduce the
// implicit device synchronisation of cudaMalloc/cudaFree into a latency-
// critical loop, or embedders that forbid the library from owning memory.
// gw_epsinv_elements_noalloc serves them: the caller passes device inputs and
// outputs, and the per-call scratch (pivots d, multipliers l, a zero-pivot
// flag) lives in one file-scope __device__ array that every GPU loading the
// library keeps until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "gw.h"
#include "gw_common.cuh"
#include "linalg.cuh"

namespace {

constexpr int kNoallocMaxK = 4096;   // largest Lanczos dimension accepted
constexpr int kMaxDevices = 64;

// [0, K) pivots d, [K, 2K) multipliers l, then the zero-pivot flag (an int).
// In host code `g_tridiag_scratch` only names the symbol; its device address
// comes from cudaGetSymbolAddress (below), once per device.
static __device__ __align__(256) double g_tridiag_scratch[2 * kNoallocMaxK + 2];

std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up on the
// first call made with that device current.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_tridiag_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" gw_status gw_epsinv_elements_noalloc(const double* alpha, const double* beta, int k, double* out,
                                                void* cuda_stream) {
  if (!alpha || !out || k < 1 || (k > 1 && !beta)) return GW_E_ARG;
  if (k > kNoallocMaxK) return GW_E_ARG;     // beyond the fixed scratch: use gw_epsinv_elements
  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return GW_E_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  double* d = scratch;
  double* l = scratch + kNoallocMaxK;
  int* flag = reinterpret_cast<int*>(scratch + 2 * kNoallocMaxK);
  // An error left pending by the caller's own earlier work is reported as it
  // is, before this launch, so that the check after the launch concerns this
  // launch alone (and the caller's error is not consumed here).
  if (cudaPeekAtLastError() != cudaSuccess) return GW_E_CUDA;
  // d, l and the flag are written by the kernel before they are read (the
  // flag on every call, 0 or 1), so the previous call's contents need no
  // clearing.
  gw::launch_tridiag_inv(s, k, alpha, beta, d, l, out, flag);
  if (cudaGetLastError() != cudaSuccess) return GW_E_CUDA;
  int hflag = 0;                               // pageable host copy: no allocation
  if (cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GW_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return GW_E_CUDA;
  return hflag ? GW_E_BREAKDOWN : GW_OK;
}
