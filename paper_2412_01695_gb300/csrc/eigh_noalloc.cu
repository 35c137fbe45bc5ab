// pwk_eigh_batched_noalloc: the batched generalized Hermitian eigensolver of pwk_eigh_batched
// without any device allocation.  Its workspace is a fixed array in the library's own device
// memory, reserved when the library is loaded on a device and held until the process exits.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they solve, e.g. a
// latency-bound serving loop (cudaMalloc and cudaFree synchronise the device and stall every
// other stream) or a process whose device memory is fully reserved by another allocator, where
// a fresh cudaMalloc would fail.  They pass inputs and outputs; the scratch is built in.
#include <mutex>

#include "solvers.h"

namespace pwk {

// 3 n^2 complex128 per problem: the Cholesky factor, L^-1 H (then Z) and the reduced matrix.
constexpr size_t kNoallocElems = 3ull * 16 * kMaxBasis * kMaxBasis;   // 19.7 MB

// The scratch array.  In host code this name is only a host-side stand-in, not a device
// address: the address is taken per device with cudaGetSymbolAddress below.
static __device__ __align__(256) double2 g_eigh_scratch[kNoallocElems];

static std::mutex g_setup_mutex;
static double2* g_scratch_addr[64] = {nullptr};

// Once per device, with that device current: the device address of the scratch array.  It
// is kept for the life of the process (a cudaDeviceReset would unload the array: the header
// tells callers not to use this entry point on a device they have reset).
static int scratch_on_current_device(double2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) {
    set_error("device index above 63");
    return PWK_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_eigh_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(eigh scratch)");
    g_scratch_addr[dev] = static_cast<double2*>(p);
  }
  *out = g_scratch_addr[dev];
  return PWK_OK;
}

}  // namespace pwk

using namespace pwk;

extern "C" int pwk_eigh_batched_noalloc(int nprob, int n, int nev, const void* H, const void* S,
                                        double* eig, void* vec, int* status, void* stream) {
  if (nprob < 0 || n < 1 || nev < 1 || nev > n || (nprob > 0 && (H == nullptr || S == nullptr ||
      eig == nullptr || vec == nullptr))) {
    set_error("null pointer or bad size (need 1 <= nev <= n)");
    return PWK_ERR_INVALID;
  }
  if (n > kMaxBasis) {
    set_error("n > 160");
    return PWK_ERR_UNSUPPORTED;
  }
  if ((size_t)nprob * 3 * n * n > kNoallocElems) {
    set_error("nprob * n^2 exceeds the built-in workspace (at most 409600, e.g. 16 problems of n = 160)");
    return PWK_ERR_UNSUPPORTED;
  }
  if (nprob == 0) return PWK_OK;
  double2* W = nullptr;
  int rc = scratch_on_current_device(&W);
  if (rc) return rc;
  return launch_rr(nprob, n, nev, nullptr, nullptr, static_cast<const double2*>(H),
                   static_cast<const double2*>(S), W, static_cast<double2*>(vec), eig, status,
                   static_cast<cudaStream_t>(stream));
}
