// Measured CUDA-core FMA throughput of the current device (FP32 and FP64): the denominator of
// the roofline fractions the library's kernels are reported against.  The fused H|psi>
// kernel, the reduced eigensolver and the CG reductions are bound by these pipes rather than
// by HBM or the tensor cores, and GB300 runs FP64 at a small fraction of its FP32 rate, so the
// two peaks are measured on the device rather than taken from a data sheet.
//
// Every thread runs kChains independent multiply-add chains a <- a b + c (b, c kernel
// arguments, |b| < 1, so the values stay bounded and no chain can be folded at compile time);
// eight CTAs of 256 threads per SM keep enough independent instructions in flight to cover
// the pipe latency.  FLOPs = 2 per FMA.
#include <algorithm>

#include "pwk_internal.h"

namespace pwk {
namespace {

constexpr int kChains = 16;
constexpr int kPeakThreads = 256;
constexpr int kCtasPerSm = 8;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(T* out, T b, T c, int iters) {
  T a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = T(threadIdx.x) * T(1e-3) + T(i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == T(-1)) out[0] = s;   // never true for these b, c; keeps the chains live
}

template <typename T>
int measure(int iters, double* flops_per_s, int* sm_count, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "device attributes");
  void* out = nullptr;
  if ((e = scratch_alloc(&out, sizeof(T), st)) != cudaSuccess) return cuda_fail(e, "scratch_alloc(peak)");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = PWK_OK;
  float best = 1e30f;
  const int blocks = sms * kCtasPerSm;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    rc = cuda_fail(e, "cudaEventCreate");
  } else {
    for (int rep = 0; rep < 4 && rc == PWK_OK; ++rep) {   // the first launch is a warm-up
      cudaEventRecord(e0, st);
      fma_peak_kernel<T><<<blocks, kPeakThreads, 0, st>>>(static_cast<T*>(out), T(0.9999), T(1e-4), iters); note_launch();
      cudaEventRecord(e1, st);
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
        rc = cuda_fail(e, "fma_peak_kernel");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) best = std::min(best, ms);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  if (rc) return rc;
  const double flops = 2.0 * kChains * (double)iters * kPeakThreads * (double)blocks;
  if (flops_per_s) *flops_per_s = flops / (best * 1e-3);
  if (sm_count) *sm_count = sms;
  return PWK_OK;
}

}  // namespace
}  // namespace pwk

extern "C" int pwk_measure_fma_peak(int precision, double* flops_per_s, int* sm_count, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (precision == PWK_FP32) return pwk::measure<float>(2048, flops_per_s, sm_count, st);
  if (precision == PWK_FP64) return pwk::measure<double>(48, flops_per_s, sm_count, st);
  pwk::set_error("precision must be PWK_FP32 or PWK_FP64");
  return PWK_ERR_INVALID;
}
