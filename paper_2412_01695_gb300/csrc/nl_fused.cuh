// Nonlocal projector terms inside the fused H|psi> kernels (paper Sec. 2.2, "Non local
// pseudopotential and overlap matrix"), so that one band-k work item reads C(G) and writes
// H C(G) (and S C(G)) once from and to HBM:
//
//   prologue  lambda_m = sum_G conj(beta_m(k+G)) C(G)           (Eq. lambdah)
//             gamma_m  = sum_n D_mn lambda_n                    (Eq. gamma)
//             delta_m  = sum_n q_mn lambda_n                    (Eq. delta_eq, with q)
//   epilogue  H C(G)  += sum_m gamma_m beta_m(k+G)              (Eq. finalnl)
//             S C(G)   = C(G) + sum_m delta_m beta_m(k+G)       (Eq. finals, with q)
//
// beta(k) is read through L1/L2 (the bands of a k-point run in neighbouring CTAs, so it
// crosses HBM about once per k-point).  The projections are computed by warps, one group of
// G projectors per warp at a time: lane l sums G = l, l + 32, ... in ascending order and the
// lanes are combined by a fixed xor tree, so lambda does not depend on the number of warps
// (every launch shape gives the same bits); gamma, delta and the add-back sum the projectors
// in ascending order.  The coefficients live in shared memory at byte offset a.nl_off:
// [0, nkb) lambda, [nkb, 2 nkb) gamma, [2 nkb, 3 nkb) delta.
#pragma once
#include "fft_line.cuh"
#include "pwk_internal.h"

namespace pwk {

// projectors per warp group in the prologue (accumulators held in registers)
template <typename T>
struct NlGroup {
  static constexpr int G = sizeof(T) == 4 ? 4 : 3;
};

// Prologue, part 1: lambda of every projector into nls[0, nkb).  C(G) is read through
// `cin`, beta(k) through `bk` ([nkb][ldb]); either may be global or shared memory.
template <typename T, typename CV>
__device__ __forceinline__ void nl_fused_project(const FusedArgs& a, const c2_t<T>* bk, int ldb,
                                                 const CV* cin, int np, c2_t<T>* nls) {
  using V = c2_t<T>;
  constexpr int G = NlGroup<T>::G;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int ngroups = (a.nkb + G - 1) / G;
  for (int grp = warp; grp < ngroups; grp += nw) {
    const int m0 = grp * G;
    const int nc = min(G, a.nkb - m0);
    T ar[G], ai[G];
#pragma unroll
    for (int j = 0; j < G; ++j) ar[j] = ai[j] = T(0);
    const V* bg = bk + (size_t)m0 * ldb;
    for (int g = lane; g < np; g += 32) {
      const CV cv = cin[g];
      const T cr = T(cv.x), ci = T(cv.y);
#pragma unroll
      for (int j = 0; j < G; ++j) {
        if (j < nc) {
          const V b = bg[(size_t)j * ldb + g];
          ar[j] += b.x * cr + b.y * ci;   // conj(beta) C
          ai[j] += b.x * ci - b.y * cr;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < G; ++j) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ar[j] += __shfl_xor_sync(0xffffffffu, ar[j], o);
        ai[j] += __shfl_xor_sync(0xffffffffu, ai[j], o);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < G; ++j)
        if (j < nc) nls[m0 + j] = V{ar[j], ai[j]};
    }
  }
}

// Prologue, part 2 (after a barrier): gamma = D lambda into nls[nkb, 2 nkb) and, with q,
// delta = q lambda into nls[2 nkb, 3 nkb).
template <typename T>
__device__ __forceinline__ void nl_fused_coef(const FusedArgs& a, c2_t<T>* nls) {
  using V = c2_t<T>;
  const int nkb = a.nkb;
  const int rows = a.qm != nullptr ? 2 * nkb : nkb;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) {
    const bool del = i >= nkb;
    const T* M = static_cast<const T*>(del ? a.qm : a.Dm) + (size_t)(del ? i - nkb : i) * nkb;
    T gr = T(0), gi = T(0);
    for (int j = 0; j < nkb; ++j) {
      const T d = M[j];
      const V l = nls[j];
      gr += d * l.x;
      gi += d * l.y;
    }
    nls[nkb + i] = V{gr, gi};
  }
}

// Epilogue for one plane wave g: the add-back sums h = sum gamma beta and, when with_q (the
// plan has q and S C is wanted), s = sum delta beta (else s = 0: S C = C).  beta(k) through
// `bk` ([nkb][ldb], global or shared memory).
template <typename T>
__device__ __forceinline__ void nl_fused_addback(const FusedArgs& a, const c2_t<T>* bk, int ldb, int g,
                                                 const c2_t<T>* nls, bool with_q, c2_t<T>& h, c2_t<T>& s) {
  using V = c2_t<T>;
  const int nkb = a.nkb;
  const V* bg = bk + g;
  T hr = T(0), hi = T(0), sr = T(0), si = T(0);
#pragma unroll 4
  for (int m = 0; m < nkb; ++m) {
    const V b = bg[(size_t)m * ldb];
    const V gm = nls[nkb + m];
    hr += gm.x * b.x - gm.y * b.y;
    hi += gm.x * b.y + gm.y * b.x;
    if (with_q) {
      const V dl = nls[2 * nkb + m];
      sr += dl.x * b.x - dl.y * b.y;
      si += dl.x * b.y + dl.y * b.x;
    }
  }
  h = V{hr, hi};
  s = V{sr, si};
}

// beta(k) ([nkb][npw_beta] contiguous) into shared memory at dst by asynchronous copies from
// every thread of the CTA (16-byte copies when the block is 16-byte aligned and sized, else one
// complex element per copy); returns once every copy has landed and the CTA has synchronised.
template <typename T>
__device__ __forceinline__ void nl_stage_beta(const FusedArgs& a, int k, c2_t<T>* dst) {
  using V = c2_t<T>;
  const V* src = static_cast<const V*>(a.beta) + (size_t)k * a.nkb * a.npw_beta;
  const size_t n = (size_t)a.nkb * a.npw_beta, bytes = n * sizeof(V);
  const unsigned d0 = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  if ((reinterpret_cast<size_t>(src) & 15) == 0 && (bytes & 15) == 0) {
    const char* s = reinterpret_cast<const char*>(src);
    for (size_t i = (size_t)threadIdx.x * 16; i < bytes; i += (size_t)blockDim.x * 16)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d0 + (unsigned)i), "l"(s + i) : "memory");
  } else {
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
      if constexpr (sizeof(V) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d0 + (unsigned)(i * 16)), "l"(src + i)
                     : "memory");
      else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d0 + (unsigned)(i * 8)), "l"(src + i)
                     : "memory");
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
}

// shared-memory bytes of the coefficients (lambda, gamma, delta) for nkb projectors
inline size_t nl_fused_bytes(int nkb, int elem_bytes) {
  return nkb > 0 ? (((size_t)3 * nkb * elem_bytes + 15) & ~(size_t)15) : 0;
}

}  // namespace pwk
