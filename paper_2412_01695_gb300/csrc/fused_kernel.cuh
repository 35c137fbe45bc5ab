// Fused local-potential kernel: one CTA applies the kinetic and local terms of H to one
// band of one k-point with a single round trip to HBM (read C, write the local part of H C).
// The nonlocal projector terms run as separate kernels around it (nonlocal.cu): their
// projections over all bands of a k-point share one staged copy of beta(k).
//
// Per work item (paper Sec. 2.2 and Sec. 4, Fig. 2 flow, here fused into one kernel):
//   1. load C(G) and scatter it onto the z-sticks held in shared memory (Sec. 3 "sets the
//      non zero elements of this grid");
//   2. inverse z transforms, only on the sticks (m1, m2) that carry coefficients (Eq. zfft);
//   3. for each chunk of L planes l3: inverse y transforms on the m1 planes that carry
//      sticks (Eq. yfft); for every x line (l2, l3): inverse x transform (Eq. xfft),
//      u'(r) = V(r) u(r) (Sec. 2.2.2), forward x transform keeping only the m1 planes that
//      are carried back; forward y transforms written back onto the sticks;
//   4. forward z transforms on the sticks (Eq. fwFFT);
//   5. gather r -> G with the 1/N_r of Eq. fwFFT and add the kinetic term |k+G|^2 C
//      (Sec. 2.2.1, Ry).
// The pruning skips transforms of lines that are identically zero or whose results are
// discarded; the result equals the full 3D transform pair exactly (up to rounding).
//
// Template parameters: T arithmetic type, TI io type (complex of TI in memory), N grid
// size, CPLXV: V is a complex128 field and the kinetic term is absent (the
// lattice-periodic dV psi product of the DFPT right-hand side, Eq. linear_system).
// The real V(r) is read from a transposed copy [l2][l3][l1] (one x-line contiguous); the
// complex dv(r) keeps the caller's [l1][l2][l3] layout.
#pragma once
#include <type_traits>

#include "fft_line.cuh"
#include "nl_fused.cuh"
#include "pwk_internal.h"

namespace pwk {

// Load the N contiguous values of one V(r) x-line (layout [l2][l3][l1], l1 fastest) with
// 16-byte vector loads when the line is 16-byte aligned (N * sizeof(T) a multiple of 16).
template <typename T, int N>
__device__ __forceinline__ void load_vline(const T* __restrict__ p, T (&w)[N]) {
  constexpr int VEC = 16 / sizeof(T);
  if constexpr ((N * sizeof(T)) % 16 == 0) {
    using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    const VT* q = reinterpret_cast<const VT*>(p);
    PWK_SFOR(N / VEC, j, {
      const VT v = __ldg(q + j);
      if constexpr (sizeof(T) == 4) {
        w[4 * j] = v.x;
        w[4 * j + 1] = v.y;
        w[4 * j + 2] = v.z;
        w[4 * j + 3] = v.w;
      } else {
        w[2 * j] = v.x;
        w[2 * j + 1] = v.y;
      }
    });
  } else {
    PWK_SFOR(N, j, w[j] = __ldg(p + j));
  }
}

// plane index p of grid slot i (signed m1 = i or i - N) in the window [m1lo, m1lo + P):
// p = (i - m1lo) mod N; the caller tests p < P.  m1lo lies in (-N/2, N/2).
template <int N>
__device__ __forceinline__ int plane_of_slot(int i, int m1lo) {
  int p = i - m1lo;
  return p < 0 ? p + N : (p >= N ? p - N : p);
}

// NL: the projector terms are applied as well (nl_fused.cuh: projections after the scatter
// from the staged C, add-back in the gather, beta(k) read through L1/L2); compiled apart.
template <typename T, typename TI, int N, bool CPLXV, bool NL>
__global__ void __launch_bounds__(256) fused_kernel(FusedArgs a) {
  using V = c2_t<T>;
  using VI = c2_t<TI>;
  extern __shared__ __align__(16) unsigned char smem_raw[];

  const int item = blockIdx.x;
  if (a.d_count != nullptr && item >= *a.d_count) return;
  int k, vin, vout;
  if (a.items != nullptr) {
    k = a.items[3 * item];
    vin = a.items[3 * item + 1];
    vout = a.items[3 * item + 2];
    if (k == -1) return;   // an empty slot of a fixed-size work list
    if (k < 0 || k >= a.nk || vin < 0 || vin >= a.nvec_in || vout < 0 || vout >= a.nvec_out) {
      if (threadIdx.x == 0 && a.err != nullptr) atomicOr(a.err, 1);
      return;
    }
  } else {
    const int kr = item / a.nvec_in;
    vin = vout = item - kr * a.nvec_in;
    k = a.k0 + kr;
  }
  const int tid = threadIdx.x, nth = blockDim.x;
  const int npi = a.npw_in[k], npo = a.npw_out[k];
  const int ns = a.nstick[k];
  const int zs = a.zs, P = a.P, L = a.L;

  V* Z = reinterpret_cast<V*>(smem_raw);
  V* Y = Z + (size_t)a.nstick_max * zs;
  V* psis = Y + (size_t)P * N * L;
  short* sid = reinterpret_cast<short*>(psis + a.npw_in_max);

  const VI* pin = static_cast<const VI*>(a.in) + ((size_t)k * a.nvec_in + vin) * a.npw_in_max;
  VI* pout = static_cast<VI*>(a.out) + ((size_t)k * a.nvec_out + vout) * a.npw_out_max;

  // ---- 0: zero the sticks, stage the stick table and C(G)
  for (int i = tid; i < ns * zs; i += nth) Z[i] = V{T(0), T(0)};
  {
    const short* sk = a.sid + (size_t)k * P * N;
    for (int i = tid; i < P * N; i += nth) sid[i] = sk[i];
  }
  for (int g = tid; g < npi; g += nth) {
    VI v = pin[g];
    psis[g] = V{T(v.x), T(v.y)};
  }
  __syncthreads();

  // ---- 1: scatter onto the sticks; with projectors, lambda = beta^H C
  constexpr bool nl = !CPLXV && NL;
  V* nls = reinterpret_cast<V*>(smem_raw + a.nl_off);
  {
    const int* gin = a.gin + (size_t)k * a.npw_in_max;
    for (int g = tid; g < npi; g += nth) {
      const int m = gin[g];
      Z[(m >> 8) * zs + (m & 255)] = psis[g];
    }
  }
  const V* nl_bk = nl ? static_cast<const V*>(a.beta) + (size_t)k * a.nkb * a.npw_beta : nullptr;
  if (nl) nl_fused_project<T>(a, nl_bk, a.npw_beta, psis, npi, nls);
  __syncthreads();
  if (nl) nl_fused_coef<T>(a, nls);   // read after the barriers that follow

  // ---- 2: inverse z transforms on the sticks
  for (int s = tid; s < ns; s += nth) {
    V x[N];
    V* zr = Z + s * zs;
    PWK_SFOR(N, j, x[j] = zr[j]);
    LineFFT<T, N, +1>::run(x);
    PWK_SFOR(N, j, zr[j] = x[OutSlot<N, j>::value]);
  }
  __syncthreads();

  // ---- 3: planes l3 in chunks of L
  for (int l0 = 0; l0 < N; l0 += L) {
    const int lc = min(L, N - l0);
    // 3a: inverse y transforms of the carried m1 planes (Eq. yfft)
    for (int t = tid; t < P * lc; t += nth) {
      const int p = t / lc, c = t - p * lc;
      V x[N];
      PWK_SFOR(N, j, {
        const int s = sid[p * N + j];
        x[j] = s >= 0 ? Z[s * zs + l0 + c] : V{T(0), T(0)};
      });
      LineFFT<T, N, +1>::run(x);
      V* yp = Y + (size_t)p * N * L + c;
      PWK_SFOR(N, l2, yp[l2 * L] = x[OutSlot<N, l2>::value]);
    }
    __syncthreads();
    // 3b: x lines: inverse x (Eq. xfft), V(r) product, forward x (Eq. fwFFT, x part)
    for (int t = tid; t < N * lc; t += nth) {
      const int l2 = t / lc, c = t - l2 * lc;
      V x[N];
      PWK_SFOR(N, i, {
        const int p = plane_of_slot<N>(i, a.m1lo);
        x[i] = ((unsigned)p < (unsigned)P) ? Y[((size_t)p * N + l2) * L + c] : V{T(0), T(0)};
      });
      LineFFT<T, N, +1>::run(x);
      V y[N];
      const size_t vb = (size_t)l2 * N + l0 + c;
      if constexpr (CPLXV) {
        const double2* dv = static_cast<const double2*>(a.V);
        PWK_SFOR(N, l1, {
          const double2 w = dv[(size_t)l1 * N * N + vb];
          const V u = x[OutSlot<N, l1>::value];
          y[l1] = V{T(u.x * w.x - u.y * w.y), T(u.x * w.y + u.y * w.x)};
        });
      } else {
        // V transposed: the x-line (l2, l3) is contiguous
        T w[N];
        load_vline<T, N>(static_cast<const T*>(a.V) + ((size_t)l2 * N + l0 + c) * N, w);
        PWK_SFOR(N, l1, {
          const V u = x[OutSlot<N, l1>::value];
          y[l1] = V{u.x * w[l1], u.y * w[l1]};
        });
      }
      LineFFT<T, N, -1>::run(y);
      PWK_SFOR(N, i, {
        const int p = plane_of_slot<N>(i, a.m1lo);
        if ((unsigned)p < (unsigned)P) Y[((size_t)p * N + l2) * L + c] = y[OutSlot<N, i>::value];
      });
    }
    __syncthreads();
    // 3c: forward y transforms, written back onto the sticks
    for (int t = tid; t < P * lc; t += nth) {
      const int p = t / lc, c = t - p * lc;
      V x[N];
      const V* yp = Y + (size_t)p * N * L + c;
      PWK_SFOR(N, l2, x[l2] = yp[l2 * L]);
      LineFFT<T, N, -1>::run(x);
      PWK_SFOR(N, j, {
        const int s = sid[p * N + j];
        if (s >= 0) Z[s * zs + l0 + c] = x[OutSlot<N, j>::value];
      });
    }
    __syncthreads();
  }

  // ---- 4: forward z transforms on the sticks
  for (int s = tid; s < ns; s += nth) {
    V x[N];
    V* zr = Z + s * zs;
    PWK_SFOR(N, j, x[j] = zr[j]);
    LineFFT<T, N, -1>::run(x);
    PWK_SFOR(N, j, zr[j] = x[OutSlot<N, j>::value]);
  }
  __syncthreads();

  // ---- 5: gather with 1/N_r; kinetic term
  {
    const int* gout = a.gout + (size_t)k * a.npw_out_max;
    const T sc = T(a.scale);
    const double* g2k = a.g2 != nullptr ? a.g2 + (size_t)k * a.npw_out_max : nullptr;
    const bool with_s = nl && a.sout != nullptr;
    VI* sout = with_s ? static_cast<VI*>(a.sout) + ((size_t)k * a.nvec_out + vout) * a.npw_out_max : nullptr;
    for (int g = tid; g < npo; g += nth) {
      const int m = gout[g];
      const V z = Z[(m >> 8) * zs + (m & 255)];
      V acc = V{z.x * sc, z.y * sc};
      if constexpr (!CPLXV) {
        if (g2k != nullptr) {
          const T t2 = T(g2k[g]);
          acc.x += t2 * psis[g].x;
          acc.y += t2 * psis[g].y;
        }
        if (nl) {   // the in and out spheres are the same here (npi == npo)
          V h, sv;
          nl_fused_addback<T>(a, nl_bk, a.npw_beta, g, nls, with_s && a.qm != nullptr, h, sv);
          acc.x += h.x;
          acc.y += h.y;
          if (with_s) {
            const VI cv = pin[g];
            sout[g] = a.qm != nullptr ? VI{cv.x + TI(sv.x), cv.y + TI(sv.y)} : cv;
          }
        }
      }
      pout[g] = VI{TI(acc.x), TI(acc.y)};
    }
    for (int g = npo + tid; g < a.npw_out_max; g += nth) {
      pout[g] = VI{TI(0), TI(0)};
      if (with_s) sout[g] = VI{TI(0), TI(0)};
    }
  }
}

template <typename T, typename TI, bool CPLXV, bool NL>
int launch_fused(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st) {
  if (nblocks <= 0) return PWK_OK;
  switch (N) {
#define PWK_CASE(n)                                                                             \
  case n: {                                                                                     \
    auto kern = fused_kernel<T, TI, n, CPLXV, NL>;                                                  \
    cudaError_t e = allow_full_smem(kern);                                                      \
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(fused)");                   \
    kern<<<nblocks, s.threads, s.smem, st>>>(a); note_launch();                                                \
    e = cudaGetLastError();                                                                     \
    if (e != cudaSuccess) return cuda_fail(e, "fused kernel launch");                           \
    return PWK_OK;                                                                              \
  }
    PWK_FOR_EACH_N(PWK_CASE)
#undef PWK_CASE
    default:
      set_error("unsupported grid size");
      return PWK_ERR_UNSUPPORTED;
  }
}

}  // namespace pwk
