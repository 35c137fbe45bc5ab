// Window-specialised fused H|psi> kernel.
//
// Same operator (kinetic and local terms) and the same one-HBM-round-trip structure as
// fused_kernel (paper Sec. 2.2 and Sec. 4; see fused_kernel.cuh), for spheres whose Miller indices all satisfy |m_i| <= W with
// W = N/4: a grid chosen to hold the differences G - G' of the basis (Sec. 4: "N_i large
// enough"), N >= 4 max|m|, always satisfies it.  With the window known at compile time:
//   * the z-sticks live in a dense (2W+1) x (2W+1) square of rows [m1][m2] (rows without a
//     stick of this k stay zero), so the y pass reads and writes them without a stick table;
//   * every transform reads only the 2W+1 window inputs (the others are literal zeros) and
//     stores only the outputs that are used later; no per-element index arithmetic or
//     predicated shared-memory access remains.
// The real sticks of the k-point (for the z passes) and the packed (row, m3) place of every
// basis vector come from the plan's window tables.
#pragma once
#include <type_traits>

#include "fft_line.cuh"
#include "fused_kernel.cuh"
#include "nl_fused.cuh"
#include "pwk_internal.h"

namespace pwk {

template <int N, int W>
struct Win {
  static constexpr int NW = 2 * W + 1;
  __host__ __device__ static constexpr bool in(int i) { return i <= W || i >= N - W; }
  __host__ __device__ static constexpr int idx(int i) { return i <= W ? i + W : i - N + W; }  // 0 .. 2W
};

// inputs outside the window, known zero in the inverse transforms (LineFFTZ prunes them)
template <int N, int W>
struct OutOfWin {
  __host__ __device__ static constexpr bool zero(int i) { return !Win<N, W>::in(i); }
};

// MODE 0: the CTA takes the l3 planes in chunks of L, with block barriers between the y, x
//         and y passes of a chunk.
// MODE 1: each warp takes its own L planes at a time (planes w L, w L + 1, ... in rounds of
//         nwarps L) through the y, x and y passes with warp-level synchronisation only; block
//         barriers remain only around the z passes.  The arithmetic of every line is the same
//         in both modes (the results are bitwise equal); only the thread mapping differs.
// The work of one band-k item (k, input slot vin, output slot vout) of the plan described
// by `a`; the kernels below decode the item and call it.
// NL: the nonlocal projector terms are applied in the epilogue (nl_fused.cuh) when the plan
//     has projectors (a.nkb > 0); the kernel without them (NL false) is compiled apart, so the
//     projector code costs it nothing.
template <typename T, typename TI, int N, int W, int MODE, bool NL>
__device__ __forceinline__ void window_body(const FusedArgs& a, int k, int vin, int vout) {
  using V = c2_t<T>;
  using VI = c2_t<TI>;
  using Wn = Win<N, W>;
  constexpr int NW = Wn::NW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int np = a.npw_in[k];
  const int ns = a.nstick[k];
  const int zs = a.zs, L = a.L, yps = a.yps;

  V* Z = reinterpret_cast<V*>(smem_raw);               // [NW*NW][zs]
  V* Y = Z + (size_t)NW * NW * zs;                      // [NW][yps] (N x L used per plane)
  // plane buffers: one [NW][yps] for the CTA (MODE 0) or one per warp (MODE 1), then the rows
  const int ycopies = MODE == 1 ? (int)(blockDim.x >> 5) : 1;
  short* rows = reinterpret_cast<short*>(Y + (size_t)ycopies * NW * yps);  // [nstick_max]

  const VI* pin = static_cast<const VI*>(a.in) + ((size_t)k * a.nvec_in + vin) * a.npw_in_max;
  VI* pout = static_cast<VI*>(a.out) + ((size_t)k * a.nvec_out + vout) * a.npw_out_max;

  // C(G) is read from global memory by the two stages that need it (scatter, kinetic term):
  // the second read hits L1/L2, and the shared memory a staged copy would take buys occupancy.
  // ---- 0: zero the stick square, stage the stick rows
  for (int i = tid; i < NW * NW * zs; i += nth) Z[i] = V{T(0), T(0)};
  {
    const short* rk = a.sid + (size_t)k * a.nstick_max;
    for (int i = tid; i < ns; i += nth) rows[i] = rk[i];
  }
  __syncthreads();

  // ---- 1: scatter
  {
    const int* gin = a.gin + (size_t)k * a.npw_in_max;
    for (int g = tid; g < np; g += nth) {
      const int m = gin[g];
      const VI v = pin[g];
      Z[(m >> 8) * zs + (m & 255)] = V{T(v.x), T(v.y)};
    }
  }
  __syncthreads();

  // ---- 2: inverse z transforms of the real sticks (inputs only in the m3 window)
  for (int s = tid; s < ns; s += nth) {
    V x[N];
    V* zr = Z + rows[s] * zs;
    PWK_SFOR(N, j, x[j] = Wn::in(j) ? zr[j] : V{T(0), T(0)});
    LineFFTZ<T, N, +1, OutOfWin<N, W>>::run(x);
    PWK_SFOR(N, j, zr[j] = x[OutSlot<N, j>::value]);
  }
  __syncthreads();

  if constexpr (MODE == 0) {
  // ---- 3: planes l3 in chunks of L
  for (int l0 = 0; l0 < N; l0 += L) {
    const int lc = min(L, N - l0);
    // 3a: inverse y transforms, inputs on the m2 window of plane p
    for (int t = tid; t < NW * lc; t += nth) {
      const int c = t / NW, p = t - c * NW;   // plane fastest: conflict-free (see window_strides)
      V x[N];
      const V* zp = Z + (size_t)p * NW * zs + l0 + c;
      PWK_SFOR(N, j, x[j] = Wn::in(j) ? zp[Wn::idx(j) * zs] : V{T(0), T(0)});
      LineFFTZ<T, N, +1, OutOfWin<N, W>>::run(x);
      V* yp = Y + (size_t)p * yps + c;
      PWK_SFOR(N, l2, yp[l2 * L] = x[OutSlot<N, l2>::value]);
    }
    __syncthreads();
    // 3b: x lines: inverse x, V(r) product, forward x (window outputs only)
    for (int t = tid; t < N * lc; t += nth) {
      const int l2 = t / lc, c = t - l2 * lc;
      // V(r) of the line is requested first: its latency hides behind the inverse transform
      T w[N];
      load_vline<T, N>(static_cast<const T*>(a.V) + ((size_t)l2 * N + l0 + c) * N, w);
      V x[N];
      const V* yl = Y + (size_t)l2 * L + c;
      PWK_SFOR(N, i, x[i] = Wn::in(i) ? yl[(size_t)Wn::idx(i) * yps] : V{T(0), T(0)});
      LineFFTZ<T, N, +1, OutOfWin<N, W>>::run(x);
      V y[N];
      PWK_SFOR(N, l1, {
        const V u = x[OutSlot<N, l1>::value];
        y[l1] = V{u.x * w[l1], u.y * w[l1]};
      });
      LineFFT<T, N, -1>::run(y);
      V* yo = Y + (size_t)l2 * L + c;
      PWK_SFOR(N, i, {
        if constexpr (Wn::in(i)) yo[(size_t)Wn::idx(i) * yps] = y[OutSlot<N, i>::value];
      });
    }
    __syncthreads();
    // 3c: forward y transforms, window outputs written back to the stick square
    for (int t = tid; t < NW * lc; t += nth) {
      const int c = t / NW, p = t - c * NW;
      V x[N];
      const V* yp = Y + (size_t)p * yps + c;
      PWK_SFOR(N, l2, x[l2] = yp[l2 * L]);
      LineFFT<T, N, -1>::run(x);
      V* zp = Z + (size_t)p * NW * zs + l0 + c;
      PWK_SFOR(N, j, {
        if constexpr (Wn::in(j)) zp[Wn::idx(j) * zs] = x[OutSlot<N, j>::value];
      });
    }
    __syncthreads();
  }
  } else {
    // ---- 3 (MODE 1): each warp carries L planes of its own through y, x, y
    const int warp = tid >> 5, lane = tid & 31, nw = nth >> 5;
    V* Yw = Y + (size_t)warp * NW * yps;        // [NW][yps]: plane p row, (l2, cc) at l2 L + cc
    for (int l0 = warp * L; l0 < N; l0 += nw * L) {
      const int lc = min(L, N - l0);
      // y inverse: lane -> (plane p, column cc), inputs on the m2 window
      for (int t = lane; t < NW * lc; t += 32) {
        const int c = t / NW, p = t - c * NW;
        V x[N];
        const V* zp = Z + (size_t)p * NW * zs + l0 + c;
        PWK_SFOR(N, j, x[j] = Wn::in(j) ? zp[Wn::idx(j) * zs] : V{T(0), T(0)});
        LineFFTZ<T, N, +1, OutOfWin<N, W>>::run(x);
        V* yp = Yw + (size_t)p * yps + c;
        PWK_SFOR(N, l2, yp[l2 * L] = x[OutSlot<N, l2>::value]);
      }
      __syncwarp();
      // x lines: inverse x, V(r) product, forward x (window outputs only)
      for (int t = lane; t < N * lc; t += 32) {
        const int l2 = t / lc, c = t - l2 * lc;
        T w[N];
        load_vline<T, N>(static_cast<const T*>(a.V) + ((size_t)l2 * N + l0 + c) * N, w);
        V x[N];
        const V* yl = Yw + (size_t)l2 * L + c;
        PWK_SFOR(N, i, x[i] = Wn::in(i) ? yl[(size_t)Wn::idx(i) * yps] : V{T(0), T(0)});
        LineFFTZ<T, N, +1, OutOfWin<N, W>>::run(x);
        V y[N];
        PWK_SFOR(N, l1, {
          const V u = x[OutSlot<N, l1>::value];
          y[l1] = V{u.x * w[l1], u.y * w[l1]};
        });
        LineFFT<T, N, -1>::run(y);
        V* yo = Yw + (size_t)l2 * L + c;
        PWK_SFOR(N, i, {
          if constexpr (Wn::in(i)) yo[(size_t)Wn::idx(i) * yps] = y[OutSlot<N, i>::value];
        });
      }
      __syncwarp();
      // y forward, window outputs back to the stick square (this warp's columns only)
      for (int t = lane; t < NW * lc; t += 32) {
        const int c = t / NW, p = t - c * NW;
        V x[N];
        const V* yp = Yw + (size_t)p * yps + c;
        PWK_SFOR(N, l2, x[l2] = yp[l2 * L]);
        LineFFT<T, N, -1>::run(x);
        V* zp = Z + (size_t)p * NW * zs + l0 + c;
        PWK_SFOR(N, j, {
          if constexpr (Wn::in(j)) zp[Wn::idx(j) * zs] = x[OutSlot<N, j>::value];
        });
      }
      __syncwarp();
    }
    __syncthreads();
  }

  // ---- 4: forward z transforms of the real sticks (window outputs only)
  for (int s = tid; s < ns; s += nth) {
    V x[N];
    V* zr = Z + rows[s] * zs;
    PWK_SFOR(N, j, x[j] = zr[j]);
    LineFFT<T, N, -1>::run(x);
    PWK_SFOR(N, j, {
      if constexpr (Wn::in(j)) zr[j] = x[OutSlot<N, j>::value];
    });
  }
  __syncthreads();

  // ---- 5: gather with 1/N_r; kinetic term
  if (!NL || a.nkb == 0) {
    const int* gout = a.gout + (size_t)k * a.npw_out_max;
    const T sc = T(a.scale);
    const double* g2k = a.g2 + (size_t)k * a.npw_out_max;
    for (int g = tid; g < np; g += nth) {
      const int m = gout[g];
      const V z = Z[(m >> 8) * zs + (m & 255)];
      const T t2 = T(g2k[g]);
      const VI cv = pin[g];
      V acc = V{z.x * sc + t2 * T(cv.x), z.y * sc + t2 * T(cv.y)};
      pout[g] = VI{TI(acc.x), TI(acc.y)};
    }
    for (int g = np + tid; g < a.npw_out_max; g += nth) pout[g] = VI{TI(0), TI(0)};
  } else if constexpr (NL) {
    // With projectors (nl_fused.cuh): the local result and C go to shared memory past the
    // stick square; once the square is read, beta(k) is staged over it, and the projections,
    // gamma (delta) and the add-back (S C) run from shared memory.
    const int* gout = a.gout + (size_t)k * a.npw_out_max;
    const T sc = T(a.scale);
    const double* g2k = a.g2 + (size_t)k * a.npw_out_max;
    V* LOC = reinterpret_cast<V*>(smem_raw + a.loc_off);   // [npw_out_max] local + kinetic
    V* Cs = LOC + a.npw_out_max;                             // [npw_out_max] C in T
    V* nls = reinterpret_cast<V*>(smem_raw + a.nl_off);
    for (int g = tid; g < np; g += nth) {
      const int m = gout[g];
      const V z = Z[(m >> 8) * zs + (m & 255)];
      const T t2 = T(g2k[g]);
      const VI cv = pin[g];
      LOC[g] = V{z.x * sc + t2 * T(cv.x), z.y * sc + t2 * T(cv.y)};
      Cs[g] = V{T(cv.x), T(cv.y)};
    }
    __syncthreads();
    V* Bs = reinterpret_cast<V*>(smem_raw);                  // [nkb][npw_beta]
    nl_stage_beta<T>(a, k, Bs);
    nl_fused_project<T>(a, Bs, a.npw_beta, Cs, np, nls);
    __syncthreads();
    nl_fused_coef<T>(a, nls);
    __syncthreads();
    const bool with_s = a.sout != nullptr;
    const bool with_q = with_s && a.qm != nullptr;
    VI* sout = with_s ? static_cast<VI*>(a.sout) + ((size_t)k * a.nvec_out + vout) * a.npw_out_max : nullptr;
    for (int g = tid; g < np; g += nth) {
      V h, sv;
      nl_fused_addback<T>(a, Bs, a.npw_beta, g, nls, with_q, h, sv);
      const V l = LOC[g];
      pout[g] = VI{TI(l.x + h.x), TI(l.y + h.y)};
      if (with_s) {
        const VI cv = pin[g];
        sout[g] = a.qm != nullptr ? VI{cv.x + TI(sv.x), cv.y + TI(sv.y)} : cv;
      }
    }
    for (int g = np + tid; g < a.npw_out_max; g += nth) {
      pout[g] = VI{TI(0), TI(0)};
      if (with_s) sout[g] = VI{TI(0), TI(0)};
    }
  }
}

// One CTA per work item of one plan: item = (k - k0) * nvec + band of a batched call, or the
// (k, in_slot, out_slot) entry of a work list.
template <typename T, typename TI, int N, int W, int MODE, bool NL>
__global__ void __launch_bounds__(256) fused_window_kernel(FusedArgs a) {
  const int item = blockIdx.x;
  if (a.d_count != nullptr && item >= *a.d_count) return;
  int k, vin, vout;
  if (a.items != nullptr) {
    k = a.items[3 * item];
    vin = a.items[3 * item + 1];
    vout = a.items[3 * item + 2];
    if (k == -1) return;
    if (k < 0 || k >= a.nk || vin < 0 || vin >= a.nvec_in || vout < 0 || vout >= a.nvec_out) {
      if (threadIdx.x == 0 && a.err != nullptr) atomicOr(a.err, 1);
      return;
    }
  } else {
    const int kr = item / a.nvec_in;
    vin = vout = item - kr * a.nvec_in;
    k = a.k0 + kr;
  }
  window_body<T, TI, N, W, MODE, NL>(a, k, vin, vout);
}

// One CTA per work item of a list that spans several plans of the same grid (cells with their
// own atoms, projectors, V(r), spheres and k-points): entry (plan, k, in_slot, out_slot) of
// a.items, the plan's arguments at a.multi[plan] (in device memory).  An entry with plan = -1
// is an empty slot; one outside the plans or the plan's k-points and slots is skipped and
// flagged in the first plan's error word.
template <typename T, typename TI, int N, int W, int MODE>
__global__ void __launch_bounds__(256) fused_window_multi_kernel(FusedArgs a0) {
  const int item = blockIdx.x;
  const int* it = a0.items + 4 * (size_t)item;
  const int p = it[0], k = it[1], vin = it[2], vout = it[3];
  if (p == -1) return;
  if (p < 0 || p >= a0.nmulti) {
    if (threadIdx.x == 0 && a0.err != nullptr) atomicOr(a0.err, 1);
    return;
  }
  const FusedArgs& a = a0.multi[p];
  if (k < 0 || k >= a.nk || vin < 0 || vin >= a.nvec_in || vout < 0 || vout >= a.nvec_out) {
    if (threadIdx.x == 0 && a0.err != nullptr) atomicOr(a0.err, 1);
    return;
  }
  window_body<T, TI, N, W, MODE, true>(a, k, vin, vout);
}

// window half-width instantiated for a grid of size N
__host__ __device__ constexpr int window_of(int N) { return N / 4; }

template <typename T, typename TI>
int launch_window_multi(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st) {
  if (nblocks <= 0) return PWK_OK;
  switch (N) {
#define PWK_WMCASE(n)                                                                           \
  case n: {                                                                                     \
    auto kern = s.kind == 2 ? fused_window_multi_kernel<T, TI, n, window_of(n), 1>              \
                            : fused_window_multi_kernel<T, TI, n, window_of(n), 0>;             \
    cudaError_t e = allow_full_smem(kern);                                                      \
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(window multi)");            \
    kern<<<nblocks, s.threads, s.smem, st>>>(a); note_launch();                                                \
    e = cudaGetLastError();                                                                     \
    if (e != cudaSuccess) return cuda_fail(e, "window multi kernel launch");                    \
    return PWK_OK;                                                                              \
  }
    PWK_FOR_EACH_N(PWK_WMCASE)
#undef PWK_WMCASE
    default:
      set_error("unsupported grid size");
      return PWK_ERR_UNSUPPORTED;
  }
}

template <typename T, typename TI, bool NL>
int launch_window(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st) {
  if (nblocks <= 0) return PWK_OK;
  switch (N) {
#define PWK_WCASE(n)                                                                            \
  case n: {                                                                                     \
    auto kern = s.kind == 2 ? fused_window_kernel<T, TI, n, window_of(n), 1, NL>                \
                            : fused_window_kernel<T, TI, n, window_of(n), 0, NL>;               \
    cudaError_t e = allow_full_smem(kern);                                                      \
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(window)");                  \
    kern<<<nblocks, s.threads, s.smem, st>>>(a); note_launch();                                                \
    e = cudaGetLastError();                                                                     \
    if (e != cudaSuccess) return cuda_fail(e, "window kernel launch");                          \
    return PWK_OK;                                                                              \
  }
    PWK_FOR_EACH_N(PWK_WCASE)
#undef PWK_WCASE
    default:
      set_error("unsupported grid size");
      return PWK_ERR_UNSUPPORTED;
  }
}

}  // namespace pwk
