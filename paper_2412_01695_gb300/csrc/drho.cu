// Induced charge density of a perturbation (paper Sec. 2.3, Eq. drho):
//
//   drho(r) = 4 sum_k w_k sum_nu conj(u_{k,nu}(r)) [P_c du_{k,nu}](r)
//
// u_{k,nu} on the k sphere (plan_k), du on the k+q sphere (plan_kq), both brought to the real-
// space grid by the inverse transform of Sec. 2.2.2 (no normalisation); P_c du = du -
// sum_v u_{k+q,v} <S u_{k+q,v}|du> (S = 1 without q).  The augmentation term is not included
// (the paper did not accelerate it).
//
// The paper keeps two full FFT grids per band in HBM for this step (Sec. 3).  Here one CTA
// takes one (k, nu) pair at a time: both coefficient sets are scattered onto the union of the
// two spheres' z-sticks in shared memory (the transfer maps of the k -> k+q pair), both are
// transformed z on the sticks, y on the carried m1 planes, x on every line, and the product
// of an x line pair is added at once to the CTA's own partial grid (FP64, in global memory,
// L2-resident).  The CTAs take the pairs in a fixed grid-stride order and the partial grids
// are summed in a fixed order by a second kernel: the result does not depend on timing.
#include <algorithm>

#include "fft_line.cuh"
#include "fused_kernel.cuh"
#include "pwk_internal.h"
#include "solvers.h"

namespace pwk {

namespace {

constexpr int kDrhoParts = 256;   // partial grids (CTAs) of the accumulation

struct DrhoArgs {
  const void* uk = nullptr;      // [nk][nocc][npw_k] complex128
  const double2* du = nullptr;   // [nk][nocc][npw_kq] complex128 (already projected)
  const double* w = nullptr;     // [nk] weights
  double2* part = nullptr;       // [kDrhoParts][N^3]
  int nk = 0, nocc = 0, npw_k = 0, npw_kq = 0;
  const int* npwk = nullptr;
  const int* npwq = nullptr;
  const int* nstick = nullptr;
  const int* gin = nullptr;      // k sphere -> sticks
  const int* gout = nullptr;     // k+q sphere -> sticks
  const short* sid = nullptr;
  int nstick_max = 0, m1lo = 0, P = 0, L = 0, zs = 0;
};

template <typename T, int N>
__global__ void __launch_bounds__(256) drho_kernel(DrhoArgs a) {
  using V = c2_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int zs = a.zs, P = a.P, L = a.L;
  V* ZA = reinterpret_cast<V*>(smem_raw);                  // [nstick_max][zs]  u
  V* ZB = ZA + (size_t)a.nstick_max * zs;                  // [nstick_max][zs]  du
  V* YA = ZB + (size_t)a.nstick_max * zs;                  // [P][N][L]
  V* YB = YA + (size_t)P * N * L;
  V* XA = YB + (size_t)P * N * L;                          // [N (l1)][N (l2)][L]
  short* sid = reinterpret_cast<short*>(XA + (size_t)N * N * L);   // [P][N]
  const int tid = threadIdx.x, nth = blockDim.x;
  double2* acc = a.part + (size_t)blockIdx.x * N * N * N;
  for (int i = tid; i < N * N * N; i += nth) acc[i] = make_double2(0.0, 0.0);
  const int npairs = a.nk * a.nocc;
  for (int pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
    const int k = pr / a.nocc, v = pr - k * a.nocc;
    const int ns = a.nstick[k];
    const int nka = a.npwk[k], nkb = a.npwq[k];
    const double wk = 4.0 * a.w[k];
    __syncthreads();   // the previous pair is done with the buffers
    for (int i = tid; i < ns * zs; i += nth) ZA[i] = ZB[i] = V{T(0), T(0)};
    {
      const short* sk = a.sid + (size_t)k * P * N;
      for (int i = tid; i < P * N; i += nth) sid[i] = sk[i];
    }
    __syncthreads();
    {
      const double2* pu = static_cast<const double2*>(a.uk) + ((size_t)k * a.nocc + v) * a.npw_k;
      const double2* pd = a.du + ((size_t)k * a.nocc + v) * a.npw_kq;
      const int* gi = a.gin + (size_t)k * a.npw_k;
      const int* go = a.gout + (size_t)k * a.npw_kq;
      for (int g = tid; g < nka; g += nth) {
        const int m = gi[g];
        const double2 c = pu[g];
        ZA[(m >> 8) * zs + (m & 255)] = V{T(c.x), T(c.y)};
      }
      for (int g = tid; g < nkb; g += nth) {
        const int m = go[g];
        const double2 c = pd[g];
        ZB[(m >> 8) * zs + (m & 255)] = V{T(c.x), T(c.y)};
      }
    }
    __syncthreads();
    // inverse z transforms of both fields on the sticks (Eq. zfft)
    for (int s = tid; s < 2 * ns; s += nth) {
      V x[N];
      V* zr = (s < ns ? ZA + s * zs : ZB + (s - ns) * zs);
      PWK_SFOR(N, j, x[j] = zr[j]);
      LineFFT<T, N, +1>::run(x);
      PWK_SFOR(N, j, zr[j] = x[OutSlot<N, j>::value]);
    }
    __syncthreads();
    for (int l0 = 0; l0 < N; l0 += L) {
      const int lc = min(L, N - l0);
      // inverse y transforms of the carried m1 planes (Eq. yfft), both fields
      for (int t = tid; t < 2 * P * lc; t += nth) {
        const int f = t / (P * lc), r = t - f * P * lc;
        const int p = r / lc, c = r - p * lc;
        const V* Z = f ? ZB : ZA;
        V x[N];
        PWK_SFOR(N, j, {
          const int s = sid[p * N + j];
          x[j] = s >= 0 ? Z[s * zs + l0 + c] : V{T(0), T(0)};
        });
        LineFFT<T, N, +1>::run(x);
        V* yp = (f ? YB : YA) + (size_t)p * N * L + c;
        PWK_SFOR(N, l2, yp[l2 * L] = x[OutSlot<N, l2>::value]);
      }
      __syncthreads();
      // x lines (Eq. xfft) of u, kept in shared memory
      for (int t = tid; t < N * lc; t += nth) {
        const int l2 = t / lc, c = t - l2 * lc;
        V x[N];
        PWK_SFOR(N, i, {
          const int p = plane_of_slot<N>(i, a.m1lo);
          x[i] = (unsigned)p < (unsigned)P ? YA[((size_t)p * N + l2) * L + c] : V{T(0), T(0)};
        });
        LineFFT<T, N, +1>::run(x);
        PWK_SFOR(N, l1, XA[((size_t)l1 * N + l2) * L + c] = x[OutSlot<N, l1>::value]);
      }
      __syncthreads();
      // x lines of du, product conj(u) du added to this CTA's grid
      for (int t = tid; t < N * lc; t += nth) {
        const int l2 = t / lc, c = t - l2 * lc;
        V x[N];
        PWK_SFOR(N, i, {
          const int p = plane_of_slot<N>(i, a.m1lo);
          x[i] = (unsigned)p < (unsigned)P ? YB[((size_t)p * N + l2) * L + c] : V{T(0), T(0)};
        });
        LineFFT<T, N, +1>::run(x);
        double2* ag = acc + (size_t)l2 * N + l0 + c;
        PWK_SFOR(N, l1, {
          const V ua = XA[((size_t)l1 * N + l2) * L + c], ub = x[OutSlot<N, l1>::value];
          const double re = (double)ua.x * ub.x + (double)ua.y * ub.y;   // conj(u) du
          const double im = (double)ua.x * ub.y - (double)ua.y * ub.x;
          double2& d = ag[(size_t)l1 * N * N];
          d.x += wk * re;
          d.y += wk * im;
        });
      }
      __syncthreads();
    }
  }
}

// drho[l] = sum_p part[p][l] in ascending p
__global__ void drho_reduce_kernel(int nr, int nparts, const double2* part, double2* out) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nr) return;
  double sx = 0.0, sy = 0.0;
  for (int p = 0; p < nparts; ++p) {
    const double2 v = part[(size_t)p * nr + l];
    sx += v.x;
    sy += v.y;
  }
  out[l] = make_double2(sx, sy);
}

// P_c du = du - sum_v u_v <su_v|du> (su = S u, or u when S = 1), one CTA per (k, nu)
__global__ void __launch_bounds__(256) conduction_kernel(int nocc, int np, const int* npw,
                                                         const double2* u, const double2* su,
                                                         const double2* du, double2* out) {
  const int k = blockIdx.x / nocc;
  const int npk = npw[k];
  __shared__ double2 mu[64];
  const double2* D = du + (size_t)blockIdx.x * np;
  const double2* U = u + (size_t)k * nocc * np;
  const double2* SU = su + (size_t)k * nocc * np;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int v = warp; v < nocc; v += nw) {
    double sx = 0, sy = 0;
    const double2* s = SU + (size_t)v * np;
    for (int g = lane; g < npk; g += 32) {
      const double2 a = s[g], b = D[g];
      sx += a.x * b.x + a.y * b.y;
      sy += a.x * b.y - a.y * b.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) mu[v] = make_double2(sx, sy);
  }
  __syncthreads();
  double2* O = out + (size_t)blockIdx.x * np;
  for (int g = threadIdx.x; g < np; g += blockDim.x) {
    if (g >= npk) {
      O[g] = make_double2(0.0, 0.0);
      continue;
    }
    double2 r = D[g];
    for (int v = 0; v < nocc; ++v) {
      const double2 p = U[(size_t)v * np + g], m = mu[v];
      r.x -= p.x * m.x - p.y * m.y;
      r.y -= p.x * m.y + p.y * m.x;
    }
    O[g] = r;
  }
}

// work list (k, nu, nu) of every pair
__global__ void pair_items_kernel(int npairs, int nocc, int* items) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npairs) return;
  items[3 * i] = i / nocc;
  items[3 * i + 1] = items[3 * i + 2] = i % nocc;
}

size_t drho_smem(int N, int elem_bytes, const SphereMap& sm, int L) {
  const int zs = (N % 2 == 0) ? N + 1 : N;
  return ((size_t)2 * sm.nstick_max * zs + (size_t)2 * sm.P * N * L + (size_t)N * N * L) * elem_bytes +
         (size_t)sm.P * N * sizeof(short) + 16;
}

template <typename T>
int launch_drho_typed(int N, const DrhoArgs& a, int nparts, size_t smem, cudaStream_t st) {
  switch (N) {
#define PWK_DCASE(n)                                                                             \
  case n: {                                                                                      \
    auto kern = drho_kernel<T, n>;                                                               \
    cudaError_t e = allow_full_smem(kern);                                                       \
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(drho)");                     \
    kern<<<nparts, 256, smem, st>>>(a); note_launch();                                                          \
    e = cudaGetLastError();                                                                      \
    return e == cudaSuccess ? PWK_OK : cuda_fail(e, "drho_kernel");                              \
  }
    PWK_FOR_EACH_N(PWK_DCASE)
#undef PWK_DCASE
    default:
      set_error("unsupported grid size");
      return PWK_ERR_UNSUPPORTED;
  }
}

}  // namespace

}  // namespace pwk

using namespace pwk;

extern "C" int pwk_drho_batched(pwk_plan* pq, pwk_plan* pk, int precision, const void* psi_k,
                                const void* psi_kq, const void* dpsi, int nocc, const double* weights,
                                void* drho, void* stream) {
  if (pq == nullptr || pk == nullptr || psi_k == nullptr || psi_kq == nullptr || dpsi == nullptr ||
      weights == nullptr || drho == nullptr || nocc < 1) {
    set_error("null pointer or nocc < 1");
    return PWK_ERR_INVALID;
  }
  if (precision != PWK_FP64 && precision != PWK_FP32_C128) {
    set_error("precision must be PWK_FP64 or PWK_FP32_C128");
    return PWK_ERR_INVALID;
  }
  if (nocc > 64) {
    set_error("nocc > 64");
    return PWK_ERR_UNSUPPORTED;
  }
  if (pq->nk != pk->nk || pq->N != pk->N) {
    set_error("plan_k and plan_kq must have the same nk and grid");
    return PWK_ERR_INVALID;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc;
  if ((rc = ensure_xfer(pq, pk))) return rc;
  const int N = pq->N, nk = pq->nk, npq = pq->npw_max, npairs = nk * nocc;
  const SphereMap& sm = pq->xfer;
  const int elem = precision == PWK_FP64 ? 16 : 8;
  int L = N;
  while (L > 1 && drho_smem(N, elem, sm, L) > 100 * 1024) --L;
  const size_t smem = drho_smem(N, elem, sm, L);
  if (smem > 227 * 1024) {
    set_error("induced-density kernel does not fit in shared memory");
    return PWK_ERR_UNSUPPORTED;
  }
  const int nparts = std::min(npairs, kDrhoParts);
  const size_t nr = (size_t)N * N * N;
  // scratch: P_c du [nk][nocc][npw_kq], S u (with q), the work list and the partial grids
  double2 *duc = nullptr, *su = nullptr, *part = nullptr;
  int* items = nullptr;
  const size_t nv = (size_t)npairs * npq;
  cudaError_t e = scratch_alloc((void**)&duc, nv * sizeof(double2), st);
  if (e == cudaSuccess) e = scratch_alloc((void**)&part, (size_t)nparts * nr * sizeof(double2), st);
  if (e == cudaSuccess && pq->d_q != nullptr) e = scratch_alloc((void**)&su, nv * sizeof(double2), st);
  if (e == cudaSuccess && pq->d_q != nullptr)
    e = scratch_alloc((void**)&items, (size_t)npairs * 3 * sizeof(int), st);
  if (e != cudaSuccess) {
    for (void* q : {(void*)duc, (void*)part, (void*)su, (void*)items})
      if (q) cudaFreeAsync(q, st);
    return cuda_fail(e, "scratch_alloc(drho)");
  }
  const double2* suv = static_cast<const double2*>(psi_kq);
  if (pq->d_q != nullptr) {   // S u_{k+q,v}: the projector terms alone
    pair_items_kernel<<<(npairs + 255) / 256, 256, 0, st>>>(npairs, nocc, items); note_launch();
    e = cudaGetLastError();
    rc = e == cudaSuccess ? run_hpsi(pq, PWK_FP64, psi_kq, nullptr, items, nullptr, npairs, nocc, nocc, st, su)
                          : cuda_fail(e, "pair_items_kernel");
    suv = su;
  }
  if (rc == PWK_OK) {
    conduction_kernel<<<npairs, 256, 0, st>>>(nocc, npq, pq->d_npw, static_cast<const double2*>(psi_kq), suv,
                                              static_cast<const double2*>(dpsi), duc); note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "conduction_kernel");
  }
  if (rc == PWK_OK) {
    DrhoArgs a;
    a.uk = psi_k;
    a.du = duc;
    a.w = weights;
    a.part = part;
    a.nk = nk;
    a.nocc = nocc;
    a.npw_k = pk->npw_max;
    a.npw_kq = npq;
    a.npwk = pk->d_npw;
    a.npwq = pq->d_npw;
    a.nstick = sm.d_nstick;
    a.gin = sm.d_gin;
    a.gout = sm.d_gout;
    a.sid = sm.d_sid;
    a.nstick_max = sm.nstick_max;
    a.m1lo = sm.m1lo;
    a.P = sm.P;
    a.L = L;
    a.zs = (N % 2 == 0) ? N + 1 : N;
    rc = precision == PWK_FP64 ? launch_drho_typed<double>(N, a, nparts, smem, st)
                               : launch_drho_typed<float>(N, a, nparts, smem, st);
  }
  if (rc == PWK_OK) {
    drho_reduce_kernel<<<(int)((nr + 255) / 256), 256, 0, st>>>((int)nr, nparts, part,
                                                                static_cast<double2*>(drho)); note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "drho_reduce_kernel");
  }
  cudaFreeAsync(duc, st);
  cudaFreeAsync(part, st);
  if (su) cudaFreeAsync(su, st);
  if (items) cudaFreeAsync(items, st);
  return rc;
}
