// Nonlocal projector terms of H and the overlap S for a list of band-k work items
// (paper Sec. 2.2, "Non local pseudopotential and overlap matrix"):
//
//   nl_project_kernel:  lambda_n = sum_G conj(beta_n(k+G)) C(G)          (Eq. lambdah)
//                       gamma_m  = sum_n D_mn lambda_n                    (Eq. gamma)
//                       delta_m  = sum_n q_mn lambda_n                    (Eq. delta_eq)
//   nl_addback_kernel:  H C(G)  += sum_m gamma_m beta_m(k+G)              (Eq. finalnl)
//                       S C(G)   = C(G) + sum_m delta_m beta_m(k+G)       (Eq. finals)
//
// The paper computes these as matrix-matrix products over the bands of a k-point.  Here one
// CTA takes eight consecutive work items (one warp each); the bands of one k share its
// projectors, so the CTA stages beta(k) through shared memory in tiles of PC projectors
// x kNlTile plane waves and every warp of that k reads the tile from there: beta(k) crosses
// L2 once per eight bands instead of once per band.  Tiles move by asynchronous copies
// (cp.async) through a ring of kNlStages buffers, so a CTA keeps two tiles in flight while it
// works on a third.  The projection runs before the local
// term (it reads C, which an in-place call overwrites); the add-back runs after it and adds to
// the output.  gamma and delta pass between the two kernels through a scratch array.
//
// Summation orders are fixed: lane l of a warp sums G = l, l + 32, ... in ascending order and
// the lanes are combined by a fixed xor tree; gamma, delta and the add-back sum over the
// projectors in ascending order.  Results do not depend on the launch.
#include <algorithm>

#include "fft_line.cuh"
#include "pwk_internal.h"

namespace pwk {

namespace {

constexpr int kNlItems = 8;     // work items (warps) per CTA
constexpr int kNlTile = 128;    // plane waves per staged tile
// projectors per staged tile (the accumulators of a chunk live in registers)
// Projectors per staged tile, PC, is a template parameter: every projector loop is unrolled
// over exactly PC accumulators.  The host picks PC from {4, 8, 9, 12, 16} so that the chunks
// cover nkb with the fewest unused slots (9 for one s+p+d atom, 12 for four such atoms).
constexpr int kNlPcs[] = {16, 12, 9, 8, 4};
int nl_pick_pc(int nkb, int max_pc) {
  int best = 4, best_waste = 1 << 30, best_chunks = 1 << 30;
  for (int pc : kNlPcs) {
    if (pc > max_pc) continue;
    const int chunks = (nkb + pc - 1) / pc, waste = chunks * pc - nkb;
    if (waste < best_waste || (waste == best_waste && chunks < best_chunks)) {
      best = pc;
      best_waste = waste;
      best_chunks = chunks;
    }
  }
  return best;
}

// (k, vin, vout) of work item `item`; k = -1 when the warp has nothing to do.
__device__ __forceinline__ void nl_item(const NlArgs& a, int item, int& k, int& vin, int& vout) {
  k = -1;
  vin = vout = 0;
  if (item >= a.nitems) return;
  if (a.d_count != nullptr && item >= *a.d_count) return;
  if (a.items != nullptr) {
    const int kk = a.items[3 * item];
    vin = a.items[3 * item + 1];
    vout = a.items[3 * item + 2];
    if (kk < 0 || kk >= a.nk || vin < 0 || vin >= a.nvec_in || vout < 0 || vout >= a.nvec_out) return;
    k = kk;
  } else {
    const int kr = item / a.nvec_in;
    vin = vout = item - kr * a.nvec_in;
    k = a.k0 + kr;
  }
}

// true for the first warp of the CTA whose item has k-point ks[w] (the CTA handles each
// distinct k-point once; ks is in shared memory, so the answer is uniform over the CTA)
__device__ __forceinline__ bool first_of_k(const int* ks, int w) {
  if (ks[w] < 0) return false;
  for (int v = 0; v < w; ++v)
    if (ks[v] == ks[w]) return false;
  return true;
}

constexpr int kNlThreads = kNlItems * 32;
constexpr int kNlStages = 3;    // tiles in flight per CTA (asynchronous copies)

// Asynchronous global -> shared copy of one complex element (8 or 16 bytes), zero-filled when
// !valid (nothing is read then; src must still point into the array).
template <int B>
__device__ __forceinline__ void cp_async_elem(void* dst, const void* src, bool valid) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  const int n = valid ? B : 0;
  if constexpr (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Shared-memory ring of kNlStages tiles: beta(k) projectors [c0, c0 + nc) x plane waves
// [g0, g0 + kNlTile) and, for the projection, the same plane waves of the CTA's input vectors.
template <typename T, typename TI, int PC>
struct NlRing {
  using V = c2_t<T>;
  using VI = c2_t<TI>;
  static constexpr int kChunk = PC;
  static constexpr size_t kBeta = (size_t)kChunk * kNlTile * sizeof(V);
  static constexpr size_t kPsi = (size_t)kNlItems * kNlTile * sizeof(VI);
  static constexpr size_t kSlot = kBeta + kPsi;
  unsigned char* base;
  __device__ V* beta(int slot) const { return reinterpret_cast<V*>(base + slot * kSlot); }
  __device__ VI* psi(int slot) const { return reinterpret_cast<VI*>(base + slot * kSlot + kBeta); }
  // issue the copies of one tile (every thread of the CTA takes part; `pin` of this warp's
  // item or null)
  __device__ __forceinline__ void issue(int slot, const V* bk, int ldb, int c0, int nc, int g0, int np,
                                        const VI* pin) const {
    V* b = beta(slot);
    for (int t = threadIdx.x; t < kChunk * kNlTile; t += kNlThreads) {
      const int i = t / kNlTile, g = g0 + (t - i * kNlTile);
      const bool ok = i < nc && g < np;
      cp_async_elem<sizeof(V)>(b + t, ok ? bk + (size_t)(c0 + i) * ldb + g : bk, ok);
    }
    if (pin != nullptr) {
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      VI* ps = psi(slot) + warp * kNlTile;
#pragma unroll
      for (int u = 0; u < kNlTile / 32; ++u) {
        const int g = g0 + lane + 32 * u;
        cp_async_elem<sizeof(VI)>(ps + lane + 32 * u, g < np ? pin + g : pin, g < np);
      }
    }
    cp_async_commit();
  }
};

template <typename T, typename TI, int PC>
__global__ void __launch_bounds__(kNlThreads, sizeof(T) == 4 ? 3 : 2) nl_project_kernel(NlArgs a) {
  using V = c2_t<T>;
  using VI = c2_t<TI>;
  using Ring = NlRing<T, TI, PC>;
  constexpr int kNlChunk = Ring::kChunk;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Ring ring{smem_raw};
  V* lam = reinterpret_cast<V*>(smem_raw + kNlStages * Ring::kSlot);   // [kNlItems][nkb]
  __shared__ int ks[kNlItems];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.x * kNlItems + warp;
  int k, vin, vout;
  nl_item(a, item, k, vin, vout);
  if (lane == 0) ks[warp] = k;
  __syncthreads();
  for (int w0 = 0; w0 < kNlItems; ++w0) {
    if (!first_of_k(ks, w0)) continue;
    const int kk = ks[w0];
    const int np = a.npw[kk];
    const int ntile = (np + kNlTile - 1) / kNlTile;
    const V* bk = static_cast<const V*>(a.beta) + (size_t)kk * a.nkb * a.npw_max;
    const bool mine = k == kk;
    const VI* pin = mine ? static_cast<const VI*>(a.in) + ((size_t)kk * a.nvec_in + vin) * a.npw_max : nullptr;
    for (int c0 = 0; c0 < a.nkb; c0 += kNlChunk) {
      const int nc = min(kNlChunk, a.nkb - c0);
      T ar[kNlChunk], ai[kNlChunk];
#pragma unroll
      for (int j = 0; j < kNlChunk; ++j) ar[j] = ai[j] = T(0);
#pragma unroll
      for (int t = 0; t < kNlStages - 1; ++t) {
        if (t < ntile) ring.issue(t, bk, a.npw_max, c0, nc, t * kNlTile, np, pin);
        else cp_async_commit();
      }
      for (int t = 0; t < ntile; ++t) {
        cp_async_wait<kNlStages - 2>();   // this thread's copies of tile t have landed
        __syncthreads();                  // everyone's have; tile t - 1 is consumed
        const int tn = t + kNlStages - 1;
        if (tn < ntile) ring.issue(tn % kNlStages, bk, a.npw_max, c0, nc, tn * kNlTile, np, pin);
        else cp_async_commit();
        if (mine) {
          const V* bt = ring.beta(t % kNlStages);
          const VI* pt = ring.psi(t % kNlStages) + warp * kNlTile;
#pragma unroll
          for (int u = 0; u < kNlTile / 32; ++u) {
            const VI cv = pt[lane + 32 * u];
            const T cr = T(cv.x), ci = T(cv.y);
#pragma unroll
            for (int j = 0; j < kNlChunk; ++j) {
              if (j < nc) {
                const V b = bt[j * kNlTile + lane + 32 * u];
                ar[j] += b.x * cr + b.y * ci;   // conj(beta) * C
                ai[j] += b.x * ci - b.y * cr;
              }
            }
          }
        }
      }
      cp_async_wait<0>();
      __syncthreads();   // the ring is free for the next chunk
      if (mine) {
#pragma unroll
        for (int j = 0; j < kNlChunk; ++j) {
          if (j < nc) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              ar[j] += __shfl_xor_sync(0xffffffffu, ar[j], o);
              ai[j] += __shfl_xor_sync(0xffffffffu, ai[j], o);
            }
            if (lane == 0) lam[warp * a.nkb + c0 + j] = V{ar[j], ai[j]};
          }
        }
      }
    }
  }
  __syncthreads();
  if (k < 0) return;
  // gamma = D lambda (Eq. gamma), delta = q lambda (Eq. delta_eq)
  const V* lw = lam + warp * a.nkb;
  V* cf = static_cast<V*>(a.coef) + (size_t)item * 2 * a.nkb;
  const T* D = static_cast<const T*>(a.D);
  const T* q = static_cast<const T*>(a.q);
  for (int i = lane; i < a.nkb; i += 32) {
    T gr = T(0), gi = T(0), dr = T(0), di = T(0);
    for (int j = 0; j < a.nkb; ++j) {
      const V l = lw[j];
      const T dm = D[(size_t)i * a.nkb + j];
      gr += dm * l.x;
      gi += dm * l.y;
      if (q != nullptr) {
        const T qm = q[(size_t)i * a.nkb + j];
        dr += qm * l.x;
        di += qm * l.y;
      }
    }
    cf[i] = V{gr, gi};
    cf[a.nkb + i] = V{dr, di};
  }
}

template <typename T, typename TI, int PC>
__global__ void __launch_bounds__(kNlThreads, sizeof(T) == 4 ? 3 : 2) nl_addback_kernel(NlArgs a) {
  using V = c2_t<T>;
  using VI = c2_t<TI>;
  using Ring = NlRing<T, TI, PC>;
  constexpr int kNlChunk = Ring::kChunk;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Ring ring{smem_raw};
  V* cfs = reinterpret_cast<V*>(smem_raw + kNlStages * Ring::kSlot);   // [kNlItems][2][nkb]
  __shared__ int ks[kNlItems];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.x * kNlItems + warp;
  int k, vin, vout;
  nl_item(a, item, k, vin, vout);
  if (lane == 0) ks[warp] = k;
  V* cw = cfs + (size_t)warp * 2 * a.nkb;
  if (k >= 0) {
    const V* cf = static_cast<const V*>(a.coef) + (size_t)item * 2 * a.nkb;
    for (int i = lane; i < 2 * a.nkb; i += 32) cw[i] = cf[i];
  }
  __syncthreads();
  const bool with_s = a.sout != nullptr;
  for (int w0 = 0; w0 < kNlItems; ++w0) {
    if (!first_of_k(ks, w0)) continue;
    const int kk = ks[w0];
    const int np = a.npw[kk];
    const int ntile = (np + kNlTile - 1) / kNlTile;
    const int nchunk = (a.nkb + kNlChunk - 1) / kNlChunk;
    const int nstep = ntile * nchunk;   // steps in the order (g tile, projector chunk)
    const V* bk = static_cast<const V*>(a.beta) + (size_t)kk * a.nkb * a.npw_max;
    const bool mine = k == kk;
    VI* pout = a.out != nullptr ? static_cast<VI*>(a.out) + ((size_t)kk * a.nvec_out + vout) * a.npw_max
                                : nullptr;   // null: S only
    VI* sout = with_s ? static_cast<VI*>(a.sout) + ((size_t)kk * a.nvec_out + vout) * a.npw_max : nullptr;
    const VI* pin = static_cast<const VI*>(a.in) + ((size_t)kk * a.nvec_in + vin) * a.npw_max;
    auto issue = [&](int st) {
      const int t = st / nchunk, c0 = (st - t * nchunk) * kNlChunk;
      ring.issue(st % kNlStages, bk, a.npw_max, c0, min(kNlChunk, a.nkb - c0), t * kNlTile, np, nullptr);
    };
#pragma unroll
    for (int st = 0; st < kNlStages - 1; ++st) {
      if (st < nstep) issue(st);
      else cp_async_commit();
    }
    V ah[kNlTile / 32], as[kNlTile / 32];
    VI hv[kNlTile / 32], cv[kNlTile / 32];
    for (int st = 0; st < nstep; ++st) {
      const int t = st / nchunk, c0 = (st - t * nchunk) * kNlChunk;
      const int nc = min(kNlChunk, a.nkb - c0);
      if (c0 == 0 && mine) {   // the output (and input) values of this tile, loaded early
#pragma unroll
        for (int u = 0; u < kNlTile / 32; ++u) {
          const int g = t * kNlTile + lane + 32 * u;
          ah[u] = as[u] = V{T(0), T(0)};
          hv[u] = (g < np && pout != nullptr) ? pout[g] : VI{TI(0), TI(0)};
          if (with_s) cv[u] = g < np ? pin[g] : VI{TI(0), TI(0)};
        }
      }
      cp_async_wait<kNlStages - 2>();
      __syncthreads();
      if (st + kNlStages - 1 < nstep) issue(st + kNlStages - 1);
      else cp_async_commit();
      if (mine) {
        const V* bt = ring.beta(st % kNlStages);
#pragma unroll
        for (int j = 0; j < kNlChunk; ++j) {
          if (j < nc) {
            const V gm = cw[c0 + j], dl = cw[a.nkb + c0 + j];
#pragma unroll
            for (int u = 0; u < kNlTile / 32; ++u) {
              const V b = bt[j * kNlTile + lane + 32 * u];
              ah[u].x += gm.x * b.x - gm.y * b.y;
              ah[u].y += gm.x * b.y + gm.y * b.x;
              if (with_s) {
                as[u].x += dl.x * b.x - dl.y * b.y;
                as[u].y += dl.x * b.y + dl.y * b.x;
              }
            }
          }
        }
        if (c0 + kNlChunk >= a.nkb) {   // last chunk of this g tile: write it
#pragma unroll
          for (int u = 0; u < kNlTile / 32; ++u) {
            const int g = t * kNlTile + lane + 32 * u;
            if (g < np) {
              if (pout != nullptr) pout[g] = VI{TI(T(hv[u].x) + ah[u].x), TI(T(hv[u].y) + ah[u].y)};
              if (with_s) sout[g] = VI{cv[u].x + TI(as[u].x), cv[u].y + TI(as[u].y)};
            }
          }
        }
      }
    }
    cp_async_wait<0>();
    __syncthreads();
    if (mine && with_s)
      for (int g = np + lane; g < a.npw_max; g += 32) sout[g] = VI{TI(0), TI(0)};
  }
}

template <typename T, typename TI, int PC>
size_t nl_smem(int nkb, bool addback) {
  return kNlStages * NlRing<T, TI, PC>::kSlot + (size_t)kNlItems * nkb * (addback ? 2 : 1) * sizeof(c2_t<T>);
}

template <typename T, typename TI, int PC>
int launch_nl_pc(const NlArgs& a, int nblocks, cudaStream_t st) {
  const size_t s1 = nl_smem<T, TI, PC>(a.nkb, false);
  const size_t s3 = nl_smem<T, TI, PC>(a.nkb, true);
  if (a.phase == 0) {
    if (cudaError_t e = allow_full_smem(nl_project_kernel<T, TI, PC>); e != cudaSuccess)
      return cuda_fail(e, "cudaFuncSetAttribute(nl_project)");
    nl_project_kernel<T, TI, PC><<<nblocks, kNlThreads, s1, st>>>(a); note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "nl_project_kernel");
  } else {
    if (cudaError_t e = allow_full_smem(nl_addback_kernel<T, TI, PC>); e != cudaSuccess)
      return cuda_fail(e, "cudaFuncSetAttribute(nl_addback)");
    nl_addback_kernel<T, TI, PC><<<nblocks, kNlThreads, s3, st>>>(a); note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "nl_addback_kernel");
  }
  return PWK_OK;
}

template <typename T>
constexpr int nl_max_pc() { return sizeof(T) == 4 ? 16 : 9; }

template <typename T, typename TI>
int launch_nl_typed(const NlArgs& a, cudaStream_t st) {
  const int nblocks = (a.nitems + kNlItems - 1) / kNlItems;
  if (nblocks == 0 || (a.nkb == 0 && (a.phase == 0 || a.sout == nullptr))) return PWK_OK;
  switch (nl_pick_pc(a.nkb, nl_max_pc<T>())) {
    case 16: return launch_nl_pc<T, TI, 16>(a, nblocks, st);
    case 12: return launch_nl_pc<T, TI, 12>(a, nblocks, st);
    case 9: return launch_nl_pc<T, TI, 9>(a, nblocks, st);
    case 8: return launch_nl_pc<T, TI, 8>(a, nblocks, st);
    default: return launch_nl_pc<T, TI, 4>(a, nblocks, st);
  }
}

template <typename T, typename TI>
size_t nl_smem_picked(int nkb) {
  switch (nl_pick_pc(nkb, nl_max_pc<T>())) {
    case 16: return nl_smem<T, TI, 16>(nkb, true);
    case 12: return nl_smem<T, TI, 12>(nkb, true);
    case 9: return nl_smem<T, TI, 9>(nkb, true);
    case 8: return nl_smem<T, TI, 8>(nkb, true);
    default: return nl_smem<T, TI, 4>(nkb, true);
  }
}

}  // namespace

size_t nl_shared_bytes(int nkb, int precision) {
  switch (precision) {
    case PWK_FP64: return nl_smem_picked<double, double>(nkb);
    case PWK_FP32: return nl_smem_picked<float, float>(nkb);
    default: return nl_smem_picked<float, double>(nkb);
  }
}

int launch_nl(int precision, const NlArgs& a, cudaStream_t st) {
  // both contractions on the tensor cores where they apply (the coefficient scratch has the
  // same layout on either path, so a phase may run on the tensor cores and the other not)
  if (a.tensor_cores && nl_tcw_applies(precision, a)) return launch_nl_tcw(precision, a, st);
  switch (precision) {
    case PWK_FP64: return launch_nl_typed<double, double>(a, st);
    case PWK_FP32: return launch_nl_typed<float, float>(a, st);
    default: return launch_nl_typed<float, double>(a, st);
  }
}

}  // namespace pwk
