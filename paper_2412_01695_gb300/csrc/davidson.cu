// Batched block-Davidson diagonalisation of H(k) for every k of a plan (paper Sec. 2.1 and
// Algorithm 2: the Davidson steps run for all N_k k-points at once).
//
// Per k the basis phi (up to max_basis vectors), H phi, the reduced matrices H~, S~ and the
// reduced eigenvectors live on the device.  Every step is a kernel over all active k:
//   resid   : residual of each Ritz vector, correction (H_diag - eps)^-1 (H - eps) phi and
//             its normalisation (Sec. 2.1, second and third steps)
//   select  : which bands still need a correction (|eps^(n+1) - eps^(n)| > eth, plus an
//             optional residual bound); a k with none left is done
//   restart : when the basis would exceed max_basis, phi <- phi v, H phi <- (H phi) v
//             (restart with the current Ritz vectors)
//   append  : new vectors at the end of the basis; H applied to them with the fused kernel
//   gram    : new rows/columns of H~ and S~ (FP64 dot products)
//   rr      : batched FP64 generalized eigensolve (rr.cu)
// The host only reads one counter per iteration (bands left) to decide whether to stop.
// A k-point whose reduced problem fails (S~ numerically singular in its leading block, or a
// non-finite eigenvector) drops the vectors of that step and restarts from its Ritz vectors; after
// more than three failures it is given up and its bands are reported unconverged.
// Mixed mode: each k-point applies H in FP32 until its bands stop moving by more than
// max(eth, 1e-4 Ry) (and ||r|| < max(res_tol, 1e-3)); then its Ritz vectors get FP64 H
// applications and it goes on in FP64 to eth (per k-point, independently of the others).  Reduced matrices, eigensolve, norms and residuals are FP64 always.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "fft_line.cuh"
#include "solvers.h"

namespace pwk {

struct DavWork {
  int nk = 0, nb = 0, MB = 0, npw_max = 0;   // nb, MB: the current call's
  int cap_nb = 0, cap_MB = 0;                // the allocated capacity
  bool has_s = false, has32 = false;         // S phi arrays, FP32 arrays allocated
  bool with_s = false;   // overlap S (plan with q): S phi kept beside H phi
  double2 *phi = nullptr, *hphi = nullptr, *corr = nullptr, *tmp1 = nullptr, *tmp2 = nullptr;
  double2 *sphi = nullptr, *tmp3 = nullptr;
  double* sdiag = nullptr;
  unsigned char* drop = nullptr;   // [nk][MB] basis vectors the last eigensolve left out
  int* lastrow = nullptr;          // [nk][nb] basis row of each band's latest correction
  // mixed mode: FP32 basis of the phase-1 k-points (same layouts as the FP64 arrays)
  bool mixed = false;
  float2 *phi32 = nullptr, *hphi32 = nullptr, *sphi32 = nullptr, *corr32 = nullptr;
  float2 *t32a = nullptr, *t32b = nullptr, *t32c = nullptr;
  float *hdiag32 = nullptr, *sdiag32 = nullptr;
  double2 *Hr = nullptr, *Sr = nullptr, *W = nullptr, *ev = nullptr;
  double *eps = nullptr, *eps_new = nullptr, *hdiag = nullptr, *rnorm = nullptr;
  int *nbase = nullptr, *nnc = nullptr, *todo = nullptr, *active = nullptr, *moved = nullptr;
  int *restart = nullptr, *items = nullptr, *iters = nullptr,
      *status = nullptr, *failcount = nullptr, *force = nullptr, *dbg = nullptr,
      *phase = nullptr, *switchk = nullptr, *iterk = nullptr, *counters = nullptr;
  std::vector<void*> ptrs;
};

void destroy_dav_work(pwk_plan* p) {
  if (p->dav == nullptr) return;
  for (void* q : p->dav->ptrs) plan_free(p, q);
  delete p->dav;
  p->dav = nullptr;
}

template <typename T>
static int dalloc(pwk_plan* p, DavWork* w, T** ptr, size_t n) {
  int rc = plan_alloc(p, (void**)ptr, n * sizeof(T));
  if (rc == PWK_OK) w->ptrs.push_back(*ptr);
  return rc;
}

// The workspace only grows: a call whose nb and MB fit the allocated capacity (and whose
// precision mode and overlap the allocated arrays cover) reuses it, so a plan that serves
// solves of different sizes allocates (and synchronises the device) only for the largest.
// The arrays are indexed with the call's nb and MB.
static int alloc_dav_work(pwk_plan* p, int nb, int MB, bool mixed, bool with_s);
static int ensure_dav_work(pwk_plan* p, int nb, int MB, bool mixed) {
  const bool with_s = p->d_q != nullptr;
  int cnb = nb, cMB = MB;
  bool cs = with_s, c32 = mixed;
  if (DavWork* w0 = p->dav) {
    if (!(w0->cap_nb >= nb && w0->cap_MB >= MB && (w0->has_s || !with_s) && (w0->has32 || !mixed))) {
      cnb = std::max(nb, w0->cap_nb);
      cMB = std::max(MB, w0->cap_MB);
      cs = with_s || w0->has_s;
      c32 = mixed || w0->has32;
      destroy_dav_work(p);
    }
  }
  if (p->dav == nullptr) {
    if (int rc = alloc_dav_work(p, cnb, cMB, c32, cs)) return rc;
  }
  DavWork* w = p->dav;
  w->nb = nb;
  w->MB = MB;
  w->with_s = with_s;
  w->mixed = mixed;
  return PWK_OK;
}

static int alloc_dav_work(pwk_plan* p, int nb, int MB, bool mixed, bool with_s) {
  DavWork* w = new DavWork();
  p->dav = w;
  w->nk = p->nk;
  w->cap_nb = nb;
  w->cap_MB = MB;
  w->npw_max = p->npw_max;
  w->has_s = with_s;
  w->has32 = mixed;
  const size_t nk = p->nk, np = p->npw_max;
  int rc;
  if (mixed && ((rc = dalloc(p, w, &w->phi32, nk * MB * np)) || (rc = dalloc(p, w, &w->hphi32, nk * MB * np)) ||
                (rc = dalloc(p, w, &w->corr32, nk * nb * np)) || (rc = dalloc(p, w, &w->t32a, nk * nb * np)) ||
                (rc = dalloc(p, w, &w->t32b, nk * nb * np)) || (rc = dalloc(p, w, &w->hdiag32, nk * np)))) {
    destroy_dav_work(p);
    return rc;
  }
  if (mixed && with_s && ((rc = dalloc(p, w, &w->sphi32, nk * MB * np)) || (rc = dalloc(p, w, &w->t32c, nk * nb * np)) ||
                          (rc = dalloc(p, w, &w->sdiag32, nk * np)))) {
    destroy_dav_work(p);
    return rc;
  }
  if (with_s && ((rc = dalloc(p, w, &w->sphi, nk * MB * np)) || (rc = dalloc(p, w, &w->tmp3, nk * nb * np)) ||
                 (rc = dalloc(p, w, &w->sdiag, nk * np)))) {
    destroy_dav_work(p);
    return rc;
  }
  if ((rc = dalloc(p, w, &w->phi, nk * MB * np)) || (rc = dalloc(p, w, &w->hphi, nk * MB * np)) ||
      (rc = dalloc(p, w, &w->corr, nk * nb * np)) || (rc = dalloc(p, w, &w->tmp1, nk * nb * np)) ||
      (rc = dalloc(p, w, &w->tmp2, nk * nb * np)) || (rc = dalloc(p, w, &w->Hr, nk * MB * MB)) ||
      (rc = dalloc(p, w, &w->Sr, nk * MB * MB)) || (rc = dalloc(p, w, &w->W, nk * 3 * MB * MB)) ||
      (rc = dalloc(p, w, &w->ev, nk * MB * nb)) || (rc = dalloc(p, w, &w->eps, nk * nb)) ||
      (rc = dalloc(p, w, &w->eps_new, nk * nb)) || (rc = dalloc(p, w, &w->hdiag, nk * np)) ||
      (rc = dalloc(p, w, &w->rnorm, nk * nb)) || (rc = dalloc(p, w, &w->nbase, nk)) ||
      (rc = dalloc(p, w, &w->nnc, nk)) || (rc = dalloc(p, w, &w->todo, nk * nb)) ||
      (rc = dalloc(p, w, &w->active, nk)) || (rc = dalloc(p, w, &w->moved, nk * nb)) ||
      (rc = dalloc(p, w, &w->restart, nk)) || (rc = dalloc(p, w, &w->items, nk * nb * 3)) ||
      (rc = dalloc(p, w, &w->iters, nk)) ||
      (rc = dalloc(p, w, &w->status, nk)) || (rc = dalloc(p, w, &w->failcount, nk)) ||
      (rc = dalloc(p, w, &w->force, nk)) || (rc = dalloc(p, w, &w->dbg, 4)) ||
      (rc = dalloc(p, w, &w->phase, nk)) || (rc = dalloc(p, w, &w->switchk, nk)) ||
      (rc = dalloc(p, w, &w->iterk, nk)) || (rc = dalloc(p, w, &w->counters, 8)) ||
      (rc = dalloc(p, w, &w->drop, nk * MB)) || (rc = dalloc(p, w, &w->lastrow, nk * nb))) {
    destroy_dav_work(p);
    return rc;
  }
  return PWK_OK;
}

// ------------------------------------------------------------------ kernels
template <typename V>
__device__ __forceinline__ V cmul_(V a, V b) {
  return V{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename V>
__device__ __forceinline__ V cmulc_(V a, V b) {  // conj(a) b
  return V{a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}
// true when k-point k takes part in a launch restricted to phase `want` (0: any phase)
__device__ __forceinline__ bool in_phase(const int* phase, int want, int k) {
  return want == 0 || phase[k] == want;
}

template <typename T>
__device__ T bsum(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  T s = T(0);
  for (int i = 0; i < nw; ++i) s += red[i];
  __syncthreads();
  return s;
}

// H_diag(G) = |k+G|^2 + <V> + sum_mn beta_m(G) D_mn conj(beta_n(G))   (diagonal of H in PWs)
// S_diag(G) = 1 + sum_mn beta_m(G) q_mn conj(beta_n(G))   (when q is given; Sec. 2.1)
__global__ void hdiag_kernel(int nk, int np, int nkb, const int* npw, const double* g2,
                             double vmean, const double2* beta, const double* D, double* hd,
                             const double* q, double* sd) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)nk * np) return;
  const int k = (int)(i / np), g = (int)(i % np);
  if (g >= npw[k]) {
    hd[i] = 0.0;
    if (sd != nullptr) sd[i] = 1.0;
    return;
  }
  double s = g2[i] + vmean, so = 1.0;
  const double2* b = beta + (size_t)k * nkb * np + g;
  for (int m = 0; m < nkb; ++m) {
    const double2 bm = b[(size_t)m * np];
    for (int n = 0; n < nkb; ++n) {
      const double dmn = D[m * nkb + n];
      const double qmn = q != nullptr ? q[m * nkb + n] : 0.0;
      if (dmn == 0.0 && qmn == 0.0) continue;
      const double2 bn = b[(size_t)n * np];
      const double re = bm.x * bn.x + bm.y * bn.y;   // Re(beta_m conj(beta_n))
      s += dmn * re;
      so += qmn * re;
    }
  }
  hd[i] = s;
  if (sd != nullptr) sd[i] = so;
}

// copy nv vectors per k between arrays with different per-k strides (and precisions)
template <typename TS, typename TD>
__global__ void copy_vecs_kernel(int nk, int nv, int np, const c2_t<TS>* src, int src_nvec,
                                 int src_off, c2_t<TD>* dst, int dst_nvec, int dst_off,
                                 const int* only, const int* phase, int want) {
  const int k = blockIdx.x / nv, j = blockIdx.x % nv;
  if ((only != nullptr && !only[k]) || !in_phase(phase, want, k)) return;
  const c2_t<TS>* s = src + ((size_t)k * src_nvec + src_off + j) * np;
  c2_t<TD>* d = dst + ((size_t)k * dst_nvec + dst_off + j) * np;
  for (int g = threadIdx.x; g < np; g += blockDim.x) d[g] = c2_t<TD>{TD(s[g].x), TD(s[g].y)};
}

// work list: (k, base[k] + t) for t < cnt[k] on k with mask[k] (and phase[k] == want_phase
// when want_phase > 0), else empty slots (k = -1)
__global__ void items_kernel(int nk, int nb, const int* active, const int* base, int base_const,
                             const int* cnt, int cnt_const, const int* phase, int want_phase,
                             int* items) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nk * nb) return;
  const int k = i / nb, t = i % nb;
  const int b = base ? base[k] : base_const;
  const int c = cnt ? cnt[k] : cnt_const;
  const bool on = active[k] && t < c && (want_phase <= 0 || phase[k] == want_phase);
  items[3 * i] = on ? k : -1;
  items[3 * i + 1] = on ? b + t : 0;
  items[3 * i + 2] = on ? b + t : 0;
}

// Compensated FP32 accumulation of products (hi + lo): a*b is split exactly into its rounded
// value and the FMA residual, and the running sum by a two-sum, so the pair carries about
// twice the FP32 precision.
struct CompSum {
  float hi = 0.f, lo = 0.f;
  // (round-to-nearest intrinsics: the compiler may not contract or reorder these steps)
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = fmaf(a, b, -p);   // exact: a * b = p + pe
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));   // hi + p = s + e
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// New columns b = base + t (t < cnt) of H~ and S~: rows a < base + cnt.  Each (a, b) is
// written by one CTA (rows a >= base only for a <= b) together with its mirror (b, a).
// S~_ab = <phi_a|S phi_b> with sphi = S phi (sphi = phi when S = 1).  T is the precision of
// the stored vectors and of the sums (FP32 for phase-1 k-points of the mixed mode); the
// reduced matrices are FP64.
template <typename T>
__global__ void __launch_bounds__(256) gram_kernel(int nb, int MB, int np, const int* npw,
                                                   const int* active, const int* base,
                                                   int base_const, const int* cnt, int cnt_const,
                                                   const c2_t<T>* phi, const c2_t<T>* hphi,
                                                   const c2_t<T>* sphi, double2* Hr, double2* Sr,
                                                   const int* phase, int want) {
  using V = c2_t<T>;
  const int k = blockIdx.x / nb, t = blockIdx.x % nb;
  if (!active[k] || !in_phase(phase, want, k)) return;
  const int b0 = base ? base[k] : base_const, c = cnt ? cnt[k] : cnt_const;
  if (t >= c) return;
  const int b = b0 + t, nrow = b0 + c, n = npw[k];
  extern __shared__ __align__(16) unsigned char gsh[];
  V* pb = reinterpret_cast<V*>(gsh);
  V* hb = pb + np;
  const V* P = phi + (size_t)k * MB * np;
  const V* HP = hphi + (size_t)k * MB * np;
  const V* SP = sphi + (size_t)k * MB * np;
  for (int g = threadIdx.x; g < n; g += blockDim.x) {
    pb[g] = SP[(size_t)b * np + g];
    hb[g] = HP[(size_t)b * np + g];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double2* H = Hr + (size_t)k * MB * MB;
  double2* S = Sr + (size_t)k * MB * MB;
  for (int a = warp; a < nrow; a += nw) {
    if (a >= b0 && a > b) continue;
    const V* pa = P + (size_t)a * np;
    double hx = 0, hy = 0, sx = 0, sy = 0;
    if constexpr (sizeof(T) == 8) {
      for (int g = lane; g < n; g += 32) {
        const V x = pa[g];
        const V h = cmulc_(x, hb[g]);
        const V s = cmulc_(x, pb[g]);
        hx += h.x;
        hy += h.y;
        sx += s.x;
        sy += s.y;
      }
    } else {
      // FP32 vectors: products and sums carried as unevaluated pairs hi + lo (error-free
      // product by FMA, two-sum), so S~ and H~ are those of the stored vectors to about
      // 1e-14 while the arithmetic stays on the FP32 pipe
      CompSum ah, bh, as, bs;
      for (int g = lane; g < n; g += 32) {
        const V x = pa[g], y = hb[g], z = pb[g];
        ah.add_prod(x.x, y.x);
        ah.add_prod(x.y, y.y);   // Re conj(x) y
        bh.add_prod(x.x, y.y);
        bh.add_prod(-x.y, y.x);  // Im conj(x) y
        as.add_prod(x.x, z.x);
        as.add_prod(x.y, z.y);
        bs.add_prod(x.x, z.y);
        bs.add_prod(-x.y, z.x);
      }
      hx = ah.value();
      hy = bh.value();
      sx = as.value();
      sy = bs.value();
    }
    for (int o = 16; o > 0; o >>= 1) {
      hx += __shfl_xor_sync(0xffffffffu, hx, o);
      hy += __shfl_xor_sync(0xffffffffu, hy, o);
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) {
      if (a == b) {
        H[a * MB + b] = make_double2(hx, 0.0);
        S[a * MB + b] = make_double2(sx, 0.0);
      } else {
        H[a * MB + b] = make_double2(hx, hy);
        H[b * MB + a] = make_double2(hx, -hy);
        S[a * MB + b] = make_double2(sx, sy);
        S[b * MB + a] = make_double2(sx, -sy);
      }
    }
  }
}

// out[k][j] = sum_{i < nbase} ev[k][i][j] in[k][i]   (j < nb), for k with only[k] != 0;
// arithmetic in the input precision TI, output converted to TO
template <typename TI, typename TO>
__global__ void __launch_bounds__(256) rotate_kernel(int nb, int MB, int np, const int* nbase,
                                                     const int* only, const double2* ev,
                                                     const c2_t<TI>* in, c2_t<TO>* out,
                                                     int out_nvec, const int* phase, int want) {
  using V = c2_t<TI>;
  const int k = blockIdx.x / nb, j = blockIdx.x % nb;
  if ((only != nullptr && !only[k]) || !in_phase(phase, want, k)) return;
  const int n = nbase[k];
  __shared__ V c[kMaxBasis];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 e = ev[((size_t)k * MB + i) * nb + j];
    c[i] = V{TI(e.x), TI(e.y)};
  }
  __syncthreads();
  const V* X = in + (size_t)k * MB * np;
  c2_t<TO>* o = out + ((size_t)k * out_nvec + j) * np;
  for (int g = threadIdx.x; g < np; g += blockDim.x) {
    TI sx = 0, sy = 0;
    for (int i = 0; i < n; ++i) {
      const V t = cmul_(c[i], X[(size_t)i * np + g]);
      sx += t.x;
      sy += t.y;
    }
    o[g] = c2_t<TO>{TO(sx), TO(sy)};
  }
}

// Correction vector of band i (Sec. 2.1): r = sum_j v_ji (H phi_j - eps_i S phi_j),
// c = r / clamp(H_diag - eps_i S_diag), c /= ||c||.  ||r|| is stored for the residual test.
// The unpreconditioned r (orthogonal to the whole basis by the Galerkin condition, so a new
// direction whenever it is not zero) is used instead when c is numerically parallel to the
// Ritz vector (|cos| > 1 - 1e-6: H diagonal in plane waves, exact preconditioner) or when the
// band's previous correction was left out of the reduced problem as dependent on the basis.
// sphi = phi and sdiag = null when S = 1.  T: precision of the vectors and the arithmetic.
template <typename T>
__global__ void __launch_bounds__(256) resid_kernel(int nb, int MB, int np, const int* npw,
                                                    const int* nbase, const int* active,
                                                    const int* moved, int all_bands,
                                                    const double2* ev, const double* eps,
                                                    const c2_t<T>* phi, const c2_t<T>* hphi,
                                                    const c2_t<T>* sphi, const T* hdiag,
                                                    const T* sdiag, const unsigned char* drop,
                                                    const int* lastrow, c2_t<T>* corr,
                                                    double* rnorm, const int* phase, int want) {
  using V = c2_t<T>;
  const int k = blockIdx.x / nb, i = blockIdx.x % nb;
  if (!active[k] || !in_phase(phase, want, k)) return;
  if (!all_bands && !moved[k * nb + i]) return;
  const int n = nbase[k], npk = npw[k];
  __shared__ V c[kMaxBasis];
  __shared__ T red[32];
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double2 e = ev[((size_t)k * MB + j) * nb + i];
    c[j] = V{T(e.x), T(e.y)};
  }
  __syncthreads();
  const T e = T(eps[k * nb + i]);
  const V* P = phi + (size_t)k * MB * np;
  const V* HP = hphi + (size_t)k * MB * np;
  const V* SP = sphi + (size_t)k * MB * np;
  V* out = corr + ((size_t)k * nb + i) * np;
  const T* hd = hdiag + (size_t)k * np;
  const T* sdk = sdiag != nullptr ? sdiag + (size_t)k * np : nullptr;
  T rr = 0, cc = 0, zz = 0, zcx = 0, zcy = 0;
  for (int g = threadIdx.x; g < npk; g += blockDim.x) {
    T rx = 0, ry = 0, zx = 0, zy = 0;
    for (int j = 0; j < n; ++j) {
      const V hp = HP[(size_t)j * np + g], p = P[(size_t)j * np + g], sp = SP[(size_t)j * np + g];
      const V d = V{hp.x - e * sp.x, hp.y - e * sp.y};
      const V t = cmul_(c[j], d);
      const V z = cmul_(c[j], p);
      rx += t.x;
      ry += t.y;
      zx += z.x;
      zy += z.y;
    }
    rr += rx * rx + ry * ry;
    T x = hd[g] - e * (sdk != nullptr ? sdk[g] : T(1));
    const T s = x >= T(0) ? T(1) : T(-1);
    x = s * fmax(fabs(x), T(1e-2));
    const V v = V{rx / x, ry / x};
    cc += v.x * v.x + v.y * v.y;
    zz += zx * zx + zy * zy;
    zcx += zx * v.x + zy * v.y;   // <ritz|v>
    zcy += zx * v.y - zy * v.x;
    out[g] = V{rx, ry};
  }
  rr = bsum(rr, red);
  cc = bsum(cc, red);
  zz = bsum(zz, red);
  zcx = bsum(zcx, red);
  zcy = bsum(zcy, red);
  const int lr = lastrow[k * nb + i];
  const bool was_dropped = lr >= 0 && lr < n && drop[(size_t)k * MB + lr] != 0;
  const bool parallel = was_dropped || (zcx * zcx + zcy * zcy) > T(1.0 - 1e-6) * T(1.0 - 1e-6) * zz * cc;
  const T nrm2 = parallel ? rr : cc;
  const T inv = nrm2 > T(0) ? T(1) / sqrt(nrm2) : T(0);
  for (int g = threadIdx.x; g < np; g += blockDim.x) {
    if (g < npk) {
      const V r = out[g];
      T sc = inv;
      if (!parallel) {
        T x = hd[g] - e * (sdk != nullptr ? sdk[g] : T(1));
        const T s = x >= T(0) ? T(1) : T(-1);
        sc = inv / (s * fmax(fabs(x), T(1e-2)));
      }
      out[g] = V{r.x * sc, r.y * sc};
    } else {
      out[g] = V{T(0), T(0)};
    }
  }
  if (threadIdx.x == 0) rnorm[k * nb + i] = sqrt((double)rr);
}

// Which bands still need a correction, per k-point and its phase (1: FP32 H, 2: FP64 H).
// counters[0] += bands to correct this step, counters[5] += those of phase-2 k-points,
// counters[6] += k-points that take a correction step,
// counters[4] += k-points switching from phase 1 to phase 2 this step (their FP32 floor is
// reached or their phase-1 iterations are used up), counters[1] += bands of k-points given up
// after repeated reduced-problem failures (counters[2], [3]: the first such k and its status).
__global__ void select_kernel(int nk, int nb, int MB, double rt1, double rt2, int cap1, int* active,
                              const int* phase, const int* moved, const double* rnorm,
                              const int* nbase, int* todo, int* nnc, int* restart, int* iters,
                              const int* status, int* force, const int* failcount, int* switchk,
                              int* iterk, int* counters) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk) return;
  switchk[k] = 0;
  iterk[k] = 0;
  if (active[k] && failcount[k] > 3) {   // give this k-point up: its bands stay unconverged
    active[k] = 0;
    nnc[k] = nb;
    restart[k] = 0;
    atomicAdd(&counters[1], nb);
    if (atomicCAS(&counters[2], -1, k) == -1) counters[3] = status[k];
    return;
  }
  if (!active[k]) {
    nnc[k] = 0;
    restart[k] = 0;
    return;
  }
  const double rt = phase[k] == 1 ? rt1 : rt2;
  int c = 0;
  for (int i = 0; i < nb; ++i) {
    const bool conv = !moved[k * nb + i] && (rt <= 0.0 || rnorm[k * nb + i] <= rt);
    if (!conv) todo[k * nb + c++] = i;
  }
  if (phase[k] == 1 && (c == 0 || iters[k] >= cap1)) {
    switchk[k] = 1;
    nnc[k] = 0;
    restart[k] = 0;
    atomicAdd(&counters[4], 1);
    return;
  }
  nnc[k] = c;
  restart[k] = (c > 0 && (nbase[k] + c > MB || force[k])) ? 1 : 0;
  force[k] = 0;
  if (c == 0) {
    active[k] = 0;
  } else {
    iters[k] += 1;
    iterk[k] = 1;
    atomicAdd(&counters[6], 1);
  }
  atomicAdd(&counters[0], c);
  if (phase[k] == 2) atomicAdd(&counters[5], c);
}

__global__ void set_value_kernel(int nk, const int* mask, int* a, int v) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nk && mask[k]) a[k] = v;
}

template <typename T>
__global__ void append_kernel(int nb, int MB, int np, const int* active, const int* nbase,
                              const int* nnc, const int* todo, const c2_t<T>* corr, c2_t<T>* phi,
                              int* lastrow, const int* phase, int want) {
  const int k = blockIdx.x / nb, t = blockIdx.x % nb;
  if (!active[k] || t >= nnc[k] || !in_phase(phase, want, k)) return;
  const int i = todo[k * nb + t];
  if (threadIdx.x == 0) lastrow[k * nb + i] = nbase[k] + t;
  const c2_t<T>* s = corr + ((size_t)k * nb + i) * np;
  c2_t<T>* d = phi + ((size_t)k * MB + nbase[k] + t) * np;
  for (int g = threadIdx.x; g < np; g += blockDim.x) d[g] = s[g];
}

// FP32 copies of the plane-wave diagonals of H and S for the phase-1 arithmetic
__global__ void to_float_kernel(size_t n, const double* a, float* b) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

__global__ void set_nbase_kernel(int nk, const int* only, int* nbase, int value, const int* add) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk || (only && !only[k])) return;
  nbase[k] = add ? nbase[k] + add[k] : value;
}

// After the eigensolve: moved = |eps_new - eps| > eth, eps = eps_new.  A k-point whose
// reduced problem failed (status != 0: the eigensolver wrote nothing) drops the vectors of
// this step (n_base -= added[k]), keeps its previous Ritz pairs, corrects every band again and
// restarts from its Ritz vectors at the next step; after more than three failures it is
// given up (reported as an error by the next select).
__global__ void update_kernel(int nk, int nb, double eth1, double eth2, const int* phase,
                              const int* mask, int force_all, const double* eps_new, double* eps,
                              int* moved, const int* status, const int* added, int* nbase,
                              int* force, int* failcount, int* dbg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nk * nb) return;
  const int k = i / nb;
  if (!mask[k]) return;
  const double eth = phase[k] == 1 ? eth1 : eth2;
  if (status[k] != 0) {
    moved[i] = 1;
    if (i % nb == 0) {
      if (atomicAdd(&dbg[0], 1) == 0) {   // first failure of the call: k, size, status
        dbg[1] = k;
        dbg[2] = nbase[k];
        dbg[3] = status[k];
      }
      if (added != nullptr) nbase[k] -= added[k];
      force[k] = 1;
      failcount[k] += 1;
    }
    return;
  }
  moved[i] = force_all ? 1 : (fabs(eps_new[i] - eps[i]) > eth);
  eps[i] = eps_new[i];
}

// phase switch: every k-point that has not been given up takes part again
__global__ void reactivate_kernel(int nk, int* active, const int* failcount) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nk) active[k] = failcount[k] <= 3 ? 1 : 0;
}

__global__ void fill_int_kernel(int n, int* a, int v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

static int blocks(size_t n, int t = 256) { return (int)((n + t - 1) / t); }

// Diagnostic: when the environment variable PWK_DUMP_RR names a directory, the reduced
// H~ and S~ (leading n x n block, complex128, row-major) of the first k-point whose reduced
// problem failed in a call are written there as rr_H_k<k>.bin and rr_S_k<k>.bin.
static void dump_reduced(const DavWork* w, int k, int n) {
  const char* dir = std::getenv("PWK_DUMP_RR");
  if (dir == nullptr || k < 0 || n <= 0 || n > w->MB) return;
  std::vector<double2> h((size_t)w->MB * w->MB), s((size_t)w->MB * w->MB);
  const size_t off = (size_t)k * w->MB * w->MB;
  if (cudaMemcpy(h.data(), w->Hr + off, h.size() * sizeof(double2), cudaMemcpyDeviceToHost) ||
      cudaMemcpy(s.data(), w->Sr + off, s.size() * sizeof(double2), cudaMemcpyDeviceToHost))
    return;
  for (int which = 0; which < 2; ++which) {
    char path[512];
    std::snprintf(path, sizeof(path), "%s/rr_%s_k%d.bin", dir, which ? "S" : "H", k);
    FILE* f = std::fopen(path, "wb");
    if (!f) continue;
    const std::vector<double2>& m = which ? s : h;
    for (int r = 0; r < n; ++r) std::fwrite(m.data() + (size_t)r * w->MB, sizeof(double2), n, f);
    std::fclose(f);
  }
}

// Diagnostic: when PWK_TRACE_RR names a directory, the reduced H~, S~ of k-point 0 at every
// eigensolve of a call are written there as trace_<step>_H.bin / trace_<step>_S.bin, with the
// eigenvalues the solver returned (trace_<step>_eps.bin, nb float64) and its status.
static void trace_reduced(const DavWork* w, int step) {
  const char* dir = std::getenv("PWK_TRACE_RR");
  if (dir == nullptr) return;
  int n = 0, status = 0;
  if (cudaMemcpy(&n, w->nbase, sizeof(int), cudaMemcpyDeviceToHost) ||
      cudaMemcpy(&status, w->status, sizeof(int), cudaMemcpyDeviceToHost) || n <= 0 || n > w->MB)
    return;
  std::vector<double2> h((size_t)w->MB * w->MB), s((size_t)w->MB * w->MB);
  std::vector<double> e(w->nb);
  if (cudaMemcpy(h.data(), w->Hr, h.size() * sizeof(double2), cudaMemcpyDeviceToHost) ||
      cudaMemcpy(s.data(), w->Sr, s.size() * sizeof(double2), cudaMemcpyDeviceToHost) ||
      cudaMemcpy(e.data(), w->eps_new, e.size() * sizeof(double), cudaMemcpyDeviceToHost))
    return;
  char path[512];
  for (int which = 0; which < 2; ++which) {
    std::snprintf(path, sizeof(path), "%s/trace_%03d_%s.bin", dir, step, which ? "S" : "H");
    FILE* f = std::fopen(path, "wb");
    if (!f) continue;
    const std::vector<double2>& m = which ? s : h;
    for (int r = 0; r < n; ++r) std::fwrite(m.data() + (size_t)r * w->MB, sizeof(double2), n, f);
    std::fclose(f);
  }
  std::snprintf(path, sizeof(path), "%s/trace_%03d_eps.bin", dir, step);
  if (FILE* f = std::fopen(path, "wb")) {
    std::fwrite(e.data(), sizeof(double), e.size(), f);
    std::fwrite(&status, sizeof(int), 1, f);
    std::fclose(f);
  }
}

#define KCHECK(what)                                 \
  do {                                               \
    cudaError_t e_ = cudaGetLastError();             \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

}  // namespace pwk

using namespace pwk;

extern "C" int pwk_davidson_batched(pwk_plan* p, int mode, void* psi_v, double* eig, int nb,
                                    double eth, double res_tol, int max_iter, int max_basis,
                                    int* iters_out, int* notconv_out, long long* napply_out,
                                    void* stream) {
  if (p == nullptr || psi_v == nullptr || eig == nullptr || nb < 1 || !(eth > 0.0) || max_iter < 1) {
    set_error("null pointer, nb < 1, eth <= 0 or max_iter < 1");
    return PWK_ERR_INVALID;
  }
  if (mode != PWK_FP64 && mode != PWK_FP32_C128) {
    set_error("mode must be PWK_FP64 or PWK_FP32_C128");
    return PWK_ERR_INVALID;
  }
  int MB = max_basis > 0 ? max_basis : std::min(4 * nb, kMaxBasis);
  if (MB < 2 * nb || MB > kMaxBasis) {
    set_error("need 2*nb <= max_basis <= 160");
    return PWK_ERR_UNSUPPORTED;
  }
  for (int k = 0; k < p->nk; ++k)
    if (p->h_npw[k] < MB) {
      set_error("max_basis exceeds the number of plane waves of a k-point");
      return PWK_ERR_INVALID;
    }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = ensure_dav_work(p, nb, MB, mode == PWK_FP32_C128);
  if (rc) return rc;
  DavWork* w = p->dav;
  const int nk = p->nk, np = p->npw_max;
  double2* psi = static_cast<double2*>(psi_v);
  const size_t gram_smem = 2 * (size_t)np * sizeof(double2);
  if (gram_smem > 227 * 1024) {
    set_error("npw_max too large for the Gram kernel (2 vectors in shared memory)");
    return PWK_ERR_UNSUPPORTED;
  }
  if (cudaError_t e = allow_full_smem(gram_kernel<double>); e != cudaSuccess)
    return cuda_fail(e, "cudaFuncSetAttribute(gram)");
  if (cudaError_t e = allow_full_smem(gram_kernel<float>); e != cudaSuccess)
    return cuda_fail(e, "cudaFuncSetAttribute(gram)");
  long long napply[2] = {0, 0};
  int total = 0, given_up = 0, host_dbg[4] = {0, 0, 0, 0};
  bool dumped = false;
  const bool mixed = w->mixed;
  // phase filters of the FP64 launches: every k in FP64 mode, the phase-2 k in mixed mode
  const int want64 = mixed ? 2 : 0;

  PhaseTimer T(p, st);                                       // pwk_plan_set_solver_timing
  double* const rr_flops = T.on ? p->d_flops : nullptr;
  double2* const sphi = w->with_s ? w->sphi : w->phi;       // S phi (S = 1: phi itself)
  float2* const sphi32 = w->with_s ? w->sphi32 : w->phi32;
  hdiag_kernel<<<blocks((size_t)nk * np), 256, 0, st>>>(nk, np, p->nkb, p->d_npw, p->d_g2, p->v_mean,
                                                        p->d_beta, p->d_D, w->hdiag, p->d_q,
                                                        w->with_s ? w->sdiag : nullptr); note_launch();
  if (mixed) {
    to_float_kernel<<<blocks((size_t)nk * np), 256, 0, st>>>((size_t)nk * np, w->hdiag, w->hdiag32); note_launch();
    if (w->with_s) { to_float_kernel<<<blocks((size_t)nk * np), 256, 0, st>>>((size_t)nk * np, w->sdiag, w->sdiag32); note_launch(); }
  }
  KCHECK("hdiag_kernel");
  fill_int_kernel<<<blocks(nk), 256, 0, st>>>(nk, w->active, 1); note_launch();
  fill_int_kernel<<<blocks(nk), 256, 0, st>>>(nk, w->iters, 0); note_launch();
  fill_int_kernel<<<blocks(nk), 256, 0, st>>>(nk, w->status, 0); note_launch();
  fill_int_kernel<<<blocks(nk), 256, 0, st>>>(nk, w->restart, 0); note_launch();
  fill_int_kernel<<<blocks(nk), 256, 0, st>>>(nk, w->force, 0); note_launch();
  fill_int_kernel<<<blocks(nk), 256, 0, st>>>(nk, w->failcount, 0); note_launch();
  fill_int_kernel<<<1, 32, 0, st>>>(4, w->dbg, 0); note_launch();
  fill_int_kernel<<<blocks((size_t)nk * nb), 256, 0, st>>>(nk * nb, w->lastrow, -1); note_launch();
  if (mixed)
    { copy_vecs_kernel<double, float><<<nk * nb, 256, 0, st>>>(nk, nb, np, psi, nb, 0, w->phi32, MB, 0, nullptr,
                                                             nullptr, 0); note_launch(); }
  else
    { copy_vecs_kernel<double, double><<<nk * nb, 256, 0, st>>>(nk, nb, np, psi, nb, 0, w->phi, MB, 0, nullptr,
                                                              nullptr, 0); note_launch(); }
  KCHECK("davidson init");

  // Phase 1 (mixed mode) stops at the FP32 noise floor: eigenvalues of the reduced problem
  // built from FP32 H applications move by ~1e-6 |H| between iterations and residuals bottom
  // out near 1e-5, so a k-point leaves phase 1 when its bands stop moving by 1e-4 Ry with
  // ||r|| < 1e-3, or after min(max_iter/2, 60) correction steps; it then restarts from its Ritz
  // vectors with FP64 H applications (phase 2) and goes on to eth and res_tol.  Each k-point
  // switches on its own: the others keep iterating in their phase.  Phase-1 k-points keep
  // their basis, H basis and corrections in FP32 and do the vector arithmetic (corrections,
  // reduced-matrix columns, rotations) in FP32; the reduced matrices and their eigensolve
  // are FP64 in both phases.
  const double eth1 = mode == PWK_FP32_C128 ? std::max(eth, 1e-4) : eth;
  const double rt1 = mode == PWK_FP32_C128 && res_tol > 0 ? std::max(res_tol, 1e-3) : res_tol;
  // a k-point still short of the FP32 floor after 60 correction steps (a slow band next to a
  // small gap) finishes in FP64 instead of spending the rest of max_iter in FP32
  const int cap1 = std::max(1, std::min(max_iter / 2, 60));
  fill_int_kernel<<<blocks(nk), 256, 0, st>>>(nk, w->phase, mixed ? 1 : 2); note_launch();
  fill_int_kernel<<<blocks(nk), 256, 0, st>>>(nk, w->switchk, 0); note_launch();
  fill_int_kernel<<<blocks(nk), 256, 0, st>>>(nk, w->iterk, 0); note_launch();

  // new columns of H~, S~ for the k-points in mask, in the precision of their phase
  auto gram = [&](const int* mask, const int* base, int base_const, const int* cnt, int cnt_const) {
    if (mixed)
      { gram_kernel<float><<<nk * nb, 256, gram_smem / 2, st>>>(nb, MB, np, p->d_npw, mask, base, base_const, cnt,
                                                             cnt_const, w->phi32, w->hphi32, sphi32, w->Hr,
                                                             w->Sr, w->phase, 1); note_launch(); }
    gram_kernel<double><<<nk * nb, 256, gram_smem, st>>>(nb, MB, np, p->d_npw, mask, base, base_const, cnt,
                                                         cnt_const, w->phi, w->hphi, sphi, w->Hr, w->Sr,
                                                         w->phase, want64); note_launch();
  };

  // H on phi[0:nb] of the k-points in mask (all in phase ph), their nb x nb reduced matrices
  // and eigensolve
  auto start_block = [&](int ph, int* mask, int count) -> int {
    items_kernel<<<blocks((size_t)nk * nb), 256, 0, st>>>(nk, nb, mask, nullptr, 0, nullptr, nb,
                                                          w->phase, 0, w->items); note_launch();
    KCHECK("items_kernel");
    cudaEvent_t th = T.mark();
    int r = ph == 1 ? run_hpsi(p, PWK_FP32, w->phi32, w->hphi32, w->items, nullptr, nk * nb, MB, MB, st,
                               w->with_s ? w->sphi32 : nullptr)
                    : run_hpsi(p, PWK_FP64, w->phi, w->hphi, w->items, nullptr, nk * nb, MB, MB, st,
                               w->with_s ? w->sphi : nullptr);
    if (r) return r;
    T.close(0, th);
    napply[ph == 2 ? 0 : 1] += (long long)count * nb;
    gram(mask, nullptr, 0, nullptr, nb);
    KCHECK("gram_kernel");
    set_nbase_kernel<<<blocks(nk), 256, 0, st>>>(nk, mask, w->nbase, nb, nullptr); note_launch();
    cudaEvent_t tr = T.mark();
    r = launch_rr(nk, MB, nb, w->nbase, mask, w->Hr, w->Sr, w->W, w->ev, w->eps_new, w->status, st,
                  w->drop, rr_flops);
    T.close(1, tr);
    return r;
  };

  if ((rc = start_block(mixed ? 1 : 2, w->active, nk))) return rc;
  update_kernel<<<blocks((size_t)nk * nb), 256, 0, st>>>(nk, nb, eth1, eth, w->phase, w->active, 1,
                                                         w->eps_new, w->eps, w->moved, w->status,
                                                         nullptr, w->nbase, w->force, w->failcount,
                                                         w->dbg); note_launch();
  KCHECK("update_kernel");

  int it = 0;
  int hc[8];
  const int allb = (rt1 > 0 || res_tol > 0) ? 1 : 0;
  for (;;) {
    if (mixed)
      { resid_kernel<float><<<nk * nb, 256, 0, st>>>(nb, MB, np, p->d_npw, w->nbase, w->active, w->moved, allb,
                                                   w->ev, w->eps, w->phi32, w->hphi32, sphi32, w->hdiag32,
                                                   w->with_s ? w->sdiag32 : nullptr, w->drop, w->lastrow,
                                                   w->corr32, w->rnorm, w->phase, 1); note_launch(); }
    resid_kernel<double><<<nk * nb, 256, 0, st>>>(nb, MB, np, p->d_npw, w->nbase, w->active, w->moved, allb,
                                                  w->ev, w->eps, w->phi, w->hphi, sphi, w->hdiag,
                                                  w->with_s ? w->sdiag : nullptr, w->drop, w->lastrow,
                                                  w->corr, w->rnorm, w->phase, want64); note_launch();
    KCHECK("resid_kernel");
    cudaMemsetAsync(w->counters, 0, 8 * sizeof(int), st);
    cudaMemsetAsync(w->counters + 2, 0xff, sizeof(int), st);
    select_kernel<<<blocks(nk), 256, 0, st>>>(nk, nb, MB, rt1, res_tol, cap1, w->active, w->phase,
                                              w->moved, w->rnorm, w->nbase, w->todo, w->nnc,
                                              w->restart, w->iters, w->status, w->force,
                                              w->failcount, w->switchk, w->iterk, w->counters); note_launch();
    KCHECK("select_kernel");
    cudaError_t ce = cudaMemcpyAsync(hc, w->counters, 8 * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(host_dbg, w->dbg, 4 * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return cuda_fail(ce, "davidson counters");
    T.harvest();
    if (host_dbg[0] > 0 && !dumped) {   // H~, S~ are still those of the failed eigensolve
      dump_reduced(w, host_dbg[1], host_dbg[2]);
      dumped = true;
    }
    if (hc[1]) {
      given_up += hc[1];
      char buf[200];
      std::snprintf(buf, sizeof(buf),
                    "k=%d given up after repeated reduced-problem failures (status %d: %s), iteration %d",
                    hc[2], hc[3], hc[3] == PWK_ERR_NUMERIC ? "non-finite eigenvector" : "S~ not positive definite",
                    it);
      set_error(buf);
    }
    total = hc[0];
    const int nswitch = hc[4], n64 = hc[5];
    if (total == 0 && nswitch == 0) break;
    if (++it > max_iter) break;
    if (nswitch > 0) {
      // FP64 refinement start of the k-points leaving phase 1: their Ritz vectors from the
      // FP32 basis, in FP64, then FP64 H on them
      rotate_kernel<float, double><<<nk * nb, 256, 0, st>>>(nb, MB, np, w->nbase, w->switchk, w->ev, w->phi32,
                                                            w->tmp1, nb, nullptr, 0); note_launch();
      copy_vecs_kernel<double, double><<<nk * nb, 256, 0, st>>>(nk, nb, np, w->tmp1, nb, 0, w->phi, MB, 0,
                                                                w->switchk, nullptr, 0); note_launch();
      set_value_kernel<<<blocks(nk), 256, 0, st>>>(nk, w->switchk, w->phase, 2); note_launch();
      KCHECK("phase switch");
      if ((rc = start_block(2, w->switchk, nswitch))) return rc;
      update_kernel<<<blocks((size_t)nk * nb), 256, 0, st>>>(nk, nb, eth1, eth, w->phase, w->switchk, 0,
                                                             w->eps_new, w->eps, w->moved, w->status,
                                                             nullptr, w->nbase, w->force, w->failcount,
                                                             w->dbg); note_launch();
      KCHECK("update_kernel");
    }
    if (total > 0) {
      // restart the k-points whose basis would overflow
      if (mixed) {
        rotate_kernel<float, float><<<nk * nb, 256, 0, st>>>(nb, MB, np, w->nbase, w->restart, w->ev, w->phi32,
                                                             w->t32a, nb, w->phase, 1); note_launch();
        rotate_kernel<float, float><<<nk * nb, 256, 0, st>>>(nb, MB, np, w->nbase, w->restart, w->ev, w->hphi32,
                                                             w->t32b, nb, w->phase, 1); note_launch();
        copy_vecs_kernel<float, float><<<nk * nb, 256, 0, st>>>(nk, nb, np, w->t32a, nb, 0, w->phi32, MB, 0,
                                                                w->restart, w->phase, 1); note_launch();
        copy_vecs_kernel<float, float><<<nk * nb, 256, 0, st>>>(nk, nb, np, w->t32b, nb, 0, w->hphi32, MB, 0,
                                                                w->restart, w->phase, 1); note_launch();
        if (w->with_s) {
          rotate_kernel<float, float><<<nk * nb, 256, 0, st>>>(nb, MB, np, w->nbase, w->restart, w->ev,
                                                               w->sphi32, w->t32c, nb, w->phase, 1); note_launch();
          copy_vecs_kernel<float, float><<<nk * nb, 256, 0, st>>>(nk, nb, np, w->t32c, nb, 0, w->sphi32, MB, 0,
                                                                  w->restart, w->phase, 1); note_launch();
        }
      }
      rotate_kernel<double, double><<<nk * nb, 256, 0, st>>>(nb, MB, np, w->nbase, w->restart, w->ev, w->phi,
                                                             w->tmp1, nb, w->phase, want64); note_launch();
      rotate_kernel<double, double><<<nk * nb, 256, 0, st>>>(nb, MB, np, w->nbase, w->restart, w->ev, w->hphi,
                                                             w->tmp2, nb, w->phase, want64); note_launch();
      copy_vecs_kernel<double, double><<<nk * nb, 256, 0, st>>>(nk, nb, np, w->tmp1, nb, 0, w->phi, MB, 0,
                                                                w->restart, w->phase, want64); note_launch();
      copy_vecs_kernel<double, double><<<nk * nb, 256, 0, st>>>(nk, nb, np, w->tmp2, nb, 0, w->hphi, MB, 0,
                                                                w->restart, w->phase, want64); note_launch();
      if (w->with_s) {
        rotate_kernel<double, double><<<nk * nb, 256, 0, st>>>(nb, MB, np, w->nbase, w->restart, w->ev,
                                                               w->sphi, w->tmp3, nb, w->phase, want64); note_launch();
        copy_vecs_kernel<double, double><<<nk * nb, 256, 0, st>>>(nk, nb, np, w->tmp3, nb, 0, w->sphi, MB, 0,
                                                                  w->restart, w->phase, want64); note_launch();
      }
      gram(w->restart, nullptr, 0, nullptr, nb);
      set_nbase_kernel<<<blocks(nk), 256, 0, st>>>(nk, w->restart, w->nbase, nb, nullptr); note_launch();
      KCHECK("davidson restart");
      // append the corrections, apply H to them (FP32 for phase-1 k, FP64 for phase-2 k)
      if (mixed)
        { append_kernel<float><<<nk * nb, 256, 0, st>>>(nb, MB, np, w->iterk, w->nbase, w->nnc, w->todo,
                                                      w->corr32, w->phi32, w->lastrow, w->phase, 1); note_launch(); }
      append_kernel<double><<<nk * nb, 256, 0, st>>>(nb, MB, np, w->iterk, w->nbase, w->nnc, w->todo, w->corr,
                                                     w->phi, w->lastrow, w->phase, want64); note_launch();
      KCHECK("davidson append");
      for (int ph = 1; ph <= 2; ++ph) {
        const int cnt = ph == 2 ? n64 : total - n64;
        if (cnt == 0) continue;
        items_kernel<<<blocks((size_t)nk * nb), 256, 0, st>>>(nk, nb, w->iterk, w->nbase, 0, w->nnc, 0,
                                                              w->phase, ph, w->items); note_launch();
        KCHECK("items_kernel");
        cudaEvent_t th = T.mark();
        if (ph == 1) {
          if ((rc = run_hpsi(p, PWK_FP32, w->phi32, w->hphi32, w->items, nullptr, nk * nb, MB, MB, st,
                             w->with_s ? w->sphi32 : nullptr)))
            return rc;
        } else {
          if ((rc = run_hpsi(p, PWK_FP64, w->phi, w->hphi, w->items, nullptr, nk * nb, MB, MB, st,
                             w->with_s ? w->sphi : nullptr)))
            return rc;
        }
        T.close(0, th);
        napply[ph == 2 ? 0 : 1] += cnt;
      }
      gram(w->iterk, w->nbase, 0, w->nnc, 0);
      set_nbase_kernel<<<blocks(nk), 256, 0, st>>>(nk, w->iterk, w->nbase, 0, w->nnc); note_launch();
      KCHECK("davidson gram");
      cudaEvent_t tr = T.mark();
      if ((rc = launch_rr(nk, MB, nb, w->nbase, w->iterk, w->Hr, w->Sr, w->W, w->ev, w->eps_new,
                          w->status, st, w->drop, rr_flops)))
        return rc;
      T.close(1, tr);
      trace_reduced(w, it);
      update_kernel<<<blocks((size_t)nk * nb), 256, 0, st>>>(nk, nb, eth1, eth, w->phase, w->iterk, 0,
                                                             w->eps_new, w->eps, w->moved, w->status,
                                                             w->nnc, w->nbase, w->force, w->failcount,
                                                             w->dbg); note_launch();
      KCHECK("update_kernel");
    }
  }
  // eigenvectors out: psi = phi v (from the FP32 basis for k-points still in phase 1);
  // eigenvalues out
  if (mixed)
    { rotate_kernel<float, double><<<nk * nb, 256, 0, st>>>(nb, MB, np, w->nbase, nullptr, w->ev, w->phi32, psi,
                                                          nb, w->phase, 1); note_launch(); }
  rotate_kernel<double, double><<<nk * nb, 256, 0, st>>>(nb, MB, np, w->nbase, nullptr, w->ev, w->phi, psi, nb,
                                                         w->phase, want64); note_launch();
  KCHECK("final rotate");
  cudaError_t ce = cudaMemcpyAsync(eig, w->eps, sizeof(double) * nk * nb, cudaMemcpyDeviceToDevice, st);
  std::vector<int> h_iters(nk), h_nnc(nk);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_iters.data(), w->iters, sizeof(int) * nk, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_nnc.data(), w->nnc, sizeof(int) * nk, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return cuda_fail(ce, "davidson results");
  T.finish();
  if (iters_out) std::memcpy(iters_out, h_iters.data(), sizeof(int) * nk);
  if (notconv_out) std::memcpy(notconv_out, h_nnc.data(), sizeof(int) * nk);
  if (napply_out) {
    napply_out[0] = napply[0];
    napply_out[1] = napply[1];
  }
  return total + given_up;
}
