// Batched DFPT Sternheimer solver (paper Sec. 2.3-2.4, Algorithm 4): for every k of the
// block and every occupied band n
//   [H_{k+q} + alpha_k Q - eps_{k,n} S] x_{k,n} = b_{k,n} = -(1 - S P_v) dV psi_{k,n}
// (Eq. linear_system with dS = 0 for a local perturbation dv; Q = sum_v S|u_v><u_v|S,
// Eqs. projector, compute_mu, use_mu, apply_s_ch; S = 1 without q, where this is
// [H + alpha P_v - eps] x = -P_c dV psi), solved by the preconditioned CG of Eqs. ax1 ..
// updatedold for all (k, n) at once.  With S, S u_v is computed once per call and
// alpha Q d = sum_v (S u_v) alpha <S u_v|d>, so S is applied to each CG direction once
// (together with H, from the same projections).
//
// Kernels (one CTA per (k, n) unless noted):
//   rhs     : fused transfer kernel (inverse transform of psi_k on the k sphere, dv(r) u(r),
//             forward transform gathered on the k+q sphere), then b = -(w - P_v w)
//   aop     : mu_v = <psi_{k+q,v}|d> (Eq. compute_mu), y = sum_v psi_v mu_v (Eq. use_mu),
//             t = H d - eps d + alpha y   (the H d part is the fused H|psi> kernel)
//   cg_dir  : d = M^-1 r (Eq. row2), rho = Re<d|r> (Eq. row3), gamma (Eq. row4), d += gamma
//             d_old (Eq. updated); ||r|| for the stopping test
//   cg_step : lambda = -Re<d|r>/Re<d|t> (Eq. lambda), x += lambda d, r += lambda t,
//             d_old = d, rho_old = rho (Eqs. updatex, updater, updatedold)
// Dot products and scalars are FP64 and stay on the device; the host reads the counters
// (pairs still iterating) every few iterations.  FP64 mode: FP64 vectors and operator.  Mixed
// mode: FP64 iterative refinement around FP32 inner solves: each round takes the true FP64
// residual r = A x - b, solves A e = -r for a correction with FP32 vectors and the FP32
// operator (H d and the valence projection alpha Q d), reducing it by 1e-6 (the FP32
// rounding allows that before the inner iteration stalls; 1e-4 took one refinement round
// more, 1e-7 more iterations), and adds e to x in FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "solvers.h"

namespace pwk {

struct CgWork {
  int nk = 0, nocc = 0, np = 0;
  bool with_s = false;    // overlap S (plan with q): S u_v and S d kept
  double2 *b = nullptr, *r = nullptr, *d = nullptr, *dold = nullptr, *t = nullptr;
  double2 *su = nullptr, *sx = nullptr;
  float2* v32 = nullptr;   // the valence set of the operator (S psi or psi) in FP32
  // mixed mode: the inner solve's vectors in FP32 (correction e, its residual r, direction
  // d, t = H d and S d)
  bool has32 = false;
  float2 *e32 = nullptr, *r32 = nullptr, *d32 = nullptr, *t32 = nullptr, *sd32 = nullptr;
  double *rho = nullptr, *rho_old = nullptr, *bnorm = nullptr, *thr = nullptr, *tkin = nullptr;
  double *rnorm = nullptr;
  int *active = nullptr, *first = nullptr, *iters = nullptr, *items = nullptr, *counters = nullptr;
  int* list = nullptr;   // pairs still iterating, compacted (cg_compact_kernel)
  int* seen = nullptr;   // iters[i] at pair i's last true residual
  std::vector<void*> ptrs;
};

void destroy_cg_work(pwk_plan* p) {
  if (p->cg == nullptr) return;
  for (void* q : p->cg->ptrs) plan_free(p, q);
  delete p->cg;
  p->cg = nullptr;
}

template <typename T>
static int calloc_(pwk_plan* p, CgWork* w, T** ptr, size_t n) {
  int rc = plan_alloc(p, (void**)ptr, n * sizeof(T));
  if (rc == PWK_OK) w->ptrs.push_back(*ptr);
  return rc;
}

// Grows only, like the Davidson workspace: a call with at most the allocated number of
// occupied bands (and an overlap the arrays cover) reuses it; arrays are indexed with the
// call's nocc.
static int ensure_cg_work(pwk_plan* p, int nocc, bool mixed) {
  const bool want_s = p->d_q != nullptr;
  if (p->cg && p->cg->nocc >= nocc && (p->cg->with_s || !want_s) && (p->cg->has32 || !mixed)) return PWK_OK;
  bool with_s = want_s, has32 = mixed;
  if (p->cg) {
    nocc = std::max(nocc, p->cg->nocc);
    with_s = with_s || p->cg->with_s;
    has32 = has32 || p->cg->has32;
  }
  destroy_cg_work(p);
  CgWork* w = new CgWork();
  p->cg = w;
  w->nk = p->nk;
  w->nocc = nocc;   // capacity
  w->np = p->npw_max;
  w->with_s = with_s;   // S arrays allocated
  const size_t nv = (size_t)p->nk * nocc, nv2 = nv * p->npw_max;
  int rc;
  if (with_s && ((rc = calloc_(p, w, &w->su, nv2)) || (rc = calloc_(p, w, &w->sx, nv2)))) {
    destroy_cg_work(p);
    return rc;
  }
  w->has32 = has32;
  if (has32 && ((rc = calloc_(p, w, &w->e32, nv2)) || (rc = calloc_(p, w, &w->r32, nv2)) ||
                (rc = calloc_(p, w, &w->d32, nv2)) || (rc = calloc_(p, w, &w->t32, nv2)) ||
                (with_s && (rc = calloc_(p, w, &w->sd32, nv2))))) {
    destroy_cg_work(p);
    return rc;
  }
  if ((rc = calloc_(p, w, &w->b, nv2)) || (rc = calloc_(p, w, &w->r, nv2)) ||
      (rc = calloc_(p, w, &w->d, nv2)) || (rc = calloc_(p, w, &w->dold, nv2)) ||
      (rc = calloc_(p, w, &w->t, nv2)) || (rc = calloc_(p, w, &w->rho, nv)) ||
      (rc = calloc_(p, w, &w->rho_old, nv)) || (rc = calloc_(p, w, &w->bnorm, nv)) ||
      (rc = calloc_(p, w, &w->thr, nv)) || (rc = calloc_(p, w, &w->tkin, nv)) ||
      (rc = calloc_(p, w, &w->rnorm, nv)) || (rc = calloc_(p, w, &w->active, nv)) ||
      (rc = calloc_(p, w, &w->first, nv)) || (rc = calloc_(p, w, &w->iters, nv)) ||
      (rc = calloc_(p, w, &w->items, nv * 3)) || (rc = calloc_(p, w, &w->list, nv)) ||
      (rc = calloc_(p, w, &w->seen, nv)) || (rc = calloc_(p, w, &w->v32, nv2)) ||
      (rc = calloc_(p, w, &w->counters, 4))) {
    destroy_cg_work(p);
    return rc;
  }
  return PWK_OK;
}

// ------------------------------------------------------------------ kernels
constexpr int kCgMaxPw = 2048;   // plane waves whose preconditioner cg_dir keeps in shared memory

__device__ __forceinline__ double2 cmc(double2 a, double2 b) {  // conj(a) b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__device__ double bsum2(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  __syncthreads();
  return s;
}

// Block sums of two doubles per thread, reduced by warp 0 alone from per-thread partials in
// shared memory (part: blockDim.x entries): the FP64 pipe runs at 1/64 of the FP32 rate on
// this GPU and an FP64 instruction costs the whole warp, so a shuffle tree in every warp
// (or every thread re-adding the warp partials) costs several times the arithmetic it
// reduces.  All threads get both sums.
__device__ double2 bsum_pair(double a, double b, double2* part, double2* out) {
  part[threadIdx.x] = make_double2(a, b);
  __syncthreads();
  if (threadIdx.x < 32) {
    double sa = 0.0, sb = 0.0;
    for (int j = threadIdx.x; j < (int)blockDim.x; j += 32) {
      sa += part[j].x;
      sb += part[j].y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
      sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    if (threadIdx.x == 0) *out = make_double2(sa, sb);
  }
  __syncthreads();
  return *out;
}

// The preconditioner of Sec. 2.4 for one plane wave, 1/M_G = 1 / max(1, |k+q+G|^2 / T_kin),
// formed in FP32 (any fixed positive M keeps the CG exact; the same expression serves every
// iteration of a solve).
__device__ __forceinline__ double precond(double g2, float itk) {
  return (double)(1.0f / fmaxf(1.0f, (float)g2 * itk));
}

// out = u + a_w ws + a_p sum_v py_v <pm_v|w>  for (k, n) with active (or all if null).
// a_w = wmode ? -eps[k][n] : -1;  a_p = pmode ? alpha[k] : 1;  u may be null (a_u = 0);
// ws null means ws = w.  With S = 1: pm = py = psi_{k+q,v}, ws = w.  With S (Eq. projector):
// pm = py = S psi_{k+q,v} and ws = S w for the operator (alpha Q w - eps S w), and pm = psi,
// py = S psi for the right-hand side -(1 - S P_v) w.  The norm of out goes to onorm.
// T is the arithmetic type (vectors are complex128 in memory): FP64, or FP32 for the operator
// inside the mixed-mode CG, whose H part is FP32 as well (the refinement's FP64 residuals
// use the FP64 form).
template <typename T>
__global__ void __launch_bounds__(512) proj_combine_kernel(int nocc, int np, const int* npw,
                                                           const int* active,
                                                           const double2* pm, const double2* py,
                                                           const double2* u, const double2* w,
                                                           const double2* ws,
                                                           int wmode, const double* eps,
                                                           int pmode, const double* alpha,
                                                           double2* out, double* onorm) {
  const int k = blockIdx.x / nocc;
  if (active != nullptr && !active[blockIdx.x]) return;
  const int npk = npw[k];
  __shared__ T mur[64], mui[64];
  __shared__ double red[32];
  const double2* W = w + (size_t)blockIdx.x * np;
  const double2* WS = ws != nullptr ? ws + (size_t)blockIdx.x * np : W;
  const double2* Pk = pm + (size_t)k * nocc * np;
  const double2* Yk = py + (size_t)k * nocc * np;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int v = warp; v < nocc; v += nw) {
    T sx = 0, sy = 0;
    const double2* pv = Pk + (size_t)v * np;
    for (int g = lane; g < npk; g += 32) {
      const double2 a = pv[g], b = W[g];   // conj(a) b
      const T ax = T(a.x), ay = T(a.y), bx = T(b.x), by = T(b.y);
      sx += ax * bx + ay * by;
      sy += ax * by - ay * bx;
    }
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) {
      mur[v] = sx;
      mui[v] = sy;
    }
  }
  __syncthreads();
  const T aw = wmode ? T(-eps[blockIdx.x]) : T(-1);
  const T ap = pmode ? T(alpha[k]) : T(1);
  const double2* U = u ? u + (size_t)blockIdx.x * np : nullptr;
  double2* O = out + (size_t)blockIdx.x * np;
  double nn = 0.0;
  for (int g = threadIdx.x; g < np; g += blockDim.x) {
    if (g >= npk) {
      O[g] = make_double2(0.0, 0.0);
      continue;
    }
    T yx = 0, yy = 0;
    for (int v = 0; v < nocc; ++v) {
      const double2 p = Yk[(size_t)v * np + g];
      const T px = T(p.x), pyv = T(p.y), mx = mur[v], my = mui[v];
      yx += px * mx - pyv * my;
      yy += px * my + pyv * mx;
    }
    const double2 wg = WS[g];
    const T ox = aw * T(wg.x) + ap * yx, oy = aw * T(wg.y) + ap * yy;
    double2 o = make_double2(double(ox), double(oy));
    if (U) {
      o.x += U[g].x;
      o.y += U[g].y;
    }
    nn += o.x * o.x + o.y * o.y;
    O[g] = o;
  }
  if (onorm != nullptr) {   // uniform over the block
    nn = bsum2(nn, red);
    if (threadIdx.x == 0) onorm[blockIdx.x] = sqrt(nn);
  }
}

// <psi_{k+q,n}|T|psi_{k+q,n}> / <psi|psi> for the preconditioner of Sec. 2.4
__global__ void tkin_kernel(int nocc, int np, const int* npw, const double* g2, const double2* psi,
                            double* tkin) {
  const int k = blockIdx.x / nocc;
  __shared__ double red[32];
  const double2* P = psi + (size_t)blockIdx.x * np;
  const double* G = g2 + (size_t)k * np;
  double a = 0.0, b = 0.0;
  for (int g = threadIdx.x; g < npw[k]; g += blockDim.x) {
    const double m = P[g].x * P[g].x + P[g].y * P[g].y;
    a += G[g] * m;
    b += m;
  }
  a = bsum2(a, red);
  b = bsum2(b, red);
  if (threadIdx.x == 0) tkin[blockIdx.x] = b > 0.0 ? a / b : 1.0;
}

// r = t - b (or -b when t is null); relative norm; thresholds and activity for the inner solve
__global__ void residual_kernel(int nocc, int np, const int* npw, const double2* t, const double2* b,
                                const double* bnorm, double tol, double eta, double2* r,
                                double* rnorm, double* thr, int* active, int* first,
                                int* counters) {
  const int i = blockIdx.x, k = i / nocc;
  __shared__ double red[32];
  const double2* T = t ? t + (size_t)i * np : nullptr;
  const double2* B = b + (size_t)i * np;
  double2* R = r + (size_t)i * np;
  double nn = 0.0;
  for (int g = threadIdx.x; g < np; g += blockDim.x) {
    double2 v = make_double2(-B[g].x, -B[g].y);
    if (T && g < npw[k]) {
      v.x += T[g].x;
      v.y += T[g].y;
    }
    R[g] = v;
    nn += v.x * v.x + v.y * v.y;
  }
  nn = bsum2(nn, red);
  if (threadIdx.x == 0) {
    const double rn = sqrt(nn), bn = bnorm[i];
    rnorm[i] = bn > 0.0 ? rn / bn : 0.0;
    const bool on = bn > 0.0 && rn > tol * bn;
    active[i] = on ? 1 : 0;
    first[i] = 1;
    const double th = fmax(tol * bn, eta * rn);
    thr[i] = th * th;
    if (on) atomicAdd(&counters[0], 1);
  }
}

// d = M^-1 r (+ gamma d_old); rho = Re<d|r>; stop when ||r||^2 <= thr
__global__ void __launch_bounds__(256) cg_dir_kernel(int nocc, int np, const int* npw,
                                                     const double* g2, const double* tkin,
                                                     const double2* r, double2* d,
                                                     const double2* dold, double* rho,
                                                     const double* rho_old, const double* thr,
                                                     int* active, int* first, int* counters) {
  const int i = blockIdx.x, k = i / nocc;
  if (!active[i]) return;
  __shared__ double red[32];
  const int npk = npw[k];
  const double* G = g2 + (size_t)k * np;
  const float itk = (float)(1.0 / tkin[i]);
  const double2* R = r + (size_t)i * np;
  // 1/M_G (Eq. row2, precond()): kept in shared memory for the update pass when the sphere
  // fits (np is uniform over the launch)
  __shared__ double im[kCgMaxPw];
  const bool keep = np <= kCgMaxPw;
  double rr = 0.0, rh = 0.0;
  for (int g = threadIdx.x; g < npk; g += blockDim.x) {
    const double2 x = R[g];
    const double mi = precond(G[g], itk);
    if (keep) im[g] = mi;
    rr += x.x * x.x + x.y * x.y;
    rh += (x.x * x.x + x.y * x.y) * mi;   // Re<M^-1 r | r>
  }
  rr = bsum2(rr, red);
  rh = bsum2(rh, red);
  if (rr <= thr[i]) {
    if (threadIdx.x == 0) active[i] = 0;
    return;
  }
  const bool f = first[i] != 0;
  const double gam = f ? 0.0 : rh / rho_old[i];
  const double2* DO = dold + (size_t)i * np;
  double2* D = d + (size_t)i * np;
  for (int g = threadIdx.x; g < np; g += blockDim.x) {
    if (g >= npk) {
      D[g] = make_double2(0.0, 0.0);
      continue;
    }
    const double mi = keep ? im[g] : precond(G[g], itk);   // im[g]: this thread's, pass 1
    double2 v = make_double2(R[g].x * mi, R[g].y * mi);
    if (!f) {
      v.x += gam * DO[g].x;
      v.y += gam * DO[g].y;
    }
    D[g] = v;
  }
  if (threadIdx.x == 0) {
    rho[i] = rh;
    first[i] = 0;
    atomicAdd(&counters[0], 1);
  }
}

__global__ void cg_items_kernel(int n_pairs, int nocc, const int* active, int* items) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pairs) return;
  const bool on = active == nullptr || active[i] != 0;   // null: every pair
  items[3 * i] = on ? i / nocc : -1;
  items[3 * i + 1] = on ? i % nocc : 0;
  items[3 * i + 2] = on ? i % nocc : 0;
}

// lambda = -Re<d|r>/Re<d|t>; x += lambda d; r += lambda t; d_old = d; rho_old = rho
__global__ void __launch_bounds__(256) cg_step_kernel(int nocc, int np, const int* npw,
                                                      int* active, const double2* d,
                                                      const double2* t, double2* x, double2* r,
                                                      double2* dold, const double* rho,
                                                      double* rho_old, int* iters,
                                                      int* counters) {
  const int i = blockIdx.x, k = i / nocc;
  if (!active[i]) return;
  __shared__ double red[32];
  const int npk = npw[k];
  const double2* D = d + (size_t)i * np;
  const double2* T = t + (size_t)i * np;
  double2* R = r + (size_t)i * np;
  double dr = 0.0, dt = 0.0;
  for (int g = threadIdx.x; g < npk; g += blockDim.x) {
    dr += D[g].x * R[g].x + D[g].y * R[g].y;
    dt += D[g].x * T[g].x + D[g].y * T[g].y;
  }
  dr = bsum2(dr, red);
  dt = bsum2(dt, red);
  if (!(dt > 0.0) || !isfinite(dr)) {   // indefinite direction or breakdown: stop this pair
    if (threadIdx.x == 0) {
      active[i] = 0;
      atomicOr(&counters[1], 1);
    }
    return;
  }
  const double lam = -dr / dt;
  double2* X = x + (size_t)i * np;
  double2* DO = dold + (size_t)i * np;
  for (int g = threadIdx.x; g < npk; g += blockDim.x) {
    const double2 dg = D[g], tg = T[g];
    X[g].x += lam * dg.x;
    X[g].y += lam * dg.y;
    R[g].x += lam * tg.x;
    R[g].y += lam * tg.y;
    DO[g] = dg;
  }
  if (threadIdx.x == 0) {
    rho_old[i] = rho[i];
    iters[i] += 1;
  }
}

// The pairs still iterating as a compact list, with their H|psi> work items (k, n, n) in the
// same order; counters[2] = their number.  Warp-aggregated: pairs keep their order within a
// warp (the bands of a k-point stay together for the projector kernels), warps in any order.
__global__ void cg_compact_kernel(int n_pairs, int nocc, const int* active, int* list, int* items,
                                  int* counters) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool on = i < n_pairs && active[i] != 0;
  const unsigned m = __ballot_sync(0xffffffffu, on);
  if (m == 0) return;   // uniform over the warp
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == 0) base = atomicAdd(&counters[2], __popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (on) {
    const int c = base + __popc(m & ((1u << lane) - 1u));
    list[c] = i;
    items[3 * c] = i / nocc;
    items[3 * c + 1] = i % nocc;
    items[3 * c + 2] = i % nocc;
  }
}

// The pairs whose x changed since their last true residual (iters[i] != seen[i]) as a
// compact list with their work items, like cg_compact_kernel; seen[i] is brought up to date.
__global__ void stale_compact_kernel(int n_pairs, int nocc, const int* iters, int* seen, int* list,
                                     int* items, int* counters) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool on = i < n_pairs && iters[i] != seen[i];
  const unsigned m = __ballot_sync(0xffffffffu, on);
  if (m == 0) return;   // uniform over the warp
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == 0) base = atomicAdd(&counters[2], __popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (on) {
    const int c = base + __popc(m & ((1u << lane) - 1u));
    list[c] = i;
    items[3 * c] = i / nocc;
    items[3 * c + 1] = i % nocc;
    items[3 * c + 2] = i % nocc;
    seen[i] = iters[i];
  }
}

// The true residual r = A x - b with the FP64 operator for the listed pairs (the first
// *count entries of list; H x and S x already applied): t = H x - eps S x + alpha sum_v py_v
// <pm_v|x> (the arithmetic of proj_combine_kernel<double>), r = t - b, ||r|| / ||b|| into
// rnorm, and the thresholds and activity of the next inner solve (as residual_kernel).
__global__ void __launch_bounds__(512) true_residual_kernel(int nocc, int np, const int* npw, const int* list,
                                                           const int* count, const double2* pm,
                                                           const double2* py, const double2* hx,
                                                           const double2* x, const double2* sx,
                                                           const double* eps, const double* alpha,
                                                           const double2* b, const double* bnorm,
                                                           double tol, double eta, double2* r,
                                                           double* rnorm, double* thr, int* active,
                                                           int* first, int* counters) {
  if ((int)blockIdx.x >= *count) return;
  const int i = list[blockIdx.x], k = i / nocc;
  const int npk = npw[k];
  __shared__ double mur[64], mui[64];
  __shared__ double red[32];
  const double2* X = x + (size_t)i * np;
  const double2* SX = sx != nullptr ? sx + (size_t)i * np : X;
  const double2* HX = hx + (size_t)i * np;
  const double2* B = b + (size_t)i * np;
  const double2* Pk = pm + (size_t)k * nocc * np;
  const double2* Yk = py + (size_t)k * nocc * np;
  double2* R = r + (size_t)i * np;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int v = warp; v < nocc; v += nw) {
    double sx_ = 0, sy_ = 0;
    const double2* pv = Pk + (size_t)v * np;
    for (int g = lane; g < npk; g += 32) {
      const double2 a = pv[g], bb = X[g];   // conj(a) x
      sx_ += a.x * bb.x + a.y * bb.y;
      sy_ += a.x * bb.y - a.y * bb.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      sx_ += __shfl_xor_sync(0xffffffffu, sx_, o);
      sy_ += __shfl_xor_sync(0xffffffffu, sy_, o);
    }
    if (lane == 0) {
      mur[v] = sx_;
      mui[v] = sy_;
    }
  }
  __syncthreads();
  const double aw = -eps[i], ap = alpha[k];
  double nn = 0.0;
  for (int g = threadIdx.x; g < np; g += blockDim.x) {
    double2 v = make_double2(-B[g].x, -B[g].y);
    if (g < npk) {
      double yx = 0, yy = 0;
      for (int u = 0; u < nocc; ++u) {
        const double2 p = Yk[(size_t)u * np + g];
        yx += p.x * mur[u] - p.y * mui[u];
        yy += p.x * mui[u] + p.y * mur[u];
      }
      const double2 wg = SX[g], h = HX[g];
      v.x += (aw * wg.x + ap * yx) + h.x;
      v.y += (aw * wg.y + ap * yy) + h.y;
    }
    R[g] = v;
    nn += v.x * v.x + v.y * v.y;
  }
  nn = bsum2(nn, red);
  if (threadIdx.x == 0) {
    const double rn = sqrt(nn), bn = bnorm[i];
    rnorm[i] = bn > 0.0 ? rn / bn : 0.0;
    const bool on = bn > 0.0 && rn > tol * bn;
    active[i] = on ? 1 : 0;
    first[i] = 1;
    const double th = fmax(tol * bn, eta * rn);
    thr[i] = th * th;
    if (on) atomicAdd(&counters[0], 1);
  }
}

// FP32 copy of n complex128 values (the valence set the mixed-mode operator reads every
// iteration, converted once per solve).
__global__ void to_c64_kernel(size_t n, const double2* in, float2* out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

// One CG iteration of a pair after H d (and S d) have been applied, in one pass over the
// pair's vectors (one CTA per listed pair, a warp per valence vector for the projections), FP64
// (the mixed mode's inner solves use cg_update32_kernel):
//   mu_v = <pm_v|d>, t = H d - eps (S) d + alpha sum_v pm_v mu_v          (Eqs. compute_mu,
//          use_mu: the operator A d)
//   lambda = -Re<d|r> / Re<d|t>, x += lambda d, r += lambda t               (Eqs. lambda,
//          updatex, updater)
//   stop if ||r||^2 <= thr; else rho' = Re<M^-1 r|r>, d = M^-1 r + (rho'/rho) d, rho = rho'
//          (Eqs. row2 - updated of the next iteration; d_old is the d just used, so no
//          separate copy is kept)
// pm is the valence set S psi_v (psi_v without S).  t and M^-1 r stay in shared memory (2 np
// complex128) between the passes; sums and updates are FMA chains (every FP64 instruction
// counts on this GPU).  counters[0] counts the pairs with a new direction, counters[1] flags a
// breakdown (Re<d|t> <= 0: the pair stops, as in cg_step_kernel).
__global__ void __launch_bounds__(512) cg_update_kernel(int nocc, int np, const int* npw, const int* list,
                                                       const double* g2, const double* tkin,
                                                       const double2* pm, const double2* hd, double2* d,
                                                       const double2* sd, const double* eps,
                                                       const double* alpha, double2* x, double2* r,
                                                       double* rho, const double* thr, int* active,
                                                       int* iters, int* counters, const int* count) {
  if ((int)blockIdx.x >= *count) return;   // the launch covers an upper bound of the list
  const int i = list[blockIdx.x], k = i / nocc;
  const int npk = npw[k];
  extern __shared__ double2 cg_sm[];
  double2* ts = cg_sm;          // t = A d
  double2* rs = cg_sm + np;     // M^-1 r of the updated r
  __shared__ double mur[64], mui[64];
  __shared__ double2 part[512], tot;
  double2* D = d + (size_t)i * np;
  const double2* HD = hd + (size_t)i * np;
  const double2* Pk = pm + (size_t)k * nocc * np;
  double2* X = x + (size_t)i * np;
  double2* R = r + (size_t)i * np;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int v = warp; v < nocc; v += nw) {
    double sx = 0, sy = 0;
    const double2* pv = Pk + (size_t)v * np;
    for (int g = lane; g < npk; g += 32) {
      const double2 a = pv[g], b = D[g];   // conj(a) b
      sx = fma(a.x, b.x, fma(a.y, b.y, sx));
      sy = fma(a.x, b.y, fma(-a.y, b.x, sy));
    }
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) {
      mur[v] = sx;
      mui[v] = sy;
    }
  }
  __syncthreads();
  const double aw = -eps[i], ap = alpha[k];
  double dr = 0.0, dt = 0.0;
  for (int g = threadIdx.x; g < npk; g += blockDim.x) {
    double yx = 0, yy = 0;
    for (int v = 0; v < nocc; ++v) {
      const double2 pv = Pk[(size_t)v * np + g];
      yx = fma(pv.x, mur[v], fma(-pv.y, mui[v], yx));
      yy = fma(pv.x, mui[v], fma(pv.y, mur[v], yy));
    }
    const double2 dg = D[g], rg = R[g];
    const double2 w = sd != nullptr ? sd[(size_t)i * np + g] : dg;
    const double2 h = HD[g];
    const double2 t = make_double2(fma(aw, w.x, fma(ap, yx, h.x)), fma(aw, w.y, fma(ap, yy, h.y)));
    ts[g] = t;
    dr = fma(dg.x, rg.x, fma(dg.y, rg.y, dr));
    dt = fma(dg.x, t.x, fma(dg.y, t.y, dt));
  }
  {
    const double2 s2 = bsum_pair(dr, dt, part, &tot);
    dr = s2.x;
    dt = s2.y;
  }
  if (!(dt > 0.0) || !isfinite(dr)) {   // indefinite direction or breakdown: stop this pair
    if (threadIdx.x == 0) {
      active[i] = 0;
      atomicOr(&counters[1], 1);
    }
    return;
  }
  const double lam = -dr / dt;
  const float itk = (float)(1.0 / tkin[i]);
  const double* G = g2 + (size_t)k * np;
  double rr = 0.0, rh = 0.0;
  for (int g = threadIdx.x; g < npk; g += blockDim.x) {
    const double2 dg = D[g], t = ts[g];
    double2 xg = X[g], rg = R[g];
    xg.x = fma(lam, dg.x, xg.x);
    xg.y = fma(lam, dg.y, xg.y);
    rg.x = fma(lam, t.x, rg.x);
    rg.y = fma(lam, t.y, rg.y);
    X[g] = xg;
    R[g] = rg;
    const double mi = precond(G[g], itk);
    rs[g] = make_double2(rg.x * mi, rg.y * mi);   // M^-1 r for the next direction
    const double q = fma(rg.x, rg.x, rg.y * rg.y);
    rr += q;
    rh = fma(q, mi, rh);
  }
  {
    const double2 s2 = bsum_pair(rr, rh, part, &tot);
    rr = s2.x;
    rh = s2.y;
  }
  if (threadIdx.x == 0) iters[i] += 1;
  if (rr <= thr[i]) {
    if (threadIdx.x == 0) active[i] = 0;
    return;
  }
  const double gam = rh / rho[i];
  for (int g = threadIdx.x; g < npk; g += blockDim.x) {
    const double2 zg = rs[g], dg = D[g];   // zg = M^-1 r
    D[g] = make_double2(fma(gam, dg.x, zg.x), fma(gam, dg.y, zg.y));
  }
  if (threadIdx.x == 0) {
    rho[i] = rh;
    atomicAdd(&counters[0], 1);
  }
}

// ------------------------------------------------------------------ mixed-mode inner solve
// The inner solve of a refinement round works on the correction e of the current x: it
// solves A e = -r (r = A x - b, the FP64 true residual) with FP32 vectors and the FP32
// operator, and the round ends with x += e in FP64.  Only the dot products are reduced in
// FP64 (each thread's FP32 partial, then an FP64 sum over the block), and the CG scalars are
// FP64; the element-wise work stays off the FP64 pipe.

// Start of an inner solve for every pair: e = 0; for the active pairs r32 = r, the first
// direction d = M^-1 r, rho = Re<M^-1 r|r>, and the stopping test (||r||^2 <= thr: the pair
// is inactive; counters[0] counts the pairs with a direction).
__global__ void __launch_bounds__(256) cg_init32_kernel(int nocc, int np, const int* npw, const double* g2,
                                                       const double* tkin, const double2* r, float2* e32,
                                                       float2* r32, float2* d32, double* rho,
                                                       const double* thr, int* active, int* counters) {
  const int i = blockIdx.x, k = i / nocc;
  __shared__ double2 part[256], tot;
  float2* E = e32 + (size_t)i * np;
  for (int g = threadIdx.x; g < np; g += blockDim.x) E[g] = make_float2(0.f, 0.f);
  if (!active[i]) return;
  const int npk = npw[k];
  const float itk = (float)(1.0 / tkin[i]);
  const double* G = g2 + (size_t)k * np;
  const double2* R = r + (size_t)i * np;
  float2* R32 = r32 + (size_t)i * np;
  float2* D32 = d32 + (size_t)i * np;
  float rr = 0.f, rh = 0.f;
  for (int g = threadIdx.x; g < np; g += blockDim.x) {
    if (g >= npk) {
      R32[g] = make_float2(0.f, 0.f);
      D32[g] = make_float2(0.f, 0.f);
      continue;
    }
    const float2 v = make_float2((float)R[g].x, (float)R[g].y);
    const float mi = 1.0f / fmaxf(1.0f, (float)G[g] * itk);
    R32[g] = v;
    D32[g] = make_float2(v.x * mi, v.y * mi);
    const float q = fmaf(v.x, v.x, v.y * v.y);
    rr += q;
    rh = fmaf(q, mi, rh);
  }
  const double2 s2 = bsum_pair((double)rr, (double)rh, part, &tot);
  if (threadIdx.x == 0) {
    if (s2.x <= thr[i]) {
      active[i] = 0;
    } else {
      rho[i] = s2.y;
      atomicAdd(&counters[0], 1);
    }
  }
}

// One FP32 CG iteration of a listed pair (the first *count entries of list): t = H d - eps S d +
// alpha sum_v pm_v <pm_v|d> from the FP32 H (and S) output, lambda = -Re<d|r>/Re<d|t>,
// e += lambda d, r += lambda t, the stopping test, the next direction d = M^-1 r + gamma d.
// Vectors and element-wise arithmetic FP32; each thread's partial dot products are summed in
// FP64 over the block; lambda, gamma, rho FP64.  Counters as in cg_update_kernel.
__global__ void __launch_bounds__(512) cg_update32_kernel(int nocc, int np, const int* npw, const int* list,
                                                         const int* count, const double* g2,
                                                         const double* tkin, const float2* pm32,
                                                         const float2* t32, float2* d32,
                                                         const float2* sd32, const double* eps,
                                                         const double* alpha, float2* e32, float2* r32,
                                                         double* rho, const double* thr, int* active,
                                                         int* iters, int* counters) {
  if ((int)blockIdx.x >= *count) return;   // the launch covers an upper bound of the list
  const int i = list[blockIdx.x], k = i / nocc;
  const int npk = npw[k];
  extern __shared__ float2 cg32_sm[];
  float2* ds = cg32_sm;            // d
  float2* ts = cg32_sm + np;       // t = A d
  float2* zs = cg32_sm + 2 * np;   // M^-1 r of the updated r
  __shared__ float mur[64], mui[64];
  __shared__ double2 part[512], tot;
  float2* D = d32 + (size_t)i * np;
  const float2* HD = t32 + (size_t)i * np;
  const float2* Pk = pm32 + (size_t)k * nocc * np;
  float2* E = e32 + (size_t)i * np;
  float2* R = r32 + (size_t)i * np;
  for (int g = threadIdx.x; g < npk; g += blockDim.x) ds[g] = D[g];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int v = warp; v < nocc; v += nw) {
    float sx = 0.f, sy = 0.f;
    const float2* pv = Pk + (size_t)v * np;
    for (int g = lane; g < npk; g += 32) {
      const float2 a = pv[g], b = ds[g];   // conj(a) b
      sx = fmaf(a.x, b.x, fmaf(a.y, b.y, sx));
      sy = fmaf(a.x, b.y, fmaf(-a.y, b.x, sy));
    }
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) {
      mur[v] = sx;
      mui[v] = sy;
    }
  }
  __syncthreads();
  const float aw = (float)(-eps[i]), ap = (float)alpha[k];
  float dr = 0.f, dt = 0.f;
  for (int g = threadIdx.x; g < npk; g += blockDim.x) {
    float yx = 0.f, yy = 0.f;
    for (int v = 0; v < nocc; ++v) {
      const float2 pv = Pk[(size_t)v * np + g];
      yx = fmaf(pv.x, mur[v], fmaf(-pv.y, mui[v], yx));
      yy = fmaf(pv.x, mui[v], fmaf(pv.y, mur[v], yy));
    }
    const float2 w = sd32 != nullptr ? sd32[(size_t)i * np + g] : ds[g];
    const float2 h = HD[g];
    const float2 t = make_float2(fmaf(aw, w.x, fmaf(ap, yx, h.x)), fmaf(aw, w.y, fmaf(ap, yy, h.y)));
    ts[g] = t;
    const float2 dg = ds[g], rg = R[g];
    dr = fmaf(dg.x, rg.x, fmaf(dg.y, rg.y, dr));
    dt = fmaf(dg.x, t.x, fmaf(dg.y, t.y, dt));
  }
  double drd, dtd;
  {
    const double2 s2 = bsum_pair((double)dr, (double)dt, part, &tot);
    drd = s2.x;
    dtd = s2.y;
  }
  if (!(dtd > 0.0) || !isfinite(drd)) {   // indefinite direction or breakdown: stop this pair
    if (threadIdx.x == 0) {
      active[i] = 0;
      atomicOr(&counters[1], 1);
    }
    return;
  }
  const float lam = (float)(-drd / dtd);
  const float itk = (float)(1.0 / tkin[i]);
  const double* G = g2 + (size_t)k * np;
  float rr = 0.f, rh = 0.f;
  for (int g = threadIdx.x; g < npk; g += blockDim.x) {
    const float2 dg = ds[g], t = ts[g];
    float2 eg = E[g], rg = R[g];
    eg.x = fmaf(lam, dg.x, eg.x);
    eg.y = fmaf(lam, dg.y, eg.y);
    rg.x = fmaf(lam, t.x, rg.x);
    rg.y = fmaf(lam, t.y, rg.y);
    E[g] = eg;
    R[g] = rg;
    const float mi = 1.0f / fmaxf(1.0f, (float)G[g] * itk);
    zs[g] = make_float2(rg.x * mi, rg.y * mi);
    const float q = fmaf(rg.x, rg.x, rg.y * rg.y);
    rr += q;
    rh = fmaf(q, mi, rh);
  }
  double rrd, rhd;
  {
    const double2 s2 = bsum_pair((double)rr, (double)rh, part, &tot);
    rrd = s2.x;
    rhd = s2.y;
  }
  if (threadIdx.x == 0) iters[i] += 1;
  if (rrd <= thr[i]) {
    if (threadIdx.x == 0) active[i] = 0;
    return;
  }
  const float gam = (float)(rhd / rho[i]);
  for (int g = threadIdx.x; g < npk; g += blockDim.x) {
    const float2 zg = zs[g], dg = ds[g];
    D[g] = make_float2(fmaf(gam, dg.x, zg.x), fmaf(gam, dg.y, zg.y));
  }
  if (threadIdx.x == 0) {
    rho[i] = rhd;
    atomicAdd(&counters[0], 1);
  }
}

// x += e for every pair (e is zero where the pair did not iterate)
__global__ void add_correction_kernel(int nocc, int np, const int* npw, const float2* e32, double2* x) {
  const int i = blockIdx.x, k = i / nocc, npk = npw[k];
  const float2* E = e32 + (size_t)i * np;
  double2* X = x + (size_t)i * np;
  for (int g = threadIdx.x; g < npk; g += blockDim.x) {
    const float2 e = E[g];
    X[g] = make_double2(X[g].x + (double)e.x, X[g].y + (double)e.y);
  }
}

// Shared memory of cg_update_kernel for spheres of np plane waves; the fused step is used
// while it fits, else the separate proj_combine, cg_step and cg_dir kernels.
static size_t cg_update_smem(int np) { return (size_t)2 * np * sizeof(double2); }
constexpr size_t kCgUpdateMaxSmem = 200 * 1024;
// CG iterations between two reads of the solver's counters by the host
constexpr int kCgBurst = 4;

// The stick maps of the pair (k sphere of plan_k -> k+q sphere of plan_kq, the union of their
// z-sticks), built once per pair of plans and kept in plan_kq.
int ensure_xfer(pwk_plan* pq, const pwk_plan* pk) {
  if (pq->xfer_src == pk) return PWK_OK;
  if (pq->xfer.d_nstick) {
    plan_free(pq, pq->xfer.d_nstick);
    plan_free(pq, pq->xfer.d_gin);
    plan_free(pq, pq->xfer.d_gout);
    plan_free(pq, pq->xfer.d_sid);
    pq->xfer = SphereMap();
    pq->xfer_src = nullptr;
  }
  int rc = build_sphere_map(pq, pq->xfer, pq->nk, pk->h_npw.data(), pk->npw_max, pk->h_miller.data(),
                            pq->h_npw.data(), pq->npw_max, pq->h_miller.data(), pk->d_npw, pq->d_npw);
  if (rc) return rc;
  pq->xshape = choose_shape(pq->N, 16, pq->xfer, 1);
  if (pq->xshape.smem > 227 * 1024) {
    set_error("transfer kernel does not fit in shared memory");
    return PWK_ERR_UNSUPPORTED;
  }
  pq->xfer_src = pk;
  return PWK_OK;
}

static int nblk(size_t n, int t = 256) { return (int)((n + t - 1) / t); }

#define KCK(what)                                      \
  do {                                                 \
    cudaError_t e_ = cudaGetLastError();               \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

}  // namespace pwk

using namespace pwk;

extern "C" int pwk_sternheimer_cg_batched(pwk_plan* pq, pwk_plan* pk, int mode, const void* psi_k_v,
                                          const double* eps_k, const void* psi_kq_v, int nocc,
                                          const double* alpha, const void* dv_r, void* dpsi_v,
                                          double tol, int max_iter, int* iters_out,
                                          double* resid_out, void* stream) {
  if (pq == nullptr || pk == nullptr || psi_k_v == nullptr || eps_k == nullptr ||
      psi_kq_v == nullptr || alpha == nullptr || dv_r == nullptr || dpsi_v == nullptr ||
      nocc < 1 || !(tol > 0.0) || max_iter < 1) {
    set_error("null pointer, nocc < 1, tol <= 0 or max_iter < 1");
    return PWK_ERR_INVALID;
  }
  if (mode != PWK_FP64 && mode != PWK_FP32_C128) {
    set_error("mode must be PWK_FP64 or PWK_FP32_C128");
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
  if ((rc = ensure_cg_work(pq, nocc, mode == PWK_FP32_C128))) return rc;
  CgWork* w = pq->cg;
  const int nk = pq->nk, np = pq->npw_max, npairs = nk * nocc;
  const double2* psi_kq = static_cast<const double2*>(psi_kq_v);
  double2* x = static_cast<double2*>(dpsi_v);
  int hc[2] = {0, 0};
  auto read_counters = [&]() -> int {
    cudaError_t e = cudaMemcpyAsync(hc, w->counters, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? PWK_OK : cuda_fail(e, "cg counters");
  };

  // ---- right-hand side: w = dV psi_k on the k+q sphere (into t), b = -(w - P_v w)
  {
    FusedArgs a;
    a.in = psi_k_v;
    a.out = w->t;
    a.nvec_in = a.nvec_out = nocc;
    a.nk = nk;
    a.npw_in_max = pk->npw_max;
    a.npw_out_max = np;
    a.npw_in = pk->d_npw;
    a.npw_out = pq->d_npw;
    a.nstick = pq->xfer.d_nstick;
    a.gin = pq->xfer.d_gin;
    a.gout = pq->xfer.d_gout;
    a.sid = pq->xfer.d_sid;
    a.nstick_max = pq->xfer.nstick_max;
    a.m1lo = pq->xfer.m1lo;
    a.P = pq->xfer.P;
    a.L = pq->xshape.L;
    a.zs = (pq->N % 2 == 0) ? pq->N + 1 : pq->N;
    a.V = dv_r;
    a.scale = 1.0 / (double)pq->Nr;
    a.err = pq->d_err;
    if ((rc = launch_fused_xfer(pq->N, a, npairs, pq->xshape, st))) return rc;
  }
  // S psi_{k+q,v} (FP64) when the plan has q; the H output of that call is not used
  const double2* su = psi_kq;
  const bool with_s = pq->d_q != nullptr;   // this call applies S (the workspace may hold more)
  if (with_s) {
    cg_items_kernel<<<nblk(npairs), 256, 0, st>>>(npairs, nocc, nullptr, w->items); note_launch();
    if ((rc = run_hpsi(pq, PWK_FP64, psi_kq, w->r, w->items, nullptr, npairs, nocc, nocc, st, w->su)))
      return rc;
    su = w->su;
  }
  double2* const sx = with_s ? w->sx : nullptr;   // S applied to the operand of A
  // one warp per valence vector for the projections mu_v (8 to 16 warps)
  const int pc_threads = 32 * std::min(std::max(nocc, 8), 16);
  proj_combine_kernel<double><<<npairs, pc_threads, 0, st>>>(nocc, np, pq->d_npw, nullptr, psi_kq, su, nullptr, w->t,
                                              nullptr, 0, nullptr, 0, nullptr, w->b, w->bnorm); note_launch();
  tkin_kernel<<<npairs, 256, 0, st>>>(nocc, np, pq->d_npw, pq->d_g2, psi_kq, w->tkin); note_launch();
  cudaMemsetAsync(w->iters, 0, sizeof(int) * npairs, st);
  cudaMemsetAsync(w->seen, 0, sizeof(int) * npairs, st);
  cudaMemsetAsync(x, 0, sizeof(double2) * (size_t)npairs * np, st);
  KCK("sternheimer setup");

  PhaseTimer T(pq, st);   // pwk_plan_set_solver_timing (H applications inside the CG)
  const size_t upd_smem = cg_update_smem(np);
  const bool fused_step = upd_smem <= kCgUpdateMaxSmem;
  // mixed mode: the inner solves on FP32 vectors (fused step only)
  const size_t upd32_smem = (size_t)3 * np * sizeof(float2);
  const bool inner32 = fused_step && mode == PWK_FP32_C128;
  if (inner32 && upd32_smem > 48 * 1024) {
    cudaError_t e = allow_full_smem(cg_update32_kernel);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(cg_update32)");
  }
  if (fused_step && upd_smem > 48 * 1024) {
    cudaError_t e = allow_full_smem(cg_update_kernel);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(cg_update)");
  }
  const int inner_prec = (mode == PWK_FP64) ? PWK_FP64 : PWK_FP32_C128;
  const double eta = (mode == PWK_FP64) ? 0.0 : 1e-6;
  // The iteration aims at half the requested residual: an FP64 operator that rounds
  // differently (another library, a dense matrix) then still finds ||A x - b|| <= tol ||b||;
  // the count returned and resid_out are measured against tol itself.
  const double tol_in = 0.5 * tol;
  // FP64 H x, S x and the true residual for the pairs whose x changed since their last one
  // (a compact list; the launches cover every pair and read the list's length on the device)
  auto true_residual = [&](double tol_r, double eta_r) -> int {
    stale_compact_kernel<<<nblk(npairs), 256, 0, st>>>(npairs, nocc, w->iters, w->seen, w->list, w->items,
                                                       w->counters); note_launch();
    cudaEvent_t th = T.mark();
    int r2 = run_hpsi(pq, PWK_FP64, x, w->t, w->items, w->counters + 2, npairs, nocc, nocc, st, sx);
    if (r2) return r2;
    T.close(0, th);
    true_residual_kernel<<<npairs, pc_threads, 0, st>>>(nocc, np, pq->d_npw, w->list, w->counters + 2, su, su,
                                                        w->t, x, sx, eps_k, alpha, w->b, w->bnorm, tol_r,
                                                        eta_r, w->r, w->rnorm, w->thr, w->active, w->first,
                                                        w->counters); note_launch();
    return PWK_OK;
  };
  if (fused_step && inner_prec != PWK_FP64) {
    const size_t nvv = (size_t)nk * nocc * np;
    to_c64_kernel<<<std::min<size_t>(nblk(nvv), 4 * 1024), 256, 0, st>>>(nvv, su, w->v32); note_launch();
  }
  bool x_zero = true;
  for (int outer = 0; outer < 8; ++outer) {
    cudaMemsetAsync(w->counters, 0, 4 * sizeof(int), st);
    if (x_zero) {
      residual_kernel<<<npairs, 256, 0, st>>>(nocc, np, pq->d_npw, nullptr, w->b, w->bnorm, tol_in, eta,
                                              w->r, w->rnorm, w->thr, w->active, w->first, w->counters); note_launch();
    } else {
      // the true residual of the pairs whose x changed in the last inner solve (the others
      // keep theirs: converged, or stopped by a breakdown at their first step)
      if ((rc = true_residual(tol_in, eta))) return rc;
    }
    KCK("sternheimer residual");
    if ((rc = read_counters())) return rc;
    T.harvest();
    if (hc[0] == 0) break;
    x_zero = false;
    if (inner32) {
      // mixed mode: the inner solve on the FP32 correction e (A e = -r), then x += e
      cudaMemsetAsync(w->counters, 0, 4 * sizeof(int), st);
      cg_init32_kernel<<<npairs, 256, 0, st>>>(nocc, np, pq->d_npw, pq->d_g2, w->tkin, w->r, w->e32, w->r32,
                                              w->d32, w->rho, w->thr, w->active, w->counters); note_launch();
      KCK("cg_init32_kernel");
      if ((rc = read_counters())) return rc;
      T.harvest();
      for (int it = 0; it < max_iter && hc[0] > 0;) {
        const int nact = hc[0];   // pairs with a direction at the last read: an upper bound after it
        for (int b = 0; b < kCgBurst && it < max_iter; ++b, ++it) {
          cudaMemsetAsync(w->counters, 0, 4 * sizeof(int), st);
          cg_compact_kernel<<<nblk(npairs), 256, 0, st>>>(npairs, nocc, w->active, w->list, w->items,
                                                          w->counters); note_launch();
          cudaEvent_t th = T.mark();
          if ((rc = run_hpsi(pq, PWK_FP32, w->d32, w->t32, w->items, w->counters + 2, nact, nocc, nocc, st,
                             with_s ? w->sd32 : nullptr)))
            return rc;
          T.close(0, th);
          cg_update32_kernel<<<nact, pc_threads, upd32_smem, st>>>(nocc, np, pq->d_npw, w->list, w->counters + 2,
                                                                   pq->d_g2, w->tkin, w->v32, w->t32, w->d32,
                                                                   with_s ? w->sd32 : nullptr, eps_k, alpha, w->e32,
                                                                   w->r32, w->rho, w->thr, w->active, w->iters,
                                                                   w->counters); note_launch();
          KCK("cg_update32_kernel");
        }
        if ((rc = read_counters())) return rc;
        T.harvest();
      }
      add_correction_kernel<<<npairs, 256, 0, st>>>(nocc, np, pq->d_npw, w->e32, x); note_launch();
      KCK("add_correction_kernel");
      continue;
    }
    // the first direction of this inner solve: d = M^-1 r (cg_dir_kernel)
    cudaMemsetAsync(w->counters, 0, 4 * sizeof(int), st);
    cg_dir_kernel<<<npairs, 256, 0, st>>>(nocc, np, pq->d_npw, pq->d_g2, w->tkin, w->r, w->d, w->dold,
                                          w->rho, w->rho_old, w->thr, w->active, w->first, w->counters); note_launch();
    KCK("cg_dir_kernel");
    if ((rc = read_counters())) return rc;
    T.harvest();
    for (int it = 0; it < max_iter && hc[0] > 0;) {
      const int nact = hc[0];   // pairs with a direction at the last read: an upper bound after it
      if (fused_step) {
        // one pass per pair and iteration: the active pairs compacted, H (and S) applied to
        // their directions, then the fused CG step that also forms the next direction.  Up to
        // kCgBurst iterations run between two reads of the counters (pairs only leave the
        // active set, so nact bounds every list of the burst; the launches read its current
        // length on the device)
        for (int b = 0; b < kCgBurst && it < max_iter; ++b, ++it) {
          cudaMemsetAsync(w->counters, 0, 4 * sizeof(int), st);
          cg_compact_kernel<<<nblk(npairs), 256, 0, st>>>(npairs, nocc, w->active, w->list, w->items,
                                                          w->counters); note_launch();
          cudaEvent_t th = T.mark();
          if ((rc = run_hpsi(pq, inner_prec, w->d, w->t, w->items, w->counters + 2, nact, nocc, nocc, st, sx)))
            return rc;
          T.close(0, th);
          // FP64 mode (the mixed mode's inner solves take the FP32 path above)
          cg_update_kernel<<<nact, pc_threads, upd_smem, st>>>(nocc, np, pq->d_npw, w->list, pq->d_g2,
                w->tkin, su, w->t, w->d, sx, eps_k, alpha, x, w->r, w->rho, w->thr, w->active, w->iters,
                w->counters, w->counters + 2); note_launch();
          KCK("cg_update_kernel");
        }
      } else {
        // spheres too large for the fused step: A d, the step and the next direction apart
        ++it;
        cudaMemsetAsync(w->counters, 0, 4 * sizeof(int), st);
        cg_items_kernel<<<nblk(npairs), 256, 0, st>>>(npairs, nocc, w->active, w->items); note_launch();
        cudaEvent_t th = T.mark();
        if ((rc = run_hpsi(pq, inner_prec, w->d, w->t, w->items, nullptr, npairs, nocc, nocc, st, sx)))
          return rc;
        T.close(0, th);
        if (inner_prec == PWK_FP64)
          { proj_combine_kernel<double><<<npairs, pc_threads, 0, st>>>(nocc, np, pq->d_npw, w->active, su, su, w->t,
                                                              w->d, sx, 1, eps_k, 1, alpha, w->t, nullptr); note_launch(); }
        else
          { proj_combine_kernel<float><<<npairs, pc_threads, 0, st>>>(nocc, np, pq->d_npw, w->active, su, su, w->t,
                                                             w->d, sx, 1, eps_k, 1, alpha, w->t, nullptr); note_launch(); }
        cg_step_kernel<<<npairs, 256, 0, st>>>(nocc, np, pq->d_npw, w->active, w->d, w->t, x, w->r, w->dold,
                                               w->rho, w->rho_old, w->iters, w->counters); note_launch();
        cudaMemsetAsync(w->counters, 0, sizeof(int), st);
        cg_dir_kernel<<<npairs, 256, 0, st>>>(nocc, np, pq->d_npw, pq->d_g2, w->tkin, w->r, w->d, w->dold,
                                              w->rho, w->rho_old, w->thr, w->active, w->first, w->counters); note_launch();
        KCK("cg_step_kernel");
      }
      if ((rc = read_counters())) return rc;
      T.harvest();
    }
  }
  // final true residual with the FP64 operator, for the pairs whose x changed since their
  // last one (the others' rnorm is that of their current x already)
  cudaMemsetAsync(w->counters, 0, 4 * sizeof(int), st);
  {
    if ((rc = true_residual(tol, 0.0))) return rc;
    KCK("sternheimer final residual");
    std::vector<double> h_rn(npairs);
    std::vector<int> h_it(npairs);
    cudaError_t e = cudaMemcpyAsync(h_rn.data(), w->rnorm, sizeof(double) * npairs, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_it.data(), w->iters, sizeof(int) * npairs, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "sternheimer results");
    T.finish();
    if (resid_out) std::memcpy(resid_out, h_rn.data(), sizeof(double) * npairs);
    if (iters_out) std::memcpy(iters_out, h_it.data(), sizeof(int) * npairs);
    int above = 0;
    for (double v : h_rn) above += (v > tol);
    return above;
  }
}
