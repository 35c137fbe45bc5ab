// Batched generalized Hermitian eigensolver for the Davidson reduced problem (paper Sec. 5):
//   H~ v = eps S~ v,   n = N_base <= 160,   lowest nb eigenpairs, one CTA per k-point, FP64.
//
// The paper runs LAPACK ZHEGV(X) converted to device routines, one thread per k, with a
// non-recursive Cholesky (ZPOTRF2 rewritten).  Here a whole CTA works on one k:
//   1. Cholesky S~ = L L^H (right-looking, column by column, lower triangle only);
//   2. C = L^-1 H~ L^-H: X = L^-1 H~ by forward substitution (one thread per column), then
//      the lower triangle of C = X L^-H by row-wise substitution (one thread per row);
//   3. Householder reduction of C to a real symmetric tridiagonal T = Q^H C Q
//      (reflectors H = I - tau v v^H, beta real, two-sided rank-2 updates of the lower
//      triangle);
//   4. the nb lowest eigenvalues of T from Sturm counts (a bracket narrowed by bisection in
//      FP32, confirmed by two FP64 counts, then safeguarded Newton steps on det(T - x) in
//      FP64 down to two ulp of |T|) and their eigenvectors by inverse iteration on T (one
//      thread per cluster of close eigenvalues, clusters in parallel; the members of a
//      cluster reorthogonalised inside the iteration);
//   5. back-transform x = L^-H Q z (reflectors applied in reverse order, then the triangular
//      solve column by column; a few lanes of one warp per vector).
// All matrices live in a per-k global workspace (L2-resident while the CTA works on it).
// The kernel is bound by the FP64 pipe (1/64 of the FP32 rate on this GPU) when the batch
// is full, so the loops count FP64 instructions: fused multiply-add chains (4 per complex
// multiply-add), triangles visited without masked lanes, reciprocal pivots formed once,
// reductions of the reflector step done by one warp.
// A dependent vector among the first nb (pivot below 1e-6 of its diagonal) marks the k-point
// with status PWK_ERR_NOT_POSDEF; a non-finite eigenvector, or eigenvectors of T that are not
// orthonormal to 1e-8, mark it PWK_ERR_NUMERIC.
#include <cmath>

#include "solvers.h"

namespace pwk {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
// accumulate with two fused multiply-adds per real component (4 FP64 instructions per
// complex multiply-add)
__device__ __forceinline__ void cfma(double2& s, double2 a, double2 b) {   // s += a b
  s.x = fma(a.x, b.x, s.x);
  s.x = fma(-a.y, b.y, s.x);
  s.y = fma(a.x, b.y, s.y);
  s.y = fma(a.y, b.x, s.y);
}
__device__ __forceinline__ void cfma_c(double2& s, double2 a, double2 b) {   // s += a conj(b)
  s.x = fma(a.x, b.x, s.x);
  s.x = fma(a.y, b.y, s.x);
  s.y = fma(a.y, b.x, s.y);
  s.y = fma(-a.x, b.y, s.y);
}
__device__ __forceinline__ void cfms(double2& s, double2 a, double2 b) {   // s -= a b
  s.x = fma(-a.x, b.x, s.x);
  s.x = fma(a.y, b.y, s.x);
  s.y = fma(-a.x, b.y, s.y);
  s.y = fma(-a.y, b.x, s.y);
}
__device__ __forceinline__ void cfms_c(double2& s, double2 a, double2 b) {   // s -= a conj(b)
  s.x = fma(-a.x, b.x, s.x);
  s.x = fma(-a.y, b.y, s.x);
  s.y = fma(-a.y, b.x, s.y);
  s.y = fma(a.x, b.y, s.y);
}

// Visit every (r, c) with 0 <= c <= r < m once, spread over the block: rows p and m-1-p are
// paired (p + 1 and m - p entries, m + 1 together), so the flat index runs over
// ceil(m/2) (m + 1) slots and the triangle masks off no lane.  Threads step their (p, o)
// position by the block size without dividing.
template <class F>
__device__ __forceinline__ void for_lower(int m, int tid, int nth, F f) {
  const int w = m + 1, total = ((m + 1) >> 1) * w;
  if (tid >= total) return;
  int p = tid / w, o = tid - p * w;
  const int dp = nth / w, dq = nth - dp * w;
  for (int i = tid; i < total; i += nth) {
    if (o <= p) f(p, o);
    else if (m - 1 - p != p) f(m - 1 - p, o - p - 1);
    p += dp;
    o += dq;
    if (o >= w) {
      o -= w;
      ++p;
    }
  }
}

// block-wide sum of a double (all threads get the result)
__device__ double block_sum(double v, double* red) {
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
__device__ double2 block_sum2(double2 v, double* red) {
  return make_double2(block_sum(v.x, red), block_sum(v.y, red));
}

// Rayleigh-Ritz of every active k (active[k] != 0).
// Hr, Sr: [nk][ld][ld] (row-major, full Hermitian in the leading n x n block)
// W: [nk][3][ld][ld] workspace; ev: [nk][ld][nb]; eps: [nk][nb]; status [nk]
// nbase == nullptr: every problem has size ld.  status may be null (not written).
// drop_out: [nk][ld] dependent-vector flags of the Cholesky step, or null.
__global__ void __launch_bounds__(256) rr_kernel(int nk, int ld, int nb, const int* nbase,
                                                 const int* active, const double2* Hr,
                                                 const double2* Sr, double2* W, double2* ev,
                                                 double* eps, int* status, unsigned char* drop_out,
                                                 double* flops) {
  const int k = blockIdx.x;
  if (k >= nk || (active != nullptr && !active[k])) return;
  const int n = nbase != nullptr ? nbase[k] : ld;
  const int tid = threadIdx.x, nth = blockDim.x;
  // algorithmic FP64 operation count of this problem (real flops, 8 per complex multiply-add):
  // Cholesky n^3/6, L^-1 H L^-H 2n^3/3, tridiagonalisation 2n^3/3, back-transform 3n^2 nb/2
  // complex multiply-adds
  if (flops != nullptr && tid == 0) atomicAdd(flops, 12.0 * n * n * n + 12.0 * n * n * nb);
  __shared__ double red[32];
  __shared__ double d[kMaxBasis], e[kMaxBasis], rc[kMaxBasis], rs[kMaxBasis];
  __shared__ double2 tau[kMaxBasis], vv[kMaxBasis], ww[kMaxBasis];
  __shared__ double lam[kMaxBasis];
  __shared__ int flag;
  __shared__ unsigned char dropped[kMaxBasis];
  const size_t ldsq = (size_t)ld * ld;
  const double2* H = Hr + k * ldsq;
  const double2* S = Sr + k * ldsq;
  double2* Lm = W + 3 * k * ldsq;     // Cholesky factor (lower), row-major
  double2* X = Lm + ldsq;             // L^-1 H, then Z (real, column-major)
  double2* C = X + ldsq;              // L^-1 H L^-H, then Householder vectors
  if (tid == 0) flag = 0;
  // ---- 1. Cholesky of S (lower).  A basis vector whose pivot falls below 1e-6 of its S~
  //      diagonal (new direction below 1e-3 of its norm) is numerically dependent on the
  //      earlier ones: it is dropped (its row and column of L become e_j and it is decoupled
  //      from the reduced problem below).  The bound sits far above the rounding noise of the
  //      Schur complement of an exactly dependent vector (seen up to 4e-8 when the earlier
  //      basis is itself ill-conditioned), which a smaller bound can mistake for a new
  //      direction and turn into a spurious Ritz value.
  //      Only the lower triangle of S and L is read or written.
  for (int i = tid; i < n * n; i += nth) {
    const int r = i / n, c = i - r * n;
    if (c <= r) Lm[r * ld + c] = S[r * ld + c];
  }
  for (int i = tid; i < n; i += nth) dropped[i] = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      const double p = Lm[j * ld + j].x;
      const bool drop = !(p > 1e-6 * S[j * ld + j].x);
      dropped[j] = drop ? 1 : 0;
      if (drop && j < nb) flag = 1;   // the leading nb vectors must be independent
      const double l = drop ? 1.0 : sqrt(p);
      Lm[j * ld + j] = make_double2(l, 0.0);
      rc[j] = 1.0 / l;
    }
    __syncthreads();
    const int m = n - j - 1;
    if (dropped[j]) {
      for (int r = j + 1 + tid; r < n; r += nth) Lm[r * ld + j] = make_double2(0.0, 0.0);
      for (int q = tid; q < j; q += nth) Lm[j * ld + q] = make_double2(0.0, 0.0);
      __syncthreads();
      continue;
    }
    const double ipiv = rc[j];
    for (int r = tid; r < m; r += nth) {
      double2 v = Lm[(j + 1 + r) * ld + j];
      v = make_double2(v.x * ipiv, v.y * ipiv);
      Lm[(j + 1 + r) * ld + j] = v;
      vv[r] = v;
    }
    __syncthreads();
    // trailing update of the lower triangle: L[r][c] -= L[r][j] conj(L[c][j]), c <= r
    double2* L22 = Lm + (size_t)(j + 1) * ld + (j + 1);
    for_lower(m, tid, nth, [&](int r, int c) { cfms_c(L22[r * ld + c], vv[r], vv[c]); });
    __syncthreads();
  }
  if (drop_out != nullptr)
    for (int i = tid; i < n; i += nth) drop_out[(size_t)k * ld + i] = dropped[i];
  if (flag) {
    if (tid == 0 && status != nullptr) status[k] = PWK_ERR_NOT_POSDEF;
    return;
  }
  // ---- 2. X = L^-1 H (forward substitution, one column of H per thread), then the lower
  //      triangle of C = X L^-H row by row: row r of C solves C[r][:] L^H = X[r][:], and its
  //      entries c <= r need only the entries before them, so the lower triangle costs n^3/6
  //      complex multiply-adds instead of the n^3/2 of a full solve.  The inverse diagonal of
  //      L (rc) was formed once by the Cholesky step.
  for (int c = tid; c < n; c += nth) {
    for (int r = 0; r < n; ++r) {
      double2 s = H[r * ld + c];
      const double2* lr = Lm + (size_t)r * ld;
      for (int q = 0; q < r; ++q) cfms(s, lr[q], X[q * ld + c]);
      const double il = rc[r];
      X[r * ld + c] = make_double2(s.x * il, s.y * il);
    }
  }
  __syncthreads();
  for (int r = tid; r < n; r += nth) {
    const double2* xr = X + (size_t)r * ld;
    double2* cr = C + (size_t)r * ld;
    for (int c = 0; c <= r; ++c) {
      double2 s = xr[c];
      const double2* lc = Lm + (size_t)c * ld;
      for (int q = 0; q < c; ++q) cfms_c(s, cr[q], lc[q]);   // s -= C[r][q] conj(L[c][q])
      const double il = rc[c];
      cr[c] = make_double2(s.x * il, c == r ? 0.0 : s.y * il);   // C is Hermitian: real diagonal
    }
  }
  __syncthreads();
  // dropped vectors: decouple their row/column and park their eigenvalue above the spectrum
  // (||C||_F from the lower triangle)
  {
    double f = 0.0;
    for_lower(n, tid, nth, [&](int r, int c) {
      const double2 v = C[r * ld + c];
      f += (r == c ? 1.0 : 2.0) * (v.x * v.x + v.y * v.y);
    });
    f = block_sum(f, red);
    const double big = 4.0 * sqrt(f) + 1.0;
    for_lower(n, tid, nth, [&](int r, int c) {
      if (dropped[r] || dropped[c]) C[r * ld + c] = make_double2(r == c ? big : 0.0, 0.0);
    });
    __syncthreads();
  }
  // ---- 3. Householder tridiagonalisation of the Hermitian C held in its lower triangle;
  //      v_j stored in C[j+1..n-1][j] with v[0] = 1.  Per step: the reflector (warp 0), the
  //      product w = tau C22 v (one row per thread, the upper half read through the lower
  //      triangle), the correction w += alpha2 v (warp 0), and the rank-2 update of the lower
  //      triangle of C22.
  for (int j = 0; j + 1 < n; ++j) {
    const int m = n - j - 1;       // length of x = C[j+1..n-1][j]
    if (tid < 32) {
      double xn2 = 0.0;
      for (int i = 1 + tid; i < m; i += 32) {
        const double2 v = C[(j + 1 + i) * ld + j];
        vv[i] = v;
        xn2 = fma(v.x, v.x, fma(v.y, v.y, xn2));
      }
      for (int o = 16; o > 0; o >>= 1) xn2 += __shfl_xor_sync(0xffffffffu, xn2, o);
      const double2 alpha = C[(j + 1) * ld + j];
      double2 t = make_double2(0.0, 0.0);
      double beta = alpha.x;
      if (xn2 > 0.0 || alpha.y != 0.0) {
        const double nrm = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn2);
        beta = alpha.x >= 0.0 ? -nrm : nrm;
        const double ib = 1.0 / beta;
        t = make_double2((beta - alpha.x) * ib, -alpha.y * ib);
        // u = x / (alpha - beta)
        const double2 den = make_double2(alpha.x - beta, alpha.y);
        const double idd = 1.0 / (den.x * den.x + den.y * den.y);
        const double2 inv = make_double2(den.x * idd, -den.y * idd);
        for (int i = 1 + tid; i < m; i += 32) {
          const double2 u = cmul(vv[i], inv);
          vv[i] = u;
          C[(j + 1 + i) * ld + j] = u;
        }
      }
      __syncwarp();   // every lane has read alpha before it is overwritten
      if (tid == 0) {
        tau[j] = t;
        e[j] = beta;
        d[j] = C[j * ld + j].x;
        C[(j + 1) * ld + j] = make_double2(1.0, 0.0);   // v[0] = 1
        vv[0] = make_double2(1.0, 0.0);
      }
    }
    __syncthreads();
    const double2 t = tau[j];
    if (t.x == 0.0 && t.y == 0.0) continue;   // uniform across the block
    // w = tau * C22 v  (C22 = C[j+1.., j+1..], Hermitian, lower triangle stored)
    const double2* C22 = C + (size_t)(j + 1) * ld + (j + 1);
    for (int r = tid; r < m; r += nth) {
      double2 s = make_double2(0.0, 0.0);
      const double2* row = C22 + (size_t)r * ld;
      for (int q = 0; q <= r; ++q) cfma(s, row[q], vv[q]);
      for (int q = r + 1; q < m; ++q) cfma_c(s, vv[q], C22[(size_t)q * ld + r]);   // conj(C[q][r]) v_q
      ww[r] = cmul(t, s);
    }
    __syncthreads();
    // alpha2 = -1/2 tau (w^H v); w += alpha2 v
    if (tid < 32) {
      double2 dot = make_double2(0.0, 0.0);
      for (int r = tid; r < m; r += 32) cfma_c(dot, vv[r], ww[r]);   // conj(w_r) v_r
      for (int o = 16; o > 0; o >>= 1) {
        dot.x += __shfl_xor_sync(0xffffffffu, dot.x, o);
        dot.y += __shfl_xor_sync(0xffffffffu, dot.y, o);
      }
      const double2 a2 = cmul(make_double2(-0.5 * t.x, -0.5 * t.y), dot);
      for (int r = tid; r < m; r += 32) cfma(ww[r], a2, vv[r]);
    }
    __syncthreads();
    // C22 -= v w^H + w v^H  (lower triangle)
    double2* C22w = C + (size_t)(j + 1) * ld + (j + 1);
    for_lower(m, tid, nth, [&](int r, int c) {
      double2& x = C22w[r * ld + c];
      cfms_c(x, vv[r], ww[c]);
      cfms_c(x, ww[r], vv[c]);
      if (r == c) x.y = 0.0;   // Hermitian: real diagonal
    });
    __syncthreads();
  }
  if (tid == 0) {
    d[n - 1] = C[(n - 1) * ld + (n - 1)].x;
    e[n - 1] = 0.0;
  }
  __syncthreads();
  // ---- 4. the nb lowest eigenpairs of the real tridiagonal T = (d, e): bisection on Sturm
  //      counts for the eigenvalues (one thread per eigenvalue: the threads of a warp work in
  //      lockstep, so every FP64 instruction serves up to 32 eigenvalues), then inverse
  //      iteration for the eigenvectors.
  double* e2 = rs;
  __shared__ double glo, ghi, pivmin, tiny, werr, atol;
  __shared__ float d32[kMaxBasis], e232[kMaxBasis];
  __shared__ float pivmin32;
  __shared__ int use32;
  if (tid == 0) {
    double lo = 1e300, hi = -1e300, emax = 0.0, dmax = 0.0;
    for (int i = 0; i < n; ++i) {
      const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
      lo = fmin(lo, d[i] - r);
      hi = fmax(hi, d[i] + r);
      dmax = fmax(dmax, fabs(d[i]));
      if (i + 1 < n) {
        e2[i] = e[i] * e[i];
        emax = fmax(emax, e2[i]);
      }
    }
    const double span = fmax(fabs(lo), fabs(hi));
    glo = lo - 1e-14 * span - 1e-300;
    ghi = hi + 1e-14 * span + 1e-300;
    pivmin = 1e-290 * fmax(1.0, emax);
    tiny = 2.2e-16 * fmax(1.0, fmax(dmax, sqrt(emax)));
    // absolute accuracy of the eigenvalues: two units in the last place of the Gershgorin
    // bound of |T| (a Sturm count is backward stable, so no bracket narrower than a few
    // ulp(|T|) is meaningful; a bound relative to |lambda| alone never ends for lambda ~ 0)
    atol = 4.4e-16 * span;
    // FP32 Sturm counts are exact for a T perturbed by at most u32 (2 dmax + |x| + 9 max|e|)
    // (u32 = 2^-24: rounding of d, e^2 to FP32 and of each step of the recurrence, whose
    // division is the fast one, within 2 ulp), so an FP32 bracket widened by werr (8 times
    // that bound, |x| <= dmax + 2 max|e|) holds the eigenvalue; the FP64 counts confirm it
    // before it is used.
    werr = 4.8e-7 * (3.0 * dmax + 11.0 * sqrt(emax));
    use32 = dmax < 1e15 && emax < 1e28;
    pivmin32 = (float)(1e-30 * fmax(1.0, emax));
  }
  __syncthreads();
  if (use32)
    for (int i = tid; i < n; i += nth) {
      d32[i] = (float)d[i];
      e232[i] = i + 1 < n ? (float)e2[i] : 0.0f;
    }
  __syncthreads();
  // bisection, one thread per eigenvalue (threads of a warp in lockstep, so every FP64
  // instruction serves up to 32 eigenvalues); FP64 throughput, not latency, bounds this
  // kernel when the batch is full, so the Sturm counts are not multiplied across threads.
  // count(x) = number of eigenvalues below x (Sturm sequence of the LDL^T factorisation of
  // T - x).  The bracket is first narrowed in FP32 (64 times the FP64 rate) down to werr;
  // the FP64 stage then starts from that bracket widened by werr on both sides.
  auto count64 = [&](double x) {
    double q = d[0] - x;
    int cnt = q < 0.0;
    for (int i = 1; i < n; ++i) {
      if (fabs(q) < pivmin) q = -pivmin;
      q = d[i] - x - e2[i - 1] / q;
      cnt += q < 0.0;
    }
    return cnt;
  };
  // The same recurrence with its derivative: the count at x, and in s the logarithmic
  // derivative of det(T - x) = prod_i q_i, s = sum_i q_i' / q_i with
  // q_i' = -1 + e_{i-1}^2 q_{i-1}' / q_{i-1}^2, so that x - 1/s is the Newton step for det.
  auto count_newton = [&](double x, double& s) {
    double q = d[0] - x, dq = -1.0;
    int cnt = q < 0.0;
    if (fabs(q) < pivmin) q = -pivmin;
    double r = 1.0 / q;
    s = dq * r;
    for (int i = 1; i < n; ++i) {
      const double t = e2[i - 1] * r;   // e_{i-1}^2 / q_{i-1}
      dq = fma(t * r, dq, -1.0);
      q = (d[i] - x) - t;
      cnt += q < 0.0;
      if (fabs(q) < pivmin) q = -pivmin;
      r = 1.0 / q;
      s = fma(dq, r, s);
    }
    return cnt;
  };
  for (int j = tid; j < nb; j += nth) {
    double a = glo, b = ghi;
    int ca = 0, cb = n;   // counts at a and b
    if (use32) {
      float a32 = __double2float_rd(glo), b32 = __double2float_ru(ghi);
      const float w32 = (float)werr;
      for (int it = 0; it < 160; ++it) {
        const float mid = 0.5f * (a32 + b32);
        if (mid <= a32 || mid >= b32 || b32 - a32 <= w32) break;
        float q = d32[0] - mid;
        int cnt = q < 0.0f;
        for (int i = 1; i < n; ++i) {
          if (fabsf(q) < pivmin32) q = -pivmin32;
          q = d32[i] - mid - __fdividef(e232[i - 1], q);
          cnt += q < 0.0f;
        }
        if (cnt > j) b32 = mid;
        else a32 = mid;
      }
      const double a1 = fmax(glo, (double)a32 - werr), b1 = fmin(ghi, (double)b32 + werr);
      const int c1 = count64(a1), c2 = count64(b1);
      if (c1 <= j && c2 > j) {
        a = a1;
        b = b1;
        ca = c1;
        cb = c2;
      }
    }
    // FP64: safeguarded Newton on det(T - x).  Every pass counts at x and shrinks the bracket
    // to the side that keeps eigenvalue j; while the bracket holds eigenvalue j alone
    // (count(a) = j, count(b) = j + 1) the Newton step is taken if it lands inside it, else
    // (and for eigenvalues not yet separated from a neighbour) the bracket is bisected.  The
    // Newton iterates approach the eigenvalue from one side, so the far end of the bracket
    // stays where it was: once a step of rounding size (at most atol) points out of the
    // bracket (the last iterate, now one end of it, is within rounding of the eigenvalue) the
    // next count is taken atol inside that end, which closes the bracket to atol instead of
    // halving it from the far end; a larger step out of the bracket is replaced by a
    // bisection.  A separated eigenvalue takes two to five passes instead of the ~30 halvings
    // from werr down.
    double x = 0.5 * (a + b), lj = x;
    for (int it = 0; it < 200; ++it) {
      const double tol = atol + 2.0 * pivmin;
      if (b - a <= tol) {
        lj = 0.5 * (a + b);
        break;
      }
      double sd;
      const int c = count_newton(x, sd);
      if (c > j) {
        b = x;
        cb = c;
      } else {
        a = x;
        ca = c;
      }
      if (ca == j && cb == j + 1) {
        const double xn = x - 1.0 / sd;
        if (xn > a && xn < b) {
          lj = xn;
          if (fabs(xn - x) <= tol) break;
          x = xn;
          continue;
        }
        if (fabs(xn - x) <= tol) {   // a rounding-size step out of the bracket
          const double xi = x == a ? x + tol : x - tol;
          if (xi > a && xi < b) {
            x = xi;
            lj = x;
            continue;
          }
        }
      }
      x = 0.5 * (a + b);
      lj = x;
      if (x <= a || x >= b) break;
    }
    lam[j] = lj;
  }
  __syncthreads();
  double* XS = reinterpret_cast<double*>(X);   // x_j at XS + j n, pivots of T - lam_j at XS + (nb + j) n
  // Clusters: consecutive eigenvalues closer than ortol = 1e-3 max(1, |lam|) (the reorthogonalisation
  // criterion of inverse iteration, relative to the spectrum the nb eigenpairs span).  Each
  // cluster is handled by one thread in order: every iterate of a member is orthogonalised
  // against the members before it, inside the iteration; eigenvalues of a cluster closer than
  // eps3 are separated by eps3 before the LDL^T factorisation.  Clusters run in parallel.
  __shared__ int ncl, cl_start[kMaxBasis + 1];
  __shared__ double ortol, eps3;
  if (tid == 0) {
    const double scale = fmax(1.0, fmax(fabs(lam[0]), fabs(lam[nb - 1])));
    ortol = 1e-3 * scale;
    eps3 = 16.0 * 2.2e-16 * scale;
    int c = 0;
    cl_start[c++] = 0;
    for (int j = 1; j < nb; ++j)
      if (lam[j] - lam[j - 1] > ortol) cl_start[c++] = j;
    cl_start[c] = nb;
    ncl = c;
  }
  __syncthreads();
  for (int c = tid; c < ncl; c += nth) {
    double lprev = -1e300;
    for (int j = cl_start[c]; j < cl_start[c + 1]; ++j) {
      double* x = XS + (size_t)j * n;
      double* Dv = XS + (size_t)(nb + j) * n;
      double lj = lam[j];
      if (j > cl_start[c] && lj < lprev + eps3) lj = lprev + eps3;
      lprev = lj;
      // LDL^T of T - lj; Dv keeps 1/D (the solves below then multiply only)
      double D = d[0] - lj;
      if (fabs(D) < tiny) D = D < 0.0 ? -tiny : tiny;
      double iD = 1.0 / D;
      Dv[0] = iD;
      for (int i = 1; i < n; ++i) {
        D = d[i] - lj - e2[i - 1] * iD;
        if (fabs(D) < tiny) D = D < 0.0 ? -tiny : tiny;
        iD = 1.0 / D;
        Dv[i] = iD;
      }
      for (int i = 0; i < n; ++i) {   // start vector: a fixed pseudo-random pattern per (i, j)
        const unsigned h = (unsigned)(i + 1) * 2654435761u ^ (unsigned)(j + 1) * 2246822519u;
        x[i] = 0.5 + (double)(h >> 8) * (1.0 / 16777216.0);
      }
      for (int iter = 0; iter < 5; ++iter) {
        for (int i = 1; i < n; ++i) x[i] -= (e[i - 1] * Dv[i - 1]) * x[i - 1];   // L y = b
        x[n - 1] *= Dv[n - 1];                                                   // D z = y, L^T x = z
        for (int i = n - 2; i >= 0; --i) x[i] = (x[i] - e[i] * x[i + 1]) * Dv[i];
        for (int q = cl_start[c]; q < j; ++q) {   // modified Gram-Schmidt against the cluster
          const double* xq = XS + (size_t)q * n;
          double s2 = 0.0;
          for (int i = 0; i < n; ++i) s2 += xq[i] * x[i];
          for (int i = 0; i < n; ++i) x[i] -= s2 * xq[i];
        }
        double nn = 0.0;
        for (int i = 0; i < n; ++i) nn += x[i] * x[i];
        if (!(nn > 0.0) || !isfinite(nn)) {
          flag = 2;   // non-finite eigenvector: report, do not use
          break;
        }
        const double inv = 1.0 / sqrt(nn);
        for (int i = 0; i < n; ++i) x[i] *= inv;
      }
    }
  }
  __syncthreads();
  // guard: the nb vectors must be orthonormal; a loss (a cluster missed by the criterion)
  // is reported like a non-finite vector and the caller drops the step
  for (int pq = tid; pq < nb * nb && flag == 0; pq += nth) {
    const int a = pq / nb, b = pq - a * nb;
    if (b > a) continue;
    const double* xa = XS + (size_t)a * n;
    const double* xb = XS + (size_t)b * n;
    double s2 = 0.0;
    for (int i = 0; i < n; ++i) s2 += xa[i] * xb[i];
    if (!(fabs(s2 - (a == b ? 1.0 : 0.0)) < 1e-8)) flag = 2;
  }
  __syncthreads();
  if (flag == 2) {
    if (tid == 0 && status != nullptr) status[k] = PWK_ERR_NUMERIC;
    return;
  }
  // ---- 5. back-transform x = L^-H Q z of the selected vectors.  G lanes of one warp per
  //      vector (G = 8 for nb <= 32, fewer for more vectors); lane c of a group holds the rows
  //      r = c, c + G, c + 2G, ... of its vector, so a reflector on rows h+1..n-1 costs each
  //      lane about (n-h-1)/G row updates and a G-lane reduction, the triangular solve
  //      (column by column: x_r, then its share subtracted from the rows above) a broadcast
  //      and about r/G updates per row, and the vectors of a warp need no block barrier.
  for (int j = tid; j < nb; j += nth) eps[k * nb + j] = lam[j];
  double2* E = ev + (size_t)k * ld * nb;
  {
    const int G = nb <= nth / 8 ? 8 : nb <= nth / 4 ? 4 : nb <= nth / 2 ? 2 : 1;
    const int c = tid % G, lane = tid & 31, ngroups = nth / G;
    const int gbase = lane & ~(G - 1);   // lane of c = 0 in this group (G divides 32)
    auto first_row = [&](int lo) { return lo <= c ? c : c + G * ((lo - c + G - 1) / G); };
    for (int j0 = 0; j0 < nb; j0 += ngroups) {   // uniform trip counts: shuffles see every lane
      const int j = j0 + tid / G;
      const bool valid = j < nb;
      if (valid)
        for (int r = c; r < n; r += G) E[r * nb + j] = make_double2(XS[(size_t)j * n + r], 0.0);
      // y = H_0 H_1 ... H_{n-2} y : apply H_{n-2} first; H_h = I - tau_h v_h v_h^H
      for (int h = n - 2; h >= 0; --h) {
        const double2 th = tau[h];
        if (th.x == 0.0 && th.y == 0.0) continue;   // uniform across the block
        double2 sv = make_double2(0.0, 0.0);      // v^H y over rows h+1..n-1
        const int r0 = first_row(h + 1);
        if (valid)
          for (int r = r0; r < n; r += G) {
            const double2 v = C[r * ld + h], y = E[r * nb + j];
            sv.x = fma(v.x, y.x, fma(v.y, y.y, sv.x));
            sv.y = fma(v.x, y.y, fma(-v.y, y.x, sv.y));
          }
        for (int o = G >> 1; o > 0; o >>= 1) {
          sv.x += __shfl_xor_sync(0xffffffffu, sv.x, o);
          sv.y += __shfl_xor_sync(0xffffffffu, sv.y, o);
        }
        const double2 ts = cmul(th, sv);
        if (valid)
          for (int r = r0; r < n; r += G) {
            const double2 v = C[r * ld + h];
            double2 y = E[r * nb + j];
            y.x = fma(-v.x, ts.x, fma(v.y, ts.y, y.x));
            y.y = fma(-v.x, ts.y, fma(-v.y, ts.x, y.y));
            E[r * nb + j] = y;
          }
      }
      // x = L^-H y: x_r = y_r / L[r][r] from the last row up, then y_q -= conj(L[r][q]) x_r
      // for the rows q < r (L^H has conj(L[r][q]) in row q, column r)
      for (int r = n - 1; r >= 0; --r) {
        const int owner = r % G;
        double2 xr = make_double2(0.0, 0.0);
        if (valid && c == owner) {
          const double il = rc[r];
          const double2 y = E[r * nb + j];
          xr = make_double2(y.x * il, y.y * il);
          E[r * nb + j] = xr;
        }
        xr.x = __shfl_sync(0xffffffffu, xr.x, gbase + owner);
        xr.y = __shfl_sync(0xffffffffu, xr.y, gbase + owner);
        if (valid) {
          const double2* lr = Lm + (size_t)r * ld;
          for (int q = c; q < r; q += G) {
            const double2 l = lr[q];
            double2 y = E[q * nb + j];
            y.x = fma(-l.x, xr.x, fma(-l.y, xr.y, y.x));
            y.y = fma(-l.x, xr.y, fma(l.y, xr.x, y.y));
            E[q * nb + j] = y;
          }
        }
      }
    }
  }
  if (tid == 0 && status != nullptr) status[k] = PWK_OK;
}

int launch_rr(int nk, int ld, int nb, const int* nbase, const int* active, const double2* Hr,
              const double2* Sr, double2* W, double2* ev, double* eps, int* status,
              cudaStream_t st, unsigned char* drop_out, double* flops) {
  rr_kernel<<<nk, 256, 0, st>>>(nk, ld, nb, nbase, active, Hr, Sr, W, ev, eps, status, drop_out, flops); note_launch();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PWK_OK : cuda_fail(e, "rr_kernel");
}

}  // namespace pwk

using namespace pwk;

// Batched generalized Hermitian eigensolver as a library entry point (workspace allocated
// per call).
extern "C" int pwk_eigh_batched(int nprob, int n, int nev, const void* H, const void* S,
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
  if (nprob == 0) return PWK_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double2* W = nullptr;
  cudaError_t e = cudaMalloc(&W, sizeof(double2) * 3 * (size_t)n * n * nprob);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(eigh workspace)");
  int rc = launch_rr(nprob, n, nev, nullptr, nullptr, static_cast<const double2*>(H),
                     static_cast<const double2*>(S), W, static_cast<double2*>(vec), eig, status, st);
  e = cudaStreamSynchronize(st);
  cudaFree(W);
  if (rc) return rc;
  return e == cudaSuccess ? PWK_OK : cuda_fail(e, "eigh");
}
