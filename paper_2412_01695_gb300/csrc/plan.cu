// Plans: the per-k tables of a block of k-points kept resident on the device (paper Sec. 3:
// projectors and wave-function layout loaded for all N_k points before the solvers run),
// the sphere -> stick maps of the pruned transforms (Sec. 4), and the H|psi> entry points.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fft_line.cuh"
#include "nl_fused.cuh"
#include "pwk_internal.h"
#include "solvers.h"

namespace pwk {

static thread_local std::string g_detail;

void set_error(const std::string& msg) { g_detail = msg; }

namespace {
std::mutex g_smem_mu;
std::map<std::pair<const void*, int>, bool> g_smem_raised;
}  // namespace

bool smem_limit_raised(const void* kern, int dev) {
  std::lock_guard<std::mutex> lock(g_smem_mu);
  return g_smem_raised.count({kern, dev}) != 0;
}
void mark_smem_limit_raised(const void* kern, int dev) {
  std::lock_guard<std::mutex> lock(g_smem_mu);
  g_smem_raised[{kern, dev}] = true;
}

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int cuda_fail(cudaError_t e, const char* what) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  set_error(buf);
  return e == cudaErrorMemoryAllocation ? PWK_ERR_NOMEM : PWK_ERR_CUDA;
}

int plan_alloc(pwk_plan* p, void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 16;
  if (p->budget != 0 && p->bytes + bytes > p->budget) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "allocation of %zu bytes exceeds the plan budget (%zu of %zu used)",
                  bytes, p->bytes, p->budget);
    set_error(buf);
    return PWK_ERR_BUDGET;
  }
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return cuda_fail(e, "cudaMalloc");
  }
  p->bytes += bytes;
  p->allocs.push_back(*ptr);
  p->alloc_sizes.push_back(bytes);
  return PWK_OK;
}

void plan_free(pwk_plan* p, void* ptr) {
  if (ptr == nullptr) return;
  for (size_t i = 0; i < p->allocs.size(); ++i) {
    if (p->allocs[i] == ptr) {
      cudaFree(ptr);
      p->bytes -= p->alloc_sizes[i];
      p->allocs.erase(p->allocs.begin() + i);
      p->alloc_sizes.erase(p->alloc_sizes.begin() + i);
      return;
    }
  }
}

bool grid_supported(int N) {
  switch (N) {
#define PWK_CASE(n) case n:
    PWK_FOR_EACH_N(PWK_CASE)
#undef PWK_CASE
    return true;
    default:
      return false;
  }
}

size_t fused_smem_bytes(int N, int elem_bytes, int nstick_max, int P, int L, int npw_in_max) {
  const int zs = (N % 2 == 0) ? N + 1 : N;
  size_t elems = (size_t)nstick_max * zs + (size_t)P * N * L + npw_in_max;
  return elems * elem_bytes + (size_t)P * N * sizeof(short) + 16;
}

// The y pass maps thread t to (plane p = t % NW, column c = t / NW) and touches element
// p * (NW * zs) + c of the stick square and p * yps + c of the chunk buffer; the x pass maps t to
// (l2 = t / L, c = t % L) and touches p * yps + l2 * L + c.  With u = NW^-1 (mod 16) (NW is
// odd), NW * zs = yps = u (mod 16) makes every y-pass address u * t plus a constant (mod 16), and
// x-pass addresses are consecutive in t: the 16 eight-byte accesses of a half-warp fall on 32
// different banks in both passes.  zs = u^2 (mod 16) is odd, so the z pass (one stick row per
// thread) stays conflict-free for consecutive sticks as well.
void window_strides(int N, int L, int* zs, int* yps) {
  const int W = N / 4, NW = 2 * W + 1;
  int u = 1;
  while ((NW * u) % 16 != 1) ++u;
  const int z_res = (u * u) % 16;
  int z = N;
  while (z % 16 != z_res) ++z;
  *zs = z;
  int y = N * L;
  while (y % 16 != u) ++y;
  *yps = y;
}

size_t window_smem_bytes(int N, int elem_bytes, int L, int nstick_max, int copies) {
  const int W = N / 4, NW = 2 * W + 1;
  int zs, yps;
  window_strides(N, L, &zs, &yps);
  size_t elems = (size_t)NW * NW * zs + (size_t)copies * NW * yps;
  return elems * elem_bytes + (size_t)nstick_max * sizeof(short) + 16;
}

// ---------------------------------------------------------------- setup kernels
// |k+G|^2 (Ry) for every basis vector of every k (paper Sec. 2.2.1), zero padding.
__global__ void kinetic_table_kernel(int nk, int npw_max, const int* npw, const double* kc,
                                     const int* miller, const double* B, double* g2) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)nk * npw_max) return;
  const int k = (int)(i / npw_max), g = (int)(i % npw_max);
  if (g >= npw[k]) {
    g2[i] = 0.0;
    return;
  }
  const int* m = miller + 3 * i;
  double q[3];
  for (int c = 0; c < 3; ++c) q[c] = kc[3 * k + c] + m[0] * B[c] + m[1] * B[3 + c] + m[2] * B[6 + c];
  g2[i] = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
}

__global__ void to_f32_kernel(size_t n, const double* in, float* out) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}

// Vt[(l2 N + l3) N + l1] = V[(l1 N + l2) N + l3]: one x-line of the grid contiguous
template <typename T>
__global__ void transpose_v_kernel(int N, const double* V, T* Vt) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t n3 = (size_t)N * N * N;
  if (i >= n3) return;
  const int l1 = (int)(i % N), l3 = (int)((i / N) % N), l2 = (int)(i / ((size_t)N * N));
  Vt[i] = (T)V[((size_t)l1 * N + l2) * N + l3];
}

// sum of n values by one CTA in a fixed order (the result is the same on every run)
__global__ void sum_kernel(size_t n, const double* in, double* out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) s += in[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

static int blocks_for(size_t n, int t = 256) { return (int)((n + t - 1) / t); }

// ---------------------------------------------------------------- sphere maps
// Build the stick tables for input spheres (miller_in) and output spheres (miller_out).
int build_sphere_map(pwk_plan* p, SphereMap& sm, int nk, const int* npw_in, int npw_in_max,
                     const int* miller_in, const int* npw_out, int npw_out_max,
                     const int* miller_out, const int* d_npw_in, const int* d_npw_out) {
  const int N = p->N;
  const int half = (N - 1) / 2;
  int m1lo = N, m1hi = -N;
  auto check_range = [&](const int* mil, const int* npw, int npw_max) -> int {
    for (int k = 0; k < nk; ++k)
      for (int g = 0; g < npw[k]; ++g)
        for (int c = 0; c < 3; ++c) {
          const int m = mil[((size_t)k * npw_max + g) * 3 + c];
          if (m < -half || m > half) {  // strictly |m| < N/2: one grid slot per index
            char buf[160];
            std::snprintf(buf, sizeof(buf), "Miller index %d (k %d, G %d) outside |m| < N/2 = %d", m, k, g, N / 2);
            set_error(buf);
            return PWK_ERR_INVALID;
          }
          if (c == 0) {
            m1lo = std::min(m1lo, m);
            m1hi = std::max(m1hi, m);
          }
        }
    return PWK_OK;
  };
  int rc = check_range(miller_in, npw_in, npw_in_max);
  if (rc) return rc;
  rc = check_range(miller_out, npw_out, npw_out_max);
  if (rc) return rc;
  const int P = m1hi - m1lo + 1;
  std::vector<int> nstick(nk), gin((size_t)nk * npw_in_max, 0), gout((size_t)nk * npw_out_max, 0);
  std::vector<short> sid((size_t)nk * P * N, (short)-1);
  int nsmax = 0;
  auto wrap = [N](int m) { return ((m % N) + N) % N; };
  for (int k = 0; k < nk; ++k) {
    std::map<std::pair<int, int>, int> st;
    for (int pass = 0; pass < 2; ++pass) {
      const int* mil = pass ? miller_out : miller_in;
      const int nmax = pass ? npw_out_max : npw_in_max;
      const int n = pass ? npw_out[k] : npw_in[k];
      for (int g = 0; g < n; ++g) {
        const int* m = mil + ((size_t)k * nmax + g) * 3;
        st.emplace(std::make_pair(m[0], m[1]), 0);
      }
    }
    int s = 0;
    for (auto& kv : st) kv.second = s++;
    nstick[k] = s;
    nsmax = std::max(nsmax, s);
    if (s >= (1 << 23) || s > 32767) {
      set_error("too many z-sticks");
      return PWK_ERR_UNSUPPORTED;
    }
    for (auto& kv : st) sid[((size_t)k * P + (kv.first.first - m1lo)) * N + wrap(kv.first.second)] = (short)kv.second;
    for (int pass = 0; pass < 2; ++pass) {
      const int* mil = pass ? miller_out : miller_in;
      const int nmax = pass ? npw_out_max : npw_in_max;
      const int n = pass ? npw_out[k] : npw_in[k];
      std::vector<int>& dst = pass ? gout : gin;
      std::vector<char> seen((size_t)s * N, 0);
      for (int g = 0; g < n; ++g) {
        const int* m = mil + ((size_t)k * nmax + g) * 3;
        const int sk = st[std::make_pair(m[0], m[1])];
        const int slot = wrap(m[2]);
        if (seen[(size_t)sk * N + slot]) {
          char buf[160];
          std::snprintf(buf, sizeof(buf), "k %d: two basis vectors map to the same grid point (G %d)", k, g);
          set_error(buf);
          return PWK_ERR_INVALID;
        }
        seen[(size_t)sk * N + slot] = 1;
        dst[(size_t)k * nmax + g] = (sk << 8) | slot;
      }
    }
  }
  sm.nstick_max = nsmax;
  sm.m1lo = m1lo;
  sm.P = P;
  sm.npw_in_max = npw_in_max;
  sm.npw_out_max = npw_out_max;
  sm.d_npw_in = d_npw_in;
  sm.d_npw_out = d_npw_out;
  if ((rc = plan_alloc(p, (void**)&sm.d_nstick, sizeof(int) * nk))) return rc;
  if ((rc = plan_alloc(p, (void**)&sm.d_gin, sizeof(int) * gin.size()))) return rc;
  if ((rc = plan_alloc(p, (void**)&sm.d_gout, sizeof(int) * gout.size()))) return rc;
  if ((rc = plan_alloc(p, (void**)&sm.d_sid, sizeof(short) * sid.size()))) return rc;
  cudaError_t e;
  if ((e = cudaMemcpy(sm.d_nstick, nstick.data(), sizeof(int) * nk, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(sm.d_gin, gin.data(), sizeof(int) * gin.size(), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(sm.d_gout, gout.data(), sizeof(int) * gout.size(), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(sm.d_sid, sid.data(), sizeof(short) * sid.size(), cudaMemcpyHostToDevice)))
    return cuda_fail(e, "cudaMemcpy(sphere map)");
  return PWK_OK;
}

// Tables of the window-specialised kernel: every Miller index of the plan within
// |m_i| <= W = N/4; the sticks of a k live at rows (m1+W)(2W+1) + (m2+W) of a dense square.
int build_window_tables(pwk_plan* p) {
  const int N = p->N, W = N / 4, NW = 2 * W + 1, nk = p->nk, np = p->npw_max;
  for (size_t i = 0; i < p->h_miller.size(); ++i) {
    const int g = (int)((i / 3) % np), k = (int)(i / 3 / np);
    if (g < p->h_npw[k] && std::abs(p->h_miller[i]) > W) return PWK_OK;   // not eligible
  }
  const int nsm = p->self.nstick_max;
  std::vector<int> gm((size_t)nk * np, 0);
  std::vector<short> rows((size_t)nk * nsm, (short)0);
  for (int k = 0; k < nk; ++k) {
    std::vector<char> seen((size_t)NW * NW, 0);
    int c = 0;
    for (int g = 0; g < p->h_npw[k]; ++g) {
      const int* m = &p->h_miller[((size_t)k * np + g) * 3];
      const int row = (m[0] + W) * NW + (m[1] + W);
      gm[(size_t)k * np + g] = (row << 8) | (((m[2] % N) + N) % N);
      if (!seen[row]) {
        seen[row] = 1;
        if (c >= nsm) return PWK_OK;   // cannot happen: same stick count as the self map
        rows[(size_t)k * nsm + c++] = (short)row;
      }
    }
  }
  int rc;
  if ((rc = plan_alloc(p, (void**)&p->d_wgmap, sizeof(int) * gm.size()))) return rc;
  if ((rc = plan_alloc(p, (void**)&p->d_wrows, sizeof(short) * rows.size()))) return rc;
  cudaError_t e;
  if ((e = cudaMemcpy(p->d_wgmap, gm.data(), sizeof(int) * gm.size(), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(p->d_wrows, rows.data(), sizeof(short) * rows.size(), cudaMemcpyHostToDevice)))
    return cuda_fail(e, "cudaMemcpy(window tables)");
  p->window_ok = true;
  return PWK_OK;
}

// Launch shape: the largest l3 chunk that keeps two CTAs per SM (FP64: one) within the
// 227 KB of shared memory per CTA, threads 256.
LaunchShape choose_shape(int N, int elem_bytes, const SphereMap& sm, int ctas_per_sm) {
  LaunchShape s;
  s.threads = 256;
  const size_t sm_total = 228 * 1024, per_cta_max = 227 * 1024;
  const size_t target = std::min(per_cta_max, sm_total / ctas_per_sm - 1024);
  int best = 1;
  for (int L = N; L >= 1; --L) {
    if (fused_smem_bytes(N, elem_bytes, sm.nstick_max, sm.P, L, sm.npw_in_max) <= target) {
      best = L;
      break;
    }
  }
  s.L = best;
  s.smem = fused_smem_bytes(N, elem_bytes, sm.nstick_max, sm.P, best, sm.npw_in_max);
  return s;
}

static NlArgs nl_args(const pwk_plan* p, int precision, const void* in, void* out, void* sout,
                      const int* items, const int* d_count, int nblocks, int nvec_in, int nvec_out,
                      int k0);

// Shared-memory layout of the local kernel with the projector terms fused in: the kernel's
// own buffers, then (window kernels) the gathered local result and C, placed past the stick
// square; beta(k) is staged at offset 0 once the square has been read; the coefficients
// (lambda, gamma, delta) last.  Returns the bytes the launch needs; *nl_off, *loc_off get the
// offsets.
static size_t fused_layout(const pwk_plan* p, int precision, const LaunchShape& s, int* nl_off, int* loc_off) {
  const size_t V = precision == PWK_FP64 ? 16 : 8;
  auto r16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
  size_t R = r16(s.smem);
  size_t loc = 0;
  if (s.kind >= 1) {
    const int N = p->N, NW = 2 * (N / 4) + 1;
    int zs = 0, yps = 0;
    window_strides(N, s.L, &zs, &yps);
    const size_t zb = r16((size_t)NW * NW * zs * V);
    const size_t lc = r16(2 * (size_t)p->npw_max * V);
    const size_t bb = r16((size_t)p->nkb * p->npw_max * V);
    R = std::max(R, std::max(bb, zb) + lc);
    loc = R - lc;
  }
  if (nl_off) *nl_off = (int)R;
  if (loc_off) *loc_off = (int)loc;
  return R + nl_fused_bytes(p->nkb, (int)V);
}

// Whether the projector terms of this precision run inside the local kernel: the plan's
// choice (set by the autotuner, or forced by pwk_plan_set_projector_path) and room in shared
// memory.
static bool nl_fused_fits(const pwk_plan* p, int precision, const LaunchShape& s) {
  return p->nkb > 0 && fused_layout(p, precision, s, nullptr, nullptr) <= 227 * 1024;
}
static bool nl_fused_for(const pwk_plan* p, int precision, const LaunchShape& s) {
  if (p->projector_path == 3) return nl_fused_fits(p, precision, s);
  if (p->projector_path != 0) return false;
  return p->nl_fused[precision] && nl_fused_fits(p, precision, s);
}

// Point the kernel arguments at the plan's projectors (the precision's copies of beta, D, q)
// and the shared-memory layout of the fused kernel.
static void set_fused_nl(const pwk_plan* p, int precision, FusedArgs& a, void* sout, const LaunchShape& s) {
  const bool f64 = precision == PWK_FP64;
  a.beta = f64 ? static_cast<const void*>(p->d_beta) : static_cast<const void*>(p->d_beta32);
  a.Dm = f64 ? static_cast<const void*>(p->d_D) : static_cast<const void*>(p->d_D32);
  a.qm = f64 ? static_cast<const void*>(p->d_q) : static_cast<const void*>(p->d_q32);
  a.sout = sout;
  a.nkb = p->nkb;
  a.npw_beta = p->npw_max;
  fused_layout(p, precision, s, &a.nl_off, &a.loc_off);
}

static int launch_variant(int precision, int N, const FusedArgs& a, int nblocks,
                          const LaunchShape& s0, cudaStream_t st) {
  LaunchShape s = s0;
  if (a.beta != nullptr) s.smem = (size_t)a.nl_off + nl_fused_bytes(a.nkb, precision == PWK_FP64 ? 16 : 8);
  const bool nl = a.beta != nullptr;
  if (s.kind >= 1) {
    switch (precision) {
      case PWK_FP64: return nl ? launch_window_f64_nl(N, a, nblocks, s, st) : launch_window_f64(N, a, nblocks, s, st);
      case PWK_FP32: return nl ? launch_window_f32_nl(N, a, nblocks, s, st) : launch_window_f32(N, a, nblocks, s, st);
      default:
        return nl ? launch_window_f32c128_nl(N, a, nblocks, s, st) : launch_window_f32c128(N, a, nblocks, s, st);
    }
  }
  switch (precision) {
    case PWK_FP64: return nl ? launch_fused_f64_nl(N, a, nblocks, s, st) : launch_fused_f64(N, a, nblocks, s, st);
    case PWK_FP32: return nl ? launch_fused_f32_nl(N, a, nblocks, s, st) : launch_fused_f32(N, a, nblocks, s, st);
    default: return nl ? launch_fused_f32c128_nl(N, a, nblocks, s, st) : launch_fused_f32c128(N, a, nblocks, s, st);
  }
}

// Point the kernel arguments at the tables of the chosen kernel kind.
static void use_kind(const pwk_plan* p, FusedArgs& a, int kind) {
  if (kind >= 1) {
    a.gin = a.gout = p->d_wgmap;
    a.sid = p->d_wrows;
    window_strides(p->N, a.L, &a.zs, &a.yps);
  } else {
    a.gin = p->self.d_gin;
    a.gout = p->self.d_gout;
    a.sid = p->self.d_sid;
    a.zs = (p->N % 2 == 0) ? p->N + 1 : p->N;
    a.yps = p->N * a.L;
  }
}

// Pick the launch shape (kernel kind, threads per CTA, l3 chunk L) of one precision, and
// whether the projector terms run inside the local kernel or in separate kernels, by timing
// them on a sample of the plan's k-points (8 zero vectors per k, up to 512 k-points in FP32
// and 96 in FP64; the work of the kernels does not depend on the values).  Every shape of a
// kind gives bitwise the same result: the arithmetic of each line and the order of every
// reduction do not depend on the shape.
int autotune_shape(pwk_plan* p, int precision) {
  const int N = p->N;
  const int elem = precision == PWK_FP64 ? 16 : 8;
  const int io_elem = precision == PWK_FP32 ? 8 : 16;
  std::vector<LaunchShape> cands;
  const int Ls[4] = {N, (N + 1) / 2, (N + 2) / 3, (N + 3) / 4};
  for (int kind = 0; kind < (p->window_ok ? 3 : 1); ++kind)
    for (int T : {96, 128, 192, 256})
      for (int li = 0; li < 4; ++li) {
        // kinds 0, 1: L planes per chunk of the CTA; kind 2: L = 1 or 2 planes per warp
        const int L = kind == 2 ? li + 1 : Ls[li];
        if (kind == 2 && L > 2) continue;
        if (kind != 2 && li > 0 && L == Ls[li - 1]) continue;
        LaunchShape c;
        c.kind = kind;
        c.threads = T;
        c.L = L;
        c.smem = kind >= 1 ? window_smem_bytes(N, elem, L, p->self.nstick_max, kind == 2 ? T / 32 : 1)
                           : fused_smem_bytes(N, elem, p->self.nstick_max, p->self.P, L, p->npw_max);
        if (c.smem <= 227 * 1024) cands.push_back(c);
      }
  if (cands.empty()) return PWK_OK;   // the default shape stands (plan creation checked it)
  const int nv = 8, nkt = std::min(p->nk, precision == PWK_FP64 ? 96 : 512);
  const size_t bytes = (size_t)nkt * nv * p->npw_max * io_elem;
  void *in = nullptr, *out = nullptr;
  if (cudaMalloc(&in, bytes) != cudaSuccess || cudaMalloc(&out, bytes) != cudaSuccess) {
    cudaFree(in);
    cudaGetLastError();
    return PWK_OK;   // no room to tune: keep the default
  }
  cudaMemset(in, 0, bytes);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  FusedArgs a = hpsi_args(p, precision, in, out);
  a.nvec_in = a.nvec_out = nv;
  // time of one call (after one untimed launch), ms; 1e30 if it fails
  auto time_it = [&](auto&& run) -> float {
    if (run() != PWK_OK) {
      cudaGetLastError();
      return 1e30f;
    }
    cudaEventRecord(e0, 0);
    for (int r = 0; r < 3; ++r) run();
    cudaEventRecord(e1, 0);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      cudaGetLastError();
      return 1e30f;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  // Two interleaved rounds over the candidates, the faster of each candidate's two timings
  // counts (a clock ramp or another process's burst during one timing does not decide).  Each
  // candidate is timed without the projector terms and, where they fit, with them fused in.
  std::vector<float> tplain(cands.size(), 1e30f), tfused(cands.size(), 1e30f);
  for (int round = 0; round < 2; ++round) {
    for (size_t ci = 0; ci < cands.size(); ++ci) {
      const LaunchShape& c = cands[ci];
      a.L = c.L;
      use_kind(p, a, c.kind);
      a.beta = nullptr;
      tplain[ci] = std::min(tplain[ci], time_it([&] { return launch_variant(precision, N, a, nkt * nv, c, 0); }));
      if (nl_fused_fits(p, precision, c)) {
        set_fused_nl(p, precision, a, nullptr, c);
        tfused[ci] = std::min(tfused[ci], time_it([&] { return launch_variant(precision, N, a, nkt * nv, c, 0); }));
        a.beta = nullptr;
      }
    }
  }
  size_t bp = 0, bf = 0;
  for (size_t ci = 0; ci < cands.size(); ++ci) {
    if (tplain[ci] < tplain[bp]) bp = ci;
    if (tfused[ci] < tfused[bf]) bf = ci;
  }
  cudaFree(in);
  cudaFree(out);
  in = out = nullptr;
  // The projector terms inside the best fused shape against the separate kernels around the
  // best plain shape (projections, local kernel, add-back; on the CUDA cores and, for the FP32
  // arithmetic where they apply, on the tensor cores), timed as whole H applications of 32
  // bands (a whole-k-point call of a band set) on a larger sample (a few waves of the
  // one-CTA-per-k-point projector kernels), where launch overheads and partial last waves no
  // longer decide.
  bool fused = false, tc = false;
  if (p->nkb > 0 && tfused[bf] < 1e29f && tplain[bp] < 1e29f) {
    const int nv2 = 32, nk2 = std::min(p->nk, precision == PWK_FP64 ? 64 : 384);
    const size_t bytes2 = (size_t)nk2 * nv2 * p->npw_max * io_elem;
    void* coef = nullptr;
    if (cudaMalloc(&in, bytes2) == cudaSuccess && cudaMalloc(&out, bytes2) == cudaSuccess &&
        cudaMalloc(&coef, (size_t)nk2 * nv2 * 2 * p->nkb * elem) == cudaSuccess) {
      cudaMemset(in, 0, bytes2);
      FusedArgs b = hpsi_args(p, precision, in, out);
      b.nvec_in = b.nvec_out = nv2;
      NlArgs n = nl_args(p, precision, in, out, nullptr, nullptr, nullptr, nk2 * nv2, nv2, nv2, 0);
      n.coef = coef;
      n.tensor_cores = true;
      const bool try_tc = precision != PWK_FP64 && nl_tcw_applies(precision, n);
      float tf = 1e30f, ts = 1e30f, tt = 1e30f;
      auto split = [&](bool on_tc) {
        const LaunchShape& cp = cands[bp];
        b.L = cp.L;
        use_kind(p, b, cp.kind);
        b.beta = nullptr;
        n.tensor_cores = on_tc;
        return time_it([&] {
          n.phase = 0;
          int r = launch_nl(precision, n, 0);
          if (r == PWK_OK) r = launch_variant(precision, N, b, nk2 * nv2, cp, 0);
          n.phase = 1;
          return r ? r : launch_nl(precision, n, 0);
        });
      };
      for (int round = 0; round < 2; ++round) {
        const LaunchShape& cf = cands[bf];
        b.L = cf.L;
        use_kind(p, b, cf.kind);
        set_fused_nl(p, precision, b, nullptr, cf);
        tf = std::min(tf, time_it([&] { return launch_variant(precision, N, b, nk2 * nv2, cf, 0); }));
        ts = std::min(ts, split(false));
        if (try_tc) tt = std::min(tt, split(true));
      }
      // the separate CUDA-core kernels unless another path is faster by more than 3 %: near
      // ties (timing noise) then resolve the same way in every process
      const float best_other = std::min(tf, tt);
      if (best_other < 0.97f * ts) {
        fused = tf <= tt;
        tc = !fused;
      }
    } else {
      cudaGetLastError();
    }
    cudaFree(coef);
    cudaFree(in);
    cudaFree(out);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (tplain[bp] < 1e29f || fused) {
    p->shape[precision] = fused ? cands[bf] : cands[bp];
    p->nl_fused[precision] = fused;
    p->nl_tc[precision] = tc;
  }
  return PWK_OK;
}

FusedArgs hpsi_args(const pwk_plan* p, int precision, const void* in, void* out) {
  FusedArgs a;
  a.in = in;
  a.out = out;
  a.nk = p->nk;
  a.npw_in_max = a.npw_out_max = p->npw_max;
  a.npw_in = a.npw_out = p->d_npw;
  a.nstick = p->self.d_nstick;
  a.gin = p->self.d_gin;
  a.gout = p->self.d_gout;
  a.sid = p->self.d_sid;
  a.nstick_max = p->self.nstick_max;
  a.m1lo = p->self.m1lo;
  a.P = p->self.P;
  a.L = p->shape[precision].L;
  a.zs = (p->N % 2 == 0) ? p->N + 1 : p->N;
  a.g2 = p->d_g2;
  a.V = precision == PWK_FP64 ? static_cast<const void*>(p->d_Vt64) : static_cast<const void*>(p->d_V32);
  a.scale = 1.0 / (double)p->Nr;
  a.err = p->d_err;
  return a;
}

// Stream-ordered pool for per-call scratch (one per device, kept for the life of the
// process).  Its release threshold is unbounded, so memory freed at the end of a call stays
// mapped and the next call's allocation is a pool hit instead of a new mapping.
cudaError_t scratch_pool(cudaMemPool_t* pool) {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) {
    *pool = it->second;
    return cudaSuccess;
  }
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  e = cudaMemPoolCreate(pool, &props);
  if (e != cudaSuccess) return e;
  unsigned long long keep = ~0ull;
  e = cudaMemPoolSetAttribute(*pool, cudaMemPoolAttrReleaseThreshold, &keep);
  if (e != cudaSuccess) return e;
  pools[dev] = *pool;
  return cudaSuccess;
}

cudaError_t scratch_alloc(void** ptr, size_t bytes, cudaStream_t st) {
  cudaMemPool_t pool;
  cudaError_t e = scratch_pool(&pool);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(ptr, bytes, pool, st);
  return e;
}

// Arguments of the separate projector kernels for a launch of run_hpsi (coef left null).
static NlArgs nl_args(const pwk_plan* p, int precision, const void* in, void* out, void* sout,
                      const int* items, const int* d_count, int nblocks, int nvec_in, int nvec_out,
                      int k0) {
  NlArgs n;
  n.in = in;
  n.out = out;
  n.sout = sout;
  n.items = items;
  n.d_count = d_count;
  n.k0 = k0;
  n.err = p->d_err;
  n.tensor_cores = p->projector_path == 1 || (p->projector_path == 0 && p->nl_tc[precision]);
  n.wait_polls = p->wait_polls;
  n.nitems = nblocks;
  n.nvec_in = nvec_in;
  n.nvec_out = nvec_out;
  n.nk = p->nk;
  n.npw_max = p->npw_max;
  n.npw = p->d_npw;
  n.nkb = p->nkb;
  const bool f64 = precision == PWK_FP64;
  n.beta = f64 ? static_cast<const void*>(p->d_beta) : static_cast<const void*>(p->d_beta32);
  n.D = f64 ? static_cast<const void*>(p->d_D) : static_cast<const void*>(p->d_D32);
  n.q = f64 ? static_cast<const void*>(p->d_q) : static_cast<const void*>(p->d_q32);
  return n;
}

int run_hpsi(pwk_plan* p, int precision, const void* in, void* out, const int* items,
             const int* d_count, int nblocks, int nvec_in, int nvec_out, cudaStream_t st,
             void* sout, int k0) {
  if (precision < 0 || precision > 2) {
    set_error("unknown precision");
    return PWK_ERR_INVALID;
  }
  if (nblocks <= 0) return PWK_OK;
  const LaunchShape& shape = p->shape[precision];
  if (out != nullptr && nl_fused_for(p, precision, shape)) {
    // one kernel: projections, local and kinetic terms, add-back (and S C)
    FusedArgs a = hpsi_args(p, precision, in, out);
    a.items = items;
    a.d_count = d_count;
    a.k0 = k0;
    a.nvec_in = nvec_in;
    a.nvec_out = nvec_out;
    use_kind(p, a, shape.kind);
    set_fused_nl(p, precision, a, sout, shape);
    return launch_variant(precision, p->N, a, nblocks, shape, st);
  }
  // separate projector kernels: coefficients gamma, delta of every item in scratch from a
  // stream-ordered pool, so concurrent calls on other streams never share it
  NlArgs n;
  const bool nl = p->nkb > 0 || sout != nullptr;   // with no projectors S C = C (phase 1 copies)
  if (nl) {
    n = nl_args(p, precision, in, out, sout, items, d_count, nblocks, nvec_in, nvec_out, k0);
    const bool f64 = precision == PWK_FP64;
    const size_t cbytes = (size_t)nblocks * 2 * p->nkb * (f64 ? 16 : 8);
    if (cbytes > 0) {
      cudaError_t e = scratch_alloc(&n.coef, cbytes, st);
      if (e != cudaSuccess) return cuda_fail(e, "scratch_alloc(projector coefficients)");
    }
    n.phase = 0;
    if (int r = launch_nl(precision, n, st)) {
      if (n.coef) cudaFreeAsync(n.coef, st);
      return r;
    }
  }
  int r = PWK_OK;
  if (out != nullptr) {   // out == null: S only (no local term, no H add-back)
    FusedArgs a = hpsi_args(p, precision, in, out);
    a.items = items;
    a.d_count = d_count;
    a.k0 = k0;
    a.nvec_in = nvec_in;
    a.nvec_out = nvec_out;
    use_kind(p, a, p->shape[precision].kind);
    r = launch_variant(precision, p->N, a, nblocks, p->shape[precision], st);
  }
  if (nl) {
    if (r == PWK_OK) {
      n.phase = 1;
      r = launch_nl(precision, n, st);
    }
    if (n.coef) {
      cudaError_t e = cudaFreeAsync(n.coef, st);
      if (r == PWK_OK && e != cudaSuccess) r = cuda_fail(e, "cudaFreeAsync(projector coefficients)");
    }
  }
  return r;
}

}  // namespace pwk

using namespace pwk;

extern "C" {

int pwk_supported_grid(int N) { return grid_supported(N) ? 1 : 0; }

const char* pwk_version(void) { return "pwk 0.1 (sm_103a)"; }

const char* pwk_last_error_detail(void) { return g_detail.c_str(); }

const char* pwk_strerror(int code) {
  switch (code) {
    case PWK_OK: return "success";
    case PWK_ERR_INVALID: return "invalid argument";
    case PWK_ERR_UNSUPPORTED: return "unsupported size or configuration";
    case PWK_ERR_NOMEM: return "device allocation failed";
    case PWK_ERR_BUDGET: return "plan HBM budget exceeded";
    case PWK_ERR_CUDA: return "CUDA error";
    case PWK_ERR_NOT_POSDEF: return "reduced overlap matrix not positive definite";
    case PWK_ERR_NUMERIC: return "numerical breakdown";
    default: return code > 0 ? "not converged" : "unknown error";
  }
}

size_t pwk_plan_device_bytes(const pwk_plan* p) { return p ? p->bytes : 0; }

int pwk_plan_set_wait_limit(pwk_plan* p, long long polls) {
  if (p == nullptr || polls < 0) {
    set_error("null plan or negative poll count");
    return PWK_ERR_INVALID;
  }
  p->wait_polls = polls;
  return PWK_OK;
}

int pwk_plan_errors(pwk_plan* p, int* flags, int clear) {
  if (p == nullptr || flags == nullptr) {
    set_error("null plan or flags");
    return PWK_ERR_INVALID;
  }
  cudaError_t e = cudaSetDevice(p->device);
  int v = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&v, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && clear) e = cudaMemset(p->d_err, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "pwk_plan_errors");
  *flags = v;
  return PWK_OK;
}

long long pwk_launch_count(void) { return pwk::g_launches.load(std::memory_order_relaxed); }

int pwk_plan_set_projector_path(pwk_plan* p, int path) {
  if (p == nullptr || path < 0 || path > 3) {
    set_error("null plan or path not 0..3");
    return PWK_ERR_INVALID;
  }
  p->projector_path = path;
  return PWK_OK;
}

int pwk_plan_projector_fused(const pwk_plan* p, int precision) {
  if (p == nullptr || precision < 0 || precision > 2) return -1;
  return nl_fused_for(p, precision, p->shape[precision]) ? 1 : 0;
}

int pwk_plan_projector_choice(const pwk_plan* p, int precision) {
  if (p == nullptr || precision < 0 || precision > 2) return -1;
  if (p->nkb == 0) return 0;
  if (nl_fused_for(p, precision, p->shape[precision])) return 3;
  const bool tc = p->projector_path == 1 || (p->projector_path == 0 && p->nl_tc[precision]);
  return tc && precision != PWK_FP64 ? 1 : 2;
}

int pwk_plan_set_launch_shape(pwk_plan* p, int precision, int kind, int threads, int l3_chunk) {
  if (p == nullptr || precision < 0 || precision > 2 || kind < 0 || kind > 2 ||
      (threads != 96 && threads != 128 && threads != 192 && threads != 256) || l3_chunk < 1 ||
      l3_chunk > p->N) {
    set_error("bad plan, precision, kind (0/1/2), threads (96/128/192/256) or l3 chunk (1..N)");
    return PWK_ERR_INVALID;
  }
  if (kind >= 1 && !p->window_ok) {
    set_error("the window kernel needs every |m_i| <= N/4");
    return PWK_ERR_UNSUPPORTED;
  }
  const int elem = precision == PWK_FP64 ? 16 : 8;
  LaunchShape c;
  c.kind = kind;
  c.threads = threads;
  c.L = l3_chunk;
  c.smem = kind >= 1 ? window_smem_bytes(p->N, elem, l3_chunk, p->self.nstick_max, kind == 2 ? threads / 32 : 1)
                     : fused_smem_bytes(p->N, elem, p->self.nstick_max, p->self.P, l3_chunk, p->npw_max);
  if (c.smem > 227 * 1024) {
    set_error("shape needs more than 227 KB of shared memory");
    return PWK_ERR_UNSUPPORTED;
  }
  p->shape[precision] = c;
  return PWK_OK;
}

int pwk_plan_launch_shape(const pwk_plan* p, int precision, int* kind, int* threads,
                          int* l3_chunk, size_t* smem_bytes) {
  if (p == nullptr || precision < 0 || precision > 2) {
    set_error("null plan or unknown precision");
    return PWK_ERR_INVALID;
  }

  if (kind) *kind = p->shape[precision].kind;
  if (threads) *threads = p->shape[precision].threads;
  if (l3_chunk) *l3_chunk = p->shape[precision].L;
  if (smem_bytes) *smem_bytes = p->shape[precision].smem;
  return PWK_OK;
}

void pwk_plan_destroy(pwk_plan* p) {
  if (p == nullptr) return;
  destroy_solver_work(p);
  if (p->copy_in != nullptr) cudaStreamDestroy(p->copy_in);
  if (p->copy_out != nullptr) cudaStreamDestroy(p->copy_out);
  if (p->compute2 != nullptr) cudaStreamDestroy(p->compute2);
  for (void* q : p->allocs) cudaFree(q);
  delete p;
}

int pwk_plan_create(pwk_plan** out, const double* A, int N1, int N2, int N3, int nk,
                    const double* kcart, const int* npw, int npw_max, const int* miller, int nkb,
                    const void* beta, const double* D, const double* vloc_r, size_t hbm_budget) {
  if (out == nullptr) {
    set_error("out is NULL");
    return PWK_ERR_INVALID;
  }
  *out = nullptr;
  if (A == nullptr || kcart == nullptr || npw == nullptr || miller == nullptr || vloc_r == nullptr ||
      (nkb > 0 && (beta == nullptr || D == nullptr)) || nk < 1 || npw_max < 1 || nkb < 0) {
    set_error("null pointer or non-positive size");
    return PWK_ERR_INVALID;
  }
  if (N1 != N2 || N2 != N3 || !grid_supported(N1)) {
    set_error("grid must be N x N x N with N in the supported set");
    return PWK_ERR_UNSUPPORTED;
  }
  for (int k = 0; k < nk; ++k)
    if (npw[k] < 1 || npw[k] > npw_max) {
      set_error("npw[k] outside [1, npw_max]");
      return PWK_ERR_INVALID;
    }
  if (nkb > 1024) {
    set_error("more than 1024 projectors");
    return PWK_ERR_UNSUPPORTED;
  }
  pwk_plan* p = new pwk_plan();
  cudaGetDevice(&p->device);
  p->N = N1;
  p->Nr = N1 * N2 * N3;
  p->nk = nk;
  p->npw_max = npw_max;
  p->nkb = nkb;
  p->budget = hbm_budget;
  std::memcpy(p->A, A, sizeof(p->A));
  {
    // reciprocal rows b_i with a_i . b_j = 2 pi delta_ij: B = 2 pi (A^-1)^T
    const double* a = A;
    const double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                       a[2] * (a[3] * a[7] - a[4] * a[6]);
    if (std::fabs(det) < 1e-12) {
      delete p;
      set_error("singular lattice");
      return PWK_ERR_INVALID;
    }
    double inv[9];
    inv[0] = (a[4] * a[8] - a[5] * a[7]) / det;
    inv[1] = (a[2] * a[7] - a[1] * a[8]) / det;
    inv[2] = (a[1] * a[5] - a[2] * a[4]) / det;
    inv[3] = (a[5] * a[6] - a[3] * a[8]) / det;
    inv[4] = (a[0] * a[8] - a[2] * a[6]) / det;
    inv[5] = (a[2] * a[3] - a[0] * a[5]) / det;
    inv[6] = (a[3] * a[7] - a[4] * a[6]) / det;
    inv[7] = (a[1] * a[6] - a[0] * a[7]) / det;
    inv[8] = (a[0] * a[4] - a[1] * a[3]) / det;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) p->B[3 * i + j] = 2.0 * kPi * inv[3 * j + i];
  }
  p->h_npw.assign(npw, npw + nk);
  p->h_kcart.assign(kcart, kcart + 3 * (size_t)nk);
  p->h_miller.assign(miller, miller + 3 * (size_t)nk * npw_max);
  if (nkb > 0) p->h_D.assign(D, D + (size_t)nkb * nkb);
  p->d_beta = static_cast<const double2*>(beta);
  p->d_V = vloc_r;

  int rc = PWK_OK;
  cudaError_t e;
  int* d_miller = nullptr;
  double* d_B = nullptr;
  double* d_vsum = nullptr;
#define TRY(x)          \
  do {                  \
    rc = (x);           \
    if (rc) goto fail;  \
  } while (0)
#define TRYC(x, what)                  \
  do {                                 \
    e = (x);                           \
    if (e != cudaSuccess) {            \
      rc = cuda_fail(e, what);         \
      goto fail;                       \
    }                                  \
  } while (0)
  TRY(plan_alloc(p, (void**)&p->d_err, sizeof(int)));
  TRYC(cudaMemset(p->d_err, 0, sizeof(int)), "cudaMemset");
  TRY(plan_alloc(p, (void**)&p->d_npw, sizeof(int) * nk));
  TRYC(cudaMemcpy(p->d_npw, npw, sizeof(int) * nk, cudaMemcpyHostToDevice), "cudaMemcpy(npw)");
  TRY(plan_alloc(p, (void**)&p->d_kcart, sizeof(double) * 3 * nk));
  TRYC(cudaMemcpy(p->d_kcart, kcart, sizeof(double) * 3 * nk, cudaMemcpyHostToDevice), "cudaMemcpy(k)");
  TRY(plan_alloc(p, (void**)&p->d_g2, sizeof(double) * (size_t)nk * npw_max));
  TRYC(cudaMalloc(&d_miller, sizeof(int) * 3 * (size_t)nk * npw_max), "cudaMalloc(tmp)");
  TRYC(cudaMalloc(&d_B, sizeof(double) * 9), "cudaMalloc(tmp)");
  TRYC(cudaMemcpy(d_miller, miller, sizeof(int) * 3 * (size_t)nk * npw_max, cudaMemcpyHostToDevice),
       "cudaMemcpy(miller)");
  TRYC(cudaMemcpy(d_B, p->B, sizeof(double) * 9, cudaMemcpyHostToDevice), "cudaMemcpy(B)");
  kinetic_table_kernel<<<blocks_for((size_t)nk * npw_max), 256>>>(nk, npw_max, p->d_npw, p->d_kcart,
                                                                  d_miller, d_B, p->d_g2); note_launch();
  TRYC(cudaGetLastError(), "kinetic_table_kernel");
  if (nkb > 0) {
    const size_t nb2 = (size_t)nk * nkb * npw_max * 2;
    TRY(plan_alloc(p, (void**)&p->d_beta32, sizeof(float) * nb2));
    to_f32_kernel<<<blocks_for(nb2), 256>>>(nb2, static_cast<const double*>(beta), (float*)p->d_beta32); note_launch();
    TRYC(cudaGetLastError(), "beta to f32");
    std::vector<float> D32(p->h_D.begin(), p->h_D.end());
    TRY(plan_alloc(p, (void**)&p->d_D, sizeof(double) * nkb * nkb));
    TRY(plan_alloc(p, (void**)&p->d_D32, sizeof(float) * nkb * nkb));
    TRYC(cudaMemcpy(p->d_D, D, sizeof(double) * nkb * nkb, cudaMemcpyHostToDevice), "cudaMemcpy(D)");
    TRYC(cudaMemcpy(p->d_D32, D32.data(), sizeof(float) * nkb * nkb, cudaMemcpyHostToDevice), "cudaMemcpy(D32)");
  }
  TRY(plan_alloc(p, (void**)&p->d_V32, sizeof(float) * (size_t)p->Nr));
  TRY(plan_alloc(p, (void**)&p->d_Vt64, sizeof(double) * (size_t)p->Nr));
  transpose_v_kernel<float><<<blocks_for(p->Nr), 256>>>(p->N, vloc_r, p->d_V32); note_launch();
  transpose_v_kernel<double><<<blocks_for(p->Nr), 256>>>(p->N, vloc_r, p->d_Vt64); note_launch();
  TRYC(cudaGetLastError(), "V transpose");
  TRYC(cudaMalloc(&d_vsum, sizeof(double)), "cudaMalloc(tmp)");
  TRYC(cudaMemset(d_vsum, 0, sizeof(double)), "cudaMemset");
  sum_kernel<<<1, 256>>>((size_t)p->Nr, vloc_r, d_vsum); note_launch();
  TRYC(cudaGetLastError(), "sum_kernel");
  TRYC(cudaMemcpy(&p->v_mean, d_vsum, sizeof(double), cudaMemcpyDeviceToHost), "cudaMemcpy(vsum)");
  p->v_mean /= (double)p->Nr;
  TRY(build_sphere_map(p, p->self, nk, npw, npw_max, miller, npw, npw_max, miller, p->d_npw, p->d_npw));
  p->shape[PWK_FP64] = choose_shape(p->N, 16, p->self, 1);
  p->shape[PWK_FP32] = choose_shape(p->N, 8, p->self, 2);
  p->shape[PWK_FP32_C128] = p->shape[PWK_FP32];
  if (p->shape[PWK_FP64].smem > 227 * 1024) {
    set_error("the z-sticks and one plane of the carried m1 window do not fit in shared memory");
    rc = PWK_ERR_UNSUPPORTED;
    goto fail;
  }
  TRY(build_window_tables(p));
  TRYC(cudaStreamSynchronize(cudaStreamLegacy), "plan setup");
  for (int prec = 0; prec < 3; ++prec) TRY(autotune_shape(p, prec));
  TRYC(cudaStreamSynchronize(cudaStreamLegacy), "plan setup");
  cudaFree(d_miller);
  cudaFree(d_B);
  cudaFree(d_vsum);
  *out = p;
  return PWK_OK;
fail:
  if (d_miller) cudaFree(d_miller);
  if (d_B) cudaFree(d_B);
  if (d_vsum) cudaFree(d_vsum);
  pwk_plan_destroy(p);
  return rc;
#undef TRY
#undef TRYC
}

int pwk_hpsi_batched(pwk_plan* p, int precision, const void* psi, void* hpsi, int nb, void* stream) {
  if (p == nullptr || psi == nullptr || hpsi == nullptr || nb < 1) {
    set_error("null pointer or nb < 1");
    return PWK_ERR_INVALID;
  }
  if (precision < 0 || precision > 2) {
    set_error("unknown precision");
    return PWK_ERR_INVALID;
  }
  const long long nblocks = (long long)p->nk * nb;
  if (nblocks > 0x7fffffffLL) {
    set_error("nk * nb too large for one launch");
    return PWK_ERR_UNSUPPORTED;
  }
  return run_hpsi(p, precision, psi, hpsi, nullptr, nullptr, (int)nblocks, nb, nb,
                  static_cast<cudaStream_t>(stream));
}

// First k-point of group c of pwk_hpsi_batched_host (group_start(nk, n, n) = nk).  With three
// or more groups the first and the last get half the weight of the others: the copy in of
// the first group and the copy out of the last are the parts of the pipeline that nothing
// overlaps, so they are kept short.
static int group_start(int nk, int n, int c) {
  if (n < 3) return (int)((long long)nk * c / n);
  const long long w2 = 2LL * (n - 1);   // total weight in halves: 1 + 2 (n - 2) + 1
  const long long h = c == 0 ? 0 : (c == n ? w2 : 2LL * c - 1);
  return (int)(nk * h / w2);
}

int pwk_hpsi_batched_host(pwk_plan* p, int precision, const void* h_psi, void* h_hpsi,
                          void* d_psi, void* d_hpsi, int nb, int nchunk, void* stream) {
  if (p == nullptr || h_psi == nullptr || h_hpsi == nullptr || d_psi == nullptr ||
      d_hpsi == nullptr || nb < 1 || nchunk < 1) {
    set_error("null pointer, nb < 1 or nchunk < 1");
    return PWK_ERR_INVALID;
  }
  if (precision < 0 || precision > 2) {
    set_error("unknown precision");
    return PWK_ERR_INVALID;
  }
  if ((long long)p->nk * nb > 0x7fffffffLL) {
    set_error("nk * nb too large for one launch");
    return PWK_ERR_UNSUPPORTED;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  {
    std::lock_guard<std::mutex> lock(p->copy_mu);
    if (p->copy_in == nullptr) {
      cudaError_t e = cudaStreamCreateWithFlags(&p->copy_in, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->copy_out, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->compute2, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithFlags(copy streams)");
    }
  }
  nchunk = std::min(nchunk, p->nk);
  const size_t per_k = (size_t)nb * p->npw_max * (precision == PWK_FP32 ? 8 : 16);
  // events: start, then per chunk "copied in" and "applied", then the ends of the three
  // helper streams
  std::vector<cudaEvent_t> ev(4 + 2 * (size_t)nchunk, nullptr);
  int rc = PWK_OK;
  cudaError_t e = cudaSuccess;
  for (auto& x : ev)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
  // the copies into d_psi and the second compute stream wait for the work already queued on
  // the caller's stream
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->copy_in, ev[0], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->compute2, ev[0], 0);
  const char* bi = static_cast<const char*>(h_psi);
  char* bo = static_cast<char*>(h_hpsi);
  char* di = static_cast<char*>(d_psi);
  char* dout = static_cast<char*>(d_hpsi);
  for (int c = 0; c < nchunk && e == cudaSuccess && rc == PWK_OK; ++c) {
    const int k0 = group_start(p->nk, nchunk, c), k1 = group_start(p->nk, nchunk, c + 1);
    const size_t off = (size_t)k0 * per_k, bytes = (size_t)(k1 - k0) * per_k;
    cudaEvent_t in_done = ev[1 + 2 * c], applied = ev[2 + 2 * c];
    // groups alternate between two compute streams, so the small grids of one group's three
    // launches fill the GPU together with the next group's
    cudaStream_t cs = (c & 1) ? p->compute2 : st;
    e = cudaMemcpyAsync(di + off, bi + off, bytes, cudaMemcpyHostToDevice, p->copy_in);
    if (e == cudaSuccess) e = cudaEventRecord(in_done, p->copy_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, in_done, 0);
    if (e != cudaSuccess) break;
    rc = run_hpsi(p, precision, d_psi, d_hpsi, nullptr, nullptr, (k1 - k0) * nb, nb, nb, cs, nullptr, k0);
    if (rc != PWK_OK) break;
    e = cudaEventRecord(applied, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->copy_out, applied, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bo + off, dout + off, bytes, cudaMemcpyDeviceToHost, p->copy_out);
  }
  // the caller's stream completes after everything this call queued on the helper streams
  // (on success the last copy back; after an error whatever was queued before it), so that a
  // synchronisation of `stream` always covers the buffers
  {
    cudaStream_t helpers[3] = {p->copy_in, p->compute2, p->copy_out};
    for (int h = 0; h < 3; ++h) {
      cudaEvent_t x = ev[ev.size() - 3 + h];
      if (x == nullptr) continue;
      cudaError_t e2 = cudaEventRecord(x, helpers[h]);
      if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(st, x, 0);
      if (e == cudaSuccess) e = e2;
    }
  }
  for (auto& x : ev)
    if (x != nullptr) cudaEventDestroy(x);   // released once the event completes
  if (rc != PWK_OK) return rc;
  return e == cudaSuccess ? PWK_OK : cuda_fail(e, "pwk_hpsi_batched_host");
}

int pwk_plan_set_overlap(pwk_plan* p, const double* q) {
  if (p == nullptr) {
    set_error("null plan");
    return PWK_ERR_INVALID;
  }
  if (cudaError_t e = cudaSetDevice(p->device); e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  if (cudaError_t e = cudaDeviceSynchronize(); e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  plan_free(p, p->d_q);
  plan_free(p, p->d_q32);
  p->d_q = nullptr;
  p->d_q32 = nullptr;
  if (q == nullptr || p->nkb == 0) return PWK_OK;
  const size_t n2 = (size_t)p->nkb * p->nkb;
  for (size_t i = 0; i < n2; ++i) {
    const size_t r = i / p->nkb, c = i % p->nkb;
    if (!std::isfinite(q[i]) || q[i] != q[c * p->nkb + r]) {
      set_error("q must be finite and symmetric");
      return PWK_ERR_INVALID;
    }
  }
  std::vector<float> q32(q, q + n2);
  int r = plan_alloc(p, (void**)&p->d_q, sizeof(double) * n2);
  if (r == PWK_OK) r = plan_alloc(p, (void**)&p->d_q32, sizeof(float) * n2);
  if (r != PWK_OK) {
    plan_free(p, p->d_q);
    p->d_q = nullptr;
    return r;
  }
  cudaError_t e = cudaMemcpy(p->d_q, q, sizeof(double) * n2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_q32, q32.data(), sizeof(float) * n2, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(q)");
  return PWK_OK;
}

int pwk_plan_has_overlap(const pwk_plan* p) { return p != nullptr && p->d_q != nullptr ? 1 : 0; }

static int check_hs(pwk_plan* p, int precision, const void* psi, const void* hpsi, const void* spsi) {
  if (p == nullptr || psi == nullptr || hpsi == nullptr || spsi == nullptr) {
    set_error("null pointer");
    return PWK_ERR_INVALID;
  }
  if (precision < 0 || precision > 2) {
    set_error("unknown precision");
    return PWK_ERR_INVALID;
  }
  if (spsi == psi || spsi == hpsi || hpsi == psi) {
    set_error("psi, hpsi and spsi must be three different buffers");
    return PWK_ERR_INVALID;
  }
  return PWK_OK;
}

int pwk_hspsi_batched(pwk_plan* p, int precision, const void* psi, void* hpsi, void* spsi, int nb,
                      void* stream) {
  if (int r = check_hs(p, precision, psi, hpsi, spsi)) return r;
  if (nb < 1) {
    set_error("nb < 1");
    return PWK_ERR_INVALID;
  }
  const long long nblocks = (long long)p->nk * nb;
  if (nblocks > 0x7fffffffLL) {
    set_error("nk * nb too large for one launch");
    return PWK_ERR_UNSUPPORTED;
  }
  return run_hpsi(p, precision, psi, hpsi, nullptr, nullptr, (int)nblocks, nb, nb,
                  static_cast<cudaStream_t>(stream), spsi);
}

int pwk_hspsi_items(pwk_plan* p, int precision, const void* psi, void* hpsi, void* spsi,
                    const int* items, int nitems, int nvec_per_k, void* stream) {
  if (int r = check_hs(p, precision, psi, hpsi, spsi)) return r;
  if ((nitems > 0 && items == nullptr) || nitems < 0 || nvec_per_k < 1) {
    set_error("null pointer or bad size");
    return PWK_ERR_INVALID;
  }
  return run_hpsi(p, precision, psi, hpsi, items, nullptr, nitems, nvec_per_k, nvec_per_k,
                  static_cast<cudaStream_t>(stream), spsi);
}

int pwk_hpsi_multi(int nplans, pwk_plan* const* plans, int precision, const void* const* psi,
                   void* const* hpsi, const int* nvec_per_k, const int* items, int nitems, void* stream) {
  if (nplans < 1 || plans == nullptr || psi == nullptr || hpsi == nullptr || nvec_per_k == nullptr ||
      nitems < 0 || (nitems > 0 && items == nullptr)) {
    set_error("null pointer, nplans < 1 or nitems < 0");
    return PWK_ERR_INVALID;
  }
  if (precision < 0 || precision > 2) {
    set_error("unknown precision");
    return PWK_ERR_INVALID;
  }
  const pwk_plan* p0 = plans[0];
  for (int i = 0; i < nplans; ++i) {
    const pwk_plan* p = plans[i];
    if (p == nullptr || psi[i] == nullptr || hpsi[i] == nullptr || nvec_per_k[i] < 1) {
      set_error("null plan or vector array, or nvec_per_k < 1");
      return PWK_ERR_INVALID;
    }
    if (p->N != p0->N || p->device != p0->device) {
      set_error("the plans of one call must share the grid and the device");
      return PWK_ERR_INVALID;
    }
    if (!p->window_ok) {
      set_error("pwk_hpsi_multi needs spheres within the window kernel's |m_i| <= N/4");
      return PWK_ERR_UNSUPPORTED;
    }
  }
  if (nitems == 0) return PWK_OK;
  // one launch shape for every plan: the first plan's window shape of this precision (or the
  // kernel's default chunk), shared memory for the largest stick set and fused layout
  LaunchShape s;
  s.kind = p0->shape[precision].kind >= 1 ? p0->shape[precision].kind : 1;
  s.threads = p0->shape[precision].kind >= 1 ? p0->shape[precision].threads : 128;
  s.L = p0->shape[precision].kind >= 1 ? p0->shape[precision].L : std::max(1, p0->N / 3);
  if (s.kind == 2) s.L = std::min(s.L, 2);
  const int elem = precision == PWK_FP64 ? 16 : 8;
  int nst = 0;
  for (int i = 0; i < nplans; ++i) nst = std::max(nst, plans[i]->self.nstick_max);
  s.smem = window_smem_bytes(p0->N, elem, s.L, nst, s.kind == 2 ? s.threads / 32 : 1);
  std::vector<FusedArgs> d(nplans);
  size_t need = s.smem;
  for (int i = 0; i < nplans; ++i) {
    pwk_plan* p = plans[i];
    FusedArgs a = hpsi_args(p, precision, psi[i], hpsi[i]);
    a.nvec_in = a.nvec_out = nvec_per_k[i];
    a.L = s.L;
    use_kind(p, a, s.kind);
    if (p->nkb > 0) {
      const size_t b = fused_layout(p, precision, s, nullptr, nullptr);
      if (b > 227 * 1024) {
        set_error("a plan's projectors do not fit in shared memory next to the kernel's buffers");
        return PWK_ERR_UNSUPPORTED;
      }
      set_fused_nl(p, precision, a, nullptr, s);
      need = std::max(need, b);
    }
    d[i] = a;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* dd = nullptr;
  cudaError_t e = scratch_alloc(&dd, sizeof(FusedArgs) * nplans, st);
  if (e != cudaSuccess) return cuda_fail(e, "scratch_alloc(plan arguments)");
  e = cudaMemcpyAsync(dd, d.data(), sizeof(FusedArgs) * nplans, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    cudaFreeAsync(dd, st);
    return cuda_fail(e, "cudaMemcpyAsync(plan arguments)");
  }
  FusedArgs a0 = d[0];
  a0.items = items;
  a0.multi = static_cast<const FusedArgs*>(dd);
  a0.nmulti = nplans;
  a0.err = p0->d_err;
  LaunchShape sl = s;
  sl.smem = need;
  int rc = launch_window_multi_prec(precision, p0->N, a0, nitems, sl, st);
  e = cudaFreeAsync(dd, st);
  if (rc == PWK_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaFreeAsync(plan arguments)");
  return rc;
}

int pwk_hpsi_items(pwk_plan* p, int precision, const void* psi, void* hpsi, const int* items,
                   int nitems, int nvec_per_k, void* stream) {
  if (p == nullptr || psi == nullptr || hpsi == nullptr || (nitems > 0 && items == nullptr) ||
      nitems < 0 || nvec_per_k < 1) {
    set_error("null pointer or bad size");
    return PWK_ERR_INVALID;
  }
  if (precision < 0 || precision > 2) {
    set_error("unknown precision");
    return PWK_ERR_INVALID;
  }
  return run_hpsi(p, precision, psi, hpsi, items, nullptr, nitems, nvec_per_k, nvec_per_k,
                  static_cast<cudaStream_t>(stream));
}

}  // extern "C"
