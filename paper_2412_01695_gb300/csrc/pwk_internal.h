// Internal declarations shared by the translation units of libpwk.so.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pwk.h"

// Grid sizes N (N1 = N2 = N3 = N) with an instantiated fused kernel.
#define PWK_FOR_EACH_N(X) X(12) X(15) X(16) X(18) X(20) X(24) X(25) X(27) X(30) X(32) X(36) X(40) X(45) X(48)

namespace pwk {

void set_error(const std::string& msg);  // thread-local detail for pwk_last_error_detail()
int cuda_fail(cudaError_t e, const char* what);
// Counts one kernel launch of the library (process-wide, read by pwk_launch_count).
void note_launch();

// Whether a kernel's shared-memory limit was already raised on a device (plan.cu; a
// process-wide table guarded by a mutex).
bool smem_limit_raised(const void* kern, int dev);
void mark_smem_limit_raised(const void* kern, int dev);

// Raises a kernel's dynamic shared-memory limit to the device's opt-in maximum (less the
// kernel's static shared memory), once per kernel and device: later launches skip the
// attribute calls (four runtime calls that cost more host time than a small launch).  The
// value set never depends on the launch, so host threads that launch the same kernel at the
// same time (one per stream in a serving loop) cannot lower the limit under one another's
// launch, and setting it twice is harmless.
template <typename K>
inline cudaError_t allow_full_smem(K kern) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const void* key = reinterpret_cast<const void*>(kern);
  if (smem_limit_raised(key, dev)) return cudaSuccess;
  cudaFuncAttributes fa;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) mark_smem_limit_raised(key, dev);
  return e;
}

// Device tables that place the coefficients of one sphere (input) on the FFT sticks and
// gather the coefficients of another (output) back: for H|psi> the two are the same
// sphere; for the DFPT right-hand side the input is the k sphere and the output the k+q one.
struct SphereMap {
  int nstick_max = 0;   // largest number of z-sticks over the k-points
  int m1lo = 0, P = 0;  // the m1 planes carried after the z-pass: m1 in [m1lo, m1lo + P)
  int npw_in_max = 0, npw_out_max = 0;
  int* d_nstick = nullptr;   // [nk]
  int* d_gin = nullptr;      // [nk][npw_in_max]  (stick << 8) | (m3 mod N)
  int* d_gout = nullptr;     // [nk][npw_out_max]
  short* d_sid = nullptr;    // [nk][P][N]: stick of (m1 = m1lo + p, m2 = slot) or -1
  const int* d_npw_in = nullptr;
  const int* d_npw_out = nullptr;
};

// Launch shape of the fused kernel for one precision.
struct LaunchShape {
  int kind = 0;         // 0: generic fused kernel, 1: window kernel, CTA-wide plane chunks,
                        // 2: window kernel, L planes per warp
  int threads = 256;
  int L = 0;            // l3 planes per chunk of the y/x passes
  size_t smem = 0;
};

struct DavWork;     // davidson.cu
struct CgWork;      // sternheimer.cu

}  // namespace pwk

struct pwk_plan {
  int device = 0;
  int N = 0, Nr = 0;
  int nk = 0, npw_max = 0, nkb = 0;
  double A[9] = {0}, B[9] = {0};
  std::vector<int> h_npw;
  std::vector<double> h_kcart;
  std::vector<int> h_miller;
  std::vector<double> h_D;
  // device tables
  int* d_npw = nullptr;
  double* d_kcart = nullptr;     // [nk][3]
  double* d_g2 = nullptr;        // [nk][npw_max] |k+G|^2
  const double2* d_beta = nullptr;   // caller-owned
  float2* d_beta32 = nullptr;
  double* d_D = nullptr;
  float* d_D32 = nullptr;
  double* d_q = nullptr;          // overlap coefficients q_mn (null: S = 1), pwk_plan_set_overlap
  float* d_q32 = nullptr;
  const double* d_V = nullptr;   // caller-owned
  float* d_V32 = nullptr;         // transposed [l2][l3][l1]
  double* d_Vt64 = nullptr;       // transposed [l2][l3][l1]
  double v_mean = 0.0;           // average of V over the grid (diagonal of the local term)
  pwk::SphereMap self;
  // window-specialised kernel tables (|m_i| <= (N-1)/4 on every sphere of the plan)
  bool window_ok = false;
  int* d_wgmap = nullptr;        // [nk][npw_max] (row << 8) | (m3 mod N), row = (m1+W)(2W+1)+(m2+W)
  short* d_wrows = nullptr;      // [nk][nstick_max] rows of the real sticks
  pwk::SphereMap xfer;           // from xfer_src's spheres to this plan's (DFPT rhs)
  const pwk_plan* xfer_src = nullptr;
  pwk::LaunchShape shape[3];     // per precision
  pwk::LaunchShape xshape;       // transfer kernel (complex dv, FP64)
  int projector_path = 0;        // 0 automatic, 1 tensor cores, 2 separate kernels, 3 fused
  bool nl_fused[3] = {false, false, false};   // automatic choice per precision (autotuner)
  bool nl_tc[3] = {false, false, false};      // separate kernels: tensor cores (autotuner)
  long long wait_polls = 1LL << 24;   // bound on the polls of each device-side wait
  int* d_err = nullptr;          // device error word (bad work items)
  // solver phase timing (pwk_plan_set_solver_timing): figures of the last solver call
  bool solver_timing = false;
  double solver_stats[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  double* d_flops = nullptr;     // device counter: FP64 flops of the reduced eigensolves
  // accounting
  size_t bytes = 0, budget = 0;
  std::vector<void*> allocs;
  std::vector<size_t> alloc_sizes;
  pwk::DavWork* dav = nullptr;
  pwk::CgWork* cg = nullptr;
  // streams of pwk_hpsi_batched_host (created on first use, non-blocking): copies in,
  // copies out, and a second compute stream for every other group of k-points
  std::mutex copy_mu;
  cudaStream_t copy_in = nullptr, copy_out = nullptr, compute2 = nullptr;
};

namespace pwk {
int plan_alloc(pwk_plan* p, void** ptr, size_t bytes);   // budget-checked cudaMalloc
void plan_free(pwk_plan* p, void* ptr);

// Arguments of the fused local-potential kernel (one CTA per work item).
struct FusedArgs {
  const void* in = nullptr;   // input vectors (complex of the io type)
  void* out = nullptr;        // output vectors
  const int* items = nullptr; // [n][3] (k, in_slot, out_slot) or null: item = (k - k0) * nvec + band
  const int* d_count = nullptr;  // if set, CTAs with blockIdx.x >= *d_count exit
  int k0 = 0;                    // first k-point of a batched (items == null) launch
  int nvec_in = 0, nvec_out = 0; // vectors per k in the in/out arrays
  int nk = 0;
  int npw_in_max = 0, npw_out_max = 0;
  const int* npw_in = nullptr;
  const int* npw_out = nullptr;
  const int* nstick = nullptr;
  const int* gin = nullptr;
  const int* gout = nullptr;
  const short* sid = nullptr;
  int nstick_max = 0, m1lo = 0, P = 0, L = 0, zs = 0;
  int yps = 0;                     // plane stride of the y/x chunk buffer (window kernel)
  const double* g2 = nullptr;      // kinetic table [nk][npw_out_max] or null
  const void* V = nullptr;         // real [N^3] of the arithmetic type, or complex128 dv
  double scale = 1.0;              // 1/N_r
  int* err = nullptr;
  // nonlocal projector terms fused into the kernel (nl_fused.cuh); beta == null: none
  const void* beta = nullptr;      // [nk][nkb][npw_beta] complex of the arithmetic type
  const void* Dm = nullptr;        // [nkb][nkb] real of the arithmetic type
  const void* qm = nullptr;        // [nkb][nkb] or null (S = 1)
  void* sout = nullptr;            // S C output (io type) or null
  int nkb = 0, npw_beta = 0;
  int nl_off = 0;                  // byte offset of the coefficients in dynamic shared memory
  int loc_off = 0;                 // window kernel: byte offset of the gathered local result and C
  // work lists over several plans (pwk_hpsi_multi): items are (plan, k, in, out) and the
  // plans' own arguments are multi[0 .. nmulti) in device memory
  const FusedArgs* multi = nullptr;
  int nmulti = 0;
};

size_t fused_smem_bytes(int N, int elem_bytes, int nstick_max, int P, int L, int npw_in_max);

// Arguments of the nonlocal projector kernels (nonlocal.cu): phase 0 computes gamma = D lambda
// and delta = q lambda of every item into coef; phase 1 adds sum gamma beta to out and, if
// sout is set, writes sout = in + sum delta beta.
struct NlArgs {
  int phase = 0;
  const void* in = nullptr;   // input vectors (complex of the io type)
  void* out = nullptr;        // H output (phase 1 adds to it)
  void* sout = nullptr;       // S output or null
  const int* items = nullptr; // [n][3] (k, in_slot, out_slot) or null: item = (k - k0) * nvec + band
  const int* d_count = nullptr;
  int k0 = 0;                  // first k-point of a batched (items == null) launch
  int nitems = 0, nvec_in = 0, nvec_out = 0, nk = 0, npw_max = 0;
  const int* npw = nullptr;
  const void* beta = nullptr;  // [nk][nkb][npw_max] complex of the arithmetic type
  const void* D = nullptr;     // [nkb][nkb] real of the arithmetic type
  const void* q = nullptr;     // [nkb][nkb] or null
  int nkb = 0;
  void* coef = nullptr;        // [nitems][2][nkb] complex of the arithmetic type
  int* err = nullptr;          // plan error word (bit 2: a tensor-core wait ran out)
  bool tensor_cores = false;   // projections on the tensor cores where they apply
  long long wait_polls = 1LL << 24;   // bound on the polls of each device-side wait
};
int launch_nl(int precision, const NlArgs& a, cudaStream_t st);
// tensor-core projection and add-back for wide projector sets (nonlocal_tcw.cu)
int nl_tcw_applies(int precision, const NlArgs& a);
int launch_nl_tcw(int precision, const NlArgs& a, cudaStream_t st);
// stream-ordered scratch from the library's per-device pool (memory returned with
// cudaFreeAsync stays mapped in the pool for later calls)
cudaError_t scratch_alloc(void** ptr, size_t bytes, cudaStream_t st);
size_t nl_shared_bytes(int nkb, int precision);

// launchers (one per arithmetic/io variant), defined in hpsi_*.cu
int launch_fused_f64(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st);
int launch_fused_f32(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st);
int launch_fused_f32c128(int N, const FusedArgs& a, int nblocks, const LaunchShape& s,
                         cudaStream_t st);
int launch_fused_xfer(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st);
int launch_window_f64(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st);
// the same kernels with the projector terms inside (a.beta set), defined in hpsi_*_nl.cu
int launch_fused_f64_nl(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st);
int launch_fused_f32_nl(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st);
int launch_fused_f32c128_nl(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st);
int launch_window_f64_nl(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st);
int launch_window_f32_nl(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st);
int launch_window_f32c128_nl(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st);
// work lists over several plans of one grid (pwk_hpsi_multi), defined in hpsi_multi.cu
int launch_window_multi_prec(int precision, int N, const FusedArgs& a, int nblocks, const LaunchShape& s,
                             cudaStream_t st);
int launch_window_f32(int N, const FusedArgs& a, int nblocks, const LaunchShape& s, cudaStream_t st);
int launch_window_f32c128(int N, const FusedArgs& a, int nblocks, const LaunchShape& s,
                          cudaStream_t st);
// copies: plane buffers (1 for a CTA-wide chunk, the warp count for per-warp planes)
size_t window_smem_bytes(int N, int elem_bytes, int L, int nstick_max, int copies);
// strides of the window kernel's shared buffers for chunk L (bank-conflict-free y/x passes)
void window_strides(int N, int L, int* zs, int* yps);

// fill FusedArgs for H|psi> with this plan
FusedArgs hpsi_args(const pwk_plan* p, int precision, const void* in, void* out);
// H (and, with sout set, S) on nblocks work items: projections, local + kinetic term,
// nonlocal add-back (three launches on st).  sout must not alias in.  out == null with sout
// set applies S alone.
// k0: first k-point of a batched launch (items == null): item i is band i % nvec_in of
// k-point k0 + i / nvec_in.
int run_hpsi(pwk_plan* p, int precision, const void* in, void* out, const int* items,
             const int* d_count, int nblocks, int nvec_in, int nvec_out, cudaStream_t st,
             void* sout = nullptr, int k0 = 0);

bool grid_supported(int N);
int build_sphere_map(pwk_plan* p, SphereMap& sm, int nk, const int* npw_in, int npw_in_max,
                     const int* miller_in, const int* npw_out, int npw_out_max,
                     const int* miller_out, const int* d_npw_in, const int* d_npw_out);
LaunchShape choose_shape(int N, int elem_bytes, const SphereMap& sm, int ctas_per_sm);
// stick maps from plan_k's spheres to plan_kq's (union of their sticks), kept in plan_kq
int ensure_xfer(pwk_plan* pq, const pwk_plan* pk);
}  // namespace pwk
