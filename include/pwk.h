/* pwk.h - C ABI of the many-k plane-wave Kohn-Sham library for one GB300 (sm_103a).
 *
 * The library applies the Kohn-Sham Hamiltonian to the Bloch wave-functions of many
 * k-points and bands at once (Gong & Dal Corso, arXiv:2412.01695, Sec. 2.2 and Sec. 3),
 * drives a batched block-Davidson eigensolver (Sec. 2.1, Algorithm 2) and a batched DFPT
 * Sternheimer preconditioned CG (Sec. 2.3-2.4, Algorithm 4) on the device.
 *
 * Units: Rydberg atomic units.  Lengths in bohr, wave-vectors in bohr^-1, energies in Ry;
 * the kinetic energy of a plane wave is |k+G|^2 (the Ry form of the paper's 1/2|k+G|^2 Ha).
 *
 * Layout conventions shared by every entry point:
 *   complex numbers are interleaved (re, im): complex128 = 2 x double, complex64 = 2 x float;
 *   wave-function arrays are [nk][nvec][npw_max], coefficient index fastest; entries
 *   beyond npw(k) are padding: they must be zero on input and are written as zero on output;
 *   real-space grids are [N1][N2][N3] with l3 fastest, r_l = sum_i (l_i/N_i) a_i (Sec. 4).
 *   Miller indices (m1, m2, m3) give G = m1 b1 + m2 b2 + m3 b3 with a_i . b_j = 2 pi delta_ij.
 *
 * Ownership: every device array passed in is owned by the caller and must stay alive and
 * unmodified for as long as the plan that references it (beta, vloc_r) or until the call
 * returns (everything else).  A plan owns only its own tables and workspaces.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 * Kernels are enqueued on it; entry points that iterate (Davidson, CG) synchronise the
 * stream internally to read convergence counters and return with results complete.
 *
 * Errors: every function returns an int.  0 = success; negative values are PWK_ERR_*
 * codes below (pwk_strerror() gives a message; pwk_last_error_detail() a detailed line
 * for the calling thread).  Positive values from the solvers count (k, band) pairs that did
 * not converge within max_iter.  Nothing throws across the ABI, nothing exits the process.
 */
#ifndef PWK_H
#define PWK_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PWK_OK 0
#define PWK_ERR_INVALID (-1)     /* bad argument (null pointer, size, index out of range) */
#define PWK_ERR_UNSUPPORTED (-2) /* valid but not supported (grid size, basis too large) */
#define PWK_ERR_NOMEM (-3)       /* device allocation failed */
#define PWK_ERR_BUDGET (-4)      /* would exceed the plan's HBM budget */
#define PWK_ERR_CUDA (-5)        /* a CUDA runtime call or kernel launch failed */
#define PWK_ERR_NOT_POSDEF (-6)  /* reduced overlap S~ not positive definite (Davidson) */
#define PWK_ERR_NUMERIC (-7)     /* CG breakdown (d^T A d <= 0) or non-finite values */

/* arithmetic of an H|psi> application */
#define PWK_FP64 0        /* complex128 in/out, FP64 arithmetic                          */
#define PWK_FP32 1        /* complex64 in/out, FP32 arithmetic                           */
#define PWK_FP32_C128 2   /* complex128 in/out, FP32 arithmetic (mixed-precision inner)  */

typedef struct pwk_plan pwk_plan; /* opaque */

/* ---------------------------------------------------------------------------- plans
 * pwk_plan_create: describe one cell, one FFT grid and one set of nk k-points with their
 * plane-wave spheres and projectors (paper Sec. 3: the data loaded on the GPU for a block
 * of N_k k-points before the Davidson or CG starts; Sec. 4 for the grids).
 *   A        host [3][3]   lattice vectors a_i as rows (bohr)
 *   N1,N2,N3               FFT grid; N1 = N2 = N3 = N with N in pwk_supported_grid()
 *   nk                     number of k-points (>= 1)
 *   kcart    host [nk][3]  k in cartesian coordinates (bohr^-1)
 *   npw      host [nk]     plane waves of each k (1 <= npw[k] <= npw_max)
 *   miller   host [nk][npw_max][3] Miller indices of the sphere of each k; every
 *                          |m_i| < N/2 and the npw[k] indices of one k distinct
 *   nkb                    total number of projectors over all atoms (0 allowed)
 *   beta     device [nk][nkb][npw_max] complex128: beta_i(k+G) (Eq. lambdah), zero padded
 *   D        host [nkb][nkb] real symmetric D^I_mn in Ry, zero between different atoms
 *   vloc_r   device [N1][N2][N3] float64: V_eff on the real-space grid (Sec. 2.2.2)
 *   hbm_budget bytes the plan may allocate on the device in total (0 = no limit)
 * The plan keeps FP32 copies of beta, D and V for the FP32 paths.  Returns PWK_OK and
 * *out, or an error (then *out is NULL).  Uses the current CUDA device; the caller must
 * make the same device current for every later call on the plan. */
int pwk_plan_create(pwk_plan** out, const double* A, int N1, int N2, int N3, int nk,
                    const double* kcart, const int* npw, int npw_max, const int* miller,
                    int nkb, const void* beta, const double* D, const double* vloc_r,
                    size_t hbm_budget);

/* Free every device table and workspace of the plan.  NULL is ignored. */
void pwk_plan_destroy(pwk_plan* plan);

/* Device bytes currently held by the plan (tables + workspaces). */
size_t pwk_plan_device_bytes(const pwk_plan* plan);

/* Launch shape of the H|psi> kernel for one precision (PWK_FP64, PWK_FP32 or PWK_FP32_C128):
 * kernel kind (0: general sphere kernel; 1: window kernel, usable when every |m_i| <= N/4,
 * the CTA taking l3 planes in chunks; 2: the window kernel with each warp taking its own
 * planes, l3_chunk = planes per warp, 1 or 2), threads per CTA, l3 planes per chunk and
 * dynamic shared memory per CTA.  pwk_plan_create times the candidate shapes on the plan's
 * own k-points and keeps the fastest; every shape computes the same operator (bitwise the
 * same result for kinds 1 and 2 and any threads / chunk; kind 0 rounds differently).
 * Any output pointer may be NULL. */
int pwk_plan_launch_shape(const pwk_plan* plan, int precision, int* kind, int* threads,
                          int* l3_chunk, size_t* smem_bytes);

/* Override the launch shape of one precision: kind 0, 1 or 2, threads 96, 128, 192 or 256,
 * 1 <= l3_chunk <= N.  Returns PWK_ERR_UNSUPPORTED if the shape does not fit in shared
 * memory or the window kernel does not apply to the plan (the shape is then unchanged). */
int pwk_plan_set_launch_shape(pwk_plan* plan, int precision, int kind, int threads, int l3_chunk);

/* How the nonlocal projector terms (Eqs. lambdah, gamma, finalnl; with q also delta_eq,
 * finals) are applied:
 *   0 (default)  automatic: path 2, unless path 3 or (FP32 arithmetic) path 1 ran more than
 *                3 % faster when pwk_plan_create timed them for each precision as whole H
 *                applications of 32 bands on the plan's own k-points (then the faster of
 *                the two; pwk_plan_projector_choice tells);
 *   1            separate kernels, both contractions of FP32 batched calls on whole k-points
 *                on the 5th-generation tensor cores where they apply (2 nkb <= 128, nb <= 128,
 *                tiles within shared memory; the S add-back stays on the CUDA cores): three
 *                TF32 products of a hi/lo split (FP32-level accuracy), FP32 accumulation in
 *                tensor memory; other calls fall back to path 2;
 *   2            separate CUDA-core kernels: projections before the local kernel, add-back
 *                after it, beta(k) staged in shared memory for eight bands at a time;
 *   3            inside the local kernel, so a band-k item makes one HBM round trip (read C,
 *                write H C and S C): after the transforms, the local result and C are kept in
 *                shared memory, beta(k) is staged into the freed buffers, and the projections,
 *                gamma (delta) and the add-back run from there.
 * Every path computes the same operator; they round differently (at FP32 or FP64 accuracy).
 * Path 3 (and 0) falls back to 2 where beta(k) does not fit in shared memory, and the S-only
 * application (drho) always uses 2.  PWK_ERR_INVALID for another value. */
int pwk_plan_set_projector_path(pwk_plan* plan, int path);
/* 1 if H|psi> of this precision applies the projector terms inside the local kernel (path 3,
 * or path 0 where the plan chose it), else 0; -1 for a null plan or unknown precision. */
int pwk_plan_projector_fused(const pwk_plan* plan, int precision);
/* The projector path H|psi> of this precision takes on whole-k-point batched calls under the
 * plan's current setting: 3 (inside the local kernel), 1 (separate tensor-core kernels), 2
 * (separate CUDA-core kernels), 0 if the plan has no projectors; -1 for a null plan or unknown
 * precision.  (Calls outside the tensor-core kernels' limits take path 2 where this says 1.) */
int pwk_plan_projector_choice(const pwk_plan* plan, int precision);

/* Device-side conditions the kernels of a plan recorded since the last clear (bit flags):
 *   PWK_FLAG_ITEM_SKIPPED  a work-list entry outside the plan was skipped (pwk_hpsi_items)
 *   PWK_FLAG_WAIT_TIMEOUT  a bounded device-side wait gave up (tensor-core projection): that
 *                          call's output is not valid; the context and the plan stay usable
 * Synchronises with the device (a blocking copy of one int); clear != 0 resets the flags. */
#define PWK_FLAG_ITEM_SKIPPED 1
#define PWK_FLAG_WAIT_TIMEOUT 2
int pwk_plan_errors(pwk_plan* plan, int* flags, int clear);

/* Bound on the polls of every device-side wait of the plan's kernels (default 2^24, a few
 * seconds).  A diagnostic: 0 makes every such wait give up at once, which exercises the error
 * path above without stalling the device.  PWK_ERR_INVALID for a negative value. */
int pwk_plan_set_wait_limit(pwk_plan* plan, long long polls);

/* 1 if an N x N x N grid is supported by the fused kernels, else 0. */
int pwk_supported_grid(int N);

/* ---------------------------------------------------------------------------- H|psi>
 * pwk_hpsi_batched: hpsi = H_KS psi for nb bands of every k of the plan (paper Sec. 2.2,
 * Sec. 3 "routine that applies H_KS ... for N_k k points"):
 *   kinetic |k+G|^2 C (Sec. 2.2.1), local V_eff by scatter G->r, inverse 3D transform,
 *   V(r) u(r), forward 3D transform with 1/N_r and gather r->G (Sec. 2.2.2, Sec. 4),
 *   nonlocal lambda = sum_G beta* C (Eq. lambdah), gamma = D lambda (Eq. gamma),
 *   add-back sum gamma beta (Eq. finalnl).  S is not applied (pwk_hspsi_batched does).
 *   precision  PWK_FP64, PWK_FP32 or PWK_FP32_C128
 *   psi        device [nk][nb][npw_max] complex128 (complex64 for PWK_FP32)
 *   hpsi       device, same shape and type; may be the same pointer as psi (in place),
 *              must not otherwise overlap it
 * Three launches on `stream` (projections, local and kinetic terms, nonlocal add-back); the
 * projector coefficients between them (2 nkb complex per band-k) take scratch for the call
 * from a stream-ordered memory pool the library keeps per device (memory returned to the
 * pool stays mapped for later calls).  Asynchronous on `stream`. */
int pwk_hpsi_batched(pwk_plan* plan, int precision, const void* psi, void* hpsi, int nb,
                     void* stream);

/* pwk_hpsi_batched_host: the operator of pwk_hpsi_batched on vectors that live in HOST
 * memory, for callers whose batches arrive from and return to the host (a serving loop):
 * the k-points are split into nchunk consecutive groups (with three or more, the first and
 * the last hold half as many k-points as the others), and the copy of group c + 1 to the
 * device, the H application of group c and the copy of group c - 1 back to the host run at
 * the same time (two copy streams and a second compute stream of the plan, created on first
 * use, ordered against `stream` by events; groups alternate between `stream` and the second
 * compute stream; the transfers are one asynchronous copy per group and direction).
 *   h_psi, h_hpsi  host [nk][nb][npw_max] complex128 (complex64 for PWK_FP32); page-locked
 *                  memory (cudaHostAlloc / cudaHostRegister) for the copies to overlap
 *   d_psi, d_hpsi  device work buffers of the same shape (the caller's; d_hpsi may equal
 *                  d_psi); on return from the stream they hold the batch and its result
 *   nchunk         groups, 1 <= nchunk (values above nk are taken as nk)
 * The result equals pwk_hpsi_batched's bit for bit (same kernels per band-k).  Asynchronous:
 * h_hpsi is complete when the work queued on `stream` by this call has completed; `stream`
 * also waits for the helper streams after an error, so its synchronisation always means the
 * buffers are no longer in use.  Errors:
 * PWK_ERR_INVALID for a null pointer, nb < 1, nchunk < 1 or an unknown precision; CUDA
 * failures as for pwk_hpsi_batched. */
int pwk_hpsi_batched_host(pwk_plan* plan, int precision, const void* h_psi, void* h_hpsi,
                          void* d_psi, void* d_hpsi, int nb, int nchunk, void* stream);

/* pwk_hpsi_items: the same operator on an explicit work list, for uneven batches (only the
 * listed vectors are transformed; the others are not touched).
 *   psi, hpsi   device [nk][nvec_per_k][npw_max] of the precision's complex type
 *   items       device int[nitems][3]: (k, in_slot, out_slot): hpsi[k][out_slot] =
 *               H(k) psi[k][in_slot].  An entry with k = -1 is an empty slot; an entry
 *               with another k outside [0, nk) or a slot outside [0, nvec_per_k) is
 *               skipped too (its output is left unchanged).
 *   nitems      number of entries (0 allowed: nothing is launched)
 * Two entries must not write the same output vector, and no output vector may be an input
 * of another entry.  Asynchronous on `stream`. */
int pwk_hpsi_items(pwk_plan* plan, int precision, const void* psi, void* hpsi, const int* items,
                   int nitems, int nvec_per_k, void* stream);

/* pwk_hpsi_multi: H|psi> on one work list whose entries belong to several plans -- cells with
 * their own atoms and projector sets (nkb may differ, 0 included), D, V(r), spheres and
 * k-points -- applied in a single launch (the paper batches the k-points of one cell, Sec. 3;
 * this extends the batch across cells that share an FFT grid, so uneven projector sets do
 * not split the work into one launch per cell).
 *   nplans      number of plans (>= 1); plans[i] the plan of cell i; all on one device with
 *               the same grid N, and every sphere within |m_i| <= N/4 (the window kernel)
 *   precision   PWK_FP64, PWK_FP32 or PWK_FP32_C128
 *   psi, hpsi   host arrays of nplans device pointers: psi[i], hpsi[i] are plan i's vectors
 *               [nk_i][nvec_per_k[i]][npw_max_i] of the precision's complex type
 *   nvec_per_k  host int[nplans]
 *   items       device int[nitems][4]: (plan, k, in_slot, out_slot): hpsi[plan][k][out_slot]
 *               = H_plan(k) psi[plan][k][in_slot].  plan = -1 marks an empty slot; an entry
 *               outside the plans, the plan's k-points or its slots is skipped (its output left
 *               unchanged) and flags PWK_FLAG_ITEM_SKIPPED on plans[0]
 *   nitems      number of entries (0: nothing is launched)
 * The projector terms run inside the kernel (one HBM round trip per item); the launch shape
 * is plans[0]'s window shape for the precision.  Two entries must not write the same output
 * vector, and no output may be an input of another entry (in place, hpsi[i] == psi[i], is
 * allowed).  The plans' arguments (a few hundred bytes each) take scratch from the library's
 * stream-ordered pool.  PWK_ERR_INVALID for mismatched plans or bad pointers,
 * PWK_ERR_UNSUPPORTED when a plan's spheres or projectors do not fit the window kernel.
 * Asynchronous on `stream`. */
int pwk_hpsi_multi(int nplans, pwk_plan* const* plans, int precision, const void* const* psi,
                   void* const* hpsi, const int* nvec_per_k, const int* items, int nitems, void* stream);

/* ---------------------------------------------------------------------------- overlap S
 * Ultrasoft / PAW overlap (paper Sec. 2.2):
 *   S C = C + sum_{I,mn} q^I_mn beta^I_m <beta^I_n|C>  (Eqs. lambdah, delta_eq, finals),
 * computed from the same projections lambda as the nonlocal term of H.
 *
 * pwk_plan_set_overlap: give the plan the coefficients q (host float64 [nkb][nkb], real
 * symmetric; block diagonal per atom like D, not enforced) or remove them (q = NULL: S = 1).
 * Copies q to the device (the caller keeps ownership of its array); synchronises the device.
 * Returns PWK_ERR_INVALID for a non-finite or non-symmetric q.  A plan with q makes
 * pwk_davidson_batched solve H x = eps S x and pwk_sternheimer_cg_batched use S (see there). */
int pwk_plan_set_overlap(pwk_plan* plan, const double* q);
/* 1 if the plan holds overlap coefficients q, else 0. */
int pwk_plan_has_overlap(const pwk_plan* plan);

/* pwk_hspsi_batched / pwk_hspsi_items: H C and S C together (one projection serves both),
 * same arguments as pwk_hpsi_batched / pwk_hpsi_items plus
 *   spsi   device, same shape and type as psi: S psi out (padding written as zero).
 * psi, hpsi and spsi must be three distinct, non-overlapping buffers (PWK_ERR_INVALID if two
 * pointers are equal).  Without q, S = 1 and spsi = psi.  Asynchronous on `stream`. */
int pwk_hspsi_batched(pwk_plan* plan, int precision, const void* psi, void* hpsi, void* spsi,
                      int nb, void* stream);
int pwk_hspsi_items(pwk_plan* plan, int precision, const void* psi, void* hpsi, void* spsi,
                    const int* items, int nitems, int nvec_per_k, void* stream);

/* ---------------------------------------------------------------------------- Davidson
 * pwk_davidson_batched: lowest nb eigenpairs of H(k) for every k of the plan by the block
 * Davidson iteration of Sec. 2.1, run for all k at once (Algorithm 2):
 *   Rayleigh-Ritz on the basis (H~ = <phi|H|phi>, S~ = <phi|S|phi>, FP64 Cholesky of S~ and
 *   Hermitian eigensolve, Sec. 5), correction vectors (H_diag - eps S_diag)^-1 (H - eps S) phi,
 *   normalisation, basis expansion, restart with the Ritz vectors when the basis would
 *   exceed max_basis, per-band test |eps^(n+1) - eps^(n)| > eth.
 *   mode     PWK_FP64: every H application in FP64.
 *            PWK_FP32_C128: expansion steps use FP32 H applications until the eigenvalue
 *            changes fall below max(eth, 1e-4 Ry) and the residuals below
 *            max(res_tol, 1e-3) (the FP32 noise floor), or for at most min(max_iter/2, 60)
 *            iterations; then the Ritz vectors get FP64 H applications and the iteration
 *            continues in FP64 to eth and res_tol (FP64 refinement).
 *            Reduced matrices, the eigensolve, norms and residuals are FP64 in both modes.
 *   psi      device [nk][nb][npw_max] complex128: trial vectors in, eigenvectors out (S-orthonormal)
 *   eig      device [nk][nb] float64: eigenvalues out (Ry), ascending per k
 *   eth      eigenvalue threshold (Ry), > 0
 *   res_tol  if > 0, a band also needs ||H phi - eps phi|| < res_tol to be converged
 *   max_iter iterations (>= 1); max_basis 2*nb <= max_basis <= 160 (0 = 4*nb, capped at 160)
 *   iters_out, notconv_out  host int[nk] or NULL: iterations used and bands left
 *                           unconverged per k
 *   napply_out host long long[2] or NULL: number of band H applications (FP64, FP32)
 * Workspaces are allocated in the plan on first use (and grown when needed).
 * Returns the number of unconverged (k, band) pairs (0 = all converged) or an error. */
int pwk_davidson_batched(pwk_plan* plan, int mode, void* psi, double* eig, int nb, double eth,
                         double res_tol, int max_iter, int max_basis, int* iters_out,
                         int* notconv_out, long long* napply_out, void* stream);

/* ---------------------------------------------------------------------------- induced density
 * pwk_drho_batched: the charge density induced by the perturbation (Eq. drho, Sec. 2.3),
 *   drho(r) = 4 sum_k w_k sum_{nu < nocc} conj(u_{k,nu}(r)) [P_c du_{k,nu}](r),
 * without the augmentation term (which the paper did not accelerate).  u(r) is the inverse
 * transform without normalisation of Sec. 2.2.2 (u on the k sphere of plan_k, du on the k+q
 * sphere of plan_kq); P_c du = du - sum_v psi_{k+q,v} <S psi_{k+q,v}|du> with the overlap of
 * plan_kq (S = 1 without q).
 *   plan_kq, plan_k  as for pwk_sternheimer_cg_batched (same nk, cell and grid)
 *   precision  PWK_FP64, or PWK_FP32_C128 (FP32 transforms, FP64 products and sums)
 *   psi_k      device [nk][nocc][npw_max(k)] complex128
 *   psi_kq     device [nk][nocc][npw_max(k+q)] complex128: valence states of k+q
 *              (S-orthonormal)
 *   dpsi       device [nk][nocc][npw_max(k+q)] complex128: du_{k,nu} (e.g. the output of
 *              pwk_sternheimer_cg_batched)
 *   weights    device float64 [nk]: w_k (1/N_k for a full unreduced grid)
 *   drho       device complex128 [N][N][N] (l3 fastest): overwritten with the result, per grid
 *              point (the 1/Omega of a density per volume is left out)
 * Each (k, nu) pair is transformed by one CTA and its product added to one of 256 partial
 * grids; the partial grids are summed in a fixed order, so the result is reproducible bit for
 * bit.  Scratch (P_c du, the partial grids) comes from the library's stream-ordered pool.
 * Asynchronous on `stream`. */
int pwk_drho_batched(pwk_plan* plan_kq, pwk_plan* plan_k, int precision, const void* psi_k,
                     const void* psi_kq, const void* dpsi, int nocc, const double* weights,
                     void* drho, void* stream);

/* pwk_eigh_batched: the batched generalized Hermitian eigensolver of the Davidson reduced
 * problem as a stand-alone call (paper Sec. 5: ZHEGV for many k-points at once).  For each
 * problem p < nprob: H_p v = eps S_p v, the nev lowest eigenpairs, FP64, one CTA per problem
 * (Cholesky of S, reduction to standard form, Householder tridiagonalisation, bisection and inverse iteration).
 *   H, S    device complex128 [nprob][n][n], row-major, full Hermitian; S positive definite
 *           (only its lower triangle is read)
 *   eig     device float64 [nprob][nev], ascending
 *   vec     device complex128 [nprob][n][nev]: column j is the eigenvector of eig[p][j],
 *           S-orthonormal
 *   status  device int [nprob] or NULL: 0, PWK_ERR_NOT_POSDEF (one of the first nev rows of
 *           S is dependent on the earlier ones) or PWK_ERR_NUMERIC (non-finite eigenvector)
 * A row j >= nev whose Cholesky pivot falls below 1e-6 S_jj is treated as dependent and left
 * out of the problem (its eigenvector entries are zero).  1 <= nev <= n <= 160.
 * Allocates a workspace of 3 n^2 complex128 per problem for the call and synchronises
 * `stream` before returning. */
int pwk_eigh_batched(int nprob, int n, int nev, const void* H, const void* S, double* eig,
                     void* vec, int* status, void* stream);

/* pwk_eigh_batched_noalloc: pwk_eigh_batched without any device allocation, for callers that
 * cannot call cudaMalloc where they solve: a latency-bound serving loop (cudaMalloc and
 * cudaFree synchronise the whole device and stall its other streams) or a process whose
 * device memory is entirely reserved by another allocator, so that a new cudaMalloc fails.
 * The paper has no counterpart: this is a deployment variant of the same eigensolver.
 * Same arguments, layouts and results as pwk_eigh_batched.  The workspace is a fixed array of
 * 19.7 MB in the library's device memory, held on every device that loads the library until
 * the process exits; it limits a call to nprob * n^2 <= 409600 (e.g. 16 problems of
 * n = 160, 256 of n = 40); larger calls return PWK_ERR_UNSUPPORTED and do nothing.
 * The first call on a device looks up the array's device address (once per device, with that
 * device current); make that first call before any stream capture.  The address is kept for
 * the life of the process: a cudaDeviceReset of a device unloads the array there, so a process
 * that resets a device must not call this entry point on that device afterwards.  Every call shares the
 * array (its previous contents are never read: the kernel writes each element before using
 * it), so calls that overlap on the GPU, on any streams, race: serialise them.
 * Asynchronous on `stream`: results are ready when the stream has synchronised. */
int pwk_eigh_batched_noalloc(int nprob, int n, int nev, const void* H, const void* S,
                             double* eig, void* vec, int* status, void* stream);

/* ---------------------------------------------------------------------------- Sternheimer
 * pwk_sternheimer_cg_batched: for every k of plan_k and every occupied band n, solve the
 * DFPT linear system of Eq. linear_system with dS = 0 (a local perturbation dv),
 *   [H_{k+q} + alpha_k Q - eps_{k,n} S] dpsi_{k,n} = -(1 - S P_v) dV psi_{k,n},
 * Q = sum_{v < nocc} S|psi_{k+q,v}><psi_{k+q,v}|S (Eq. projector, Eqs. compute_mu, use_mu,
 * apply_s_ch), P_v = sum_v |psi_{k+q,v}><psi_{k+q,v}|, dV = e^{iq.r} dv(r); S is the
 * overlap of plan_kq (S = 1 without q: [H + alpha P_v - eps] dpsi = -P_c dV psi; with q the
 * psi_{k+q,v} must be S-orthonormal), by the preconditioned CG of
 * Sec. 2.4 (Eqs. ax1 .. updatedold) for all (k, n) at once (Algorithm 4), with the
 * preconditioner M_GG = max(1, |k+q+G|^2 / <psi_{k+q,n}|T|psi_{k+q,n}>).
 *   plan_kq   plan of the k+q points (the operator); plan_k  plan of the k points; both
 *             have the same nk, cell and grid, point i of plan_kq being k_i + q
 *   mode      PWK_FP64: FP64 operator and CG vectors.  PWK_FP32_C128: FP64 iterative
 *             refinement (true residual with the FP64 operator, x in FP64) around an inner
 *             PCG on the correction with the FP32 operator and FP32 vectors; dot products
 *             are FP64 sums (of per-thread FP32 partials in the inner PCG) and the CG
 *             scalars are FP64 in both modes.
 *   psi_k     device [nk][nocc][npw_max(k)] complex128    occupied states at k
 *   eps_k     device [nk][nocc] float64                   their eigenvalues (Ry)
 *   psi_kq    device [nk][nocc][npw_max(k+q)] complex128  occupied states at k+q
 *   alpha     device [nk] float64                         alpha of each k (Ry)
 *   dv_r      device [N1][N2][N3] complex128              lattice-periodic part of dV
 *   dpsi      device [nk][nocc][npw_max(k+q)] complex128  solution out
 *   tol       relative residual ||A x - b|| / ||b|| to reach, per (k, n); the iteration aims
 *             at tol/2, so that an FP64 operator rounding differently still finds <= tol
 *   max_iter  CG iterations per solve (per refinement step in mixed mode)
 *   iters_out host int[nk*nocc] or NULL: CG iterations used
 *   resid_out host double[nk*nocc] or NULL: final true relative residual (FP64 operator)
 * Workspaces are allocated in plan_kq on first use.  Returns the number of (k, n) pairs
 * above tol, or an error. */
int pwk_sternheimer_cg_batched(pwk_plan* plan_kq, pwk_plan* plan_k, int mode,
                               const void* psi_k, const double* eps_k, const void* psi_kq,
                               int nocc, const double* alpha, const void* dv_r, void* dpsi,
                               double tol, int max_iter, int* iters_out, double* resid_out,
                               void* stream);

/* ---------------------------------------------------------------------------- solver timing
 * Where a solver call spends its device time (the paper splits its run times the same way:
 * H and S application, FFTs, reduced diagonalisation; Sec. 6, Tables 1-3).
 * pwk_plan_set_solver_timing(plan, 1) makes pwk_davidson_batched and
 * pwk_sternheimer_cg_batched (plan_kq) record CUDA events around their phases on their stream
 * (read after the synchronisations the solvers make anyway; 8 bytes of device memory for a
 * counter, allocated on the first switch-on); 0 switches it off.  pwk_plan_solver_stats then
 * gives the figures of the last such call on the plan:
 *   stats[0]  ms of device time in H (and S) applications
 *   stats[1]  ms in the batched reduced eigensolver (Davidson; 0 for the CG)
 *   stats[2]  ms from the call's first kernel to its last (device)
 *   stats[3]  algorithmic FP64 flops of the reduced eigensolves: 12 n^3 + 12 n^2 nb per
 *             problem of order n (the dense counts of Cholesky, reduction to standard form,
 *             tridiagonalisation and back-transform of nb vectors, 8 flops per complex
 *             multiply-add)
 *   stats[4]  stats[2] - stats[0] - stats[1]: the vector kernels and gaps
 * stats is host double[5].  PWK_ERR_INVALID for a null pointer. */
int pwk_plan_set_solver_timing(pwk_plan* plan, int on);
int pwk_plan_solver_stats(const pwk_plan* plan, double* stats);

/* ---------------------------------------------------------------------------- measurement
 * pwk_measure_fma_peak: the CUDA-core multiply-add throughput of the current device in FLOP/s
 * (2 per FMA), measured by a kernel that keeps every SM busy with independent FMA chains
 * (eight CTAs of 256 threads per SM, sixteen chains per thread), best of three timed launches
 * after a warm-up, CUDA events on `stream`.  The roofline denominator of the kernels bound by
 * these pipes: the transforms of the H|psi> kernel (FP32 or FP64), the reduced eigensolver
 * and the CG reductions (FP64); the paper states its peaks per node (Sec. 6) but no per-kernel
 * fraction, so this has no counterpart there.
 *   precision   PWK_FP32 or PWK_FP64 (PWK_ERR_INVALID otherwise)
 *   flops_per_s host double out (may be NULL)
 *   sm_count    host int out: the device's multiprocessor count (may be NULL)
 * Takes about 0.1-0.3 s; synchronises `stream`; 8 bytes of scratch from the library's pool. */
int pwk_measure_fma_peak(int precision, double* flops_per_s, int* sm_count, void* stream);

/* pwk_launch_count: how many kernels the library has launched in this process since it was
 * loaded (every launch of every entry point, counted on the host as it is queued; all devices
 * and threads together).  The difference of two readings around a region counts that region's
 * launches.  Never fails. */
long long pwk_launch_count(void);

/* ---------------------------------------------------------------------------- misc */
const char* pwk_strerror(int code);
/* Last detailed error message of the calling thread ("" if none). */
const char* pwk_last_error_detail(void);
/* Library version string. */
const char* pwk_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PWK_H */
