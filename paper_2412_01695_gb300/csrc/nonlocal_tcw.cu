// Projector contractions on the 5th-generation tensor cores for wide projector sets (paper
// Sec. 2.2, Eqs. lambdah, gamma, finalnl: per k-point an (N_kb x npw) by (npw x N_b) product
// and an (npw x N_kb) by (N_kb x N_b) product), in FP32 arithmetic from TF32 inputs by the
// split x = hi + lo (hi rounded to TF32, lo = x - hi exact in FP32):
//   A B^T ~ A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T, accumulated in FP32 in tensor memory.
// One CTA per k-point of a batched call; the complex products are real GEMMs over the
// interleaved (re, im) values:
//
// Projection (nl_project_tcw_kernel), D = A B^T with M = 128 rows of projectors, N = bands
// (rounded up to 16), K = the plane waves of the k-point in blocks of 16 (32 floats: one
// 128-byte row of a 128-byte-swizzled K-major tile):
//   A row m        = [ Re b_m(G),  Im b_m(G), ...]   -> Re lambda_m     (m < nkb)
//   A row nkb + m  = [-Im b_m(G),  Re b_m(G), ...]   -> Im lambda_m
//   B row n        = [ Re C_n(G),  Im C_n(G), ...]
// so D[m][n] = Re lambda_m(n), D[nkb + m][n] = Im lambda_m(n) (lambda = sum_G conj(beta) C);
// gamma = D lambda and delta = q lambda follow on the CUDA cores into the coefficient scratch
// the add-back reads.  Pipeline: asynchronous copies of raw blocks into a ring, seven producer
// warps splitting them into hi/lo tiles of a stage, one lane issuing the stage's MMAs,
// mbarriers between them, every wait bounded (polls and wall time).
//
// Add-back (nl_addback_tcw_kernel), D = A B^T with M = 128 plane waves per tile, N = 2 nb
// (rounded up to 16: the real and imaginary part of each band), K = the projectors in blocks
// of 16 (32 floats):
//   A row G               = [ Re b_m(G), Im b_m(G), ...]          (m in the block)
//   B row 2n   (Re part)  = [ Re gamma_m(n), -Im gamma_m(n), ...]
//   B row 2n+1 (Im part)  = [ Im gamma_m(n),  Re gamma_m(n), ...]
// so D[G][2n + c] is part c of sum_m gamma_m(n) beta_m(G), added to H C_n(G).  The B tiles of
// every projector block are built once per CTA from the coefficient scratch; the A tiles come
// from beta(k) block by block (a gather of 16 projector rows into plane-wave rows).
//
// Padding rows (projectors beyond nkb, bands beyond nb) are zero in every tile, so the MMAs
// read only defined values and the unused rows and columns of D are zero.
#include <cstdint>

#include "fft_line.cuh"
#include "pwk_internal.h"

namespace pwk {

namespace {

constexpr int kThreads = 256;
constexpr int kProducers = 224;          // warps 0..6 copy and split; warp 7 issues the MMAs
constexpr int kStages = 3;               // hi/lo tile stages
constexpr int kTileA = 128 * 128;        // bytes of a 128-row tile
// dynamic shared memory a CTA may use (227 KB less the kernels' static shared memory)
constexpr size_t kSmemCap = 226 * 1024;
// polls of the final wait for MMAs already issued when a kernel gives up (so that tensor
// memory is never freed under a running MMA), independent of the plan's wait bound
constexpr long long kDrainPolls = 1LL << 22;

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(saddr(mbar))
               : "memory");
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bounded wait for phase `parity` of an mbarrier: at most `polls` polls of at most about a
// microsecond each (the suspend-time hint) and at most kWaitNs of wall time; false if it ran out
constexpr uint64_t kWaitNs = 2000000000ull;
__device__ __forceinline__ bool wait_parity(uint64_t* mbar, uint32_t parity, long long polls) {
  uint32_t done = 0;
  const uint64_t t0 = polls > 0 ? now_ns() : 0;
  for (long long it = 0; it < polls && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(saddr(mbar)), "r"(parity), "r"(1000u)
        : "memory");
    if (!done && (it & 255) == 255 && now_ns() - t0 > kWaitNs) break;
  }
  return done != 0;
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void split4(float a, float b, float c, float d, float4& hi, float4& lo) {
  hi = make_float4(to_tf32(a), to_tf32(b), to_tf32(c), to_tf32(d));
  lo = make_float4(a - hi.x, b - hi.y, c - hi.z, d - hi.w);
}

// the 16-byte chunk c (0..7) of row r of a 128-byte-swizzled tile
__device__ __forceinline__ float4* chunk(unsigned char* tile, int r, int c) {
  return reinterpret_cast<float4*>(tile + r * 128 + ((c ^ (r & 7)) << 4));
}

template <int B>
__device__ __forceinline__ void cp_async(void* dst, const void* src, int src_bytes) {
  if constexpr (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(saddr(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}

// tensor-memory columns for N accumulator columns (a power of two, at least 32)
__host__ __device__ constexpr uint32_t tmem_cols(int n) {
  return n <= 32 ? 32u : n <= 64 ? 64u : n <= 128 ? 128u : 256u;
}

// 16 consecutive FP32 columns of this warp's 32 lanes of tensor memory
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ int round16(int n) { return (n + 15) & ~15; }

// ----------------------------------------------------------------------------- projection
template <typename TI, int RING>
__global__ void __launch_bounds__(kThreads, 1) nl_project_tcw_kernel(NlArgs a) {
  using VI = c2_t<TI>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
  __shared__ uint32_t tmem_base;
  __shared__ int failed, pfail[2], last_issued;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kr = blockIdx.x, k = a.k0 + kr;
  const int nb = a.nvec_in, nkb = a.nkb, np = a.npw[k];
  const int NB = round16(nb);
  const int nblk = (np + 15) / 16;
  const int b_bytes = NB * 128;
  const int stage_bytes = 2 * kTileA + 2 * b_bytes;
  unsigned char* base = smem_raw + ((1024u - (saddr(smem_raw) & 1023u)) & 1023u);
  const int raw_c = nb * 16 * (int)sizeof(VI), raw_slot = raw_c + nkb * 16 * (int)sizeof(float2);
  unsigned char* ring = base + kStages * stage_bytes;
  auto a_hi = [&](int s) { return base + s * stage_bytes; };
  auto a_lo = [&](int s) { return base + s * stage_bytes + kTileA; };
  auto b_hi = [&](int s) { return base + s * stage_bytes + 2 * kTileA; };
  auto b_lo = [&](int s) { return base + s * stage_bytes + 2 * kTileA + b_bytes; };
  const uint32_t ncol = tmem_cols(NB);

  // padding rows, zero in every stage: projector rows 2 nkb .. 127 of A, band rows nb .. NB-1 of B
  for (int i = tid; i < kStages * 2 * (128 + NB) * 8; i += kThreads) {
    const int c = i & 7, rr = i >> 3;
    const int rows = 128 + NB;
    const int s = rr / (2 * rows), t = (rr / rows) & 1, r = rr % rows;
    float4* p = nullptr;
    if (r < 128) {
      if (r >= 2 * nkb) p = reinterpret_cast<float4*>((t ? a_lo(s) : a_hi(s)) + r * 128) + c;
    } else if (r - 128 >= nb) {
      p = reinterpret_cast<float4*>((t ? b_lo(s) : b_hi(s)) + (r - 128) * 128) + c;
    }
    if (p) *p = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(&tmem_base)),
                 "r"(ncol));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    failed = 0;
    pfail[0] = pfail[1] = 0;
    last_issued = -1;
    for (int j = 0; j < kStages; ++j) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(saddr(&full[j])), "r"(kProducers));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(saddr(&empty[j])), "r"(1));
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;

  const VI* cin = static_cast<const VI*>(a.in) + (size_t)k * a.nvec_in * a.npw_max;
  const float2* bin = static_cast<const float2*>(a.beta) + (size_t)k * nkb * a.npw_max;
  // block b into ring slot b % RING: nb rows of 16 coefficients, nkb rows of 16 projector
  // values (one complex element per copy; zero-filled past npw(k))
  // 8-byte elements (FP32 coefficients, beta) go two plane waves per 16-byte copy when every
  // row starts on a 16-byte boundary (even npw_max, aligned bases); the part of a pair past
  // npw(k) is zero-filled
  const bool pairs = (a.npw_max % 2 == 0) && ((reinterpret_cast<uintptr_t>(a.in) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(a.beta) & 15) == 0);
  auto fetch = [&](int b) {
    if (b < nblk) {
      unsigned char* slot = ring + (b % RING) * raw_slot;
      if (pairs) {
        constexpr int per = sizeof(VI) == 8 ? 8 : 16;   // copies per band row
        for (int t = tid; t < per * nb + 8 * nkb; t += kProducers) {
          if (t < per * nb) {
            const int r = t / per, j = t - r * per;
            if constexpr (sizeof(VI) == 8) {
              const int g = 16 * b + 2 * j, nin = g + 1 < np ? 2 : (g < np ? 1 : 0);
              cp_async<16>(slot + (r * 16 + 2 * j) * 8, cin + (size_t)r * a.npw_max + (nin ? g : 0), 8 * nin);
            } else {
              const int g = 16 * b + j;
              const bool in = g < np;
              cp_async<16>(slot + (r * 16 + j) * 16, cin + (size_t)r * a.npw_max + (in ? g : 0), in ? 16 : 0);
            }
          } else {
            const int u = t - per * nb, m = u >> 3, j = u & 7;
            const int g = 16 * b + 2 * j, nin = g + 1 < np ? 2 : (g < np ? 1 : 0);
            cp_async<16>(slot + raw_c + (m * 16 + 2 * j) * 8, bin + (size_t)m * a.npw_max + (nin ? g : 0), 8 * nin);
          }
        }
      } else {
        for (int t = tid; t < 16 * (nb + nkb); t += kProducers) {
          const int r = t >> 4, j = t & 15, g = 16 * b + j;
          const bool in = g < np;
          if (r < nb) {
            cp_async<sizeof(VI)>(slot + (r * 16 + j) * sizeof(VI), cin + (size_t)r * a.npw_max + (in ? g : 0),
                                 in ? (int)sizeof(VI) : 0);
          } else {
            const int m = r - nb;
            cp_async<8>(slot + raw_c + (m * 16 + j) * 8, bin + (size_t)m * a.npw_max + (in ? g : 0), in ? 8 : 0);
          }
        }
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  // split tasks: four plane waves of a band row (B) or of a projector (two A rows)
  const int ntask = 4 * (nb + nkb);
  auto split = [&](int b, int s) {
    const unsigned char* slot = ring + (b % RING) * raw_slot;
    for (int t = tid; t < ntask; t += kProducers) {
      const bool is_c = t < 4 * nb;
      const int row = is_c ? (t >> 2) : ((t - 4 * nb) >> 2);
      const int grp = t & 3;
      float2 v[4];
      if (is_c) {
        const VI* x = reinterpret_cast<const VI*>(slot) + row * 16 + 4 * grp;
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = make_float2(float(x[j].x), float(x[j].y));
      } else {
        const float2* x = reinterpret_cast<const float2*>(slot + raw_c) + row * 16 + 4 * grp;
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = x[j];
      }
      float4 h0, l0, h1, l1;
      split4(v[0].x, v[0].y, v[1].x, v[1].y, h0, l0);
      split4(v[2].x, v[2].y, v[3].x, v[3].y, h1, l1);
      if (is_c) {   // B row `row`: [re, im] of plane waves 4 grp .. 4 grp + 3
        *chunk(b_hi(s), row, 2 * grp) = h0;
        *chunk(b_hi(s), row, 2 * grp + 1) = h1;
        *chunk(b_lo(s), row, 2 * grp) = l0;
        *chunk(b_lo(s), row, 2 * grp + 1) = l1;
      } else {      // A row m: [re b, im b];  A row nkb + m: [-im b, re b]
        *chunk(a_hi(s), row, 2 * grp) = h0;
        *chunk(a_hi(s), row, 2 * grp + 1) = h1;
        *chunk(a_lo(s), row, 2 * grp) = l0;
        *chunk(a_lo(s), row, 2 * grp + 1) = l1;
        split4(-v[0].y, v[0].x, -v[1].y, v[1].x, h0, l0);
        split4(-v[2].y, v[2].x, -v[3].y, v[3].x, h1, l1);
        *chunk(a_hi(s), nkb + row, 2 * grp) = h0;
        *chunk(a_hi(s), nkb + row, 2 * grp + 1) = h1;
        *chunk(a_lo(s), nkb + row, 2 * grp) = l0;
        *chunk(a_lo(s), nkb + row, 2 * grp + 1) = l1;
      }
    }
  };
  const uint32_t idesc = idesc_tf32(128, NB);
  auto issue = [&](int s, int b) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t ah = saddr(a_hi(s)), al = saddr(a_lo(s)), bh = saddr(b_hi(s)), bl = saddr(b_lo(s));
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {   // K steps of 8 floats within the 128-byte row
      const uint32_t o = 32u * ks;
      mma_tf32(tmem, desc_sw128(ah + o), desc_sw128(bh + o), idesc, (b > 0 || ks > 0) ? 1u : 0u);
      mma_tf32(tmem, desc_sw128(ah + o), desc_sw128(bl + o), idesc, 1u);
      mma_tf32(tmem, desc_sw128(al + o), desc_sw128(bh + o), idesc, 1u);
    }
    mma_commit(&empty[s]);
  };

  if (warp < kProducers / 32) {
#pragma unroll 1
    for (int j = 0; j < RING - 1; ++j) fetch(j);
#pragma unroll 1
    for (int b = 0; b < nblk; ++b) {
      const int s = b % kStages;
      if (b >= kStages && !wait_parity(&empty[s], (uint32_t)(((b - kStages) / kStages) & 1), a.wait_polls))
        pfail[b & 1] = 1;
      asm volatile("cp.async.wait_group %0;\n" ::"n"(RING - 2) : "memory");
      asm volatile("bar.sync 1, %0;\n" ::"n"(kProducers) : "memory");
      if (pfail[b & 1]) break;
      fetch(b + RING - 1);
      split(b, s);
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(saddr(&full[s]))
                   : "memory");
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (pfail[0] | pfail[1]) failed = 1;
  } else if (lane == 0) {
#pragma unroll 1
    for (int b = 0; b < nblk; ++b) {
      const int s = b % kStages;
      if (!wait_parity(&full[s], (uint32_t)((b / kStages) & 1), a.wait_polls)) {
        failed = 1;
        break;
      }
      issue(s, b);
      last_issued = b;
    }
  }
  __syncwarp();
  __syncthreads();
  // the last commit covers every MMA issued before it (after a failure this drains what was
  // issued before tensor memory is released; the bound is at least kDrainPolls)
  {
    const int lb = last_issued;
    if (lb >= 0) {
      const bool ok = wait_parity(&empty[lb % kStages], (uint32_t)((lb / kStages) & 1),
                                  a.wait_polls > kDrainPolls ? a.wait_polls : kDrainPolls);
      if (!ok || lb != nblk - 1) failed = 1;
    } else if (nblk > 0) {
      failed = 1;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  // lambda to shared memory (the stages are free now): lam[m'][n], m' < 2 nkb, n < nb
  float* lam = reinterpret_cast<float*>(base);
  if (!failed && warp < 4) {
    const int row = 32 * warp + lane;
    for (int c0 = 0; c0 < NB; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
      if (row < 2 * nkb) {
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (c0 + i < nb) lam[row * nb + c0 + i] = v[i];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (failed) {
    if (tid == 0 && a.err != nullptr) atomicOr(a.err, 2);
  } else {
    // gamma = D lambda (Eq. gamma), delta = q lambda (Eq. delta_eq), projectors in ascending order
    const float* D = static_cast<const float*>(a.D);
    const float* q = static_cast<const float*>(a.q);
    for (int t = tid; t < nb * nkb; t += kThreads) {
      const int n = t / nkb, i = t - n * nkb;
      float gr = 0.f, gi = 0.f, dr = 0.f, di = 0.f;
      for (int j = 0; j < nkb; ++j) {
        const float lr = lam[j * nb + n], li = lam[(nkb + j) * nb + n];
        const float dm = D[(size_t)i * nkb + j];
        gr += dm * lr;
        gi += dm * li;
        if (q != nullptr) {
          const float qm = q[(size_t)i * nkb + j];
          dr += qm * lr;
          di += qm * li;
        }
      }
      float2* cf = static_cast<float2*>(a.coef) + ((size_t)kr * a.nvec_in + n) * 2 * nkb;
      cf[i] = make_float2(gr, gi);
      cf[nkb + i] = make_float2(dr, di);
    }
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncol));
}

// copy-ring depth of the projection: 8 raw blocks in flight where shared memory allows, else 4
int project_tcw_ring(int nb, int nkb, int io_bytes);
size_t project_tcw_smem_ring(int nb, int nkb, int io_bytes, int ring) {
  const int NB = (nb + 15) & ~15;
  const size_t stages = (size_t)kStages * (2 * kTileA + 2 * NB * 128);
  const size_t rbytes = (size_t)ring * (nb * 16 * io_bytes + nkb * 16 * 8);
  const size_t lam = (size_t)2 * nkb * nb * 4;   // reuses the stages
  return (stages > lam ? stages : lam) + rbytes + 1024;
}
int project_tcw_ring(int nb, int nkb, int io_bytes) {
  return project_tcw_smem_ring(nb, nkb, io_bytes, 8) <= kSmemCap ? 8 : 4;
}
size_t project_tcw_smem(int nb, int nkb, int io_bytes) {
  return project_tcw_smem_ring(nb, nkb, io_bytes, project_tcw_ring(nb, nkb, io_bytes));
}

// ----------------------------------------------------------------------------- add-back
// Shared-memory layout of the add-back: the B hi/lo tiles of every projector block, two A
// buffers (hi/lo), two raw beta blocks ([16 projectors][128 plane waves] float2) and, when it
// fits, the tile of H C being updated ([nb][128] elements of the I/O type).
constexpr int kRawBlock = 16 * 128 * 8;
__host__ __device__ constexpr size_t addback_base_bytes(int nb, int nkb) {
  return (size_t)((nkb + 15) / 16) * 2 * ((2 * nb + 15) & ~15) * 128 + 2 * 2 * kTileA + 2 * kRawBlock + 1024;
}
__host__ __device__ constexpr size_t addback_hbuf_bytes(int nb, int io_bytes) { return (size_t)128 * nb * io_bytes; }
__host__ __device__ constexpr bool addback_uses_hbuf(int nb, int nkb, int io_bytes) {
  return addback_base_bytes(nb, nkb) + addback_hbuf_bytes(nb, io_bytes) <= kSmemCap;
}

// One CTA per k-point.  Per tile of 128 plane waves and per block of 16 projectors: the block
// of beta(k) (16 rows of 128 values, copied one step ahead into the other raw buffer) is split
// and transposed into an A tile (plane-wave rows), and one lane issues the tile's 12 MMAs
// (4 K steps x 3 products) against the block's B tile.  The tile of H C is copied into shared
// memory while the MMAs run; after the last block all eight warps add the accumulator (128
// plane waves x N) to it and store the sum.  Two A buffers alternate, so the split of a block
// overlaps the MMAs of the previous one.
template <typename TI>
__global__ void __launch_bounds__(kThreads, 1) nl_addback_tcw_kernel(NlArgs a) {
  using VI = c2_t<TI>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t done[2];
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kr = blockIdx.x, k = a.k0 + kr;
  const int nb = a.nvec_in, nkb = a.nkb, np = a.npw[k];
  const int N2 = round16(2 * nb);
  const int nkblk = (nkb + 15) / 16;
  const int b_tile = N2 * 128;
  const bool use_hbuf = addback_uses_hbuf(nb, nkb, (int)sizeof(VI));
  unsigned char* base = smem_raw + ((1024u - (saddr(smem_raw) & 1023u)) & 1023u);
  unsigned char* btiles = base;
  unsigned char* abuf = base + (size_t)nkblk * 2 * b_tile;
  unsigned char* raw = abuf + 2 * 2 * kTileA;
  VI* hbuf = reinterpret_cast<VI*>(raw + 2 * kRawBlock);
  auto bh = [&](int j) { return btiles + (size_t)j * 2 * b_tile; };
  auto bl = [&](int j) { return btiles + (size_t)j * 2 * b_tile + b_tile; };
  auto ah = [&](int u) { return abuf + u * 2 * kTileA; };
  auto al = [&](int u) { return abuf + u * 2 * kTileA + kTileA; };
  const uint32_t ncol = tmem_cols(N2);

  // B tiles from gamma of the k-point's bands: row 2n = [Re g, -Im g], row 2n+1 = [Im g, Re g]
  // for the 16 projectors of block j; rows >= 2 nb and projectors >= nkb zero
  const float2* cf = static_cast<const float2*>(a.coef) + (size_t)kr * a.nvec_in * 2 * nkb;
  for (int t = tid; t < nkblk * N2 * 4; t += kThreads) {
    const int j = t / (N2 * 4), rem = t - j * N2 * 4, row = rem >> 2, grp = rem & 3;
    const int n = row >> 1, im = row & 1;
    float x[8];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int m = 16 * j + 4 * grp + u;
      float2 g = make_float2(0.f, 0.f);
      if (n < nb && m < nkb) g = cf[(size_t)n * 2 * nkb + m];
      x[2 * u] = im ? g.y : g.x;
      x[2 * u + 1] = im ? g.x : -g.y;
    }
    float4 h0, l0, h1, l1;
    split4(x[0], x[1], x[2], x[3], h0, l0);
    split4(x[4], x[5], x[6], x[7], h1, l1);
    *chunk(bh(j), row, 2 * grp) = h0;
    *chunk(bh(j), row, 2 * grp + 1) = h1;
    *chunk(bl(j), row, 2 * grp) = l0;
    *chunk(bl(j), row, 2 * grp + 1) = l1;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(&tmem_base)),
                 "r"(ncol));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    failed = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(saddr(&done[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(saddr(&done[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_tf32(128, N2);
  const float2* bk = static_cast<const float2*>(a.beta) + (size_t)k * nkb * a.npw_max;
  VI* hout = static_cast<VI*>(a.out) + (size_t)k * a.nvec_out * a.npw_max;
  const int ntile = (np + 127) / 128;
  const int nstep = ntile * nkblk;
  // beta block of step s (tile s / nkblk, projector block s % nkblk) into raw buffer s & 1
  // (zero outside the k-point's plane waves and projectors); one commit group per call
  auto fetch_block = [&](int s) {
    if (s < nstep) {
      const int t = s / nkblk, j = s - t * nkblk;
      unsigned char* dst = raw + (s & 1) * kRawBlock;
      for (int e = tid; e < 16 * 128; e += kThreads) {
        const int m = 16 * j + (e >> 7), g = 128 * t + (e & 127);
        const bool in = m < nkb && g < np;
        cp_async<8>(dst + e * 8, bk + (in ? (size_t)m * a.npw_max + g : 0), in ? 8 : 0);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  // the tile of H C (bands x 128 plane waves) into hbuf; one commit group per call
  auto fetch_h = [&](int t) {
    if (use_hbuf && t < ntile) {
      for (int e = tid; e < nb * 128; e += kThreads) {
        const int n = e >> 7, g = 128 * t + (e & 127);
        const bool in = g < np;
        cp_async<sizeof(VI)>(hbuf + e, hout + (size_t)n * a.npw_max + (in ? g : 0), in ? (int)sizeof(VI) : 0);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  auto wait_groups = [&](int pending) {   // all but the `pending` most recent groups complete
    if (pending <= 0) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    else if (pending == 1) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    else asm volatile("cp.async.wait_group 2;\n" ::: "memory");
  };
  // per A buffer: a commit not yet waited for, and the parity of its completion (every thread
  // keeps the same copy: the control flow is uniform)
  bool pend[2] = {false, false};
  uint32_t ph[2] = {0u, 0u};
  auto wait_buf = [&](int u, long long polls) {
    if (!pend[u]) return true;
    if (!wait_parity(&done[u], ph[u], polls)) return false;
    ph[u] ^= 1u;
    pend[u] = false;
    return true;
  };
  // groups in order: block 0, H tile 0, block 1, [H tile 1 after the epilogue of tile 0], ...
  fetch_block(0);
  fetch_h(0);
  int step = 0;
  // `failed` is read only right after a barrier that follows every write to it, and the
  // decision is kept in `stop`, so every thread leaves the loops at the same barrier
  bool stop = false;
#pragma unroll 1
  for (int t = 0; t < ntile && !stop; ++t) {
    const int g0 = 128 * t;
#pragma unroll 1
    for (int j = 0; j < nkblk; ++j, ++step) {
      const int u = step & 1;
      // A buffer u is free once its previous MMA group has completed
      if (!wait_buf(u, a.wait_polls)) failed = 1;
      fetch_block(step + 1);
      // groups issued after this step's block: the next block, and H tile t at j == 0
      wait_groups(j == 0 ? 2 : 1);
      __syncthreads();
      if (failed) {
        stop = true;
        break;
      }
      // A rows = plane waves: row r, chunks 2 grp, 2 grp + 1 = projectors 4 grp .. 4 grp + 3
      // of the block as [re, im, re, im]
      const float2* x = reinterpret_cast<const float2*>(raw + (step & 1) * kRawBlock);
      for (int e = tid; e < 128 * 4; e += kThreads) {
        const int r = e >> 2, grp = e & 3;
        const float2 v0 = x[(4 * grp) * 128 + r], v1 = x[(4 * grp + 1) * 128 + r];
        const float2 v2 = x[(4 * grp + 2) * 128 + r], v3 = x[(4 * grp + 3) * 128 + r];
        float4 h0, l0, h1, l1;
        split4(v0.x, v0.y, v1.x, v1.y, h0, l0);
        split4(v2.x, v2.y, v3.x, v3.y, h1, l1);
        *chunk(ah(u), r, 2 * grp) = h0;
        *chunk(ah(u), r, 2 * grp + 1) = h1;
        *chunk(al(u), r, 2 * grp) = l0;
        *chunk(al(u), r, 2 * grp + 1) = l1;
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t a_h = saddr(ah(u)), a_l = saddr(al(u)), b_h = saddr(bh(j)), b_l = saddr(bl(j));
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint32_t o = 32u * ks;
          mma_tf32(tmem, desc_sw128(a_h + o), desc_sw128(b_h + o), idesc, (j > 0 || ks > 0) ? 1u : 0u);
          mma_tf32(tmem, desc_sw128(a_h + o), desc_sw128(b_l + o), idesc, 1u);
          mma_tf32(tmem, desc_sw128(a_l + o), desc_sw128(b_h + o), idesc, 1u);
        }
        mma_commit(&done[u]);
      }
      pend[u] = true;
    }
    if (stop) break;
    // the tile's accumulator is complete when both buffers' last groups have completed; the
    // H tile when every group but the next block's has
    if (!wait_buf(0, a.wait_polls) || !wait_buf(1, a.wait_polls)) failed = 1;
    wait_groups(1);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (failed) {
      stop = true;
      break;
    }
    // H C_n(G) += D[G][2n] + i D[G][2n+1]: warp w reads tensor-memory lanes 32 (w % 4) ..
    // (its plane waves) and every other 16-column chunk from w / 4
    {
      const int row = 32 * (warp & 3) + lane, g = g0 + row;
      for (int c0 = 16 * (warp >> 2); c0 < N2; c0 += 32) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0, v);
        if (g < np) {
          VI h[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int n = c0 / 2 + i;
            if (n < nb) h[i] = use_hbuf ? hbuf[n * 128 + row] : hout[(size_t)n * a.npw_max + g];
          }
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int n = c0 / 2 + i;
            if (n < nb) hout[(size_t)n * a.npw_max + g] = VI{h[i].x + TI(v[2 * i]), h[i].y + TI(v[2 * i + 1])};
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    fetch_h(t + 1);   // hbuf is free again
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  // after a failure: drain the MMA groups already issued before tensor memory is released
  wait_buf(0, kDrainPolls);
  wait_buf(1, kDrainPolls);
  if (failed && tid == 0 && a.err != nullptr) atomicOr(a.err, 2);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncol));
}

size_t addback_tcw_smem(int nb, int nkb, int io_bytes) {
  return addback_base_bytes(nb, nkb) + (addback_uses_hbuf(nb, nkb, io_bytes) ? addback_hbuf_bytes(nb, io_bytes) : 0);
}

}  // namespace

// The wide tensor-core kernels apply to FP32 arithmetic (PWK_FP32, PWK_FP32_C128) on batched
// calls over whole k-points, 2 nkb <= 128 projector rows, nb <= 128 bands, and shapes whose
// tiles fit in shared memory.
int nl_tcw_applies(int precision, const NlArgs& a) {
  if (precision == PWK_FP64 || a.items != nullptr || a.d_count != nullptr) return 0;
  if (a.nkb < 1 || 2 * a.nkb > 128 || a.nvec_in != a.nvec_out || a.nvec_in < 1 || a.nvec_in > 128) return 0;
  if (a.nitems % a.nvec_in != 0) return 0;
  if (a.phase == 1 && a.sout != nullptr) return 0;   // S C: the CUDA-core add-back
  const int io = precision == PWK_FP32 ? 8 : 16;
  if (project_tcw_smem(a.nvec_in, a.nkb, io) > kSmemCap) return 0;
  if (addback_tcw_smem(a.nvec_in, a.nkb, io) > kSmemCap) return 0;
  return 1;
}

int launch_nl_tcw(int precision, const NlArgs& a, cudaStream_t st) {
  const int nkl = a.nitems / a.nvec_in;
  if (nkl == 0) return PWK_OK;
  cudaError_t e;
  const bool f32 = precision == PWK_FP32;
  if (a.phase == 0) {
    const int io = f32 ? 8 : 16;
    const size_t smem = project_tcw_smem(a.nvec_in, a.nkb, io);
    const bool deep = project_tcw_ring(a.nvec_in, a.nkb, io) == 8;
    auto go = [&](auto kern) -> cudaError_t {
      cudaError_t e2 = allow_full_smem(kern);
      if (e2 != cudaSuccess) return e2;
      kern<<<nkl, kThreads, smem, st>>>(a); note_launch();
      return cudaSuccess;
    };
    if (f32) e = deep ? go(nl_project_tcw_kernel<float, 8>) : go(nl_project_tcw_kernel<float, 4>);
    else e = deep ? go(nl_project_tcw_kernel<double, 8>) : go(nl_project_tcw_kernel<double, 4>);
    if (e != cudaSuccess) return cuda_fail(e, "attr(tcw)");
  } else {
    const size_t smem = addback_tcw_smem(a.nvec_in, a.nkb, f32 ? 8 : 16);
    if (f32) {
      if ((e = allow_full_smem(nl_addback_tcw_kernel<float>)) != cudaSuccess) return cuda_fail(e, "attr(tcw)");
      nl_addback_tcw_kernel<float><<<nkl, kThreads, smem, st>>>(a); note_launch();
    } else {
      if ((e = allow_full_smem(nl_addback_tcw_kernel<double>)) != cudaSuccess) return cuda_fail(e, "attr(tcw)");
      nl_addback_tcw_kernel<double><<<nkl, kThreads, smem, st>>>(a); note_launch();
    }
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? PWK_OK : cuda_fail(e, "tensor-core projector kernel");
}

}  // namespace pwk
