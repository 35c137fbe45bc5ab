// Projections lambda = beta^H C (Eq. lambdah) on the 5th-generation tensor cores, for the FP32
// arithmetic of the batched H|psi> (paper Sec. 2.2: per k a product of the N_kb x npw
// projector matrix and the npw x N_b coefficient matrix).
//
// One CTA per k-point.  The complex product is one real GEMM with the interleaved (re, im)
// coefficients as the K dimension:
//   A (M = bands, padded to 128 rows) row n = [Re C_n(G0), Im C_n(G0), Re C_n(G1), ...]
//   B (N = 32 rows) row m      = [Re b_m(G0),  Im b_m(G0),  ...]   -> Re lambda_m
//         row 16 + m           = [-Im b_m(G0), Re b_m(G0),  ...]   -> Im lambda_m
// so D = A B^T holds Re lambda in columns 0..15 and Im lambda in columns 16..31 (N_kb <= 16).
// FP32 accuracy from TF32 inputs by the split x = hi + lo (hi rounded to TF32, lo = x - hi
// exact in FP32): A B^T ~ A_hi B_hi + A_hi B_lo + A_lo B_hi, accumulated in FP32 in tensor
// memory (three kind::tf32 MMAs per K step of 8).
//
// The K dimension runs over blocks of 16 plane waves (32 floats = one 128-byte row of a
// 128-byte-swizzled K-major tile).  The raw coefficients and projectors of a block arrive by
// asynchronous copies in a ring of kTcRing blocks (kTcRing - 1 blocks in flight).  The CTA is
// warp-specialised: seven producer warps split the raw values of a block and write the
// swizzled hi/lo tiles of one of kTcStages shared-memory stages, then arrive on the stage's
// "full" mbarrier; one lane of the eighth warp waits on it, issues the 12 MMAs of the block
// and commits them to the stage's "empty" mbarrier, which the producers wait on before they
// overwrite the stage kTcStages blocks later.  The MMA issue thus overlaps the preparation of
// the next blocks.
// Every wait is bounded: a wait that runs out sets the plan's error word and the CTA stops
// issuing work.
//
// Rows of A beyond the bands of the k-point are not written: the MMA reads whatever bytes
// follow the A tile in shared memory there (the layout keeps those reads inside the CTA's
// allocation), and those rows of D are never read.  Each product row depends on its own A
// row only, so they cannot disturb the bands' rows.
#include <cstdint>

#include "fft_line.cuh"
#include "pwk_internal.h"

namespace pwk {

namespace {

constexpr int kTcThreads = 256;
constexpr int kTcProducers = 224;        // warps 0..6 copy and split; warp 7 issues the MMAs
constexpr int kTcN = 32;            // MMA N: 16 projectors, real and imaginary rows
constexpr int kTcMaxProj = 16;
constexpr int kTcTileB = kTcN * 128;   // bytes of one B tile (32 rows x 128 B)
constexpr uint32_t kTcTmemCols = 32;
constexpr int kTcRing = 6;                 // raw blocks in the asynchronous-copy ring
constexpr int kTcStages = 3;               // hi/lo tile stages (MMAs of kTcStages - 1 blocks in flight)

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B
// apart (the leading-byte offset is not used by this layout).
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of this architecture
  d |= (uint64_t)2 << 61;   // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_addr(mbar))
               : "memory");
}

// bounded wait for the completion of phase `parity` of an mbarrier (at most `polls` polls);
// false if it ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, long long polls) {
  uint32_t done = 0;
  for (long long it = 0; it < polls && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
  }
  return done != 0;
}

__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// the 16-byte chunk c (0..7) of row r of a 128-byte-swizzled tile
__device__ __forceinline__ float4* sw_chunk(unsigned char* tile, int r, int c) {
  return reinterpret_cast<float4*>(tile + r * 128 + ((c ^ (r & 7)) << 4));
}

// asynchronous copy of B (8 or 16) bytes global -> shared; src_bytes 0 zero-fills
template <int B>
__device__ __forceinline__ void tc_cp_async(void* dst, const void* src, int src_bytes) {
  if constexpr (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem_addr(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ void split4(float a, float b, float c, float d, float4& hi, float4& lo) {
  hi = make_float4(tf32_hi(a), tf32_hi(b), tf32_hi(c), tf32_hi(d));
  lo = make_float4(a - hi.x, b - hi.y, c - hi.z, d - hi.w);
}

template <typename TI>
__global__ void __launch_bounds__(kTcThreads, 3) nl_project_tc_kernel(NlArgs a) {
  using VI = c2_t<TI>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kTcStages], empty[kTcStages];
  __shared__ uint32_t tmem_base;
  // pfail[b & 1]: set by a producer before its barrier of block b, read by all after it (two
  // slots, so a producer already at block b + 1 cannot change the value block b reads)
  __shared__ int failed, pfail[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kr = blockIdx.x, k = a.k0 + kr;
  const int nb = a.nvec_in, nkb = a.nkb, np = a.npw[k];
  const int nblk = (np + 15) / 16;
  const int ra = (nb + 7) & ~7;          // A rows written (8-row groups)
  const int a_bytes = ra * 128;
  const int stage_bytes = 2 * a_bytes + 2 * kTcTileB;
  unsigned char* base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  // raw ring after the two stages (it also covers the rows the MMA reads past an A tile)
  const int raw_a = nb * 16 * (int)sizeof(VI), raw_slot = raw_a + nkb * 16 * (int)sizeof(float2);
  unsigned char* ring = base + kTcStages * stage_bytes;
  auto a_hi = [&](int s) { return base + s * stage_bytes; };
  auto a_lo = [&](int s) { return base + s * stage_bytes + a_bytes; };
  auto b_hi = [&](int s) { return base + s * stage_bytes + 2 * a_bytes; };
  auto b_lo = [&](int s) { return base + s * stage_bytes + 2 * a_bytes + kTcTileB; };

  // B rows of projectors beyond nkb stay zero in both stages (2 stages x hi/lo x 32 rows x 8 chunks)
  for (int i = tid; i < kTcStages * 2 * kTcN * 8; i += kTcThreads) {
    const int s = i >> 9, t = (i >> 8) & 1, r = (i >> 3) & 31, c = i & 7;
    if ((r & 15) >= nkb) {
      unsigned char* tile = t == 0 ? b_hi(s) : b_lo(s);
      reinterpret_cast<float4*>(tile + r * 128)[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tmem_base)),
                 "r"(kTcTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    failed = 0;
    pfail[0] = pfail[1] = 0;
    for (int j = 0; j < kTcStages; ++j) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(&full[j])), "r"(kTcProducers));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(&empty[j])), "r"(1));
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;

  // copies of block b into ring slot b % kTcRing by the producers: nb rows of 16
  // coefficients, nkb rows of 16 projector values (one element per copy; zero past npw(k))
  const VI* cin = static_cast<const VI*>(a.in) + (size_t)k * a.nvec_in * a.npw_max;
  const float2* bin = static_cast<const float2*>(a.beta) + (size_t)k * nkb * a.npw_max;
  // 16-byte copies (one complex128 or two complex64 values) when every row of both arrays
  // starts on a 16-byte boundary (the projectors are complex64: npw_max must be even)
  const bool pairs = a.npw_max % 2 == 0 && (reinterpret_cast<uintptr_t>(a.in) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(a.beta) & 15) == 0;
  auto fetch = [&](int b) {
    if (b < nblk) {
      unsigned char* slot = ring + (b % kTcRing) * raw_slot;
      if (pairs) {   // A: 16 bytes = one complex128 or two complex64; beta: two complex64
        constexpr int per_a = sizeof(VI) == 16 ? 16 : 8;   // copies per A row of 16 plane waves
        const int na = nb * per_a;
        for (int t = tid; t < na + 8 * nkb; t += kTcProducers) {
          if (t < na) {
            const int r = t / per_a, j = (t - r * per_a) * (16 / (int)sizeof(VI)), g = 16 * b + j;
            const int nv = min(16 / (int)sizeof(VI), max(0, np - g));   // valid elements of the copy
            tc_cp_async<16>(slot + (r * 16 + j) * sizeof(VI), cin + (size_t)r * a.npw_max + (nv > 0 ? g : 0),
                            nv * (int)sizeof(VI));
          } else {
            const int m = (t - na) >> 3, j = 2 * ((t - na) & 7), g = 16 * b + j;
            const int nv = min(2, max(0, np - g));
            tc_cp_async<16>(slot + raw_a + (m * 16 + j) * 8, bin + (size_t)m * a.npw_max + (nv > 0 ? g : 0), nv * 8);
          }
        }
      } else {
        for (int t = tid; t < 16 * (nb + nkb); t += kTcProducers) {
          const int r = t >> 4, j = t & 15, g = 16 * b + j;
          const bool in = g < np;
          if (r < nb) {
            tc_cp_async<sizeof(VI)>(slot + (r * 16 + j) * sizeof(VI), cin + (size_t)r * a.npw_max + (in ? g : 0),
                                    in ? (int)sizeof(VI) : 0);
          } else {
            const int m = r - nb;
            tc_cp_async<8>(slot + raw_a + (m * 16 + j) * 8, bin + (size_t)m * a.npw_max + (in ? g : 0), in ? 8 : 0);
          }
        }
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  // this thread's split task: four plane waves of an A row (band) or of a projector
  const int ntask = 4 * (nb + nkb);
  const bool has_task = tid < ntask;
  const bool is_a = tid < 4 * nb;
  const int row = is_a ? (tid >> 2) : ((tid - 4 * nb) >> 2);
  const int grp = tid & 3;
  auto split = [&](int b, int s) {
    if (!has_task) return;
    const unsigned char* slot = ring + (b % kTcRing) * raw_slot;
    float2 v[4];
    if (is_a) {
      const VI* x = reinterpret_cast<const VI*>(slot) + row * 16 + 4 * grp;
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = make_float2(float(x[j].x), float(x[j].y));
    } else {
      const float2* x = reinterpret_cast<const float2*>(slot + raw_a) + row * 16 + 4 * grp;
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = x[j];
    }
    float4 h0, l0, h1, l1;
    split4(v[0].x, v[0].y, v[1].x, v[1].y, h0, l0);
    split4(v[2].x, v[2].y, v[3].x, v[3].y, h1, l1);
    if (is_a) {   // chunks 2 grp, 2 grp + 1 of row `row`: [re, im] of plane waves 4 grp .. 4 grp + 3
      *sw_chunk(a_hi(s), row, 2 * grp) = h0;
      *sw_chunk(a_hi(s), row, 2 * grp + 1) = h1;
      *sw_chunk(a_lo(s), row, 2 * grp) = l0;
      *sw_chunk(a_lo(s), row, 2 * grp + 1) = l1;
    } else {      // row m: [re b, im b];  row 16 + m: [-im b, re b]
      *sw_chunk(b_hi(s), row, 2 * grp) = h0;
      *sw_chunk(b_hi(s), row, 2 * grp + 1) = h1;
      *sw_chunk(b_lo(s), row, 2 * grp) = l0;
      *sw_chunk(b_lo(s), row, 2 * grp + 1) = l1;
      split4(-v[0].y, v[0].x, -v[1].y, v[1].x, h0, l0);
      split4(-v[2].y, v[2].x, -v[3].y, v[3].x, h1, l1);
      *sw_chunk(b_hi(s), 16 + row, 2 * grp) = h0;
      *sw_chunk(b_hi(s), 16 + row, 2 * grp + 1) = h1;
      *sw_chunk(b_lo(s), 16 + row, 2 * grp) = l0;
      *sw_chunk(b_lo(s), 16 + row, 2 * grp + 1) = l1;
    }
  };
  constexpr uint32_t idesc = umma_idesc_tf32(128, kTcN);
  auto issue = [&](int s, int b) {   // one thread: the 12 MMAs of block b from stage s
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t ah = smem_addr(a_hi(s)), al = smem_addr(a_lo(s));
    const uint32_t bh = smem_addr(b_hi(s)), bl = smem_addr(b_lo(s));
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {   // K steps of 8 floats (32 bytes) within the 128-byte row
      const uint32_t o = 32u * ks;
      umma_tf32(tmem, umma_desc_sw128(ah + o), umma_desc_sw128(bh + o), idesc, (b > 0 || ks > 0) ? 1u : 0u);
      umma_tf32(tmem, umma_desc_sw128(ah + o), umma_desc_sw128(bl + o), idesc, 1u);
      umma_tf32(tmem, umma_desc_sw128(al + o), umma_desc_sw128(bh + o), idesc, 1u);
    }
    umma_commit(&empty[s]);
  };

  if (warp < kTcProducers / 32) {
    // producers: copies kTcRing - 1 blocks ahead, then per block the split into stage b % kTcStages
#pragma unroll 1
    for (int j = 0; j < kTcRing - 1; ++j) fetch(j);
#pragma unroll 1
    for (int b = 0; b < nblk; ++b) {
      const int s = b % kTcStages;
      // stage s is free once the MMAs of block b - kTcStages have completed
      if (b >= kTcStages && !mbar_wait(&empty[s], (uint32_t)(((b - kTcStages) / kTcStages) & 1), a.wait_polls)) pfail[b & 1] = 1;
      asm volatile("cp.async.wait_group %0;\n" ::"n"(kTcRing - 2) : "memory");   // own copies of block b landed
      asm volatile("bar.sync 1, %0;\n" ::"n"(kTcProducers) : "memory");         // everyone's; slot b - 1 consumed
      if (pfail[b & 1]) break;   // the same value for every producer
      fetch(b + kTcRing - 1);
      split(b, s);
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // generic writes -> tensor-core reads
      asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_addr(&full[s]))
                   : "memory");
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (pfail[0] | pfail[1]) failed = 1;
  } else if (lane == 0) {
    // the MMA warp: per block, wait for the producers' stage, issue its 12 MMAs, commit
#pragma unroll 1
    for (int b = 0; b < nblk; ++b) {
      const int s = b % kTcStages;
      if (!mbar_wait(&full[s], (uint32_t)((b / kTcStages) & 1), a.wait_polls)) {
        failed = 1;
        break;
      }
      issue(s, b);
    }
  }
  __syncwarp();
  // the last block's commit covers every MMA issued before it
  if (!failed && nblk > 0 && !mbar_wait(&empty[(nblk - 1) % kTcStages], (uint32_t)(((nblk - 1) / kTcStages) & 1), a.wait_polls))
    failed = 1;
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (failed) {
    if (tid == 0 && a.err != nullptr) atomicOr(a.err, 2);
  } else if (warp < 4) {
    // rows 32 warp + lane of D: Re lambda in columns 0..15, Im lambda in 16..31
    uint32_t v[32];
    const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    const int band = 32 * warp + lane;
    if (band < nb) {
      // gamma = D lambda (Eq. gamma), delta = q lambda (Eq. delta_eq), as the CUDA-core kernel
      const float* D = static_cast<const float*>(a.D);
      const float* q = static_cast<const float*>(a.q);
      float2* cf = static_cast<float2*>(a.coef) + ((size_t)kr * a.nvec_in + band) * 2 * nkb;
      for (int i = 0; i < nkb; ++i) {
        float gr = 0.f, gi = 0.f, dr = 0.f, di = 0.f;
#pragma unroll
        for (int j = 0; j < kTcMaxProj; ++j) {
          if (j < nkb) {
            const float lr = __uint_as_float(v[j]), li = __uint_as_float(v[16 + j]);
            const float dm = D[(size_t)i * nkb + j];
            gr += dm * lr;
            gi += dm * li;
            if (q != nullptr) {
              const float qm = q[(size_t)i * nkb + j];
              dr += qm * lr;
              di += qm * li;
            }
          }
        }
        cf[i] = make_float2(gr, gi);
        cf[nkb + i] = make_float2(dr, di);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTcTmemCols));
}

size_t tc_smem_bytes(int nb, int nkb, int io_bytes) {
  const int ra = (nb + 7) & ~7;
  const size_t ring = (size_t)kTcRing * (nb * 16 * io_bytes + nkb * 16 * 8);
  // the stages, then the raw ring, at least 16 KB (the MMA reads 128 rows from an A tile
  // start), alignment slack
  return (size_t)kTcStages * (2 * ra * 128 + 2 * kTcTileB) + (ring > 16384 ? ring : 16384) + 1024;
}

}  // namespace

// 1 when the tensor-core projection applies to this launch (FP32 arithmetic, batched items of
// whole k-points, every task of a block in one thread, N_kb <= 16)
int nl_project_tc_applies(int precision, const NlArgs& a) {
  if (precision == PWK_FP64 || a.phase != 0 || a.items != nullptr || a.d_count != nullptr) return 0;
  if (a.nkb < 1 || a.nkb > kTcMaxProj || a.nvec_in != a.nvec_out || a.nvec_in < 1 || a.nvec_in > 128) return 0;
  if (4 * (a.nvec_in + a.nkb) > kTcProducers || a.nitems % a.nvec_in != 0) return 0;
  if (tc_smem_bytes(a.nvec_in, a.nkb, precision == PWK_FP32 ? 8 : 16) > 227 * 1024) return 0;
  return 1;
}

int launch_nl_project_tc(int precision, const NlArgs& a, cudaStream_t st) {
  const int nkl = a.nitems / a.nvec_in;
  if (nkl == 0) return PWK_OK;
  const size_t smem = tc_smem_bytes(a.nvec_in, a.nkb, precision == PWK_FP32 ? 8 : 16);
  cudaError_t e;
  if (precision == PWK_FP32) {
    if ((e = allow_full_smem(nl_project_tc_kernel<float>)) != cudaSuccess)
      return cuda_fail(e, "cudaFuncSetAttribute(nl_project_tc)");
    nl_project_tc_kernel<float><<<nkl, kTcThreads, smem, st>>>(a);
  } else {
    if ((e = allow_full_smem(nl_project_tc_kernel<double>)) != cudaSuccess)
      return cuda_fail(e, "cudaFuncSetAttribute(nl_project_tc)");
    nl_project_tc_kernel<double><<<nkl, kTcThreads, smem, st>>>(a);
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? PWK_OK : cuda_fail(e, "nl_project_tc_kernel");
}

}  // namespace pwk
