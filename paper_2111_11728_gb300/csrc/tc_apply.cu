// Tensor-core form of the local dual-operator product (the precision form):
//
//   Y_b(s) = D_s^{1/2} Fhat_s D_s^{1/2} X_b(s),   Fhat_s = D_s^{-1/2} F_s D_s^{-1/2},
//
// with D_s = diag(F_s).  Fhat_s is kept in TF32 or BF16 (and, for the split
// products, the rounding of its remainder to the same format), the product
// runs on the 5th-generation tensor cores (tcgen05.mma kind::tf32, or
// kind::f16 with BF16 inputs) with FP32 accumulation in tensor memory,
// operands staged by TMA into 128-byte-swizzled shared memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "fpconv.cuh"
#include "kernels.h"

namespace feti {

namespace {

constexpr int TC_M = 128;
constexpr int TC_NMAX = 256;
constexpr int TC_MAX_NC = 64;        // primal DOFs per subdomain carried in the K-extension
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_TMEM_COLS = 256;
constexpr unsigned long long TC_WAIT_NS = 1000000000ull;   // every pipeline wait gives up after 1 s
constexpr long long TC_SPIN_LIMIT = 1ll << 32;              // backstop on the number of polls
constexpr int TC_STAGES1 = 2;       // ring depth, one pass (48 KB per stage; two CTAs per SM)
constexpr int TC_STAGES3 = 2;       // ring depth, split product (96 KB per stage)
constexpr int TCP_STAGES1 = 4;      // persistent kernel: one pass, 4 x 48 KB
constexpr int TCP_STAGES3 = 2;      // persistent kernel: split product, 2 x 96 KB

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// UMMA shared-memory matrix descriptor: K-major operand in 128-byte swizzled
// rows, 8-row groups 1024 bytes apart (stride byte offset), descriptor
// version 1, layout type SWIZZLE_128B.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;
  d |= static_cast<uint64_t>(1024 >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(2) << 61;
  return d;
}

// Instruction descriptor: D = F32, A = B = TF32 (kind::tf32, format 2) or
// BF16 (kind::f16, format 1), both K-major, M = 128, N = n.
template <int FMT>
__device__ __forceinline__ uint32_t idesc_of(int n) {
  constexpr uint32_t ab = FMT == 0 ? 2u : 1u;
  return (1u << 4) | (ab << 7) | (ab << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(TC_M >> 4) << 24);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the phase `phase` of an mbarrier: true when it completed,
// false after TC_WAIT_NS of wall time (measured on the global nanosecond timer).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
  const unsigned long long t0 = global_ns();
  for (long long it = 0; it < TC_SPIN_LIMIT; ++it) {
    if ((it & 15) == 15 && global_ns() - t0 > TC_WAIT_NS) return false;
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    if (ok) return true;
  }
  return false;
}


// Operand formats.  FMT 0: TF32 values stored as FP32 bit patterns (32 per
// 128-byte row, K = 8 per MMA); FMT 1: BF16 (64 per row, K = 16 per MMA).
// Either way one MMA consumes 32 bytes of every operand row.
template <int FMT>
struct TcFmt;
template <>
struct TcFmt<0> {
  using T = float;
  static constexpr int KC = 32;
  __device__ static T round(float v) { return to_tf32(v); }
  __device__ static float value(T x) { return x; }
};
template <>
struct TcFmt<1> {
  using T = __nv_bfloat16;
  static constexpr int KC = 64;
  __device__ static T round(float v) { return __float2bfloat16_rn(v); }
  __device__ static float value(T x) { return __bfloat162float(x); }
};

// K extent of a subdomain in the tensor-core operands: n_b rounded up to the
// format's chunk kc, plus the corner coupling (n_c columns, rounded up to kc)
// when appended.
__host__ __device__ __forceinline__ int k_extent(int nb, int nc, int aug, int kc) {
  return (nb + kc - 1) / kc * kc + ((aug && nc > 0) ? (nc + kc - 1) / kc * kc : 0);
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

template <int FMT>
__device__ __forceinline__ void mma_issue(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  if (FMT == 0)
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (one per thread).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
        "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
        "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Operands of the tensor-core product, laid out for TMA:
//
//   A: the scaled blocks Fhat_s of every module, one row of the "arena" per
//      block row, a common pitch P and zero beyond n_b.  FETI-DP appends,
//      after n_b rounded up to the K chunk KC (32 TF32 or 64 BF16 values), the
//      row's scaled primal coupling Frc_hat_s = D_s^{-1/2} F_rc,s (n_c <= 64
//      columns -- 8 to 24 corners, up to 60 with edge averages -- rounded up
//      to KC).  Tensor map: dims {P, rows}, box {KC, 128}, 128-byte swizzle.
//   B: the gathered, scaled directions D_s^{1/2} B^sT X, one column per
//      direction over the padded interface space (each subdomain's range
//      rounded up to KC entries, zero in the padding), followed for FETI-DP
//      by the subdomain's coarse correction V_s (the K-extension matching
//      Frc_hat).  Tensor map: dims {padded total, m}, box {KC, 256}.
//
// With the K-extension one product gives the whole local FETI-DP operator
// D^{1/2} [Fhat | Frc_hat] [D^{1/2} X_b ; V_s] = F_s X_b + F_rc,s V_s.
//
// Both are stored as TF32 or BF16 high parts (and, for the split product,
// low parts in the same format).  One CTA computes a 128-row x 256-column output tile of one
// subdomain: thread 0 streams K chunks of 32 through a STAGES-deep ring of
// shared-memory buffers (full / empty mbarriers), thread 32 issues the MMAs
// (4 K=8 steps x PASSES per chunk) and frees a buffer by committing to its
// empty barrier; the final commit releases the epilogue, in which each warp
// reads its 32 TMEM lanes and writes FP32 rows scaled by D_s^{1/2}.
// Every wait is bounded: on time-out the CTA records an error code, waits
// (bounded) for its copies and MMAs in flight, frees its tensor memory and
// returns.
template <int FMT, int PASSES, int STAGES>
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_apply(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAl,
    const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmBl,
    const DevType* __restrict__ types, const DevSub* __restrict__ subs, const int* __restrict__ frow,
    const int64_t* __restrict__ bpad, const double* __restrict__ sqrtD, float* __restrict__ Yb, int64_t nbt,
    int m, int n_cb, int aug, int* __restrict__ status, int skip_chunk) {
  constexpr uint32_t A_BYTES = TC_M * 128, B_BYTES = TC_NMAX * 128;
  constexpr uint32_t STAGE_BYTES = (PASSES == 3 ? 2 : 1) * (A_BYTES + B_BYTES);
  constexpr int KC = TcFmt<FMT>::KC;
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  unsigned char* base = tc_smem_raw + ((1024 - (smem_u32(tc_smem_raw) & 1023)) & 1023);
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int fail_sh, consumed_sh;

  const int sidx = blockIdx.y;
  const int cb = blockIdx.x % n_cb, rb = blockIdx.x / n_cb;
  const DevSub S = subs[sidx];
  const DevType T = types[S.type];
  const int nb = T.n_b;
  const int row0 = rb * TC_M;
  if (row0 >= nb) return;                              // block-uniform
  const int col0 = cb * TC_NMAX;
  const int ncols = min(TC_NMAX, m - col0);
  const int np = ((ncols + 15) / 16) * 16;
  const int nk = k_extent(nb, T.n_c, aug, KC) / KC;
  const int arow = frow[S.module] + row0;
  const int bx0 = (int)bpad[sidx];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int i = 0; i < STAGES; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_bar[i])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty_bar[i])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done_bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fail_sh = 0;
    consumed_sh = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;

  int issued = 0;                                      // producer's count of chunks in flight or consumed
  if (tid == 0) {
    // ---- producer: TMA loads of A and B chunks into the ring ----
    for (int kc = 0; kc < nk; ++kc) {
      const int st = kc % STAGES, it = kc / STAGES;
      // test hook: the first tile stops before this chunk's copy, so the MMA
      // lane's bounded wait for it runs out (nothing is left in flight)
      if (kc == skip_chunk && blockIdx.x == 0 && blockIdx.y == 0) break;
      if (kc >= STAGES && !mbar_wait(smem_u32(&empty_bar[st]), (uint32_t)((it - 1) & 1))) {
        atomicExch(&fail_sh, 1);
        break;
      }
      if (*(volatile int*)&fail_sh) break;
      unsigned char* sb = base + st * STAGE_BYTES;
      const uint32_t fb = smem_u32(&full_bar[st]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(STAGE_BYTES) : "memory");
      tma_load_2d(smem_u32(sb), &tmA, kc * KC, arow, fb);
      tma_load_2d(smem_u32(sb + A_BYTES), &tmB, bx0 + kc * KC, col0, fb);
      if (PASSES == 3) {
        tma_load_2d(smem_u32(sb + A_BYTES + B_BYTES), &tmAl, kc * KC, arow, fb);
        tma_load_2d(smem_u32(sb + 2 * A_BYTES + B_BYTES), &tmBl, bx0 + kc * KC, col0, fb);
      }
      issued = kc + 1;
    }
  } else if (tid == 32) {
    // ---- MMA issuer ----
    const uint32_t idesc = idesc_of<FMT>(np);
    int kc = 0;
    for (; kc < nk; ++kc) {
      const int st = kc % STAGES, it = kc / STAGES;
      if (!mbar_wait(smem_u32(&full_bar[st]), (uint32_t)(it & 1))) {
        atomicExch(&fail_sh, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(base + st * STAGE_BYTES);
      const uint32_t sbh = sa + A_BYTES;
      const uint32_t sal = sa + A_BYTES + B_BYTES;
      const uint32_t sbl = sa + 2 * A_BYTES + B_BYTES;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {                 // 32 bytes of each row per MMA
#pragma unroll
        for (int pass = 0; pass < PASSES; ++pass) {
          // split product: lo x hi, hi x lo, then hi x hi (small terms first)
          const uint32_t ap = (PASSES == 3 && pass == 0) ? sal : sa;
          const uint32_t bp = (PASSES == 3 && pass == 1) ? sbl : sbh;
          const uint32_t acc = (kc > 0 || kk > 0 || pass > 0) ? 1u : 0u;
          mma_issue<FMT>(tmem, desc_sw128(ap + kk * 32), desc_sw128(bp + kk * 32), idesc, acc);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&empty_bar[st]))
                   : "memory");
    }
    consumed_sh = kc;
    // arrives once every MMA issued above has completed (also after a failure)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&done_bar))
                 : "memory");
  }
  __syncwarp();
  const bool ok = mbar_wait(smem_u32(&done_bar), 0u);
  const bool failed = __syncthreads_or(!ok || fail_sh != 0);
  if (failed) {
    if (tid == 0) {
      atomicCAS(status, 0, 3000000 + sidx);
      // wait for the copies that were issued but never consumed
      for (int kc = consumed_sh; kc < issued; ++kc)
        mbar_wait(smem_u32(&full_bar[kc % STAGES]), (uint32_t)((kc / STAGES) & 1));
    }
    if (!ok) mbar_wait(smem_u32(&done_bar), 0u);
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- epilogue: warp w owns TMEM lanes [32w, 32w+32) = output rows ----
    const int r = row0 + warp * 32 + lane;
    const float sd = r < nb ? static_cast<float>(sqrtD[S.b_off + r]) : 0.0f;
    float* yrow = Yb + S.b_off + r;
    for (int jc = 0; jc < np; jc += 32) {
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)jc, v);
      if (r < nb) {
#pragma unroll
        for (int c = 0; c < 32; ++c)
          if (jc + c < ncols) yrow[(int64_t)(col0 + jc + c) * nbt] = sd * __uint_as_float(v[c]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

// Persistent, warp-specialised form of the same product.  One CTA per SM walks
// a static list of (subdomain, row tile, column tile) triples (CTA c takes
// tiles c, c + G, c + 2G, ...).  Warp 0 (one lane) streams A and B chunks of
// every tile through a STAGES-deep ring (full / empty mbarriers); warp 1 owns
// the tensor memory (two 256-column FP32 accumulators) and one of its lanes
// issues the MMAs, alternating accumulators from tile to tile; warps 2-5 read
// a finished accumulator (tmem_full), scale and store its rows and hand it back
// (tmem_empty, 128 arrivals) while the next tile accumulates in the other one.
// Every wait is bounded; on a time-out the CTA records an error code, stops
// issuing, waits (bounded) for its copies and MMAs in flight, frees its tensor
// memory and returns.
constexpr int TCP_THREADS = 192;
constexpr uint32_t TCP_TMEM_COLS = 512;

template <int FMT, int PASSES, int STAGES>
__global__ void __launch_bounds__(TCP_THREADS, 1) k_tc_apply_p(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAl,
    const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmBl,
    const int4* __restrict__ tiles, int n_tiles, const DevType* __restrict__ types,
    const DevSub* __restrict__ subs, const int* __restrict__ frow, const int64_t* __restrict__ bpad,
    const double* __restrict__ sqrtD, float* __restrict__ Yb, int64_t nbt, int m, int aug,
    int* __restrict__ status, int fcrow0, double* __restrict__ Cb, int64_t nct) {
  constexpr uint32_t A_BYTES = TC_M * 128, B_BYTES = TC_NMAX * 128;
  constexpr uint32_t STAGE_BYTES = (PASSES == 3 ? 2 : 1) * (A_BYTES + B_BYTES);
  constexpr int KC = TcFmt<FMT>::KC;
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  unsigned char* base = tc_smem_raw + ((1024 - (smem_u32(tc_smem_raw) & 1023)) & 1023);
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], tfull_bar[2], tempty_bar[2], drain_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int fail_sh;
  __shared__ long long consumed_sh;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(TCP_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < STAGES; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_bar[i])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty_bar[i])) : "memory");
    }
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tfull_bar[i])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_u32(&tempty_bar[i])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&drain_bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fail_sh = 0;
    consumed_sh = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;

  long long issued = 0;                         // producer: chunks issued
  if (warp == 0) {
    if (lane == 0) {
      long long g = 0;
      for (int t = blockIdx.x; t < n_tiles; t += G) {
        const int4 tl = tiles[t];
        const DevSub S = subs[tl.x];
        const DevType T = types[S.type];
        // corner tile (tl.w = 1): the module's Frc_hat^T block times the operand's b part
        const int nk = tl.w ? k_extent(T.n_b, 0, 0, KC) / KC : k_extent(T.n_b, T.n_c, aug, KC) / KC;
        const int arow = tl.w ? fcrow0 + S.module * TC_M : frow[S.module] + tl.y * TC_M;
        const int bx0 = (int)bpad[tl.x];
        const int col0 = tl.z * TC_NMAX;
        for (int kc = 0; kc < nk; ++kc, ++g) {
          const int st = (int)(g % STAGES);
          const long long it = g / STAGES;
          if (g >= STAGES && !mbar_wait(smem_u32(&empty_bar[st]), (uint32_t)((it - 1) & 1))) {
            atomicExch(&fail_sh, 1);
            break;
          }
          if (*(volatile int*)&fail_sh) break;
          unsigned char* sb = base + st * STAGE_BYTES;
          const uint32_t fb = smem_u32(&full_bar[st]);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(STAGE_BYTES)
                       : "memory");
          tma_load_2d(smem_u32(sb), &tmA, kc * KC, arow, fb);
          tma_load_2d(smem_u32(sb + A_BYTES), &tmB, bx0 + kc * KC, col0, fb);
          if (PASSES == 3) {
            tma_load_2d(smem_u32(sb + A_BYTES + B_BYTES), &tmAl, kc * KC, arow, fb);
            tma_load_2d(smem_u32(sb + 2 * A_BYTES + B_BYTES), &tmBl, bx0 + kc * KC, col0, fb);
          }
          issued = g + 1;
        }
        if (*(volatile int*)&fail_sh) break;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      long long g = 0;
      int lt = 0;
      for (int t = blockIdx.x; t < n_tiles; t += G, ++lt) {
        const int4 tl = tiles[t];
        const DevSub S = subs[tl.x];
        const DevType T = types[S.type];
        const int nk = tl.w ? k_extent(T.n_b, 0, 0, KC) / KC : k_extent(T.n_b, T.n_c, aug, KC) / KC;
        const int ncols = min(TC_NMAX, m - tl.z * TC_NMAX);
        const uint32_t idesc = idesc_of<FMT>(((ncols + 15) / 16) * 16);
        const int ab = lt & 1, use = lt >> 1;
        if (use > 0 && !mbar_wait(smem_u32(&tempty_bar[ab]), (uint32_t)((use - 1) & 1))) {
          atomicExch(&fail_sh, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dacc = tmem + (uint32_t)(ab * TC_NMAX);
        bool ok = true;
        for (int kc = 0; kc < nk; ++kc, ++g) {
          const int st = (int)(g % STAGES);
          if (!mbar_wait(smem_u32(&full_bar[st]), (uint32_t)((g / STAGES) & 1))) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = smem_u32(base + st * STAGE_BYTES);
          const uint32_t sbh = sa + A_BYTES;
          const uint32_t sal = sa + A_BYTES + B_BYTES;
          const uint32_t sbl = sa + 2 * A_BYTES + B_BYTES;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
            for (int pass = 0; pass < PASSES; ++pass) {
              const uint32_t ap = (PASSES == 3 && pass == 0) ? sal : sa;
              const uint32_t bp = (PASSES == 3 && pass == 1) ? sbl : sbh;
              const uint32_t acc = (kc > 0 || kk > 0 || pass > 0) ? 1u : 0u;
              mma_issue<FMT>(dacc, desc_sw128(ap + kk * 32), desc_sw128(bp + kk * 32), idesc, acc);
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&empty_bar[st]))
                       : "memory");
          consumed_sh = g + 1;
        }
        if (!ok) {
          atomicExch(&fail_sh, 1);
          break;
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&tfull_bar[ab]))
                     : "memory");
        if (*(volatile int*)&fail_sh) break;
      }
      // arrives once every MMA issued above has completed
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&drain_bar))
                   : "memory");
    }
  } else {
    // ---- epilogue warps 2..5: TMEM lanes 32 * (warp % 4) ... + 31 ----
    const int lq = warp & 3;
    int lt = 0;
    for (int t = blockIdx.x; t < n_tiles; t += G, ++lt) {
      const int ab = lt & 1, use = lt >> 1;
      const bool ok = mbar_wait(smem_u32(&tfull_bar[ab]), (uint32_t)(use & 1));
      if (!__all_sync(0xffffffffu, ok) || *(volatile int*)&fail_sh) {
        atomicExch(&fail_sh, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int4 tl = tiles[t];
      const DevSub S = subs[tl.x];
      const int nb = types[S.type].n_b;
      const int col0 = tl.z * TC_NMAX;
      const int ncols = min(TC_NMAX, m - col0);
      const int np = ((ncols + 15) / 16) * 16;
      if (tl.w) {
        // corner tile: row r of the accumulator is C_s(r, .) = (F_rc^T X_b)(r, .)
        const int r = lq * 32 + lane;
        const bool live = r < types[S.type].n_c;
        double* crow = Cb + S.c_off + r;
        for (int jc = 0; jc < np; jc += 32) {
          uint32_t v[32];
          tmem_ld32(tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(ab * TC_NMAX + jc), v);
          if (live) {
#pragma unroll
            for (int c = 0; c < 32; ++c)
              if (jc + c < ncols) crow[(int64_t)(col0 + jc + c) * nct] = static_cast<double>(__uint_as_float(v[c]));
          }
        }
      } else {
        const int r = tl.y * TC_M + lq * 32 + lane;
        const float sd = r < nb ? static_cast<float>(sqrtD[S.b_off + r]) : 0.0f;
        float* yrow = Yb + S.b_off + r;
        for (int jc = 0; jc < np; jc += 32) {
          uint32_t v[32];
          tmem_ld32(tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(ab * TC_NMAX + jc), v);
          if (r < nb) {
#pragma unroll
            for (int c = 0; c < 32; ++c)
              if (jc + c < ncols) yrow[(int64_t)(col0 + jc + c) * nbt] = sd * __uint_as_float(v[c]);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty_bar[ab])) : "memory");
    }
  }
  __syncwarp();
  __syncthreads();
  if (fail_sh) {
    if (tid == 0) {
      atomicCAS(status, 0, 3000000 + blockIdx.x);
      for (long long g = consumed_sh; g < issued; ++g)
        mbar_wait(smem_u32(&full_bar[g % STAGES]), (uint32_t)((g / STAGES) & 1));
    }
  }
  if (tid == 32) mbar_wait(smem_u32(&drain_bar), 0u);   // every MMA of this CTA has completed
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCP_TMEM_COLS)
                 : "memory");
  }
}

// B operand: xb[j][bpad(s) + k] = parts of sqrt(D_s)[k] (B^sT X)[b, j] in
// the operand format for k < n_b(s), zero for the padding up to the next
// multiple of the format's chunk (zeroed once when the buffer is allocated).
constexpr int SP_J = 32;               // directions per block
constexpr int SP_THREADS = 512;
constexpr int SP_LD = SP_J * kSpreadRows / SP_THREADS;   // loads per thread
constexpr int SP_QL = 64;              // slots handled side by side
constexpr int SP_ME = 4;               // rows of a cross-point slot held in registers

// The operand slots of range r, directions j0 .. j0 + jn - 1, from the range's
// rows in shared memory (xs[c][i] = X(row0[r] + i, j0 + c) in FP32): SP_QL
// consecutive slots side by side (those with one row first, each class in
// position order), each group of SP_QL threads a share of the directions.
// x = sqrt(D) * (sum of the slot's signed rows): a DOF with one row takes that
// row, a cross-point DOF the sum of its rows, in the order of its row list.
template <int FMT, int PASSES>
__device__ __forceinline__ void spread_slots(const float (*xs)[kSpreadRows + 1], int r, int j0, int jn,
                                             const int* __restrict__ slot_off, const int* __restrict__ pos,
                                             const float* __restrict__ sd, const int* __restrict__ ent_off,
                                             const short* __restrict__ ent, typename TcFmt<FMT>::T* __restrict__ xb_hi,
                                             typename TcFmt<FMT>::T* __restrict__ xb_lo, int64_t nbp) {
  using F = TcFmt<FMT>;
  constexpr int NG = SP_THREADS / SP_QL, PER = SP_J / NG;
  const int q0 = slot_off[r], nq = slot_off[r + 1] - q0;
  const int g = threadIdx.x / SP_QL;
  const int64_t cstride = (int64_t)NG * nbp;
  for (int qq = threadIdx.x % SP_QL; qq < nq; qq += SP_QL) {
    const int q = q0 + qq;
    const int e0 = ent_off[q], ne = ent_off[q + 1] - e0;
    const float w = sd[q];
    const int64_t o0 = (int64_t)(j0 + g) * nbp + pos[q];
    const float* xg = &xs[g][0];
    if (ne == 1) {                       // one row: a signed copy
      const int u = ent[e0];
      const float* xr = xg + (u >= 0 ? u : ~u);
      const float ws = u >= 0 ? w : -w;
#pragma unroll
      for (int t = 0; t < PER; ++t) {
        if (g + NG * t >= jn) break;
        const float y = xr[t * NG * (kSpreadRows + 1)] * ws;
        const typename F::T h = F::round(y);
        xb_hi[o0 + t * cstride] = h;
        if (PASSES == 3) xb_lo[o0 + t * cstride] = F::round(y - F::value(h));
      }
    } else {                             // several rows, summed in list order
      int ev[SP_ME];
#pragma unroll
      for (int k = 0; k < SP_ME; ++k) ev[k] = k < ne ? ent[e0 + k] : 0;
#pragma unroll
      for (int t = 0; t < PER; ++t) {
        if (g + NG * t >= jn) break;
        const float* xc = xg + t * NG * (kSpreadRows + 1);
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < SP_ME; ++k)
          if (k < ne) acc += ev[k] >= 0 ? xc[ev[k]] : -xc[~ev[k]];
        for (int k = SP_ME; k < ne; ++k) {
          const int u = ent[e0 + k];
          acc += u >= 0 ? xc[u] : -xc[~u];
        }
        const float y = acc * w;
        const typename F::T h = F::round(y);
        xb_hi[o0 + t * cstride] = h;
        if (PASSES == 3) xb_lo[o0 + t * cstride] = F::round(y - F::value(h));
      }
    }
  }
}

// It is built from the multiplier side, one range of consecutive multiplier
// rows (at most kSpreadRows, every interface DOF's rows inside one range) and
// SP_J directions per block: the block reads X(l, j) of its rows once
// (consecutive threads, consecutive rows: coalesced; all SP_LD loads of a
// thread in flight together; FP64 -> FP32) into shared memory, then writes
// every operand slot of the range (spread_slots).
template <int FMT, int PASSES>
__global__ void __launch_bounds__(SP_THREADS) k_spread_tc(int m, const int* __restrict__ row0,
                                                          const int* __restrict__ slot_off,
                                                          const int* __restrict__ pos, const float* __restrict__ sd,
                                                          const int* __restrict__ ent_off,
                                                          const short* __restrict__ ent,
                                                          const double* __restrict__ X, int64_t ldx,
                                                          typename TcFmt<FMT>::T* __restrict__ xb_hi,
                                                          typename TcFmt<FMT>::T* __restrict__ xb_lo, int64_t nbp) {
  static_assert(SP_THREADS % kSpreadRows == 0 && SP_THREADS % SP_QL == 0, "block shape");
  constexpr int CSTEP = SP_THREADS / kSpreadRows;
  __shared__ float xs[SP_J][kSpreadRows + 1];
  const int r = blockIdx.x;
  const int l0 = row0[r], nr = row0[r + 1] - l0;
  const int j0 = blockIdx.y * SP_J, jn = min(SP_J, m - j0);
  {
    const int i = threadIdx.x % kSpreadRows, cb = threadIdx.x / kSpreadRows;
    double v[SP_LD];
    const double* x = X + (int64_t)(l0 + i) + (int64_t)(j0 + cb) * ldx;
#pragma unroll
    for (int t = 0; t < SP_LD; ++t)
      v[t] = (i < nr && cb + CSTEP * t < jn) ? __ldcs(x + (int64_t)(CSTEP * t) * ldx) : 0.0;
#pragma unroll
    for (int t = 0; t < SP_LD; ++t) xs[cb + CSTEP * t][i] = f64_to_f32_rn(v[t]);
  }
  __syncthreads();
  spread_slots<FMT, PASSES>(xs, r, j0, jn, slot_off, pos, sd, ent_off, ent, xb_hi, xb_lo, nbp);
}

// sqrt(D) of every operand slot's interface DOF in FP32 (refreshed at every
// factorization with the new diagonal).
__global__ void k_spread_weights(int n, const int* __restrict__ b, const double* __restrict__ sqrtD,
                                 float* __restrict__ sd) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) sd[q] = f64_to_f32_rn(sqrtD[b[q]]);
}

// A operand: arena rows of Fhat_s = D^{-1/2} F_s D^{-1/2} in the operand
// format (and, with aug, Frc_hat_s = D^{-1/2} F_rc,s after column n_b rounded
// up to the format's chunk).
template <int FMT>
__global__ void k_make_arena(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                             const double* __restrict__ mem, const int* __restrict__ frow, int64_t pitch, int aug,
                             typename TcFmt<FMT>::T* __restrict__ fa_hi, typename TcFmt<FMT>::T* __restrict__ fa_lo) {
  using F = TcFmt<FMT>;
  const DevModule M = mods[blockIdx.y];
  const DevType T = types[M.type];
  const int n = T.n_b, nc = (aug ? T.n_c : 0);
  const int ncol = n + nc;
  const int c0 = k_extent(n, 0, 0, F::KC);
  const double* Fm = mem + M.F;
  const double* Frc = mem + M.Frc;                  // [n x nc] row-major
  const int64_t total = (int64_t)n * ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / ncol), j = (int)(e % ncol);
    const double di = sqrt(Fm[(int64_t)i * n + i]);
    float v;
    int64_t o;
    if (j < n) {
      v = static_cast<float>(Fm[(int64_t)i * n + j] / (di * sqrt(Fm[(int64_t)j * n + j])));
      o = (int64_t)(frow[blockIdx.y] + i) * pitch + j;
    } else {
      v = static_cast<float>(Frc[(int64_t)i * nc + (j - n)] / di);
      o = (int64_t)(frow[blockIdx.y] + i) * pitch + c0 + (j - n);
    }
    const typename F::T hi = F::round(v);
    fa_hi[o] = hi;
    if (fa_lo) fa_lo[o] = F::round(v - F::value(hi));
  }
}

// Corner blocks of the arena (FETI-DP): module q's rows fcrow0 + 128 q + c hold
// Frc_hat_s^T (c < n_c): entry k < n_b is F_rc(k, c) / sqrt(F_s(k, k)); the rest of
// the 128-row block stays zero.  A corner tile multiplies it with the gathered
// operand's b part: C_s = Frc_hat^T (D^{1/2} X_b) = F_rc^T X_b.
template <int FMT>
__global__ void k_make_arena_corner(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                                    const double* __restrict__ mem, int fcrow0, int64_t pitch,
                                    typename TcFmt<FMT>::T* __restrict__ fa_hi,
                                    typename TcFmt<FMT>::T* __restrict__ fa_lo) {
  using F = TcFmt<FMT>;
  const DevModule M = mods[blockIdx.y];
  const DevType T = types[M.type];
  const int n = T.n_b, nc = T.n_c;
  const double* Fm = mem + M.F;
  const double* Frc = mem + M.Frc;                  // [n x nc] row-major
  const int64_t total = (int64_t)nc * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / n), k = (int)(e % n);
    const float v = static_cast<float>(Frc[(int64_t)k * nc + c] / sqrt(Fm[(int64_t)k * n + k]));
    const int64_t o = (int64_t)(fcrow0 + blockIdx.y * TC_M + c) * pitch + k;
    const typename F::T hi = F::round(v);
    fa_hi[o] = hi;
    if (fa_lo) fa_lo[o] = F::round(v - F::value(hi));
  }
}

// Corner reduction of the precision form, FP32 on the CUDA cores:
// C_s = F_rc,s^T X_b(s) = Frc_hat_s^T (D^{1/2} X_b(s)), read from the gathered
// operand (high + low parts) and the FP32 copy of Frc_hat.  One block per
// subdomain and 128 directions; K is staged 32 rows at a time, the next chunk's
// operand loaded into registers (16-byte loads) while the current one is
// multiplied.  A thread owns 4 directions x NCM/NCH corner columns over one of
// KS interleaved K slices (register tile); the slices are summed by warp
// shuffles at the end (fixed order: deterministic).
template <int FMT, int NCM>
__global__ void __launch_bounds__(256) k_frct_lowp(const DevType* __restrict__ types,
                                                   const DevModule* __restrict__ mods,
                                                   const DevSub* __restrict__ subs, const float* __restrict__ fmem,
                                                   const int64_t* __restrict__ bpad,
                                                   const typename TcFmt<FMT>::T* __restrict__ xb_hi,
                                                   const typename TcFmt<FMT>::T* __restrict__ xb_lo, int64_t nbp,
                                                   int m, double* __restrict__ Cb, int64_t nct) {
  using F = TcFmt<FMT>;
  using T = typename F::T;
  constexpr int NCH = NCM == 64 ? 4 : 2;            // corner groups
  constexpr int NQ = NCM / NCH;                     // corner columns per thread (12 or 16)
  constexpr int KS = 8 / NCH;                       // K slices (4 or 2)
  constexpr int EV = 16 / sizeof(T);                // operand elements per 16-byte load (8 or 4)
  constexpr int NV = 32 * 128 / EV / 256;           // 16-byte loads per thread per chunk (2 or 4)
  constexpr int NF = 32 * NCM / 256;                // corner-block entries per thread per chunk (3 or 8)
  __shared__ __align__(16) float fs[32][NCM];
  __shared__ float xs[128][33];
  const DevSub S = subs[blockIdx.y];
  const DevType Tt = types[S.type];
  const int nb = Tt.n_b, nc = Tt.n_c;
  if (nc == 0) return;
  const float* Fr = fmem + mods[S.module].Frc;      // [nb x nc] row-major
  const int j0 = blockIdx.x * 128;
  const int tid = threadIdx.x;
  const int ks = tid % KS, cq = (tid / KS) % 32, ch = tid / (KS * 32);
  const T* xh = xb_hi + bpad[blockIdx.y];
  const T* xl = xb_lo ? xb_lo + bpad[blockIdx.y] : nullptr;
  // the padded operand extends to a multiple of the format's chunk (>= 32 rows):
  // a 16-byte load at k0 + 8 i stays inside it and the padding reads as zero
  const int nbp_s = k_extent(nb, 0, 0, F::KC);
  uint4 vh[NV], vl[NV];
  float vf[NF];
  auto load_chunk = [&](int k0) {
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const int v = tid + 256 * t, j = v / (32 / EV), kk = (v % (32 / EV)) * EV;
      const int64_t o = (int64_t)(j0 + j) * nbp + k0 + kk;
      const bool ok = j0 + j < m && k0 + kk < nbp_s;
      vh[t] = ok ? *reinterpret_cast<const uint4*>(xh + o) : make_uint4(0, 0, 0, 0);
      vl[t] = (ok && xl) ? *reinterpret_cast<const uint4*>(xl + o) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int t = 0; t < NF; ++t) {
      const int e = tid + 256 * t, kk = e / NCM, c = e % NCM, k = k0 + kk;
      vf[t] = (k < nb && c < nc) ? Fr[(int64_t)k * nc + c] : 0.0f;
    }
  };
  auto store_chunk = [&]() {
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const int v = tid + 256 * t, j = v / (32 / EV), kk = (v % (32 / EV)) * EV;
      const T* ph = reinterpret_cast<const T*>(&vh[t]);
      const T* pl = reinterpret_cast<const T*>(&vl[t]);
#pragma unroll
      for (int i = 0; i < EV; ++i) xs[j][kk + i] = F::value(ph[i]) + F::value(pl[i]);
    }
#pragma unroll
    for (int t = 0; t < NF; ++t) {
      const int e = tid + 256 * t;
      fs[e / NCM][e % NCM] = vf[t];
    }
  };
  float acc[4][NQ];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[c][q] = 0.f;
  load_chunk(0);
  for (int k0 = 0; k0 < nb; k0 += 32) {
    store_chunk();
    __syncthreads();
    if (k0 + 32 < nb) load_chunk(k0 + 32);            // in flight while this chunk is multiplied
#pragma unroll
    for (int t = 0; t < 32 / KS; ++t) {
      const int kk = ks + KS * t;
      float x[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) x[c] = xs[cq * 4 + c][kk];
#pragma unroll
      for (int q4 = 0; q4 < NQ / 4; ++q4) {
        const float4 f = *reinterpret_cast<const float4*>(&fs[kk][ch * NQ + q4 * 4]);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          acc[c][q4 * 4 + 0] = fmaf(f.x, x[c], acc[c][q4 * 4 + 0]);
          acc[c][q4 * 4 + 1] = fmaf(f.y, x[c], acc[c][q4 * 4 + 1]);
          acc[c][q4 * 4 + 2] = fmaf(f.z, x[c], acc[c][q4 * 4 + 2]);
          acc[c][q4 * 4 + 3] = fmaf(f.w, x[c], acc[c][q4 * 4 + 3]);
        }
      }
    }
    __syncthreads();
  }
  // sum the K slices (adjacent lanes), slice 0 writes
#pragma unroll
  for (int o = 1; o < KS; o <<= 1)
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc[c][q] += __shfl_xor_sync(0xffffffffu, acc[c][q], o);
  if (ks != 0) return;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int j = j0 + cq * 4 + c;
    if (j >= m) continue;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int cc = ch * NQ + q;
      if (cc < nc) Cb[S.c_off + cc + (int64_t)j * nct] = static_cast<double>(acc[c][q]);
    }
  }
}

// The K-extension of the operand: V_s (the coarse correction at the
// subdomain's corners) in the chunks after its b range, zero past n_c.
// blockDim.x covers the widest extension; each subdomain (blockIdx.y) writes
// its own, PV_J directions per block.
constexpr int PV_J = 64;
template <int FMT, int PASSES>
__global__ void k_put_v(const DevType* __restrict__ types, const DevSub* __restrict__ subs,
                        const int64_t* __restrict__ bpad, const int* __restrict__ cg, const double* __restrict__ V,
                        int np, int m, typename TcFmt<FMT>::T* __restrict__ xb_hi,
                        typename TcFmt<FMT>::T* __restrict__ xb_lo, int64_t nbp) {
  using F = TcFmt<FMT>;
  const DevSub S = subs[blockIdx.y];
  const DevType T = types[S.type];
  const int c = threadIdx.x;
  if (T.n_c == 0 || c >= (T.n_c + F::KC - 1) / F::KC * F::KC) return;
  const int cgl = c < T.n_c ? cg[S.c_off + c] : 0;
  const int64_t o0 = bpad[blockIdx.y] + k_extent(T.n_b, 0, 0, F::KC) + c;
  const int j1 = min(m, (int)(blockIdx.x + 1) * PV_J);
  for (int j = blockIdx.x * PV_J + threadIdx.y; j < j1; j += blockDim.y) {
    const float v = c < T.n_c ? f64_to_f32_rn(V[cgl + (int64_t)j * np]) : 0.0f;
    const int64_t o = (int64_t)j * nbp + o0;
    const typename F::T hi = F::round(v);
    xb_hi[o] = hi;
    if (PASSES == 3) xb_lo[o] = F::round(v - F::value(hi));
  }
}

// FP32 copy of the coarse inverse (precision form).
__global__ void k_to_f32(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = static_cast<float>(x[i]);
}

// V = Kbar^{-1} Vraw in FP32 arithmetic (the precision form's coarse
// correction).  A = Kbar^{-1} in FP32 (n x n, symmetric: read as row k gives
// column k), B = Vraw in FP32 (n x m, column-major, ld n).  128 x 128 output
// tiles, 256 threads with 8 x 8 outputs each (rows tx*4.. and 64+tx*4.., so
// that every thread stores four consecutive rows of a column at once), K
// staged CG_K at a time (the next stage loaded into registers while the
// current one is multiplied), split in CG_SPLIT ranges (blockIdx.z) whose FP32
// partial products go to P [CG_SPLIT x m x ldp], ldp = n rounded up to 4;
// k_coarse_sum adds them in a fixed order into V (FP64).
constexpr int CG_T = 128, CG_K = 8, CG_SPLIT = 4;
__global__ void __launch_bounds__(256, 2) k_sgemm_coarse(int n, int m, int ldp, const float* __restrict__ A,
                                                         const float* __restrict__ B, float* __restrict__ P) {
  __shared__ __align__(16) float As[2][CG_K][CG_T];
  __shared__ __align__(16) float Bs[2][CG_K][CG_T];
  const int i0 = blockIdx.x * CG_T, j0 = blockIdx.y * CG_T;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[r][q] = 0.0f;
  const int kper = ((n + CG_SPLIT * CG_K - 1) / (CG_SPLIT * CG_K)) * CG_K;
  const int kbeg = blockIdx.z * kper, kend = min(n, kbeg + kper);
  float ra[4], rb[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = tid + 256 * t, ii = e & (CG_T - 1), kk = e >> 7, i = i0 + ii, k = k0 + kk;
      ra[t] = (i < n && k < kend) ? A[(int64_t)k * n + i] : 0.0f;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = tid + 256 * t, kk = e & (CG_K - 1), jj = e >> 3, k = k0 + kk, j = j0 + jj;
      rb[t] = (k < kend && j < m) ? B[(int64_t)j * n + k] : 0.0f;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = tid + 256 * t;
      As[buf][e >> 7][e & (CG_T - 1)] = ra[t];
      Bs[buf][e & (CG_K - 1)][e >> 3] = rb[t];
    }
  };
  if (kbeg < kend) {
    load(kbeg);
    store(0);
  }
  __syncthreads();
  int buf = 0;
  for (int k0 = kbeg; k0 < kend; k0 += CG_K) {
    const bool more = k0 + CG_K < kend;
    if (more) load(k0 + CG_K);
#pragma unroll
    for (int kk = 0; kk < CG_K; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][tx * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + tx * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][ty * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + ty * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[r][q] = fmaf(av[r], bv[q], acc[r][q]);
    }
    if (more) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  float* Pz = P + (int64_t)blockIdx.z * ldp * m;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int j = j0 + (q < 4 ? ty * 4 + q : 64 + ty * 4 + q - 4);
    if (j >= m) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = i0 + h * 64 + tx * 4;          // i, ldp multiples of 4: i < ldp covers i + 3
      if (i < ldp)
        *reinterpret_cast<float4*>(Pz + (int64_t)j * ldp + i) =
            make_float4(acc[4 * h][q], acc[4 * h + 1][q], acc[4 * h + 2][q], acc[4 * h + 3][q]);
    }
  }
}

// V(i, j) = sum over the K ranges z, in order, of P_z(i, j); widened exactly.
__global__ void k_coarse_sum(int n, int m, int ldp, const float* __restrict__ P, double* __restrict__ V) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= n) return;
  float v = 0.0f;
#pragma unroll
  for (int z = 0; z < CG_SPLIT; ++z) v += P[((int64_t)z * m + j) * ldp + i];
  V[(int64_t)j * n + i] = f32_to_f64(v);
}

// y = x in FP32 on the integer pipe (the coarse product's right-hand sides).
__global__ void k_f32_of(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = f64_to_f32_rn(x[i]);
}

// Shat = D_S^{-1/2} S_bb D_S^{-1/2} (FP32) per module, for the preconditioner
// block of the precision form, and Frc_hat = D_F^{-1/2} F_rc (FP32) for the
// corner reduction.
__global__ void k_make_lowp(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                            const double* __restrict__ mem, float* __restrict__ fmem) {
  const DevModule M = mods[blockIdx.y];
  const DevType T = types[M.type];
  const int n = T.n_b, nbc = T.n_b + T.n_c;
  const double* Sm = mem + M.S;
  const double* F = mem + M.F;
  const int nc = T.n_c;
  if (nc > 0) {
    const double* Frc = mem + M.Frc;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * nc;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int i = (int)(e / nc);
      fmem[M.Frc + e] = static_cast<float>(Frc[e] / sqrt(F[(int64_t)i * n + i]));
    }
  }
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    const double sv = Sm[(int64_t)i * nbc + j] / sqrt(Sm[(int64_t)i * nbc + i] * Sm[(int64_t)j * nbc + j]);
    fmem[M.W + e] = static_cast<float>(sv);
  }
}

// per global b: sqrt(F_s(k,k)) and sqrt(S_s(k,k))
__global__ void k_sqrt_diag(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                            const DevSub* __restrict__ subs, const double* __restrict__ mem,
                            double* __restrict__ sqrtDF, double* __restrict__ sqrtDS) {
  const DevSub S = subs[blockIdx.y];
  const DevType T = types[S.type];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= T.n_b) return;
  const DevModule M = mods[S.module];
  const int n = T.n_b, nbc = T.n_b + T.n_c;
  sqrtDF[S.b_off + k] = sqrt(mem[M.F + (int64_t)k * n + k]);
  sqrtDS[S.b_off + k] = sqrt(mem[M.S + (int64_t)k * nbc + k]);
}

// xh = D_S^{1/2} x_b in FP32 (the scaled right-hand side of the
// preconditioner block, converted once per entry on the integer pipe).
__global__ void k_scale_x32(int64_t nbt, const double* __restrict__ sqrtDS, const double* __restrict__ x,
                            float* __restrict__ xh) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b < nbt) xh[b] = f64_to_f32_rn(sqrtDS[b] * x[b]);
}

// y_b(s) = D_S^{1/2} Shat_s xh(s) in FP32 arithmetic (preconditioner block of
// the precision form), one warp per row.
__global__ void k_sub_gemv_lowp(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                                const DevSub* __restrict__ subs, const float* __restrict__ fmem,
                                const double* __restrict__ sqrtDS, const float* __restrict__ xh,
                                double* __restrict__ y) {
  const DevSub S = subs[blockIdx.y];
  const DevType T = types[S.type];
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  const int n = T.n_b;
  if (row >= n) return;
  const float* a = fmem + mods[S.module].W + (int64_t)row * n;
  const float* xs = xh + S.b_off;
  float acc = 0.0f;
  for (int k = lane; k < n; k += 32) acc = fmaf(a[k], xs[k], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) y[S.b_off + row] = sqrtDS[S.b_off + row] * f32_to_f64(acc);
}

}  // namespace

int tc_tile_rows() { return TC_M; }

size_t tc_apply_smem_bytes(int passes) {
  const size_t stage = (passes == 3 ? 2 : 1) * (size_t)(TC_M * 128 + TC_NMAX * 128);
  return 1024 + (passes == 3 ? TC_STAGES3 : TC_STAGES1) * stage;
}

namespace {

// Format and pass count of the context's precision option.
int tc_format(const Ctx& c) { return (c.opt.precision == FETI_BF16 || c.opt.precision == FETI_BF16X3) ? 1 : 0; }
bool tc_split(const Ctx& c) { return c.opt.precision == FETI_TF32X3 || c.opt.precision == FETI_BF16X3; }

}  // namespace

int tc_chunk(int precision) { return (precision == FETI_BF16 || precision == FETI_BF16X3) ? 64 : 32; }
size_t tc_elem_bytes(int precision) { return (precision == FETI_BF16 || precision == FETI_BF16X3) ? 2 : 4; }
int tc_k_extent(int nb, int nc, int aug, int kc) { return k_extent(nb, nc, aug, kc); }

cudaError_t tc_prepare(const Ctx& c, cudaStream_t st) {
  k_make_lowp<<<dim3(64, c.n_mod), 256, 0, st>>>(c.d_types, c.d_mods, c.d_modmem, c.d_fmem);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const bool split = tc_split(c);
  if (tc_format(c) == 0)
    k_make_arena<0><<<dim3(64, c.n_mod), 256, 0, st>>>(c.d_types, c.d_mods, c.d_modmem, c.d_frow, c.fa_pitch,
                                                      c.tc_aug, static_cast<float*>(c.d_fa_hi),
                                                      split ? static_cast<float*>(c.d_fa_lo) : nullptr);
  else
    k_make_arena<1><<<dim3(64, c.n_mod), 256, 0, st>>>(c.d_types, c.d_mods, c.d_modmem, c.d_frow, c.fa_pitch,
                                                      c.tc_aug, static_cast<__nv_bfloat16*>(c.d_fa_hi),
                                                      split ? static_cast<__nv_bfloat16*>(c.d_fa_lo) : nullptr);
  note_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (c.n_ctiles_rows > 0) {
    if (tc_format(c) == 0)
      k_make_arena_corner<0><<<dim3(32, c.n_mod), 256, 0, st>>>(c.d_types, c.d_mods, c.d_modmem, c.fcrow0,
                                                               c.fa_pitch, static_cast<float*>(c.d_fa_hi),
                                                               split ? static_cast<float*>(c.d_fa_lo) : nullptr);
    else
      k_make_arena_corner<1><<<dim3(32, c.n_mod), 256, 0, st>>>(c.d_types, c.d_mods, c.d_modmem, c.fcrow0,
                                                               c.fa_pitch, static_cast<__nv_bfloat16*>(c.d_fa_hi),
                                                               split ? static_cast<__nv_bfloat16*>(c.d_fa_lo)
                                                                     : nullptr);
    note_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_sqrt_diag<<<dim3((c.max_nb + 127) / 128, c.hp.n_sub), 128, 0, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_modmem,
                                                                        c.d_sqrtDF, c.d_sqrtDS);
  note_launches(1);
  const int nsl = std::max(c.n_spread_slots, 1);
  k_spread_weights<<<(unsigned)((nsl + 255) / 256), 256, 0, st>>>(c.n_spread_slots, c.d_sp_b, c.d_sqrtDF, c.d_sp_sd);
  note_launches(1);
  return cudaGetLastError();
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Row-major matrix [rows x pitch] of the operand format read in boxes of one
// 128-byte row segment x box_rows with the 128-byte swizzle; outside the
// matrix the box is filled with zeros.
template <int FMT>
bool make_map(CUtensorMap* map, const void* base, int64_t pitch, int64_t rows, uint32_t box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  const size_t eb = FMT == 0 ? 4 : 2;
  const cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch * eb};
  const cuuint32_t box[2] = {(cuuint32_t)TcFmt<FMT>::KC, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, FMT == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
            const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

template <int FMT, int PASSES, int STAGES>
cudaError_t launch_tc(const Ctx& c, int m, float* Yb, cudaStream_t st) {
  static bool attr_set = false;
  const size_t smem = tc_apply_smem_bytes(PASSES);
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_apply<FMT, PASSES, STAGES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  CUtensorMap ta, tal, tb, tbl;
  const void* alo = PASSES == 3 ? c.d_fa_lo : c.d_fa_hi;
  const void* blo = PASSES == 3 ? c.d_xb_lo : c.d_xb_hi;
  if (!make_map<FMT>(&ta, c.d_fa_hi, c.fa_pitch, c.fa_rows, TC_M) ||
      !make_map<FMT>(&tal, alo, c.fa_pitch, c.fa_rows, TC_M) ||
      !make_map<FMT>(&tb, c.d_xb_hi, c.nbp_total, m, TC_NMAX) || !make_map<FMT>(&tbl, blo, c.nbp_total, m, TC_NMAX))
    return cudaErrorInvalidValue;
  const int n_cb = (m + TC_NMAX - 1) / TC_NMAX;
  const int n_rb = (c.max_nb + TC_M - 1) / TC_M;
  dim3 grid(n_cb * n_rb, c.hp.n_sub);
  k_tc_apply<FMT, PASSES, STAGES><<<grid, TC_THREADS, smem, st>>>(ta, tal, tb, tbl, c.d_types, c.d_subs, c.d_frow,
                                                                  c.d_bpad, c.d_sqrtDF, Yb, c.hp.n_b_total, m, n_cb,
                                                                  c.tc_aug, c.d_status, c.test_skip_chunk);
  note_launches(1);
  return cudaGetLastError();
}

template <int FMT, int PASSES, int STAGES>
cudaError_t launch_tc_p(const Ctx& c, int m, float* Yb, cudaStream_t st, bool corner = false) {
  static bool attr_set = false;
  const size_t smem = 1024 + (size_t)STAGES * (PASSES == 3 ? 2 : 1) * (TC_M * 128 + TC_NMAX * 128);
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_apply_p<FMT, PASSES, STAGES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  CUtensorMap ta, tal, tb, tbl;
  const void* alo = PASSES == 3 ? c.d_fa_lo : c.d_fa_hi;
  const void* blo = PASSES == 3 ? c.d_xb_lo : c.d_xb_hi;
  if (!make_map<FMT>(&ta, c.d_fa_hi, c.fa_pitch, c.fa_rows, TC_M) ||
      !make_map<FMT>(&tal, alo, c.fa_pitch, c.fa_rows, TC_M) ||
      !make_map<FMT>(&tb, c.d_xb_hi, c.nbp_total, m, TC_NMAX) || !make_map<FMT>(&tbl, blo, c.nbp_total, m, TC_NMAX))
    return cudaErrorInvalidValue;
  const int ntl = corner ? c.n_ctiles : c.n_tiles;
  const int4* tl = corner ? c.d_tiles + c.n_tiles : c.d_tiles;
  const int grid = std::min(ntl, std::max(1, c.n_sm));
  if (grid <= 0) return cudaSuccess;
  k_tc_apply_p<FMT, PASSES, STAGES><<<grid, TCP_THREADS, smem, st>>>(ta, tal, tb, tbl, tl, ntl, c.d_types,
                                                                     c.d_subs, c.d_frow, c.d_bpad, c.d_sqrtDF, Yb,
                                                                     c.hp.n_b_total, m, c.tc_aug, c.d_status,
                                                                     c.fcrow0, c.d_Cb, c.n_c_total);
  note_launches(1);
  return cudaGetLastError();
}

template <int FMT, int PASSES>
cudaError_t launch_gather(const Ctx& c, const double* X, int64_t ldx, int m, cudaStream_t st) {
  using T = typename TcFmt<FMT>::T;
  dim3 g((unsigned)c.n_spread_ranges, (m + SP_J - 1) / SP_J);
  k_spread_tc<FMT, PASSES><<<g, SP_THREADS, 0, st>>>(m, c.d_sp_row0, c.d_sp_slot_off, c.d_sp_pos, c.d_sp_sd,
                                                     c.d_sp_ent_off, c.d_sp_ent, X, ldx, static_cast<T*>(c.d_xb_hi),
                                                     PASSES == 3 ? static_cast<T*>(c.d_xb_lo) : nullptr,
                                                     c.nbp_total);
  return cudaGetLastError();
}

template <int FMT, int PASSES>
void launch_put_v(const Ctx& c, const double* V, int m, cudaStream_t st) {
  using T = typename TcFmt<FMT>::T;
  constexpr int KC = TcFmt<FMT>::KC;
  const int ext = (c.max_nc + KC - 1) / KC * KC;      // widest corner extension (<= 64)
  dim3 g((m + PV_J - 1) / PV_J, c.hp.n_sub);
  k_put_v<FMT, PASSES><<<g, dim3(ext, 8), 0, st>>>(
      c.d_types, c.d_subs, c.d_bpad, c.d_c_glob, V, c.hp.n_primal, m, static_cast<T*>(c.d_xb_hi),
      PASSES == 3 ? static_cast<T*>(c.d_xb_lo) : nullptr, c.nbp_total);
}

}  // namespace

// The persistent kernel's work list for m directions: (subdomain, row tile,
// column tile) for every row tile that holds interface rows; consecutive
// entries share the subdomain (B chunks reused from L2) and the row tile (A
// chunks reused).  Rebuilt only when the number of column tiles changes.
cudaError_t tc_prepare_tiles(Ctx& c, int m) {
  const int n_cb = (m + TC_NMAX - 1) / TC_NMAX;
  if (c.tiles_ncb == n_cb) return cudaSuccess;
  std::vector<int4> tl;
  for (int s = 0; s < c.hp.n_sub; ++s) {
    const int nb = c.h_types[c.h_subs[s].type].n_b;
    for (int rb = 0; rb * TC_M < nb; ++rb)
      for (int cb = 0; cb < n_cb; ++cb) tl.push_back(make_int4(s, rb, cb, 0));
  }
  const int n_main = (int)tl.size();
  // corner tiles (FETI-DP): one row tile per subdomain with primal DOFs
  if (c.n_ctiles_rows > 0)
    for (int s = 0; s < c.hp.n_sub; ++s)
      if (c.h_types[c.h_subs[s].type].n_c > 0)
        for (int cb = 0; cb < n_cb; ++cb) tl.push_back(make_int4(s, 0, cb, 1));
  if ((int64_t)tl.size() > c.tiles_cap) {
    if (c.d_tiles) {
      cudaError_t e = cudaStreamSynchronize(c.stream);
      if (e != cudaSuccess) return e;
      dev_free(c, c.d_tiles, (size_t)c.tiles_cap * sizeof(int4));
    }
    c.d_tiles = nullptr;
    c.tiles_cap = 0;
    void* q = nullptr;
    cudaError_t e = dev_alloc(c, &q, std::max<size_t>(tl.size(), 1) * sizeof(int4));
    if (e != cudaSuccess) return e;
    c.d_tiles = static_cast<int4*>(q);
    c.tiles_cap = (int64_t)std::max<size_t>(tl.size(), 1);
  }
  cudaError_t e = cudaMemcpy(c.d_tiles, tl.data(), tl.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  if (c.n_sm <= 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    e = cudaDeviceGetAttribute(&c.n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  c.n_tiles = n_main;
  c.n_ctiles = (int)tl.size() - n_main;
  c.tiles_ncb = n_cb;
  return cudaSuccess;
}

// xb = parts of D^{1/2} B^T X in the operand format and padded layout.
cudaError_t tc_gather(const Ctx& c, const double* X, int64_t ldx, int m, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  if (m > c.xb_cap) return cudaErrorInvalidValue;
  const int f = tc_format(c);
  const bool split = tc_split(c);
  cudaError_t e;
  if (f == 0) e = split ? launch_gather<0, 3>(c, X, ldx, m, st) : launch_gather<0, 1>(c, X, ldx, m, st);
  else e = split ? launch_gather<1, 3>(c, X, ldx, m, st) : launch_gather<1, 1>(c, X, ldx, m, st);
  note_launches(1);
  return e;
}

// Cb = F_rc^T X_b per subdomain (FP32) from the gathered operand, then the
// corner assembly Vraw = sum over the copies of each primal DOF.
template <int FMT, int NCM>
void launch_frct_lowp(const Ctx& c, int m, cudaStream_t st) {
  using T = typename TcFmt<FMT>::T;
  dim3 g((m + 127) / 128, c.hp.n_sub);
  k_frct_lowp<FMT, NCM><<<g, 256, 0, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_fmem, c.d_bpad,
                                           static_cast<const T*>(c.d_xb_hi),
                                           tc_split(c) ? static_cast<const T*>(c.d_xb_lo) : nullptr, c.nbp_total, m,
                                           c.d_Cb, c.n_c_total);
}

cudaError_t tc_corner_reduce(const Ctx& c, int m, double* Vraw, cudaStream_t st) {
  if (c.max_nc > TC_MAX_NC) return cudaErrorInvalidValue;
  if (c.n_ctiles > 0 && c.tiles_ncb == (m + TC_NMAX - 1) / TC_NMAX) {
    // on the tensor cores: the corner tiles of the persistent product
    const bool split = tc_split(c);
    cudaError_t e;
    if (tc_format(c) == 0)
      e = split ? launch_tc_p<0, 3, TCP_STAGES3>(c, m, nullptr, st, true)
                : launch_tc_p<0, 1, TCP_STAGES1>(c, m, nullptr, st, true);
    else
      e = split ? launch_tc_p<1, 3, TCP_STAGES3>(c, m, nullptr, st, true)
                : launch_tc_p<1, 1, TCP_STAGES1>(c, m, nullptr, st, true);
    if (e != cudaSuccess) return e;
    return corner_assemble(c, m, Vraw, st);
  }
  const bool wide = c.max_nc > 24;                   // edge averages: up to 64 primal DOFs per subdomain
  if (tc_format(c) == 0) wide ? launch_frct_lowp<0, 64>(c, m, st) : launch_frct_lowp<0, 24>(c, m, st);
  else wide ? launch_frct_lowp<1, 64>(c, m, st) : launch_frct_lowp<1, 24>(c, m, st);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return corner_assemble(c, m, Vraw, st);
}

// The coarse correction V into the K-extension of the operand.
cudaError_t tc_put_v(const Ctx& c, const double* V, int m, cudaStream_t st) {
  if (!c.tc_aug) return cudaSuccess;
  const int f = tc_format(c);
  const bool split = tc_split(c);
  if (f == 0) split ? launch_put_v<0, 3>(c, V, m, st) : launch_put_v<0, 1>(c, V, m, st);
  else split ? launch_put_v<1, 3>(c, V, m, st) : launch_put_v<1, 1>(c, V, m, st);
  note_launches(1);
  return cudaGetLastError();
}

// FP32 scratch of the coarse product for n primal DOFs and cap directions:
// the split-K partials, then the right-hand sides in FP32.
int64_t tc_coarse_scratch(int n, int cap) { return ((int64_t)CG_SPLIT * ((n + 3) / 4 * 4) + n) * cap; }

cudaError_t tc_coarse_prepare(const Ctx& c, cudaStream_t st) {
  const int64_t n = (int64_t)c.hp.n_primal * c.hp.n_primal;
  k_to_f32<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(n, c.d_Kbar_inv, c.d_Kbar_inv32);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t tc_coarse_apply(const Ctx& c, const double* Vraw, double* V, int m, cudaStream_t st) {
  const int n = c.hp.n_primal;
  if (!c.d_Kbar_inv32 || n <= 0 || m <= 0) return cudaErrorInvalidValue;
  if (!c.d_coarse_part || m > c.blk_cap) return cudaErrorInvalidValue;
  const int ldp = (n + 3) / 4 * 4;
  float* P = c.d_coarse_part;
  float* B32 = c.d_coarse_part + (int64_t)CG_SPLIT * ldp * c.blk_cap;
  const int64_t nm = (int64_t)n * m;
  k_f32_of<<<(unsigned)((nm + 255) / 256), 256, 0, st>>>(nm, Vraw, B32);
  dim3 g((n + CG_T - 1) / CG_T, (m + CG_T - 1) / CG_T, CG_SPLIT);
  k_sgemm_coarse<<<g, 256, 0, st>>>(n, m, ldp, c.d_Kbar_inv32, B32, P);
  k_coarse_sum<<<dim3((n + 255) / 256, m), 256, 0, st>>>(n, m, ldp, P, V);
  note_launches(3);
  return cudaGetLastError();
}

// Yb (FP32) = D^{1/2} [Fhat | Frc_hat] xb for every subdomain (tensor cores).
cudaError_t tc_product(const Ctx& c, int m, float* Yb, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  if (m > c.xb_cap) return cudaErrorInvalidValue;
  if (c.tiles_ncb != (m + TC_NMAX - 1) / TC_NMAX) return cudaErrorInvalidValue;   // tile list not prepared
  prof_begin(st, c.fl_tc * m, 1);
  cudaError_t e;
  const bool split = tc_split(c);
  // measured choice (3D, 512 directions): BF16 operands run faster in the
  // persistent kernel (0.56 vs 0.71 ms one pass, 1.20 vs 1.64 ms split), TF32
  // operands -- twice the bytes per MMA -- in the one-tile-per-CTA kernel with
  // two CTAs per SM (1.35 vs 1.54 ms, 2.97 vs 3.12 ms)
  if (tc_format(c) == 0)
    e = split ? launch_tc<0, 3, TC_STAGES3>(c, m, Yb, st) : launch_tc<0, 1, TC_STAGES1>(c, m, Yb, st);
  else
    e = split ? launch_tc_p<1, 3, TCP_STAGES3>(c, m, Yb, st) : launch_tc_p<1, 1, TCP_STAGES1>(c, m, Yb, st);
  prof_end(st);
  return e;
}

cudaError_t lowp_gemv_S(const Ctx& c, const double* xb, float* xh, double* yb, cudaStream_t st) {
  const int64_t nbt = c.hp.n_b_total;
  k_scale_x32<<<(unsigned)((nbt + 255) / 256), 256, 0, st>>>(nbt, c.d_sqrtDS, xb, xh);
  k_sub_gemv_lowp<<<dim3((c.max_nb + 7) / 8, c.hp.n_sub), 256, 0, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_fmem,
                                                                         c.d_sqrtDS, xh, yb);
  note_launches(2);
  return cudaGetLastError();
}

}  // namespace feti
