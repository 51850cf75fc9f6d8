// Tensor-core form of the local dual-operator product (the precision form):
//
//   Y_b(s) = D_s^{1/2} Fhat_s D_s^{1/2} X_b(s),   Fhat_s = D_s^{-1/2} F_s D_s^{-1/2},
//
// with D_s = diag(F_s).  Fhat_s is stored in FP32 (rounded to TF32), the
// product runs on the 5th-generation tensor cores (tcgen05.mma kind::tf32)
// with FP32 accumulation in tensor memory.  X_b(s) = B^sT X is gathered from
// the multiplier space straight into shared memory (signed, scaled by
// D^{1/2}, rounded to TF32) -- no interface-space copy of X is written.
//
// One CTA of 128 threads computes a 128-row tile of one subdomain's output for
// up to 256 direction columns.  K is streamed in chunks of 32 FP32 values (one
// 128-byte swizzle row); thread 0 issues four K=8 MMAs per chunk and commits
// them to an mbarrier that the CTA waits on (bounded: on time-out the kernel
// records an error code, waits once more, frees its tensor memory and exits).
#include <cstdint>

#include "kernels.h"

namespace feti {

namespace {

constexpr int TC_M = 128;
constexpr int TC_KC = 32;           // FP32 elements per 128-byte row
constexpr int TC_NMAX = 256;
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_TMEM_COLS = 256;
constexpr long long TC_SPIN_LIMIT = 1ll << 22;

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

// Instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(TC_M >> 4) << 24);
}

// Byte offset of element (row, k) of a K-major tile with 128-byte rows and the
// 128-byte swizzle (16-byte chunk index XOR row % 8).
__device__ __forceinline__ uint32_t sw128_offset(int row, int k) {
  const int chunk = (k >> 2) ^ (row & 7);
  return static_cast<uint32_t>((row >> 3) * 1024 + (row & 7) * 128 + chunk * 16 + (k & 3) * 4);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
  for (long long it = 0; it < TC_SPIN_LIMIT; ++it) {
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

// PASSES = 1: one TF32 product.  PASSES = 3: the split-TF32 product
// a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi with a_hi = tf32(a), a_lo =
// tf32(a - a_hi), which carries FP32-class accuracy on the tensor cores.
template <int PASSES>
__global__ void __launch_bounds__(TC_THREADS) k_tc_apply_tf32(
    const DevType* __restrict__ types, const DevModule* __restrict__ mods, const DevSub* __restrict__ subs,
    const float* __restrict__ fmem, const double* __restrict__ X, int64_t ldx, int m,
    const int* __restrict__ b2l_off, const int* __restrict__ b2l_lam, const signed char* __restrict__ b2l_sign,
    const double* __restrict__ sqrtD, double* __restrict__ Yb, int64_t nbt, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  // 1024-byte aligned staging: A chunk [128 x 128 B], B chunk [256 x 128 B]
  // (PASSES = 3: followed by the low parts A_lo, B_lo)
  unsigned char* base = tc_smem_raw + ((1024 - (smem_u32(tc_smem_raw) & 1023)) & 1023);
  unsigned char* As = base;
  unsigned char* Bs = base + TC_M * 128;
  unsigned char* Al = Bs + TC_NMAX * 128;
  unsigned char* Bl = Al + TC_M * 128;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base_sh;

  const DevSub S = subs[blockIdx.y];
  const DevType T = types[S.type];
  const int nb = T.n_b;
  const int row0 = blockIdx.x * TC_M;
  const int col0 = blockIdx.z * TC_NMAX;
  if (row0 >= nb || col0 >= m) return;
  const int ncols = min(TC_NMAX, m - col0);
  const int np = ((ncols + 15) / 16) * 16;
  const float* F = fmem + mods[S.module].F;          // Fhat_s, nb x nb row-major FP32
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;
  const uint32_t bar = smem_u32(&mbar);
  const uint32_t idesc = idesc_tf32(np);
  uint32_t phase = 0;
  bool failed = false;

  for (int k0 = 0; k0 < nb; k0 += TC_KC) {
    // ---- stage A: 128 rows x 32 K of Fhat (zero outside the matrix) ----
    for (int e = tid; e < TC_M * TC_KC; e += TC_THREADS) {
      const int r = e >> 5, k = e & 31;
      const int gr = row0 + r, gk = k0 + k;
      const float v = (gr < nb && gk < nb) ? F[(int64_t)gr * nb + gk] : 0.0f;
      const float hi = to_tf32(v);
      *reinterpret_cast<float*>(As + sw128_offset(r, k)) = hi;
      if (PASSES == 3) *reinterpret_cast<float*>(Al + sw128_offset(r, k)) = to_tf32(v - hi);
    }
    // ---- stage B: direction j, K index k: D^{1/2} (B^sT X)[b, j], b = b_off + k0 + k ----
    for (int e = tid; e < np * TC_KC; e += TC_THREADS) {
      const int j = e >> 5, k = e & 31;
      const int gk = k0 + k, gj = col0 + j;
      float v = 0.0f;
      if (gk < nb && gj < m) {
        const int64_t b = S.b_off + gk;
        const double* x = X + (int64_t)gj * ldx;
        double acc = 0.0;
        for (int q = b2l_off[b]; q < b2l_off[b + 1]; ++q) acc += b2l_sign[q] > 0 ? x[b2l_lam[q]] : -x[b2l_lam[q]];
        v = static_cast<float>(acc * sqrtD[b]);
      }
      const float hi = to_tf32(v);
      *reinterpret_cast<float*>(Bs + sw128_offset(j, k)) = hi;
      if (PASSES == 3) *reinterpret_cast<float*>(Bl + sw128_offset(j, k)) = to_tf32(v - hi);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < TC_KC / 8; ++kk) {
#pragma unroll
        for (int pass = 0; pass < PASSES; ++pass) {
          // pass 0: lo x hi, pass 1: hi x lo, last pass: hi x hi (small terms first)
          const unsigned char* Ap = (PASSES == 3 && pass == 0) ? Al : As;
          const unsigned char* Bp = (PASSES == 3 && pass == 1) ? Bl : Bs;
          const uint64_t ad = desc_sw128(smem_u32(Ap) + kk * 32);
          const uint64_t bd = desc_sw128(smem_u32(Bp) + kk * 32);
          const uint32_t acc = (k0 > 0 || kk > 0 || pass > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\t"
              "setp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                   : "memory");
    }
    __syncwarp();
    const bool ok = mbar_wait(bar, phase);
    if (__syncthreads_or(!ok)) {           // block-uniform decision
      failed = true;
      if (tid == 0) atomicCAS(status, 0, 3000000 + blockIdx.y);
      if (!ok) mbar_wait(bar, phase);      // one more bounded wait for the MMAs in flight
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }

  if (!failed) {
    // ---- epilogue: warp w owns TMEM lanes [32w, 32w+32) = output rows ----
    const int r = row0 + warp * 32 + lane;
    const double sd = r < nb ? sqrtD[S.b_off + r] : 0.0;
    for (int jc = 0; jc < np; jc += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)jc;
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
      if (r < nb) {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int gj = col0 + jc + c;
          if (jc + c < ncols) Yb[S.b_off + r + (int64_t)gj * nbt] = sd * (double)__uint_as_float(v[c]);
        }
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

// Fhat = D^{-1/2} F D^{-1/2} (FP32, rounded to TF32) and D^{1/2} per module;
// Shat likewise for the preconditioner block S_bb (its own diagonal).
__global__ void k_make_lowp(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                            const double* __restrict__ mem, float* __restrict__ fmem) {
  const DevModule M = mods[blockIdx.y];
  const DevType T = types[M.type];
  const int n = T.n_b, nbc = T.n_b + T.n_c;
  const double* F = mem + M.F;
  const double* Sm = mem + M.S;
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    const double fv = F[e] / sqrt(F[(int64_t)i * n + i] * F[(int64_t)j * n + j]);
    fmem[M.F + e] = static_cast<float>(fv);
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

// y_b(s) = D_S^{1/2} Shat_s D_S^{1/2} x_b(s) in FP32 arithmetic (preconditioner
// block of the precision form), one warp per row.
__global__ void k_sub_gemv_lowp(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                                const DevSub* __restrict__ subs, const float* __restrict__ fmem,
                                const double* __restrict__ sqrtDS, const double* __restrict__ x,
                                double* __restrict__ y) {
  const DevSub S = subs[blockIdx.y];
  const DevType T = types[S.type];
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  const int n = T.n_b;
  if (row >= n) return;
  const float* a = fmem + mods[S.module].W + (int64_t)row * n;
  const double* xs = x + S.b_off;
  const double* ds = sqrtDS + S.b_off;
  float acc = 0.0f;
  for (int k = lane; k < n; k += 32) acc = fmaf(a[k], static_cast<float>(ds[k] * xs[k]), acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) y[S.b_off + row] = ds[row] * (double)acc;
}

}  // namespace

size_t tc_apply_smem_bytes(int passes) { return 1024 + (passes == 3 ? 2 : 1) * (TC_M * 128 + TC_NMAX * 128); }

cudaError_t tc_prepare(const Ctx& c, cudaStream_t st) {
  k_make_lowp<<<dim3(64, c.n_mod), 256, 0, st>>>(c.d_types, c.d_mods, c.d_modmem, c.d_fmem);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sqrt_diag<<<dim3((c.max_nb + 127) / 128, c.hp.n_sub), 128, 0, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_modmem,
                                                                        c.d_sqrtDF, c.d_sqrtDS);
  note_launches(1);
  return cudaGetLastError();
}

// Yb = D^{1/2} Fhat D^{1/2} B^T X for every subdomain (tensor cores).
cudaError_t tc_apply_local(const Ctx& c, const double* X, int64_t ldx, int m, double* Yb, cudaStream_t st) {
  static bool attr_set = false;
  const size_t sm1 = tc_apply_smem_bytes(1), sm3 = tc_apply_smem_bytes(3);
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_apply_tf32<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tc_apply_tf32<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((c.max_nb + TC_M - 1) / TC_M, c.hp.n_sub, (m + TC_NMAX - 1) / TC_NMAX);
  if (c.opt.precision == FETI_TF32X3)
    k_tc_apply_tf32<3><<<grid, TC_THREADS, sm3, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_fmem, X, ldx, m,
                                                      c.d_b2l_off, c.d_b2l_lam, c.d_b2l_sign, c.d_sqrtDF, Yb,
                                                      c.hp.n_b_total, c.d_status);
  else
    k_tc_apply_tf32<1><<<grid, TC_THREADS, sm1, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_fmem, X, ldx, m,
                                                      c.d_b2l_off, c.d_b2l_lam, c.d_b2l_sign, c.d_sqrtDF, Yb,
                                                      c.hp.n_b_total, c.d_status);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t lowp_gemv_S(const Ctx& c, const double* xb, double* yb, cudaStream_t st) {
  k_sub_gemv_lowp<<<dim3((c.max_nb + 7) / 8, c.hp.n_sub), 256, 0, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_fmem,
                                                                         c.d_sqrtDS, xb, yb);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace feti
