// Reduced-precision block update of the precision form: C -= A B with FP64
// storage and FP32 products and sums (CUDA cores).
//
// Inside the refinement's inner solves (reduced-precision dual operator), the
// full orthogonalization's block updates W_{i+1} -= W_j Psi_j of Algorithm 1
// are plain products, not inner products: the coefficients Psi_j = Q_j^T W_{i+1}
// stay FP64, the update of the direction block is rounded like the operator's
// own local products (an FP32-class error in W_{i+1}, removed by the next FP64
// refinement step like every other error of the inner solve).
//
// Tiles of 128 x 128 outputs, 256 threads with 8 x 8 outputs each, K staged 8
// at a time in two shared buffers (the next stage loaded into registers while
// the current one is multiplied); operands converted FP64 -> FP32 on the
// integer pipe (fpconv.cuh).
#include "kernels.h"
#include "fpconv.cuh"

namespace feti {

namespace {

constexpr int SU_BM = 128, SU_BN = 128, SU_BK = 8;

__global__ void __launch_bounds__(256, 2) k_sgemm_sub(int64_t n, int m, int k, const double* __restrict__ A,
                                                   int64_t lda, const double* __restrict__ B, int64_t ldb,
                                                   double* __restrict__ C, int64_t ldc) {
  __shared__ __align__(16) float As[2][SU_BK][SU_BM];
  __shared__ __align__(16) float Bs[2][SU_BK][SU_BN];
  const int64_t i0 = (int64_t)blockIdx.x * SU_BM;
  const int j0 = blockIdx.y * SU_BN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[r][q] = 0.0f;
  double ra[4], rb[4];
  auto load = [&](int l0) {                     // the next K stage into registers
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = tid + 256 * t, r = e & (SU_BM - 1), kk = e >> 7;
      const int64_t i = i0 + r;
      const int l = l0 + kk;
      ra[t] = (i < n && l < k) ? A[i + (int64_t)l * lda] : 0.0;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = tid + 256 * t, kk = e & (SU_BK - 1), cc = e >> 3;
      const int j = j0 + cc, l = l0 + kk;
      rb[t] = (j < m && l < k) ? B[l + (int64_t)j * ldb] : 0.0;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = tid + 256 * t;
      As[buf][e >> 7][e & (SU_BM - 1)] = f64_to_f32_rn(ra[t]);
      Bs[buf][e & (SU_BK - 1)][e >> 3] = f64_to_f32_rn(rb[t]);
    }
  };
  load(0);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int l0 = 0; l0 < k; l0 += SU_BK) {
    const bool more = l0 + SU_BK < k;
    if (more) load(l0 + SU_BK);                 // in flight while this stage is multiplied
#pragma unroll
    for (int kk = 0; kk < SU_BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][tx * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + tx * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][ty * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + ty * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[r][q] = fmaf(a[r], b[q], acc[r][q]);
    }
    if (more) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int j = j0 + (q < 4 ? ty * 4 + q : 64 + ty * 4 + q - 4);
    if (j >= m) continue;
    double* c = C + (int64_t)j * ldc;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int64_t i = i0 + (r < 4 ? tx * 4 + r : 64 + tx * 4 + r - 4);
      if (i < n) c[i] -= f32_to_f64(acc[r][q]);          // exact widening on the integer pipe
    }
  }
}

}  // namespace

cudaError_t sgemm_sub(int64_t n, int m, int k, const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                      int64_t ldc, cudaStream_t st) {
  if (n <= 0 || m <= 0 || k <= 0) return cudaSuccess;
  dim3 g((unsigned)((n + SU_BM - 1) / SU_BM), (unsigned)((m + SU_BN - 1) / SU_BN));
  k_sgemm_sub<<<g, 256, 0, st>>>(n, m, k, A, lda, B, ldb, C, ldc);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace feti
