// Dual-operator kernels: the hot path of Algorithm 1.
//
//   Y = F X:  gather X into the interface ("b") space of every subdomain
//             (B^sT X, signed), multiply by the dense local blocks, scatter
//             back with B^s.  FETI-DP (Eq. 12, u_c condensed) adds the corner
//             correction F_rc Kbar_cc^{-1} F_rc^T X between the two halves.
//   Z = [B~^s S^s B~^sT r]_s: the same gather with the scaling weights of
//             Eq. (15), one dense S^s product per subdomain, and a scatter that
//             keeps each subdomain's contribution in its own column (Section 3.3).
//
// Every multiplier row has at most two entries, so the scatter is a gather
// from the multiplier side: deterministic, no atomics.
#include <algorithm>

#include "fpconv.cuh"
#include "kernels.h"

namespace feti {

namespace {

__global__ void k_gather(int64_t nbt, int m, const int* __restrict__ off, const int* __restrict__ lam,
                         const signed char* __restrict__ sg, const double* __restrict__ X, int64_t ldx,
                         double* __restrict__ Xb) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (b >= nbt || j >= m) return;
  const double* x = X + (int64_t)j * ldx;
  double v = 0.0;
  for (int e = off[b]; e < off[b + 1]; ++e) v += sg[e] > 0 ? x[lam[e]] : -x[lam[e]];
  Xb[b + (int64_t)j * nbt] = v;
}

// Each thread serves SC_J consecutive columns, reading the row's entries once.
constexpr int SC_J = 8;
constexpr int SC_Z = 64;            // FP32 scatter: directions per block
template <typename TY>
__global__ void k_scatter(int64_t nl, int m, const int* __restrict__ b0, const signed char* __restrict__ s0,
                          const int* __restrict__ b1, const signed char* __restrict__ s1,
                          const TY* __restrict__ Yb, int64_t nbt, double* __restrict__ Y, int64_t ldy) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int j0 = blockIdx.y * SC_J;
  if (l >= nl) return;
  const int jn = min(SC_J, m - j0);
  const int p0 = b0[l], p1 = b1[l];
  const bool n0 = s0[l] < 0, n1 = p1 >= 0 && s1[l] < 0;
#pragma unroll
  for (int u = 0; u < SC_J; ++u) {
    if (u >= jn) break;
    const TY* yb = Yb + (int64_t)(j0 + u) * nbt;
    const double a = static_cast<double>(yb[p0]);
    double v = n0 ? -a : a;
    if (p1 >= 0) {
      const double c = static_cast<double>(yb[p1]);
      v += n1 ? -c : c;
    }
    Y[l + (int64_t)(j0 + u) * ldy] = v;
  }
}

// rb[b] = sum over rows of b of w * sign * r  (B~^sT r)
__global__ void k_gather_weighted(int64_t nbt, const int* __restrict__ off, const int* __restrict__ lam,
                                  const signed char* __restrict__ sg, const int* __restrict__ lb0,
                                  const double* __restrict__ w0, const double* __restrict__ w1,
                                  const double* __restrict__ r, double* __restrict__ rb) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= nbt) return;
  double v = 0.0;
  for (int e = off[b]; e < off[b + 1]; ++e) {
    const int l = lam[e];
    const double w = lb0[l] == (int)b ? w0[l] : w1[l];
    const double t = w * r[l];
    v += sg[e] > 0 ? t : -t;
  }
  rb[b] = v;
}

// Z[l, sub] = w * sign * zb[b] for each entry of row l; z[l] = row sum.
__global__ void k_prec_scatter(int64_t nl, const int* __restrict__ b0, const signed char* __restrict__ s0,
                               const int* __restrict__ b1, const signed char* __restrict__ s1,
                               const double* __restrict__ w0, const double* __restrict__ w1,
                               const int* __restrict__ bsub, const double* __restrict__ zb,
                               double* __restrict__ Z, int64_t ldz, double* __restrict__ z) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= nl) return;
  const int q0 = b0[l];
  double v0 = w0[l] * zb[q0];
  if (s0[l] < 0) v0 = -v0;
  double v = v0;
  if (Z) Z[l + (int64_t)bsub[q0] * ldz] = v0;
  const int q1 = b1[l];
  if (q1 >= 0) {
    double v1 = w1[l] * zb[q1];
    if (s1[l] < 0) v1 = -v1;
    v += v1;
    if (Z) Z[l + (int64_t)bsub[q1] * ldz] = v1;
  }
  if (z) z[l] = v;
}

// y_b(s) = A_s x_b(s) (+ beta y) with A_s = F_s (which 0), S_bb (which 1);
// one warp per row.
__global__ void k_sub_gemv(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                           const DevSub* __restrict__ subs, const double* __restrict__ mem, int which,
                           const double* __restrict__ x, double* __restrict__ y, double beta) {
  const DevSub S = subs[blockIdx.y];
  const DevType T = types[S.type];
  const DevModule M = mods[S.module];
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  const int n = T.n_b;
  if (row >= n) return;
  // which: 0 F_s, 1 S_s (b-b block of the n_bc-wide Schur complement), 2 K_bb (lumped)
  const double* A = mem + (which == 0 ? M.F : which == 1 ? M.S : M.Kl);
  const int64_t ld = which == 1 ? (int64_t)(T.n_b + T.n_c) : n;
  const double* a = A + (int64_t)row * ld;
  const double* xs = x + S.b_off;
  double acc = 0.0;
  for (int k = lane; k < n; k += 32) acc = fma(a[k], xs[k], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    double* yp = y + S.b_off + row;
    *yp = beta != 0.0 ? fma(beta, *yp, acc) : acc;
  }
}

// Cb[c_off(s) + c + j*nct] = sum_k F_rc,s(k, c) X_b(s)[k, j]: the thin corner
// product (n_c <= 24 rows), one thread per (column j, subdomain) with all
// n_c sums in registers, so no FP64 work is spent on tile padding.
template <int NC>
__global__ void k_frct(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                       const DevSub* __restrict__ subs, const double* __restrict__ mem,
                       const double* __restrict__ Xb, int64_t nbt, int m, double* __restrict__ Cb, int64_t nct) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const DevSub S = subs[blockIdx.y];
  if (j >= m) return;
  const DevType T = types[S.type];
  const int nc = T.n_c, nb = T.n_b;
  const double* F = mem + mods[S.module].Frc;    // [nb x nc] row-major
  const double* x = Xb + S.b_off + (int64_t)j * nbt;
  double acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0;
  for (int k = 0; k < nb; ++k) {
    const double xv = x[k];
    const double* fr = F + (int64_t)k * nc;
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (c < nc) acc[c] = fma(fr[c], xv, acc[c]);
  }
  double* out = Cb + S.c_off + (int64_t)j * nct;
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (c < nc) out[c] = acc[c];
}

// One direction: C_s = F_rc,s^T x_b(s) with one block of 128 threads per
// subdomain (the rows split across the threads, partial sums reduced in a
// fixed order): the one-direction variants would otherwise leave a single
// thread per subdomain walking every row.
template <int NC>
__global__ void __launch_bounds__(128) k_frct_one(const DevType* __restrict__ types,
                                                  const DevModule* __restrict__ mods,
                                                  const DevSub* __restrict__ subs, const double* __restrict__ mem,
                                                  const double* __restrict__ Xb, double* __restrict__ Cb) {
  const DevSub S = subs[blockIdx.x];
  const DevType T = types[S.type];
  const int nc = T.n_c, nb = T.n_b;
  const double* F = mem + mods[S.module].Frc;    // [nb x nc] row-major
  const double* x = Xb + S.b_off;
  double acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    const double xv = x[k];
    const double* fr = F + (int64_t)k * nc;
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (c < nc) acc[c] = fma(fr[c], xv, acc[c]);
  }
  __shared__ double red[NC][4];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if ((int)threadIdx.x < nc)
    Cb[S.c_off + threadIdx.x] = (red[threadIdx.x][0] + red[threadIdx.x][1]) + (red[threadIdx.x][2] + red[threadIdx.x][3]);
}

// Vraw[g + j*np] = sum over the corner copies of g of Cb[src + j*nct]
__global__ void k_corner_gather(int np, int m, const int* __restrict__ poff, const int* __restrict__ psrc,
                                const double* __restrict__ Cb, int64_t nct, double* __restrict__ V) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (g >= np || j >= m) return;
  double v = 0.0;
  for (int a = poff[g]; a < poff[g + 1]; ++a) v += Cb[psrc[a] + (int64_t)j * nct];
  V[g + (int64_t)j * np] = v;
}

// Vc[k + j*nct] = V[c_glob[k] + j*np]
__global__ void k_corner_spread(int64_t nct, int m, const int* __restrict__ cg, const double* __restrict__ V,
                                int np, double* __restrict__ Vc) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (k >= nct || j >= m) return;
  Vc[k + (int64_t)j * nct] = V[cg[k] + (int64_t)j * np];
}

}  // namespace

cudaError_t gather_lam_to_b(const Ctx& c, const double* X, int64_t ldx, int m, double* Xb, cudaStream_t st) {
  const int64_t nbt = c.hp.n_b_total;
  dim3 g((unsigned)((nbt + 255) / 256), m);
  k_gather<<<g, 256, 0, st>>>(nbt, m, c.d_b2l_off, c.d_b2l_lam, c.d_b2l_sign, X, ldx, Xb);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t scatter_b_to_lam(const Ctx& c, const double* Yb, int m, double* Y, int64_t ldy, cudaStream_t st) {
  const int64_t nl = c.hp.n_lam;
  dim3 g((unsigned)((nl + 255) / 256), (m + SC_J - 1) / SC_J);
  k_scatter<double><<<g, 256, 0, st>>>(nl, m, c.d_lam_b0, c.d_lam_s0, c.d_lam_b1, c.d_lam_s1, Yb, c.hp.n_b_total, Y,
                                       ldy);
  note_launches(1);
  return cudaGetLastError();
}

namespace {

// Y[l, j] = sum of the signed FP32 interface entries of row l, summed in FP32
// and widened exactly on the integer pipe (the reduced-precision operator's
// scatter; FP64 arithmetic here would bind it to the small FP64 unit).
__global__ void k_scatter32(int64_t nl, int m, const int* __restrict__ b0, const signed char* __restrict__ s0,
                            const int* __restrict__ b1, const signed char* __restrict__ s1,
                            const float* __restrict__ Yb, int64_t nbt, double* __restrict__ Y, int64_t ldy) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= nl) return;
  const int p0 = b0[l], p1 = b1[l];
  const bool n0 = s0[l] < 0, n1 = p1 >= 0 && s1[l] < 0;
  // SC_Z directions per block in groups of SC_J (few, long-lived blocks)
  const int jend = min(m, (int)(blockIdx.y + 1) * SC_Z);
  for (int j0 = blockIdx.y * SC_Z; j0 < jend; j0 += SC_J) {
    const int jn = min(SC_J, m - j0);
#pragma unroll
    for (int u = 0; u < SC_J; ++u) {
      if (u >= jn) break;
      const float* yb = Yb + (int64_t)(j0 + u) * nbt;
      const float a = yb[p0];
      float v = n0 ? -a : a;
      if (p1 >= 0) {
        const float c = yb[p1];
        v += n1 ? -c : c;
      }
      Y[l + (int64_t)(j0 + u) * ldy] = f32_to_f64(v);
    }
  }
}

}  // namespace

// Same, from an FP32 interface-space block (the tensor-core product's output).
cudaError_t scatter_b_to_lam32(const Ctx& c, const float* Yb, int m, double* Y, int64_t ldy, cudaStream_t st) {
  const int64_t nl = c.hp.n_lam;
  dim3 g((unsigned)((nl + 255) / 256), (m + SC_Z - 1) / SC_Z);
  k_scatter32<<<g, 256, 0, st>>>(nl, m, c.d_lam_b0, c.d_lam_s0, c.d_lam_b1, c.d_lam_s1, Yb, c.hp.n_b_total, Y, ldy);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t apply_local_F(Ctx& c, const double* /*Xb*/, double* /*Yb*/, int m, double beta, cudaStream_t st) {
  // descriptors point at c.d_Xb / c.d_Yb (fixed buffers); a batch's column
  // chunk may cap each subdomain's N at its own problem's directions
  if (c.gemm_F_active) return dgemm_batched(c.gemm_F_active, c.hp.n_sub, c.max_nb, m, 0, 1.0, beta, st, c.fl_F * m);
  return dgemm_batched(c.d_gemm_F, c.hp.n_sub, c.max_nb, c.max_nb, m, 1.0, beta, st, c.fl_F * m);
}

cudaError_t corner_reduce(Ctx& c, const double* /*Xb*/, int m, double* /*Cb*/, double* Vraw, cudaStream_t st) {
  cudaError_t e;
  if (m == 1 && c.max_nc <= 24) {
    if (c.max_nc <= 8) k_frct_one<8><<<c.hp.n_sub, 128, 0, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_modmem, c.d_Xb, c.d_Cb);
    else k_frct_one<24><<<c.hp.n_sub, 128, 0, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_modmem, c.d_Xb, c.d_Cb);
    note_launches(1);
    e = cudaGetLastError();
  } else if (c.max_nc <= 8) {
    k_frct<8><<<dim3((m + 63) / 64, c.hp.n_sub), 64, 0, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_modmem, c.d_Xb,
                                                             c.hp.n_b_total, m, c.d_Cb, c.n_c_total);
    note_launches(1);
    e = cudaGetLastError();
  } else if (c.max_nc <= 24) {
    k_frct<24><<<dim3((m + 63) / 64, c.hp.n_sub), 64, 0, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_modmem, c.d_Xb,
                                                              c.hp.n_b_total, m, c.d_Cb, c.n_c_total);
    note_launches(1);
    e = cudaGetLastError();
  } else {
    e = dgemm_batched(c.d_gemm_FrcT, c.hp.n_sub, c.max_nc, c.max_nb, m, 1.0, 0.0, st, c.fl_FrcT * m);
  }
  if (e != cudaSuccess) return e;
  return corner_assemble(c, m, Vraw, st);
}

// Vraw[g, j] = sum of Cb over the corner copies of primal DOF g.
cudaError_t corner_assemble(const Ctx& c, int m, double* Vraw, cudaStream_t st) {
  const int np = c.hp.n_primal;
  dim3 g((np + 127) / 128, m);
  k_corner_gather<<<g, 128, 0, st>>>(np, m, c.d_prim_off, c.d_prim_src, c.d_Cb, c.n_c_total, Vraw);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t corner_gather_vec(const Ctx& c, const double* src, double* out, cudaStream_t st) {
  const int np = c.hp.n_primal;
  k_corner_gather<<<(np + 127) / 128, 128, 0, st>>>(np, 1, c.d_prim_off, c.d_prim_src, src,
                                                    std::max<int64_t>(c.n_c_total, 1), out);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t corner_expand(Ctx& c, const double* V, int m, double* Vc, double* /*Yb*/, cudaStream_t st) {
  const int64_t nct = c.n_c_total;
  dim3 g((unsigned)((nct + 255) / 256), m);
  k_corner_spread<<<g, 256, 0, st>>>(nct, m, c.d_c_glob, V, c.hp.n_primal, Vc);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return dgemm_batched(c.d_gemm_Frc, c.hp.n_sub, c.max_nb, c.max_nb, m, 1.0, 1.0, st, c.fl_Frc * m);
}

namespace {

// Vector-load variant of k_sub_gemv (two doubles per lane per load); needs an
// even row length, which every 2D interface has (2 DOF per node).
__global__ void k_sub_gemv2(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                            const DevSub* __restrict__ subs, const double* __restrict__ mem, int which,
                            const double* __restrict__ x, double* __restrict__ y, double beta) {
  const DevSub S = subs[blockIdx.y];
  const DevType T = types[S.type];
  const DevModule M = mods[S.module];
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  const int n = T.n_b;
  if (row >= n) return;
  // which: 0 F_s, 1 S_s (b-b block of the n_bc-wide Schur complement), 2 K_bb (lumped)
  const double* A = mem + (which == 0 ? M.F : which == 1 ? M.S : M.Kl);
  const int64_t ld = which == 1 ? (int64_t)(T.n_b + T.n_c) : n;
  const double* a = A + (int64_t)row * ld;
  const double* xs = x + S.b_off;
  double acc = 0.0;
  if ((n & 1) == 0 && (ld & 1) == 0 && (S.b_off & 1) == 0) {
    const double2* a2 = reinterpret_cast<const double2*>(a);
    const double2* x2 = reinterpret_cast<const double2*>(xs);
    for (int k = lane; k < n / 2; k += 32) {
      const double2 av = a2[k], xv = x2[k];
      acc = fma(av.x, xv.x, acc);
      acc = fma(av.y, xv.y, acc);
    }
  } else {
    for (int k = lane; k < n; k += 32) acc = fma(a[k], xs[k], acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    double* yp = y + S.b_off + row;
    *yp = beta != 0.0 ? fma(beta, *yp, acc) : acc;
  }
}

}  // namespace

// config = warps per CTA (4, 8 or 16) + 100 * (vector loads)
static cudaError_t launch_gemv_cfg(const Ctx& c, int cfg, int which, const double* xb, double* yb, double beta,
                                   cudaStream_t st) {
  const int warps = cfg % 100, vec = cfg / 100;
  dim3 g((c.max_nb + warps - 1) / warps, c.hp.n_sub);
  if (vec) k_sub_gemv2<<<g, warps * 32, 0, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_modmem, which, xb, yb, beta);
  else k_sub_gemv<<<g, warps * 32, 0, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_modmem, which, xb, yb, beta);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t batched_gemv(const Ctx& c, int which, const double* xb, double* yb, double beta, cudaStream_t st) {
  return launch_gemv_cfg(c, c.gemv_cfg > 0 ? c.gemv_cfg : 8, which, xb, yb, beta, st);
}

// Autotuner: time every launch shape of the per-subdomain matrix-vector
// product on this problem (CUDA events, median of 5) and keep the fastest.
cudaError_t autotune_gemv(Ctx& c, cudaStream_t st) {
  const int cands[6] = {4, 8, 16, 104, 108, 116};
  cudaEvent_t e0, e1;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) return e;
  float best = 1e30f;
  int best_cfg = 8;
  for (int ci = 0; ci < 6 && e == cudaSuccess; ++ci) {
    float ts[5];
    for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
      cudaEventRecord(e0, st);
      e = launch_gemv_cfg(c, cands[ci], 0, c.d_pb0, c.d_pb1, 0.0, st);
      cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ts[r], e0, e1);
    }
    if (e != cudaSuccess) break;
    std::sort(ts, ts + 5);
    if (ts[2] < best) { best = ts[2]; best_cfg = cands[ci]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) {
    c.gemv_cfg = best_cfg;
    c.gemv_ms = best;
  }
  return e;
}

cudaError_t batched_gemv_F(Ctx& c, const double* xb, double* yb, cudaStream_t st) {
  return batched_gemv(c, 0, xb, yb, 0.0, st);
}

namespace {

// zb = diag(K_bb) rb: the super-lumped local block (diagonal stiffness of each
// interface copy, also the k-scaling weight source).
__global__ void k_diag_mul(int64_t n, const double* __restrict__ d, const double* __restrict__ x,
                           double* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = d[i] * x[i];
}

}  // namespace

// zb = P_s rb per subdomain with the configured local block (Dirichlet S_s,
// lumped K_bb or super-lumped diag K_bb).
static cudaError_t local_precond_block(const Ctx& c, const double* rb, double* zb, cudaStream_t st) {
  if (c.opt.precond == FETI_PRECOND_SUPERLUMPED) {
    const int64_t nbt = c.hp.n_b_total;
    k_diag_mul<<<(unsigned)((nbt + 255) / 256), 256, 0, st>>>(nbt, c.d_diagKb, rb, zb);
    note_launches(1);
    return cudaGetLastError();
  }
  return batched_gemv(c, c.opt.precond == FETI_PRECOND_LUMPED ? 2 : 1, rb, zb, 0.0, st);
}

cudaError_t precond_apply(Ctx& c, const double* r, double* Z, int64_t ldz, double* z, cudaStream_t st) {
  return precond_apply_cols(c, r, Z, ldz, c.hp.n_sub, c.d_b_sub, z, st);
}

// The block preconditioner in the work vectors rb, zb ([n_b_total] each, fully
// overwritten): column bcol[b] of Z for the b-space entry b (the subdomain, or
// its index inside its problem for a batch), ncols columns of Z cleared first.
static cudaError_t precond_core(const Ctx& c, const double* r, double* Z, int64_t ldz, int ncols, const int* bcol,
                                double* z, double* rb, double* zb, cudaStream_t st) {
  const int64_t nbt = c.hp.n_b_total, nl = c.hp.n_lam;
  k_gather_weighted<<<(unsigned)((nbt + 255) / 256), 256, 0, st>>>(nbt, c.d_b2l_off, c.d_b2l_lam, c.d_b2l_sign,
                                                                   c.d_lam_b0, c.d_w0, c.d_w1, r, rb);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = local_precond_block(c, rb, zb, st);
  if (e != cudaSuccess) return e;
  if (Z) {
    e = cudaMemsetAsync(Z, 0, sizeof(double) * (size_t)ldz * ncols, st);
    if (e != cudaSuccess) return e;
  }
  k_prec_scatter<<<(unsigned)((nl + 255) / 256), 256, 0, st>>>(nl, c.d_lam_b0, c.d_lam_s0, c.d_lam_b1, c.d_lam_s1,
                                                               c.d_w0, c.d_w1, bcol, zb, Z, ldz, z);
  note_launches(1);
  return cudaGetLastError();
}

// The block preconditioner in the context's own work vectors.
cudaError_t precond_apply_cols(Ctx& c, const double* r, double* Z, int64_t ldz, int ncols, const int* bcol,
                               double* z, cudaStream_t st) {
  return precond_core(c, r, Z, ldz, ncols, bcol, z, c.d_pb0, c.d_pb1, st);
}

// The block preconditioner (one column per subdomain) with caller-provided
// work vectors rb, zb; used by the allocation-free entry point.
cudaError_t precond_apply_scratch(const Ctx& c, const double* r, double* Z, int64_t ldz, double* z, double* rb,
                                  double* zb, cudaStream_t st) {
  return precond_core(c, r, Z, ldz, c.hp.n_sub, c.d_b_sub, z, rb, zb, st);
}

namespace {

// Yb[b_off(s) + k + j*nbt] += sum_c F_rc,s(k, c) V[c_glob(s, c) + j*np]; one
// thread per interface row, 32 columns per thread.
__global__ void k_frc_expand(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                             const DevSub* __restrict__ subs, const double* __restrict__ mem,
                             const int* __restrict__ cg, const double* __restrict__ V, int np, int m,
                             double* __restrict__ Yb, int64_t nbt) {
  const DevSub S = subs[blockIdx.y];
  const DevType T = types[S.type];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= T.n_b) return;
  const int nc = T.n_c;
  if (nc == 0) return;
  const double* fr = mem + mods[S.module].Frc + (int64_t)k * nc;
  double f[24];
  int g[24];
  for (int c = 0; c < nc && c < 24; ++c) { f[c] = fr[c]; g[c] = cg[S.c_off + c]; }
  const int j0 = blockIdx.z * 32, j1 = min(m, j0 + 32);
  for (int j = j0; j < j1; ++j) {
    double acc = 0.0;
    for (int c = 0; c < nc && c < 24; ++c) acc = fma(f[c], V[g[c] + (int64_t)j * np], acc);
    Yb[S.b_off + k + (int64_t)j * nbt] += acc;
  }
}

}  // namespace

cudaError_t corner_expand_thin(Ctx& c, const double* V, int m, double* Yb, cudaStream_t st) {
  if (c.max_nc > 24) return corner_expand(c, V, m, c.d_Vc, Yb, st);
  dim3 g((c.max_nb + 127) / 128, c.hp.n_sub, (m + 31) / 32);
  k_frc_expand<<<g, 128, 0, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_modmem, c.d_c_glob, V, c.hp.n_primal, m, Yb,
                                  c.hp.n_b_total);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t precond_apply_lowp(Ctx& c, const double* r, double* Z, int64_t ldz, double* z, cudaStream_t st) {
  // the reduced-precision copy exists for the Dirichlet block only; the lumped
  // blocks are cheap enough in FP64
  if (c.opt.precond != FETI_PRECOND_DIRICHLET) return precond_apply(c, r, Z, ldz, z, st);
  const int64_t nbt = c.hp.n_b_total, nl = c.hp.n_lam;
  double* rb = c.d_pb0;
  double* zb = c.d_pb1;
  k_gather_weighted<<<(unsigned)((nbt + 255) / 256), 256, 0, st>>>(nbt, c.d_b2l_off, c.d_b2l_lam, c.d_b2l_sign,
                                                                   c.d_lam_b0, c.d_w0, c.d_w1, r, rb);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = lowp_gemv_S(c, rb, c.d_pbh, zb, st);
  if (e != cudaSuccess) return e;
  if (Z) {
    e = cudaMemsetAsync(Z, 0, sizeof(double) * (size_t)ldz * c.hp.n_sub, st);
    if (e != cudaSuccess) return e;
  }
  k_prec_scatter<<<(unsigned)((nl + 255) / 256), 256, 0, st>>>(nl, c.d_lam_b0, c.d_lam_s0, c.d_lam_b1, c.d_lam_s1,
                                                               c.d_w0, c.d_w1, c.d_b_sub, zb, Z, ldz, z);
  note_launches(1);
  return cudaGetLastError();
}

namespace {

// y[r] = sum_k Kinv_p(r - off_p, k) x[off_p + k], p = problem of primal row r
// (the coarse inverse is block diagonal over the problems of a batch); one
// warp per row.
__global__ void k_coarse_gemv(int np_total, const int* __restrict__ row_prob, const int* __restrict__ poff,
                              const int64_t* __restrict__ koff, const double* __restrict__ Kinv,
                              const double* __restrict__ x, double* __restrict__ y) {
  const int r = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (r >= np_total) return;
  const int p = row_prob[r];
  const int o = poff[p], n = poff[p + 1] - o;
  const double* a = Kinv + koff[p] + (int64_t)(r - o) * n;
  const double* xs = x + o;
  double acc = 0.0;
  for (int k = lane; k < n; k += 32) acc = fma(a[k], xs[k], acc);
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) y[r] = acc;
}

// Kbar_p = sum over the problem's subdomains of B_c^sT Kbar_s B_c^s (gather
// over corner copies); grid.y = problem.
__global__ void k_coarse_assemble_batch(const int* __restrict__ ppoff, const int64_t* __restrict__ koff,
                                        const int* __restrict__ poff, const int* __restrict__ psrc,
                                        const int* __restrict__ c_sub, const DevSub* __restrict__ subs,
                                        const DevModule* __restrict__ mods, const DevType* __restrict__ types,
                                        const double* __restrict__ mem, double* __restrict__ K) {
  const int p = blockIdx.y;
  const int o = ppoff[p], n = ppoff[p + 1] - o;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int g1 = o + (int)(e / n), g2 = o + (int)(e % n);
  double v = 0.0;
  for (int a = poff[g1]; a < poff[g1 + 1]; ++a) {
    const int s = c_sub[psrc[a]];
    const DevSub S = subs[s];
    const int k1 = psrc[a] - (int)S.c_off;
    for (int b = poff[g2]; b < poff[g2 + 1]; ++b) {
      if (c_sub[psrc[b]] != s) continue;
      const int k2 = psrc[b] - (int)S.c_off;
      const int nc = types[S.type].n_c;
      v += mem[mods[S.module].Kb + (int64_t)k1 * nc + k2];
    }
  }
  K[koff[p] + e] = v;
}

}  // namespace

cudaError_t coarse_assemble_batch(const Ctx& c, cudaStream_t st) {
  dim3 g((unsigned)(((int64_t)c.max_np * c.max_np + 255) / 256), c.hp.n_prob);
  k_coarse_assemble_batch<<<g, 256, 0, st>>>(c.d_prob_primal_off, c.d_kbar_off, c.d_prim_off, c.d_prim_src,
                                             c.d_c_sub, c.d_subs, c.d_mods, c.d_types, c.d_modmem, c.d_Kbar);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t coarse_matvec(const Ctx& c, const double* x, double* y, cudaStream_t st) {
  const int np = c.hp.n_primal;
  k_coarse_gemv<<<(np + 7) / 8, 256, 0, st>>>(np, c.d_row_prob, c.d_prob_primal_off, c.d_kbar_off, c.d_Kbar_inv, x,
                                              y);
  note_launches(1);
  return cudaGetLastError();
}

// V = Kbar^{-1} Vraw for m columns (block diagonal over a batch's problems)
cudaError_t coarse_apply(const Ctx& c, const double* Vraw, double* V, int m, cudaStream_t st) {
  const int np = c.hp.n_primal;
  if (m == 1) return coarse_matvec(c, Vraw, V, st);
  if (c.hp.n_prob == 1) {
    GemmDesc d{};
    d.A = c.d_Kbar_inv; d.B = Vraw; d.C = V; d.M = np; d.N = m; d.K = np;
    d.ars = np; d.acs = 1; d.brs = 1; d.bcs = np; d.crs = 1; d.ccs = np;
    return dgemm_split(d, 1, nullptr, 1.0, 0.0, st);
  }
  return dgemm_batched(c.d_gemm_coarse, c.hp.n_prob, c.max_np, m, m, 1.0, 0.0, st);
}

}  // namespace feti
