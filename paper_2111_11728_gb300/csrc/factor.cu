// Factorization kernels, all FP64 (GB300's FP64 pipe sets their speed).
//
// Per module (one distinct subdomain matrix):
//   K_ii = L L^T            banded Cholesky, one CTA per module
//   Y    = L^{-1} K_{i,bc}  banded forward substitution, one thread per column
//   S    = K_{bc,bc} - Y^T Y  (Schur complement onto interface + corners)
//   F    = S_bb^{-1}        dense Cholesky, triangular inverse, L^{-T} L^{-1}
// FETI-DP additionally forms F_rc = F S_bc and the local coarse block
// Kbar_s = S_cc - S_cb F_rc (Eq. 12); the global Kbar_cc is assembled by a
// gather over the corner copies (deterministic) and inverted the same way.
#include <algorithm>
#include <vector>

#include "kernels.h"

namespace feti {

namespace {

constexpr int NT = 256;

// Right-looking banded Cholesky in the column band (Lcol[j*W + t] = L(j+t, j)).
__global__ void __launch_bounds__(NT) k_band_chol(const DevType* __restrict__ types,
                                                  const DevModule* __restrict__ mods, double* __restrict__ mem,
                                                  int* __restrict__ status) {
  const DevModule M = mods[blockIdx.x];
  const DevType T = types[M.type];
  const int n = T.n_i, bw = T.bw, W = bw + 1;
  double* L = mem + M.lcol;
  extern __shared__ double col[];
  const int tid = threadIdx.x;
  for (int j = 0; j < n; ++j) {
    const int len = min(bw, n - 1 - j);
    const double piv = L[(int64_t)j * W];
    __syncthreads();   // every thread holds the pivot before column j is overwritten
    if (!(piv > 0.0)) {
      if (tid == 0) atomicCAS(status, 0, 1000000 + blockIdx.x);
      return;
    }
    const double dj = sqrt(piv);
    const double rd = 1.0 / dj;
    for (int t = tid; t <= len; t += NT) {
      const double v = t == 0 ? dj : L[(int64_t)j * W + t] * rd;
      col[t] = v;
      L[(int64_t)j * W + t] = v;
    }
    __syncthreads();
    for (int e = tid; e < len * len; e += NT) {
      const int a = e / len + 1, b = e % len + 1;
      if (b >= a) L[(int64_t)(j + a) * W + (b - a)] = fma(-col[a], col[b], L[(int64_t)(j + a) * W + (b - a)]);
    }
    __syncthreads();
  }
}

// Row band copy Lrow[j*W + d] = L(j, j-d) and reciprocal diagonal.
__global__ void k_band_rows(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                            double* __restrict__ mem) {
  const DevModule M = mods[blockIdx.y];
  const DevType T = types[M.type];
  const int W = T.bw + 1;
  const int64_t total = (int64_t)T.n_i * W;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / W), d = (int)(e % W);
    mem[M.lrow + e] = d <= j ? mem[M.lcol + (int64_t)(j - d) * W + d] : 0.0;
    if (d == 0) mem[M.rdiag + j] = 1.0 / mem[M.lcol + (int64_t)j * W];
  }
}

// Y = L^{-1} Y for the n_bc right-hand sides of one module; each thread
// marches down one column keeping the last bw values in shared memory.
__global__ void k_band_fwd_multi(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                                 double* __restrict__ mem) {
  const DevModule M = mods[blockIdx.y];
  const DevType T = types[M.type];
  const int nbc = T.n_b + T.n_c;
  const int col = blockIdx.x * 64 + threadIdx.x;
  if (col >= nbc) return;
  const int n = T.n_i, bw = T.bw, W = bw + 1;
  extern __shared__ double win[];   // [W][64]
  const double* __restrict__ Lr = mem + M.lrow;
  const double* __restrict__ rd = mem + M.rdiag;
  double* __restrict__ Y = mem + M.Y;
  const int tc = threadIdx.x;
  int slot = 0;
  for (int j = 0; j < n; ++j) {
    double acc0 = Y[(int64_t)j * nbc + col], acc1 = 0.0;
    const double* lr = Lr + (int64_t)j * W;
    const int dmax = min(j, bw);
    int sl = slot;
    int d = 1;
    for (; d + 1 <= dmax; d += 2) {
      sl = sl == 0 ? W - 1 : sl - 1;
      acc0 = fma(-lr[d], win[sl * 64 + tc], acc0);
      sl = sl == 0 ? W - 1 : sl - 1;
      acc1 = fma(-lr[d + 1], win[sl * 64 + tc], acc1);
    }
    if (d <= dmax) {
      sl = sl == 0 ? W - 1 : sl - 1;
      acc0 = fma(-lr[d], win[sl * 64 + tc], acc0);
    }
    const double y = (acc0 + acc1) * rd[j];
    win[slot * 64 + tc] = y;
    Y[(int64_t)j * nbc + col] = y;
    slot = slot + 1 == W ? 0 : slot + 1;
  }
}

// Dense Cholesky (lower, in place, row-major with ld), one CTA per matrix.
__global__ void __launch_bounds__(NT) k_dense_chol(const DenseDesc* __restrict__ descs, int* __restrict__ status) {
  const DenseDesc D = descs[blockIdx.x];
  const int n = D.n, ld = D.ld;
  const int nf = D.n_full > n ? D.n_full : n;
  double* A = D.A;
  extern __shared__ double col[];
  const int tid = threadIdx.x;
  for (int j = 0; j < n; ++j) {
    const int len = nf - 1 - j;
    const double piv = A[(int64_t)j * ld + j];
    __syncthreads();   // every thread holds the pivot before column j is overwritten
    if (!(piv > 0.0)) {
      if (tid == 0) atomicCAS(status, 0, 2000000 + D.tag);
      return;
    }
    const double dj = sqrt(piv), rd = 1.0 / dj;
    for (int t = tid; t <= len; t += NT) {
      const double v = t == 0 ? dj : A[(int64_t)(j + t) * ld + j] * rd;
      col[t] = v;
      A[(int64_t)(j + t) * ld + j] = v;
    }
    __syncthreads();
    // lower triangle of the trailing block, row by row
    for (int a = 1 + tid / 32; a <= len; a += NT / 32) {
      const double ca = col[a];
      double* row = A + (int64_t)(j + a) * ld + j;
      for (int b = 1 + (tid & 31); b <= a; b += 32) row[b] = fma(-ca, col[b], row[b]);
    }
    __syncthreads();
  }
}

// Linv = L^{-1} (row-major, zero above the diagonal); one thread per column.
__global__ void k_tri_inv(const DenseDesc* __restrict__ descs) {
  const DenseDesc D = descs[blockIdx.y];
  const int n = D.n, ld = D.ld;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double* L = D.A;
  double* X = D.Linv;
  for (int i = 0; i < j; ++i) X[(int64_t)i * n + j] = 0.0;
  X[(int64_t)j * n + j] = 1.0 / L[(int64_t)j * ld + j];
  for (int i = j + 1; i < n; ++i) {
    const double* Li = L + (int64_t)i * ld;
    double a0 = 0.0, a1 = 0.0;
    int k = j;
    for (; k + 1 < i; k += 2) {
      a0 = fma(Li[k], X[(int64_t)k * n + j], a0);
      a1 = fma(Li[k + 1], X[(int64_t)(k + 1) * n + j], a1);
    }
    if (k < i) a0 = fma(Li[k], X[(int64_t)k * n + j], a0);
    X[(int64_t)i * n + j] = -(a0 + a1) / Li[i];
  }
}

// out = Linv^T Linv, restricted to k >= max(i, j) (Linv is lower triangular).
__global__ void __launch_bounds__(256) k_lt_l(const DenseDesc* __restrict__ descs) {
  const DenseDesc D = descs[blockIdx.z];
  const int n = D.n;
  const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16;
  if (i0 >= n || j0 >= n) return;
  const int ti = threadIdx.x / 16, tj = threadIdx.x % 16;
  const int i = i0 + ti, j = j0 + tj;
  __shared__ double As[16][17], Bs[16][17];
  double acc = 0.0;
  const int kstart = max(i0, j0) / 16 * 16;
  for (int k0 = kstart; k0 < n; k0 += 16) {
    // As[kk][ti] = Linv(k0+kk, i0+ti); Bs[kk][tj] = Linv(k0+kk, j0+tj)
    const int kk = threadIdx.x / 16, cc = threadIdx.x % 16;
    const int kr = k0 + kk;
    As[kk][cc] = (kr < n && i0 + cc < n) ? D.Linv[(int64_t)kr * n + i0 + cc] : 0.0;
    Bs[kk][cc] = (kr < n && j0 + cc < n) ? D.Linv[(int64_t)kr * n + j0 + cc] : 0.0;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 16; ++t) acc = fma(As[t][ti], Bs[t][tj], acc);
    __syncthreads();
  }
  if (i < n && j < n) D.out[(int64_t)i * n + j] = acc;
}

// Kbar_cc = sum over subdomains of B_c^sT Kbar_s B_c^s, as a gather over the
// corner copies shared by each pair of primal DOFs.
__global__ void k_coarse_assemble(int np, const int* __restrict__ poff, const int* __restrict__ psrc,
                                  const int* __restrict__ c_sub, const int64_t* __restrict__ c_off_sub,
                                  const DevSub* __restrict__ subs, const DevModule* __restrict__ mods,
                                  const DevType* __restrict__ types, const double* __restrict__ mem,
                                  double* __restrict__ K) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)np * np) return;
  const int g1 = (int)(e / np), g2 = (int)(e % np);
  double v = 0.0;
  for (int a = poff[g1]; a < poff[g1 + 1]; ++a) {
    const int s = c_sub[psrc[a]];
    const int k1 = psrc[a] - (int)c_off_sub[s];
    for (int b = poff[g2]; b < poff[g2 + 1]; ++b) {
      if (c_sub[psrc[b]] != s) continue;
      const int k2 = psrc[b] - (int)c_off_sub[s];
      const DevSub S = subs[s];
      const int nc = types[S.type].n_c;
      v += mem[mods[S.module].Kb + (int64_t)k1 * nc + k2];
    }
  }
  K[e] = v;
}

// h_s = L^{-1} f_i,s: one warp per subdomain, lane-parallel band dot products.
__global__ void k_band_fwd_single(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                                  const DevSub* __restrict__ subs, const double* __restrict__ mem,
                                  const double* __restrict__ floc, int nld, const int64_t* __restrict__ ioff,
                                  double* __restrict__ h, int n_sub) {
  const int s = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (s >= n_sub) return;
  const int lane = threadIdx.x & 31;
  const DevSub S = subs[s];
  const DevModule M = mods[S.module];
  const DevType T = types[S.type];
  const int n = T.n_i, bw = T.bw, W = bw + 1;
  const double* Lr = mem + M.lrow;
  const double* rd = mem + M.rdiag;
  double* hs = h + ioff[s];
  const double* fs = floc + (int64_t)s * nld;
  for (int j = 0; j < n; ++j) {
    const double* lr = Lr + (int64_t)j * W;
    const int dmax = min(j, bw);
    double acc = 0.0;
    for (int d = 1 + lane; d <= dmax; d += 32) acc = fma(lr[d], hs[j - d], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) hs[j] = (fs[T.ilist[j]] - acc) * rd[j];
    __syncwarp();
  }
}

// f~_bc = f_bc - Y^T h per subdomain (b part into ft[b_off], c part into ft[nbt + c_off]).
__global__ void k_condense_load(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                                const DevSub* __restrict__ subs, const double* __restrict__ mem,
                                const double* __restrict__ floc, int nld, const int64_t* __restrict__ ioff,
                                const double* __restrict__ h, int64_t nbt, double* __restrict__ ft) {
  const DevSub S = subs[blockIdx.y];
  const DevModule M = mods[S.module];
  const DevType T = types[S.type];
  const int nbc = T.n_b + T.n_c;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nbc) return;
  const double* Y = mem + M.Y;
  const double* hs = h + ioff[blockIdx.y];
  double acc = 0.0;
  for (int k = 0; k < T.n_i; ++k) acc = fma(Y[(int64_t)k * nbc + j], hs[k], acc);
  const int ld = j < T.n_b ? T.blist[j] : T.clist[j - T.n_b];
  const double v = floc[(int64_t)blockIdx.y * nld + ld] - acc;
  if (j < T.n_b) ft[S.b_off + j] = v;
  else ft[nbt + S.c_off + (j - T.n_b)] = v;
}

// which 0: W = S (n_bc x n_bc); which 1: Kb = trailing n_c x n_c block of the
// partially factorised W (its lower triangle, mirrored).
__global__ void k_copy_block(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                             double* __restrict__ mem, int which) {
  const DevModule M = mods[blockIdx.y];
  const DevType T = types[M.type];
  const int nb = T.n_b, nc = T.n_c, nbc = nb + nc;
  const int n = which == 0 ? nbc : nc;
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / n), q = (int)(e % n);
    if (which == 0) {
      mem[M.W + e] = mem[M.S + e];
    } else {
      const int hi = r > q ? r : q, lo = r > q ? q : r;
      mem[M.Kb + e] = mem[M.W + (int64_t)(nb + hi) * nbc + nb + lo];
    }
  }
}

}  // namespace

cudaError_t launch_band_chol(const Ctx& c, cudaStream_t st) {
  int maxbw = 1;
  for (auto& t : c.h_types) maxbw = std::max(maxbw, t.bw);
  size_t sm = (size_t)(maxbw + 1) * sizeof(double);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_band_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_band_chol<<<c.n_mod, NT, sm, st>>>(c.d_types, c.d_mods, c.d_modmem, c.d_status);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_band_rows<<<dim3(64, c.n_mod), 256, 0, st>>>(c.d_types, c.d_mods, c.d_modmem);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_band_fwd_multi(const Ctx& c, cudaStream_t st) {
  int maxbw = 1, maxbc = 1;
  for (auto& t : c.h_types) { maxbw = std::max(maxbw, t.bw); maxbc = std::max(maxbc, t.n_b + t.n_c); }
  size_t sm = (size_t)(maxbw + 1) * 64 * sizeof(double);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_band_fwd_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  k_band_fwd_multi<<<dim3((maxbc + 63) / 64, c.n_mod), 64, sm, st>>>(c.d_types, c.d_mods, c.d_modmem);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_copy_block(const Ctx& c, int which, cudaStream_t st) {
  k_copy_block<<<dim3(64, c.n_mod), 256, 0, st>>>(c.d_types, c.d_mods, c.d_modmem, which);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t dense_spd_inverse(const DenseDesc* d_desc, const DenseDesc* h_desc, int count, int* d_status,
                              cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int maxn = 1, maxf = 1;
  for (int i = 0; i < count; ++i) {
    maxn = std::max(maxn, h_desc[i].n);
    maxf = std::max(maxf, std::max(h_desc[i].n, h_desc[i].n_full));
  }
  size_t sm = (size_t)(maxf + 1) * sizeof(double);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_dense_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_dense_chol<<<count, NT, sm, st>>>(d_desc, d_status);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_tri_inv<<<dim3((maxn + 63) / 64, count), 64, 0, st>>>(d_desc);
  note_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 g((maxn + 15) / 16, (maxn + 15) / 16, count);
  k_lt_l<<<g, 256, 0, st>>>(d_desc);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_coarse_assemble_impl(const Ctx& c, const int* d_c_sub, const int64_t* d_c_off, double* K,
                                        cudaStream_t st) {
  const int np = c.hp.n_primal;
  const int64_t tot = (int64_t)np * np;
  k_coarse_assemble<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(np, c.d_prim_off, c.d_prim_src, d_c_sub, d_c_off,
                                                                   c.d_subs, c.d_mods, c.d_types, c.d_modmem, K);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_band_fwd_single(const Ctx& c, cudaStream_t st) {
  const int ns = c.hp.n_sub;
  k_band_fwd_single<<<(ns + 3) / 4, 128, 0, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_modmem, c.d_floc,
                                                   c.hp.n_loc_dofs, c.d_ioff, c.d_h, ns);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_condense_load(const Ctx& c, cudaStream_t st) {
  int maxbc = 1;
  for (auto& t : c.h_types) maxbc = std::max(maxbc, t.n_b + t.n_c);
  k_condense_load<<<dim3((maxbc + 63) / 64, c.hp.n_sub), 64, 0, st>>>(
      c.d_types, c.d_mods, c.d_subs, c.d_modmem, c.d_floc, c.hp.n_loc_dofs, c.d_ioff, c.d_h, c.hp.n_b_total,
      c.d_ft);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace feti
