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

// Banded Cholesky in the column band (Lcol[j*W + t] = L(j+t, j)), blocked by
// panels of BC_PB columns.  Warp 0 factors a panel (each column first takes the
// panel's earlier columns, then its pivot); then all warps apply the panel's
// rank-BC_PB update to the band columns that follow it.  Every entry receives
// the updates of the columns before it in ascending column order, as in the
// unblocked right-looking elimination, so the factor is the same bit for bit;
// the block-wide barriers drop from three per column to two per panel.
constexpr int BC_PB = 8;

__global__ void __launch_bounds__(NT) k_band_chol(const DevType* __restrict__ types,
                                                  const DevModule* __restrict__ mods, double* __restrict__ mem,
                                                  int* __restrict__ status) {
  const DevModule M = mods[blockIdx.x];
  const DevType T = types[M.type];
  const int n = T.n_i, bw = T.bw, W = bw + 1;
  double* L = mem + M.lcol;
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) s_ok = 1;
  __syncthreads();
  for (int p0 = 0; p0 < n; p0 += BC_PB) {
    const int pw = min(BC_PB, n - p0);
    if (warp == 0) {
      for (int j = p0; j < p0 + pw; ++j) {
        const int len = min(bw, n - 1 - j);
        // updates from the panel's earlier columns k (ascending): L(j+t, j) -= L(j+t, k) L(j, k)
        for (int k = max(p0, j - bw); k < j; ++k) {   // L(j, k) = 0 outside the band
          const double ljk = L[(int64_t)k * W + (j - k)];
          for (int t = lane; t <= len; t += 32) {
            const int off = j + t - k;               // row j+t in column k
            if (off <= bw) L[(int64_t)j * W + t] = fma(-ljk, L[(int64_t)k * W + off], L[(int64_t)j * W + t]);
          }
          __syncwarp();
        }
        double dj = 0.0, rd = 0.0;
        int ok = 1;
        if (lane == 0) {
          const double piv = L[(int64_t)j * W];
          ok = piv > 0.0;
          if (ok) {
            dj = sqrt(piv);
            rd = 1.0 / dj;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          if (lane == 0) {
            s_ok = 0;
            atomicCAS(status, 0, 1000000 + blockIdx.x);
          }
          break;
        }
        dj = __shfl_sync(0xffffffffu, dj, 0);
        rd = __shfl_sync(0xffffffffu, rd, 0);
        for (int t = lane; t <= len; t += 32) L[(int64_t)j * W + t] = t == 0 ? dj : L[(int64_t)j * W + t] * rd;
        __syncwarp();
      }
    }
    __syncthreads();
    if (!s_ok) return;
    // rank-pw update of band columns l in [p0+pw, p0+pw-1+bw]: for i >= l,
    // L(i, l) -= sum_k L(i, k) L(l, k) over the panel columns k (ascending)
    const int c0 = p0 + pw, c1 = min(n - 1, p0 + pw - 1 + bw);
    for (int l = c0 + warp; l <= c1; l += NT / 32) {
      const int imax = min(c1, l + bw);
      for (int i = l + lane; i <= imax; i += 32) {
        double acc = L[(int64_t)l * W + (i - l)];
        for (int k = p0; k < p0 + pw; ++k) {
          if (i - k <= bw && l - k <= bw) acc = fma(-L[(int64_t)k * W + (l - k)], L[(int64_t)k * W + (i - k)], acc);
        }
        L[(int64_t)l * W + (i - l)] = acc;
      }
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
// marches down one column keeping the last bw values in shared memory.  One
// warp of FW_COLS columns per block, so that the few distinct modules still
// spread over every SM (the substitution is FP64-bound per SM).
constexpr int FW_COLS = 32;
__global__ void k_band_fwd_multi(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                                 double* __restrict__ mem) {
  const DevModule M = mods[blockIdx.y];
  const DevType T = types[M.type];
  const int nbc = T.n_b + T.n_c;
  const int col = blockIdx.x * FW_COLS + threadIdx.x;
  if (col >= nbc) return;
  const int n = T.n_i, bw = T.bw, W = bw + 1;
  extern __shared__ double win[];   // [W][FW_COLS]
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
      acc0 = fma(-lr[d], win[sl * FW_COLS + tc], acc0);
      sl = sl == 0 ? W - 1 : sl - 1;
      acc1 = fma(-lr[d + 1], win[sl * FW_COLS + tc], acc1);
    }
    if (d <= dmax) {
      sl = sl == 0 ? W - 1 : sl - 1;
      acc0 = fma(-lr[d], win[sl * FW_COLS + tc], acc0);
    }
    const double y = (acc0 + acc1) * rd[j];
    win[slot * FW_COLS + tc] = y;
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
  __shared__ double s_dj, s_rd;
  __shared__ int s_ok;
  const int tid = threadIdx.x;
  for (int j = 0; j < n; ++j) {
    const int len = nf - 1 - j;
    if (tid == 0) {                      // one thread: square root and reciprocal of the pivot
      const double piv = A[(int64_t)j * ld + j];
      s_ok = piv > 0.0;
      if (s_ok) {
        s_dj = sqrt(piv);
        s_rd = 1.0 / s_dj;
      }
    }
    __syncthreads();   // the pivot is read before column j is overwritten
    if (!s_ok) {
      if (tid == 0) atomicCAS(status, 0, 2000000 + D.tag);
      return;
    }
    const double dj = s_dj, rd = s_rd;
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
// A warp walks the rows of its 32 columns together, starting at its first
// column, so every load of Linv is one contiguous row segment (the entries
// above a column's diagonal are zero and add nothing).
__global__ void k_tri_inv(const DenseDesc* __restrict__ descs) {
  const DenseDesc D = descs[blockIdx.y];
  const int n = D.n, ld = D.ld;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int j0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31);
  if (j0 >= n) return;
  const bool act = j < n;
  const double* L = D.A;
  double* X = D.Linv;
  if (act) {
    for (int i = 0; i < j; ++i) X[(int64_t)i * n + j] = 0.0;
    X[(int64_t)j * n + j] = 1.0 / L[(int64_t)j * ld + j];
  }
  __syncwarp();
  for (int i = j0 + 1; i < n; ++i) {
    const double* Li = L + (int64_t)i * ld;
    double a0 = 0.0, a1 = 0.0;
    int k = j0;
    for (; k + 1 < i; k += 2) {
      a0 = fma(Li[k], act ? X[(int64_t)k * n + j] : 0.0, a0);
      a1 = fma(Li[k + 1], act ? X[(int64_t)(k + 1) * n + j] : 0.0, a1);
    }
    if (k < i) a0 = fma(Li[k], act ? X[(int64_t)k * n + j] : 0.0, a0);
    if (act && i > j) X[(int64_t)i * n + j] = -(a0 + a1) / Li[i];
    __syncwarp();
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
  const double* fs = floc + S.loc_off;
  (void)nld;
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
  const double v = floc[S.loc_off + ld] - acc;
  (void)nld;
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

// Diagonal block [c0, c0+nb) of a row-major n x n matrix: Cholesky in shared
// memory, written back (lower triangle), and its inverse into Dinv (nb x nb
// row-major, ld 64).  One CTA of 256 threads.
__global__ void __launch_bounds__(256) k_diag_block(double* __restrict__ A, int n, int c0, int nb,
                                                   double* __restrict__ Dinv, int* __restrict__ status, int tag) {
  __shared__ double S[64][65];
  __shared__ double X[64][65];
  const int tid = threadIdx.x;
  for (int e = tid; e < nb * nb; e += 256) {
    const int r = e / nb, q = e % nb;
    S[r][q] = A[(int64_t)(c0 + r) * n + c0 + q];
  }
  __syncthreads();
  __shared__ double s_dj, s_rd;
  __shared__ int s_ok;
  for (int j = 0; j < nb; ++j) {
    if (tid == 0) {                      // one thread: square root and reciprocal of the pivot
      const double piv = S[j][j];
      s_ok = piv > 0.0;
      if (s_ok) {
        s_dj = sqrt(piv);
        s_rd = 1.0 / s_dj;
      }
    }
    __syncthreads();
    if (!s_ok) {
      if (tid == 0) atomicCAS(status, 0, 2000000 + tag);
      return;
    }
    const double dj = s_dj, rd = s_rd;
    for (int t = j + tid; t < nb; t += 256) S[t][j] = t == j ? dj : S[t][j] * rd;
    __syncthreads();
    for (int e = tid; e < (nb - 1 - j) * (nb - 1 - j); e += 256) {
      const int a = j + 1 + e / (nb - 1 - j), b = j + 1 + e % (nb - 1 - j);
      if (b <= a) S[a][b] = fma(-S[a][j], S[b][j], S[a][b]);
    }
    __syncthreads();
  }
  // inverse of the lower-triangular block, one thread per column
  if (tid < nb) {
    const int c = tid;
    for (int i = 0; i < c; ++i) X[i][c] = 0.0;
    X[c][c] = 1.0 / S[c][c];
    for (int i = c + 1; i < nb; ++i) {
      double acc = 0.0;
      for (int k = c; k < i; ++k) acc = fma(S[i][k], X[k][c], acc);
      X[i][c] = -acc / S[i][i];
    }
  }
  __syncthreads();
  for (int e = tid; e < nb * nb; e += 256) {
    const int r = e / nb, q = e % nb;
    if (q <= r) A[(int64_t)(c0 + r) * n + c0 + q] = S[r][q];
    Dinv[r * 64 + q] = X[r][q];
  }
}

__global__ void k_copy_rows(const double* __restrict__ src, int64_t lds, double* __restrict__ dst, int64_t ldd,
                            int rows, int cols, double scale) {
  const int64_t total = (int64_t)rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / cols), q = (int)(e % cols);
    dst[r * ldd + q] = scale * src[r * lds + q];
  }
}

}  // namespace

// Blocked right-looking Cholesky of one SPD n x n row-major matrix A (full
// symmetric storage; on return its lower triangle holds L), then
// X = L^{-1} block row by block row, then out = X^T X = A^{-1}.  All large
// products go through the FP64 GEMM, so the whole GPU works on it.
// work: 64 * n * 2 + ceil(n/64) * 4096 doubles.
cudaError_t dense_spd_inverse_blocked(double* A, double* X, double* out, int n, double* work, int* status,
                                      const DenseDesc* d_desc_for_ltl, cudaStream_t st) {
  const int NB = 64;
  const int nbk = (n + NB - 1) / NB;
  double* Dinv = work;                       // nbk x 64 x 64
  double* R = work + (int64_t)nbk * 4096;    // 64 x n
  cudaError_t e;
  for (int kb = 0; kb < nbk; ++kb) {
    const int c0 = kb * NB, nb = std::min(NB, n - c0);
    k_diag_block<<<1, 256, 0, st>>>(A, n, c0, nb, Dinv + (int64_t)kb * 4096, status, 999999);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int r0 = c0 + nb, rest = n - r0;
    if (rest <= 0) break;
    // panel: L21 = A21 L11^{-T}   (in place: each CTA owns its 64 rows and all nb columns)
    GemmDesc p{};
    p.A = A + (int64_t)r0 * n + c0; p.B = Dinv + (int64_t)kb * 4096; p.C = A + (int64_t)r0 * n + c0;
    p.M = rest; p.N = nb; p.K = nb;
    p.ars = n; p.acs = 1; p.brs = 1; p.bcs = 64; p.crs = n; p.ccs = 1;
    if ((e = dgemm_split(p, 1, nullptr, 1.0, 0.0, st)) != cudaSuccess) return e;
    // trailing update: A22 -= L21 L21^T
    GemmDesc t{};
    t.A = A + (int64_t)r0 * n + c0; t.B = A + (int64_t)r0 * n + c0; t.C = A + (int64_t)r0 * n + r0;
    t.M = rest; t.N = rest; t.K = nb;
    t.ars = n; t.acs = 1; t.brs = 1; t.bcs = n; t.crs = n; t.ccs = 1;
    if ((e = dgemm_split(t, 1, nullptr, -1.0, 1.0, st)) != cudaSuccess) return e;
  }
  // X = L^{-1}: X_ii = Dinv_i; X[i, 0:i] = -Dinv_i (L[i, 0:i] X[0:i, 0:i])
  if ((e = cudaMemsetAsync(X, 0, sizeof(double) * (size_t)n * n, st)) != cudaSuccess) return e;
  for (int ib = 0; ib < nbk; ++ib) {
    const int r0 = ib * NB, nb = std::min(NB, n - r0);
    k_copy_rows<<<16, 256, 0, st>>>(Dinv + (int64_t)ib * 4096, 64, X + (int64_t)r0 * n + r0, n, nb, nb, 1.0);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (r0 == 0) continue;
    GemmDesc a{};   // R = L[i, 0:r0] X[0:r0, 0:r0]
    a.A = A + (int64_t)r0 * n; a.B = X; a.C = R;
    a.M = nb; a.N = r0; a.K = r0;
    a.ars = n; a.acs = 1; a.brs = n; a.bcs = 1; a.crs = n; a.ccs = 1;
    if ((e = dgemm_split(a, 1, nullptr, 1.0, 0.0, st)) != cudaSuccess) return e;
    GemmDesc b{};   // X[i, 0:r0] = -Dinv_i R
    b.A = Dinv + (int64_t)ib * 4096; b.B = R; b.C = X + (int64_t)r0 * n;
    b.M = nb; b.N = r0; b.K = nb;
    b.ars = 64; b.acs = 1; b.brs = n; b.bcs = 1; b.crs = n; b.ccs = 1;
    if ((e = dgemm_split(b, 1, nullptr, -1.0, 0.0, st)) != cudaSuccess) return e;
  }
  dim3 g((n + 15) / 16, (n + 15) / 16, 1);
  k_lt_l<<<g, 256, 0, st>>>(d_desc_for_ltl);
  note_launches(1);
  (void)out;
  return cudaGetLastError();
}

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
  size_t sm = (size_t)(maxbw + 1) * FW_COLS * sizeof(double);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_band_fwd_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  k_band_fwd_multi<<<dim3((maxbc + FW_COLS - 1) / FW_COLS, c.n_mod), FW_COLS, sm, st>>>(c.d_types, c.d_mods,
                                                                                      c.d_modmem);
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
  // one warp (subdomain) per block: the warps' FP64 shuffle sums do not share an SM
  k_band_fwd_single<<<ns, 32, 0, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_modmem, c.d_floc, c.hp.n_loc_dofs,
                                        c.d_ioff, c.d_h, ns);
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
