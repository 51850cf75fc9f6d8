// Krylov helpers for Algorithm 1 (Section 3.3): the rank-revealing pivoted
// Cholesky of the Gram matrix Delta = Q^T W with the F-orthonormalising
// transform it implies, and the vector kernels of the step (all FP64, all
// reductions in a fixed order so that runs are bit-reproducible).
#include <algorithm>

#include "kernels.h"

namespace feti {

namespace {

constexpr double EPS2 = 4.930380657631324e-32;   // (2^-52)^2

// Pivot rule: the largest ratio of the remaining Schur-complement diagonal to
// the column's initial diagonal, exact ties to the lowest original column; stop
// when it is <= rr_tol.
//
// Blocked form.  Everything is indexed by the original column (no physical
// swaps): A holds the lower triangle of Delta by original index, updated once
// per panel of RR_PB pivots (a rank-RR_PB update of the rows and columns still
// unchosen); within a panel each new column of L subtracts only the panel's
// earlier columns; the remaining diagonal d is updated after every column and
// drives the pivot choice.  Every entry receives the same fused multiply-adds
// in the same order as the unblocked right-looking elimination.
//
// One launch sequence per call: k_rr_setup, then per panel k_rr_panel (one CTA
// per matrix: the RR_PB pivot steps, which are sequential) and k_rr_update (the
// panel's rank-RR_PB trailing update, RR_UB CTAs per matrix: the FP64 work,
// spread over as many SMs), then k_rr_finish.  The state between launches
// lives in the work buffer (rr_work_doubles(m) doubles per matrix):
//   A [m*m] | Lg [m*m] | rdiag [m] | d [m] | d0 [m] | Lp [RR_PB*m] |
//   perm, alive, chosen [m ints each] | k, stop, jn (ints)
// Output T (column-major, ld m, k columns) = N^T [L~^{-T}; 0] and *d_k = k.
constexpr int RR_THREADS = 1024;
constexpr int RR_PB = 16;                       // panel width (pivots per trailing update)
constexpr int RR_UB = 16;                       // CTAs per matrix in the trailing update
constexpr int RR_UT = 256;                      // threads per trailing-update CTA

struct RrState {
  double *A, *Lg, *rdiag, *d, *d0, *Lp;
  int *perm, *alive, *chosen, *k, *stop, *jn;
};

__device__ __forceinline__ RrState rr_state(double* work, int m) {
  RrState S;
  S.A = work;
  S.Lg = S.A + (int64_t)m * m;
  S.rdiag = S.Lg + (int64_t)m * m;
  S.d = S.rdiag + m;
  S.d0 = S.d + m;
  S.Lp = S.d0 + m;
  S.perm = reinterpret_cast<int*>(S.Lp + (int64_t)RR_PB * m);
  S.alive = S.perm + m;
  S.chosen = S.alive + m;
  S.k = S.chosen + m;
  S.stop = S.k + 1;
  S.jn = S.k + 2;
  return S;
}

// A = lower triangle of Delta, d = d0 = its diagonal, the live columns (initial
// diagonal above EPS2 times the largest), nothing chosen.
__global__ void __launch_bounds__(RR_THREADS) k_rr_setup(const RrDesc* __restrict__ descs, RrDesc one) {
  const RrDesc D = descs ? descs[blockIdx.x] : one;
  const int m = D.m, ld = D.ld;
  const RrState S = rr_state(D.work, m);
  __shared__ double rv[32];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
    const int a = (int)(e / m), b = (int)(e % m);
    if (b <= a) S.A[e] = D.Delta[a + (int64_t)b * ld];
  }
  double mx = 0.0;
  for (int t = tid; t < m; t += nt) {
    const double v = D.Delta[t + (int64_t)t * ld];
    S.d[t] = S.d0[t] = v;
    S.chosen[t] = 0;
    mx = fmax(mx, v);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) rv[wid] = mx;
  __syncthreads();
  double dmax = 0.0;
  for (int w = 0; w < nw; ++w) dmax = fmax(dmax, rv[w]);
  for (int t = tid; t < m; t += nt) {
    const double v = D.Delta[t + (int64_t)t * ld];
    S.alive[t] = (dmax > 0.0 && v > EPS2 * dmax) ? 1 : 0;
  }
  if (tid == 0) {
    *S.k = 0;
    *S.stop = 0;
    *S.jn = 0;
  }
}

// The pivot steps of the panel starting at position p0; the panel's columns of
// L go to Lg and Lp.  Sets *stop when no column qualifies.
__global__ void __launch_bounds__(RR_THREADS) k_rr_panel(const RrDesc* __restrict__ descs, RrDesc one, int p0,
                                                         double rr_tol) {
  const RrDesc D = descs ? descs[blockIdx.x] : one;
  const int m = D.m;
  const RrState S = rr_state(D.work, m);
  if (p0 >= m || *S.stop) return;
  extern __shared__ double rr_sh[];             // Lp[q][id], q < RR_PB
  double* Lp = rr_sh;
  __shared__ double d[1024], d0[1024];
  __shared__ unsigned char alive[1024], chosen[1024];
  __shared__ double rv[32];
  __shared__ int rp[32];
  __shared__ int s_bp, s_k;
  __shared__ double s_best, s_piv, s_rpiv;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5;
  // warps that own at least one column (m <= blockDim.x): only they take part
  // in the pivot reduction -- FP64 work is scarce on this part, so nothing is
  // computed redundantly by idle threads
  const int aw = (m + 31) / 32;
  const double* A = S.A;
  for (int t = tid; t < m; t += nt) {
    d[t] = S.d[t];
    d0[t] = S.d0[t];
    alive[t] = (unsigned char)S.alive[t];
    chosen[t] = (unsigned char)S.chosen[t];
  }
  if (tid == 0) s_k = *S.k;
  __syncthreads();
  const int pend = min(p0 + RR_PB, m);
  int jn = 0;
  bool stop = false;
  for (int j = p0; j < pend; ++j) {
    // --- pivot: max d/d0 over the unchosen live columns, ties to the lowest
    // id.  Ratios <= 0 never qualify (the stop test needs > rr_tol >= 0), so
    // they enter as 0 and the comparison runs on the bit patterns of the
    // non-negative doubles (integer pipe; same order as the values).
    if (wid < aw) {
      long long bv = -1;
      int bp = 0x7fffffff;
      for (int t = tid; t < m; t += aw * 32) {
        if (!alive[t] || chosen[t]) continue;
        const double ratio = d[t] / d0[t];
        const long long key = ratio > 0.0 ? __double_as_longlong(ratio) : 0ll;
        if (key > bv || (key == bv && t < bp)) { bv = key; bp = t; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int op = __shfl_xor_sync(0xffffffffu, bp, o);
        if (ov > bv || (ov == bv && op < bp)) { bv = ov; bp = op; }
      }
      if (lane == 0) { rv[wid] = __longlong_as_double(bv < 0 ? 0ll : bv); rp[wid] = bv < 0 ? 0x7fffffff : bp; }
    }
    __syncthreads();
    if (tid == 0) {
      long long v = -1;
      int pp = 0x7fffffff;
      for (int w = 0; w < aw; ++w) {
        const long long kw = rp[w] == 0x7fffffff ? -1 : __double_as_longlong(rv[w]);
        if (kw > v || (kw == v && rp[w] < pp)) { v = kw; pp = rp[w]; }
      }
      s_best = v < 0 ? -1.0 : __longlong_as_double(v);
      s_bp = pp == 0x7fffffff ? -1 : pp;
      if (s_bp >= 0 && s_best > rr_tol) {
        s_piv = sqrt(d[s_bp]);
        s_rpiv = 1.0 / s_piv;
      }
    }
    __syncthreads();
    if (s_bp < 0 || !(s_best > rr_tol)) { stop = true; break; }
    const int pj = s_bp;
    const int jq = j - p0;
    const double piv = s_piv;
    const double rpiv = s_rpiv;
    // --- column j of L for every unchosen live column r != pj
    for (int r = tid; r < m; r += nt) {
      if (r == pj || !alive[r] || chosen[r]) continue;
      double acc = r > pj ? A[(int64_t)r * m + pj] : A[(int64_t)pj * m + r];
      for (int q = 0; q < jq; ++q) acc = fma(-Lp[q * m + r], Lp[q * m + pj], acc);
      const double l = acc * rpiv;
      Lp[jq * m + r] = l;
      d[r] = fma(-l, l, d[r]);
    }
    if (tid == 0) {
      Lp[jq * m + pj] = piv;
      chosen[pj] = 1;
      S.perm[j] = pj;
      s_k = j + 1;
    }
    jn = jq + 1;
    __syncthreads();
  }
  // --- the panel's columns into Lg (rows of ids chosen earlier in the panel
  // hold stale values past their own column; those entries are never read)
  // and into Lp for the trailing update; the state back
  for (int e = tid; e < jn * m; e += nt) {
    const int q = e / m, id = e % m;
    const double v = Lp[q * m + id];
    S.Lg[(int64_t)id * m + p0 + q] = v;
    S.Lp[q * m + id] = v;
  }
  for (int t = tid; t < m; t += nt) {
    S.d[t] = d[t];
    S.chosen[t] = chosen[t];
  }
  if (tid == 0) {
    *S.k = s_k;
    *S.jn = jn;
    if (stop || s_k >= m) *S.stop = stop ? 1 : 0;
  }
}

// The panel's rank-jn update of the unchosen live rows and columns (lower
// triangle), RR_UB CTAs per matrix, one warp per row; skipped once the
// factorization has stopped.
__global__ void __launch_bounds__(RR_UT) k_rr_update(const RrDesc* __restrict__ descs, RrDesc one, int p0) {
  const RrDesc D = descs ? descs[blockIdx.y] : one;
  const int m = D.m;
  const RrState S = rr_state(D.work, m);
  if (p0 >= m || *S.stop) return;
  const int jn = *S.jn;
  extern __shared__ double rr_sh[];
  double* Lp = rr_sh;                           // [jn][m]
  unsigned char* live = reinterpret_cast<unsigned char*>(Lp + (int64_t)RR_PB * m);
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int e = tid; e < jn * m; e += nt) Lp[e] = S.Lp[e];
  for (int t = tid; t < m; t += nt) live[t] = S.alive[t] && !S.chosen[t];
  __syncthreads();
  double* A = S.A;
  for (int a = blockIdx.x * nw + wid; a < m; a += gridDim.x * nw) {
    if (!live[a]) continue;
    double* row = A + (int64_t)a * m;
    for (int b0 = 0; b0 <= a; b0 += 32 * 4) {
      double v[4];
      bool on[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int b = b0 + u * 32 + lane;
        on[u] = b <= a && live[b];
        v[u] = on[u] ? row[b] : 0.0;
      }
      for (int q = 0; q < jn; ++q) {
        const double la = Lp[q * m + a];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (on[u]) v[u] = fma(-la, Lp[q * m + b0 + u * 32 + lane], v[u]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (on[u]) row[b0 + u * 32 + lane] = v[u];
    }
  }
}

// Positions >= k: the remaining columns in increasing order; the reciprocals
// of the pivots (diagonal of L~) for the inverse kernel; perm and k out.
__global__ void __launch_bounds__(RR_THREADS) k_rr_finish(const RrDesc* __restrict__ descs, RrDesc one) {
  const RrDesc D = descs ? descs[blockIdx.x] : one;
  const int m = D.m;
  const RrState S = rr_state(D.work, m);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int k = *S.k;
  if (tid == 0) {
    int pos = k;
    for (int t = 0; t < m; ++t)
      if (!S.chosen[t]) S.perm[pos++] = t;
  }
  __syncthreads();
  for (int q = tid; q < k; q += nt) S.rdiag[q] = 1.0 / S.Lg[(int64_t)S.perm[q] * m + q];
  for (int t = tid; t < m; t += nt) D.perm[t] = S.perm[t];
  if (tid == 0) *D.k = k;
}

// U = L~^{-T} (upper triangular, column-major, ld m): T[jj + i*m] = X[i][jj]
// with X = L~^{-1}, L~(i, q) = Lg[perm[i]][q].  Column blocks of X are
// independent: CTA b owns columns [16b, 16b + 16) and runs the right-looking
// elimination on them (row q of X is final once scaled by 1 / L~(q, q); it then
// updates every later row), with column q + 1 of L~ prefetched into a shared
// double buffer while step q computes.  Same fused multiply-adds in the same
// order as a single-CTA right-looking inverse.
constexpr int RI_CB = 16;
constexpr int RI_THREADS = 256;

// grid: x = column block, y = matrix (descs[blockIdx.y] when descs is given, else `one`)
__global__ void __launch_bounds__(RI_THREADS) k_rr_inverse(const RrDesc* __restrict__ descs, RrDesc one) {
  const RrDesc D = descs ? descs[blockIdx.y] : one;
  const double* __restrict__ work = D.work;
  const int m = D.m;
  const int* __restrict__ perm_g = D.perm;
  double* __restrict__ T = D.T;
  extern __shared__ double ri_sh[];
  const int k = *D.k;
  const int c0 = blockIdx.x * RI_CB;
  if (c0 >= k) return;                           // block-uniform
  const double* Lg = work + (int64_t)m * m;
  const double* rdiag = work + 2 * (int64_t)m * m;
  const int rows = k - c0;
  double* xs = ri_sh;                            // [rows x RI_CB]: X[c0 + r][c0 + cc]
  double* lbuf = ri_sh + (int64_t)m * RI_CB;     // [2 x m]: column q of L~ over rows
  const int tid = threadIdx.x;
  for (int e = tid; e < rows * RI_CB; e += RI_THREADS) {
    const int r = e / RI_CB, cc = e % RI_CB;
    xs[e] = r == cc ? 1.0 : 0.0;
  }
  for (int i = c0 + 1 + tid; i < k; i += RI_THREADS) lbuf[i] = Lg[(int64_t)perm_g[i] * m + c0];
  __syncthreads();
  for (int q = c0; q < k; ++q) {
    const int cur = (q - c0) & 1;
    const double* lq = lbuf + cur * m;
    double* lnext = lbuf + (cur ^ 1) * m;
    if (tid < RI_CB && c0 + tid <= q) xs[(q - c0) * RI_CB + tid] *= rdiag[q];
    for (int i = q + 2 + tid; i < k; i += RI_THREADS) lnext[i] = Lg[(int64_t)perm_g[i] * m + q + 1];
    __syncthreads();
    const double* xq = xs + (q - c0) * RI_CB;
    for (int e = tid; e < (k - q - 1) * RI_CB; e += RI_THREADS) {
      const int i = q + 1 + e / RI_CB, cc = e % RI_CB;
      if (c0 + cc <= q) {
        double* xi = xs + (i - c0) * RI_CB + cc;
        *xi = fma(-lq[i], xq[cc], *xi);
      }
    }
    __syncthreads();
  }
  // T[jj + i*m] for the block's columns jj, all rows i < k
  const int nc = min(RI_CB, k - c0);
  for (int e = tid; e < k * RI_CB; e += RI_THREADS) {
    const int i = e / RI_CB, cc = e % RI_CB, jj = c0 + cc;
    if (cc < nc) T[jj + (int64_t)i * m] = (i >= c0 && jj <= i) ? xs[(i - c0) * RI_CB + cc] : 0.0;
  }
}

// out[j] = W[:, j] . r  (one block per column, fixed-order reduction)
__global__ void k_gemv_t(const double* __restrict__ W, int64_t ld, int64_t n, const double* __restrict__ r,
                         double* __restrict__ out) {
  const int j = blockIdx.x;
  const double* w = W + (int64_t)j * ld;
  double acc = 0.0;
  for (int64_t l = threadIdx.x; l < n; l += blockDim.x) acc = fma(w[l], r[l], acc);
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) s += red[w2];
    out[j] = s;
  }
}

__global__ void k_step(const double* __restrict__ W, const double* __restrict__ Q, int64_t ld, int64_t n, int k,
                       const double* __restrict__ g, double* __restrict__ lam_t, double* __restrict__ r,
                       double* __restrict__ qout) {
  __shared__ double gs[1024];
  for (int t = threadIdx.x; t < k; t += blockDim.x) gs[t] = g[t];
  __syncthreads();
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= n) return;
  double aw = 0.0, aq = 0.0;
  for (int j = 0; j < k; ++j) {
    aw = fma(W[l + (int64_t)j * ld], gs[j], aw);
    aq = fma(Q[l + (int64_t)j * ld], gs[j], aq);
  }
  lam_t[l] += aw;
  if (qout) qout[l] = aq;
  else r[l] -= aq;
}

__global__ void k_dot_partial(const double* __restrict__ x, const double* __restrict__ y, int64_t n,
                              double* __restrict__ part) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc = fma(x[i], y[i], acc);
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

__global__ void k_sum(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s;
  }
}

// One-direction forms of the block products (PCG and FO carry one direction):
// C = A[:, perm[0]] * U[0] (the F-orthonormal transform), and
// C = alpha * A[:, 0] * b[0] + beta * C (a rank-one update).  Padded 64 x 64
// GEMM tiles would spend 4096 FP64 FMAs per useful one here.
__global__ void k_scale_col(int64_t n, const double* __restrict__ A, int64_t lda, const int* __restrict__ perm,
                            const double* __restrict__ U, double* __restrict__ C) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) C[i] = A[i + (int64_t)perm[0] * lda] * U[0];
}

__global__ void k_axpy_scalar(int64_t n, double alpha, const double* __restrict__ A, const double* __restrict__ b,
                              double beta, double* __restrict__ C) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = alpha * A[i] * b[0];
  C[i] = beta != 0.0 ? fma(beta, C[i], v) : v;
}

__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = fma(a, x[i], b * y[i]);
}

__global__ void k_gemv_dense(const double* __restrict__ A, int n, int ld, const double* __restrict__ x,
                             double* __restrict__ y, double beta) {
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* a = A + (int64_t)row * ld;
  double acc = 0.0;
  for (int k = lane; k < n; k += 32) acc = fma(a[k], x[k], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) y[row] = beta != 0.0 ? fma(beta, y[row], acc) : acc;
}

}  // namespace

namespace {

cudaError_t rr_launch(const RrDesc* d_desc, const RrDesc& one, int n, int max_m, double rr_tol, cudaStream_t st) {
  if (max_m > 1024) return cudaErrorInvalidValue;
  if (n <= 0 || max_m <= 0) return cudaSuccess;
  static bool attr_set = false;
  const size_t psmem = (size_t)RR_PB * max_m * sizeof(double);
  const size_t usmem = psmem + (size_t)max_m;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_rr_panel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(RR_PB * 1024 * sizeof(double)));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_rr_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(RR_PB * 1024 * sizeof(double) + 1024));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_rr_setup<<<n, RR_THREADS, 0, st>>>(d_desc, one);
  // the pivot steps are bound by their block-wide barriers: no more threads
  // than columns
  const int pt = std::min(RR_THREADS, std::max(64, (max_m + 31) / 32 * 32));
  int nl = 1;
  for (int p0 = 0; p0 < max_m; p0 += RR_PB) {
    k_rr_panel<<<n, pt, psmem, st>>>(d_desc, one, p0, rr_tol);
    k_rr_update<<<dim3(RR_UB, n), RR_UT, usmem, st>>>(d_desc, one, p0);
    nl += 2;
  }
  k_rr_finish<<<n, RR_THREADS, 0, st>>>(d_desc, one);
  note_launches(nl + 1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  static bool inv_attr = false;
  const size_t ismem = (size_t)(RI_CB + 2) * 1024 * sizeof(double);
  if (!inv_attr) {
    e = cudaFuncSetAttribute(k_rr_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ismem);
    if (e != cudaSuccess) return e;
    inv_attr = true;
  }
  k_rr_inverse<<<dim3((max_m + RI_CB - 1) / RI_CB, n), RI_THREADS, (size_t)(RI_CB + 2) * max_m * sizeof(double),
                 st>>>(d_desc, one);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace

int64_t rr_work_doubles(int m) { return 2 * (int64_t)m * m + (int64_t)(4 + RR_PB) * m + (3 * (int64_t)m + 4) / 2 + 1; }

cudaError_t rr_cholesky(const double* Delta, int m, int ld, double rr_tol, double* work, double* T, int* d_k,
                        int* d_perm, cudaStream_t st) {
  RrDesc one{Delta, m, ld, work, T, d_k, d_perm};
  return rr_launch(nullptr, one, 1, m, rr_tol, st);
}

cudaError_t rr_cholesky_batched(const RrDesc* d_desc, int n, int max_m, double rr_tol, cudaStream_t st) {
  RrDesc one{};
  return rr_launch(d_desc, one, n, max_m, rr_tol, st);
}

cudaError_t gemv_t(const double* W, int64_t ld, int64_t n, int k, const double* r, double* out, cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  k_gemv_t<<<k, 256, 0, st>>>(W, ld, n, r, out);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t step_update(const double* W, const double* Q, int64_t ld, int64_t n, int k, const double* g,
                        double* lam_t, double* r, double* qout, cudaStream_t st) {
  if (k > 1024) return cudaErrorInvalidValue;
  k_step<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(W, Q, ld, n, k, g, lam_t, r, qout);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t dot(const double* x, const double* y, int64_t n, double* work, double* out, cudaStream_t st) {
  const int blocks = 256;
  k_dot_partial<<<blocks, 256, 0, st>>>(x, y, n, work);
  note_launches(1);
  k_sum<<<1, 32, 0, st>>>(work, blocks, out);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t scale_col(int64_t n, const double* A, int64_t lda, const int* perm, const double* U, double* C,
                      cudaStream_t st) {
  k_scale_col<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, A, lda, perm, U, C);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t axpy_scalar(int64_t n, double alpha, const double* A, const double* b, double beta, double* C,
                        cudaStream_t st) {
  k_axpy_scalar<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, alpha, A, b, beta, C);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st) {
  k_axpby<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, a, x, b, y);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t gemv_dense(const double* A, int n, int ld, const double* x, double* y, double beta, cudaStream_t st) {
  k_gemv_dense<<<(n + 7) / 8, 256, 0, st>>>(A, n, ld, x, y, beta);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace feti
