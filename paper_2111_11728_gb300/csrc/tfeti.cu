// Total FETI pieces (Section 2.1): the generalised inverse of each floating
// subdomain on its interface, the coarse operator G = -R^T B^T, e = -R^T f,
// and the rigid-body part of the recovered displacement.
//
// Generalised inverse: with S_b the Schur complement of K^s onto the DOFs
// touched by B (singular; its null space is spanned by the rigid modes
// restricted to those DOFs, R_b) and Rhat an orthonormal basis of span(R_b),
// F_s = (S_b + Rhat Rhat^T)^{-1} satisfies S_b F_s S_b = S_b.  Extended to the
// interior by block elimination it is a generalised inverse K^# of K^s; any
// K^# gives the same projected iterates (its null-space terms lie in
// range(G^T) and are removed by P) and the same u (alpha absorbs them).
#include <algorithm>

#include "kernels.h"

namespace feti {

namespace {

__global__ void k_add_rrt(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                          double* __restrict__ mem, int nr) {
  const DevModule M = mods[blockIdx.y];
  const DevType T = types[M.type];
  const int n = T.n_b, ld = T.n_b + T.n_c;
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    double v = 0.0;
    for (int q = 0; q < nr; ++q) v = fma(T.Rhat[i * nr + q], T.Rhat[j * nr + q], v);
    mem[M.W + (int64_t)i * ld + j] += v;
  }
}

// t[:, jj] = v e_{J0 + jj} for jj < nj (t column-major, ld n).
__global__ void k_unit_cols(int n, int nj, int J0, double v, double* __restrict__ t) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * nj) return;
  const int i = (int)(e % n), jj = (int)(e / n);
  t[e] = i == J0 + jj ? v : 0.0;
}

// The projector's coarse products without forming G: G X is a per-subdomain
// reduction of the gathered block, t[(s, q), j] = -sum_k R_b^s(k, q) (B^sT X)(k, j),
// and G^T t a per-multiplier combination of the rigid modes at the row's
// entries.  One block per (subdomain, column); the rigid modes are read per
// type (nr <= 6).
__global__ void __launch_bounds__(128) k_G_apply(int nr, const DevType* __restrict__ types,
                                                 const DevSub* __restrict__ subs, const double* __restrict__ Xb,
                                                 int64_t nbt, double* __restrict__ t, int n_coarse) {
  const int s = blockIdx.x, j = blockIdx.y;
  const DevSub S = subs[s];
  const DevType T = types[S.type];
  const double* R = T.Rraw;
  const double* x = Xb + (int64_t)j * nbt + S.b_off;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int k = threadIdx.x; k < T.n_b; k += blockDim.x) {
    const double v = x[k];
#pragma unroll
    for (int q = 0; q < 6; ++q)
      if (q < nr) acc[q] = fma(R[k * nr + q], v, acc[q]);
  }
  __shared__ double red[6][4];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < nr)
    t[(int64_t)j * n_coarse + s * nr + threadIdx.x] =
        -(red[threadIdx.x][0] + red[threadIdx.x][1] + red[threadIdx.x][2] + red[threadIdx.x][3]);
}

// X[l, j] -= (G^T t)[l, j] = sum over the entries (b, sign) of row l of
// sign * sum_q R_b^s(k, q) t[(s, q), j]   (G = -R^T B^T).
__global__ void k_Gt_sub(int64_t n_lam, int m, int nr, const int* __restrict__ b0, const signed char* __restrict__ s0,
                         const int* __restrict__ b1, const signed char* __restrict__ s1,
                         const int* __restrict__ bsub, const DevSub* __restrict__ subs,
                         const DevType* __restrict__ types, const double* __restrict__ t, int n_coarse,
                         double* __restrict__ X, int64_t ldx) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (l >= n_lam || j >= m) return;
  double v = 0.0;
  for (int e = 0; e < 2; ++e) {
    const int b = e == 0 ? b0[l] : b1[l];
    if (b < 0) continue;
    const int s = bsub[b];
    const DevSub S = subs[s];
    const double* R = types[S.type].Rraw + (int64_t)(b - S.b_off) * nr;
    const double* ts = t + (int64_t)j * n_coarse + s * nr;
    double y = 0.0;
    for (int q = 0; q < nr; ++q) y = fma(R[q], ts[q], y);
    v += (e == 0 ? s0[l] : s1[l]) > 0 ? y : -y;
  }
  X[(int64_t)j * ldx + l] += v;
}

// Rigid mode q of a subdomain at local DOF (node coordinates c, direction d).
__device__ __forceinline__ double rbm(int dim, int q, const int c[3], int d) {
  if (dim == 2) {
    if (q < 2) return d == q ? 1.0 : 0.0;
    return d == 0 ? -(double)c[1] : (double)c[0];
  }
  if (q < 3) return d == q ? 1.0 : 0.0;
  const double x = c[0], y = c[1], z = c[2];
  if (q == 3) return d == 1 ? -z : (d == 2 ? y : 0.0);
  if (q == 4) return d == 0 ? z : (d == 2 ? -x : 0.0);
  return d == 0 ? -y : (d == 1 ? x : 0.0);
}

// e[(s, q)] = -sum_a R^s(a, q) f^s(a); one block per subdomain.
__global__ void k_build_e(int dim, int nr, const DevType* __restrict__ types, const DevSub* __restrict__ subs,
                          const double* __restrict__ floc, double* __restrict__ e) {
  const int s = blockIdx.x;
  const DevSub S = subs[s];
  const DevType T = types[S.type];
  const int nld = T.n_loc, ln0 = T.ln[0], ln1 = T.ln[1];
  __shared__ double red[6][32];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int a = threadIdx.x; a < nld; a += blockDim.x) {
    const double f = floc[S.loc_off + a];
    if (f == 0.0) continue;
    const int node = a / dim, d = a % dim;
    const int c[3] = {node % ln0, (node / ln0) % ln1, node / (ln0 * ln1)};
    for (int q = 0; q < nr; ++q) acc[q] = fma(rbm(dim, q, c, d), f, acc[q]);
  }
  for (int q = 0; q < nr; ++q) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < nr) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
    e[s * nr + threadIdx.x] = -v;
  }
}

// uloc(s, a) += sum_q R^s(a, q) alpha(s, q)
__global__ void k_add_rbm(int dim, int nr, const DevType* __restrict__ types, const DevSub* __restrict__ subs,
                          const double* __restrict__ alpha, double* __restrict__ uloc) {
  const int s = blockIdx.y;
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const DevSub S = subs[s];
  const DevType T = types[S.type];
  const int nld = T.n_loc, ln0 = T.ln[0], ln1 = T.ln[1];
  if (a >= nld) return;
  const int node = a / dim, d = a % dim;
  const int c[3] = {node % ln0, (node / ln0) % ln1, node / (ln0 * ln1)};
  double v = 0.0;
  for (int q = 0; q < nr; ++q) v = fma(rbm(dim, q, c, d), alpha[s * nr + q], v);
  uloc[S.loc_off + a] += v;
}

}  // namespace

cudaError_t tfeti_add_rrt(const Ctx& c, cudaStream_t st) {
  k_add_rrt<<<dim3(64, c.n_mod), 256, 0, st>>>(c.d_types, c.d_mods, c.d_modmem, c.hp.n_rbm);
  note_launches(1);
  return cudaGetLastError();
}

// G G^T (column-major n_coarse^2 in Kbar) from the sparse G, nj <= ldw coarse
// columns at a time through the multiplier-space work block W [n_lam x ldw]:
// W = G^T E_J (as X -= G^T t with t = -E_J on a zero block), then G W.
cudaError_t tfeti_ggt(const Ctx& c, double* W, int ldw, double* t1, double* t2, double* Xb, double* Kbar,
                      cudaStream_t st) {
  const int nco = c.n_coarse;
  const int64_t nl = c.hp.n_lam;
  for (int J0 = 0; J0 < nco; J0 += ldw) {
    const int nj = std::min(ldw, nco - J0);
    const int64_t ne = (int64_t)nco * nj;
    k_unit_cols<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(nco, nj, J0, -1.0, t1);
    note_launches(1);
    cudaError_t e = cudaMemsetAsync(W, 0, sizeof(double) * (size_t)nl * nj, st);
    if (e == cudaSuccess) e = tfeti_Gt_sub(c, t1, nj, W, nl, st);
    if (e == cudaSuccess) e = gather_lam_to_b(c, W, nl, nj, Xb, st);
    if (e == cudaSuccess) e = tfeti_G_apply(c, Xb, nj, t2, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(Kbar + (int64_t)J0 * nco, t2, sizeof(double) * (size_t)ne, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t tfeti_G_apply(const Ctx& c, const double* Xb, int m, double* t, cudaStream_t st) {
  if (c.hp.n_rbm > 6) return cudaErrorInvalidValue;
  k_G_apply<<<dim3(c.hp.n_sub, m), 128, 0, st>>>(c.hp.n_rbm, c.d_types, c.d_subs, Xb, c.hp.n_b_total, t,
                                                 c.n_coarse);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t tfeti_Gt_sub(const Ctx& c, const double* t, int m, double* X, int64_t ldx, cudaStream_t st) {
  const int64_t n = c.hp.n_lam;
  k_Gt_sub<<<dim3((unsigned)((n + 255) / 256), m), 256, 0, st>>>(n, m, c.hp.n_rbm, c.d_lam_b0, c.d_lam_s0,
                                                                 c.d_lam_b1, c.d_lam_s1, c.d_b_sub, c.d_subs,
                                                                 c.d_types, t, c.n_coarse, X, ldx);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t tfeti_build_e(const Ctx& c, double* e, cudaStream_t st) {
  k_build_e<<<c.hp.n_sub, 256, 0, st>>>(c.hp.dim, c.hp.n_rbm, c.d_types, c.d_subs, c.d_floc, e);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t tfeti_add_rbm(const Ctx& c, const double* alpha, cudaStream_t st) {
  const int nld = c.hp.n_loc_dofs;
  k_add_rbm<<<dim3((nld + 127) / 128, c.hp.n_sub), 128, 0, st>>>(c.hp.dim, c.hp.n_rbm, c.d_types, c.d_subs,
                                                                 alpha, c.d_uloc);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace feti
