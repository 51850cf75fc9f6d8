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

// G[(s*nr + q) * n_lam + l] = -sign * R_b^s(k, q) for each entry (b, sign) of row l.
__global__ void k_build_G(int64_t n_lam, int nr, const int* __restrict__ b0, const signed char* __restrict__ s0,
                          const int* __restrict__ b1, const signed char* __restrict__ s1,
                          const int* __restrict__ bsub, const DevSub* __restrict__ subs,
                          const DevType* __restrict__ types, double* __restrict__ G) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= n_lam) return;
  for (int t = 0; t < 2; ++t) {
    const int b = t == 0 ? b0[l] : b1[l];
    if (b < 0) continue;
    const int sg = t == 0 ? s0[l] : s1[l];
    const int s = bsub[b];
    const DevSub S = subs[s];
    const int k = (int)(b - S.b_off);
    const double* R = types[S.type].Rraw;
    for (int q = 0; q < nr; ++q) {
      const double v = R[k * nr + q];
      G[((int64_t)s * nr + q) * n_lam + l] = sg > 0 ? -v : v;
    }
  }
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

cudaError_t tfeti_build_G(const Ctx& c, double* G, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(G, 0, sizeof(double) * (size_t)c.n_coarse * c.hp.n_lam, st);
  if (e != cudaSuccess) return e;
  const int64_t n = c.hp.n_lam;
  k_build_G<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, c.hp.n_rbm, c.d_lam_b0, c.d_lam_s0, c.d_lam_b1,
                                                         c.d_lam_s1, c.d_b_sub, c.d_subs, c.d_types, G);
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
