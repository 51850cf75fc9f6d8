// Recovery of the primal solution (FETI-DP): u_c from the second row of
// Eq. (12), then every subdomain's r-DOFs from the second row of Eq. (11),
//   K_rr u_r = f_r - K_rc u_c - B_r^T lambda,
// solved by block elimination with the stored factors:
//   x_b = F_s (f~_b - S_bc u_c - (B_r^T lambda)_b)
//   x_i = L^{-T} (L^{-1} f_i - Y_b x_b - Y_c u_c).
#include <algorithm>

#include "kernels.h"

namespace feti {

cudaError_t gemv_dense(const double* A, int n, int ld, const double* x, double* y, double beta, cudaStream_t st);
cudaError_t batched_gemv(const Ctx& c, int which, const double* xb, double* yb, double beta, cudaStream_t st);
cudaError_t axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st);

namespace {

// g_b = f~_b - S_bc u_c(s) - lam_b
__global__ void k_recover_gb(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                             const DevSub* __restrict__ subs, const double* __restrict__ mem,
                             const double* __restrict__ ft, const double* __restrict__ lamb,
                             const int* __restrict__ cg, const double* __restrict__ uc, double* __restrict__ g) {
  const DevSub S = subs[blockIdx.y];
  const DevType T = types[S.type];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= T.n_b) return;
  const int nb = T.n_b, nbc = nb + T.n_c;
  const double* Srow = mem + mods[S.module].S + (int64_t)k * nbc + nb;
  double v = ft[S.b_off + k] - lamb[S.b_off + k];
  for (int c = 0; c < T.n_c; ++c) v = fma(-Srow[c], uc[cg[S.c_off + c]], v);
  g[S.b_off + k] = v;
}

// t_i = h_i - Y_b x_b - Y_c u_c(s)
__global__ void k_recover_t(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                            const DevSub* __restrict__ subs, const double* __restrict__ mem,
                            const int64_t* __restrict__ ioff, const double* __restrict__ h,
                            const double* __restrict__ xb, const int* __restrict__ cg, const double* __restrict__ uc,
                            double* __restrict__ t) {
  const DevSub S = subs[blockIdx.y];
  const DevType T = types[S.type];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= T.n_i) return;
  const int nb = T.n_b, nbc = nb + T.n_c;
  const double* Yrow = mem + mods[S.module].Y + (int64_t)k * nbc;
  const int64_t o = ioff[blockIdx.y];
  double v = h[o + k];
  const double* x = xb + S.b_off;
  for (int j = 0; j < nb; ++j) v = fma(-Yrow[j], x[j], v);
  for (int c = 0; c < T.n_c; ++c) v = fma(-Yrow[nb + c], uc[cg[S.c_off + c]], v);
  t[o + k] = v;
}

// x = L^{-T} t in place, one warp per subdomain (column band of L).
__global__ void k_band_bwd_single(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                                  const DevSub* __restrict__ subs, const double* __restrict__ mem,
                                  const int64_t* __restrict__ ioff, double* __restrict__ t, int n_sub) {
  const int s = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (s >= n_sub) return;
  const int lane = threadIdx.x & 31;
  const DevSub S = subs[s];
  const DevModule M = mods[S.module];
  const DevType T = types[S.type];
  const int n = T.n_i, bw = T.bw, W = bw + 1;
  const double* Lc = mem + M.lcol;
  const double* rd = mem + M.rdiag;
  double* x = t + ioff[s];
  for (int j = n - 1; j >= 0; --j) {
    const double* lc = Lc + (int64_t)j * W;
    const int dmax = min(bw, n - 1 - j);
    double acc = 0.0;
    for (int d = 1 + lane; d <= dmax; d += 32) acc = fma(lc[d], x[j + d], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) x[j] = (x[j] - acc) * rd[j];
    __syncwarp();
  }
}

__global__ void k_write_uloc(const DevType* __restrict__ types, const DevSub* __restrict__ subs, int nld,
                             const int64_t* __restrict__ ioff, const double* __restrict__ xi,
                             const double* __restrict__ xb, const int* __restrict__ cg, const double* __restrict__ uc,
                             double* __restrict__ uloc) {
  const int s = blockIdx.y;
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const DevSub S = subs[s];
  const DevType T = types[S.type];
  if (a >= T.n_loc || a >= nld) return;
  const int ci = T.cls_idx[a];
  const int cls = ci >> 24, idx = ci & 0xffffff;
  double v = 0.0;
  if (cls == CLS_I) v = xi[ioff[s] + idx];
  else if (cls == CLS_B) v = xb[S.b_off + idx];
  else if (cls == CLS_C) v = uc[cg[S.c_off + idx]];
  uloc[S.loc_off + a] = v;
}

}  // namespace

// Assumes c.d_Xb holds B^T lambda (column 0).  uc: global primal values
// (FETI-DP) or null (TFETI, no corners).
static cudaError_t recover_local(Ctx& c, const double* uc, cudaStream_t st) {
  cudaError_t e;
  double* g = c.d_pb0;
  double* xb = c.d_pb1;
  int maxb = 1, maxi = 1;
  for (auto& t : c.h_types) { maxb = std::max(maxb, t.n_b); maxi = std::max(maxi, t.n_i); }
  k_recover_gb<<<dim3((maxb + 127) / 128, c.hp.n_sub), 128, 0, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_modmem,
                                                                     c.d_ft, c.d_Xb, c.d_c_glob, uc, g);
  note_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = batched_gemv(c, 0, g, xb, 0.0, st)) != cudaSuccess) return e;
  // edge averages: back to nodal values (xb in place, the c slots per subdomain)
  const int* cg = c.d_c_glob;
  if (c.max_avg > 0 && uc) {
    if ((e = launch_edge_unmap(c, uc, xb, c.d_ucl, st)) != cudaSuccess) return e;
    cg = c.d_c_iota;
    uc = c.d_ucl;
  }
  double* t = c.d_t;
  k_recover_t<<<dim3((maxi + 127) / 128, c.hp.n_sub), 128, 0, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_modmem,
                                                                    c.d_ioff, c.d_h, xb, cg, uc, t);
  note_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // one warp (subdomain) per block: the warps' FP64 shuffle sums do not share an SM
  k_band_bwd_single<<<c.hp.n_sub, 32, 0, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_modmem, c.d_ioff, t,
                                                c.hp.n_sub);
  note_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int nld = 1;
  for (auto& tt : c.h_types) nld = std::max(nld, tt.n_loc);
  k_write_uloc<<<dim3((nld + 127) / 128, c.hp.n_sub), 128, 0, st>>>(c.d_types, c.d_subs, nld, c.d_ioff, t, xb,
                                                                    cg, uc, c.d_uloc);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t recover_fetidp(Ctx& c, const double* lam, cudaStream_t st) {
  const int np = c.hp.n_primal;
  cudaError_t e;
  // u_c = Kbar^{-1} (fbar + F_rc^T lambda)
  if ((e = gather_lam_to_b(c, lam, c.hp.n_lam, 1, c.d_Xb, st)) != cudaSuccess) return e;
  double* Vraw = c.d_Vraw;
  double* uc = c.d_V;
  if ((e = corner_reduce(c, c.d_Xb, 1, c.d_Cb, Vraw, st)) != cudaSuccess) return e;
  if ((e = axpby(np, 1.0, c.d_fbar, 1.0, Vraw, st)) != cudaSuccess) return e;
  if ((e = coarse_matvec(c, Vraw, uc, st)) != cudaSuccess) return e;
  return recover_local(c, uc, st);
}

cudaError_t tfeti_add_rbm(const Ctx& c, const double* alpha, cudaStream_t st);

cudaError_t recover_tfeti(Ctx& c, const double* lam, const double* alpha, cudaStream_t st) {
  cudaError_t e;
  if ((e = gather_lam_to_b(c, lam, c.hp.n_lam, 1, c.d_Xb, st)) != cudaSuccess) return e;
  if ((e = recover_local(c, nullptr, st)) != cudaSuccess) return e;
  return tfeti_add_rbm(c, alpha, st);
}

}  // namespace feti
