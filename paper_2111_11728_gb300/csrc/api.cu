// C ABI entry points and the host driver of Algorithm 1.
//
// The host only sequences kernels and reads two scalars per Krylov iteration
// (the retained rank k_i and sqrt(r^T z)); every arithmetic step runs on the
// device in FP64.
#include <algorithm>
#include <memory>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "kernels.h"

using namespace feti;

struct feti_ctx {
  Ctx c;
};

namespace feti {

cudaError_t dev_alloc(Ctx& c, void** p, size_t bytes) {
  *p = nullptr;
  if (c.have_user_alloc) {
    *p = c.user_alloc.alloc(c.user_alloc.user, bytes, static_cast<void*>(c.stream));
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
  }
  cudaError_t e = cudaMallocAsync(p, bytes, c.stream);
  if (e != cudaSuccess) return e;
  // ordered on the context stream; synchronised so that host-side copies made
  // right after the allocation (set-up uploads) may use it too
  return cudaStreamSynchronize(c.stream);
}

void dev_free(Ctx& c, void* p, size_t bytes) {
  if (!p) return;
  if (c.have_user_alloc) c.user_alloc.free(c.user_alloc.user, p, bytes, static_cast<void*>(c.stream));
  else cudaFreeAsync(p, c.stream);
}

}  // namespace feti

namespace {

#define TRY(expr)                              \
  do {                                         \
    feti_status _s = (expr);                   \
    if (_s != FETI_OK) return _s;              \
  } while (0)
#define CU(expr) FETI_CUDA_TRY(&c, expr)

template <class T>
feti_status dalloc(Ctx& c, T*& p, size_t n) {
  p = nullptr;
  if (n == 0) n = 1;
  void* q = nullptr;
  cudaError_t e = dev_alloc(c, &q, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    c.err = "device allocation of " + std::to_string(n * sizeof(T)) + " bytes failed: " + cudaGetErrorString(e);
    return FETI_ENOMEM;
  }
  c.allocs.push_back(q);
  c.alloc_bytes.push_back(n * sizeof(T));
  c.device_bytes += n * sizeof(T);
  p = static_cast<T*>(q);
  return FETI_OK;
}

feti_status dalloc_bytes(Ctx& c, void*& p, size_t bytes) {
  unsigned char* q = nullptr;
  TRY(dalloc(c, q, bytes));
  p = q;
  return FETI_OK;
}

bool split_precision(int p) { return p == FETI_TF32X3 || p == FETI_BF16X3; }

template <class T>
feti_status upload(Ctx& c, T*& p, const std::vector<T>& v) {
  TRY(dalloc(c, p, v.size()));
  if (!v.empty()) CU(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return FETI_OK;
}

void free_all(Ctx& c) {
  cudaStreamSynchronize(c.stream);        // nothing in flight uses the memory any more
  for (size_t i = 0; i < c.allocs.size(); ++i) dev_free(c, c.allocs[i], c.alloc_bytes[i]);
  c.allocs.clear();
  c.alloc_bytes.clear();
  c.device_bytes = 0;
  c.hist_W.clear();
  c.hist_Q.clear();
  c.hist_k.clear();
  c.blk_cap = 0;
  c.kr_cap = 0;
  c.split_cap = 0;
  c.xb_cap = 0;
  if (c.d_tiles) dev_free(c, c.d_tiles, (size_t)c.tiles_cap * sizeof(int4));
  c.d_tiles = nullptr;
  c.tiles_cap = 0;
  cudaStreamSynchronize(c.stream);
  cudaGetLastError();
  c.n_tiles = 0;
  c.tiles_ncb = 0;
}

inline int64_t align32(int64_t x) { return (x + 31) / 32 * 32; }

constexpr int kGgtCols = 64;           // coarse columns per block when G G^T is formed (TFETI)
constexpr int BATCH_CHUNK = 128;        // columns per dual-operator apply in the batched Algorithm 1
constexpr int64_t BATCH_KCHUNK = 8192;  // rows per split-K chunk of its Gram products
constexpr int64_t BATCH_RCHUNK = 4096;  // rows per entry of its block updates, until autotuned

feti_status sync_check(Ctx& c) {
  CU(cudaStreamSynchronize(c.stream));
  CU(cudaGetLastError());
  return FETI_OK;
}

// ---- GEMM descriptor builders -------------------------------------------------------
feti_status build_block_descs(Ctx& c) {
  const HostProblem& hp = c.hp;
  const int64_t nbt = hp.n_b_total, nct = std::max<int64_t>(c.n_c_total, 1);
  std::vector<GemmDesc> dF(hp.n_sub), dFrcT(hp.n_sub), dFrc(hp.n_sub);
  for (int s = 0; s < hp.n_sub; ++s) {
    const DevSub& S = c.h_subs[s];
    const DevModule& M = c.h_mods[S.module];
    const DevType& T = c.h_types[S.type];
    GemmDesc g{};
    g.A = c.d_modmem + M.F; g.B = c.d_Xb + S.b_off; g.C = c.d_Yb + S.b_off;
    g.M = T.n_b; g.N = 1; g.K = T.n_b;
    g.ars = T.n_b; g.acs = 1; g.brs = 1; g.bcs = nbt; g.crs = 1; g.ccs = nbt;
    dF[s] = g;
    GemmDesc h{};
    h.A = c.d_modmem + M.Frc; h.B = c.d_Xb + S.b_off; h.C = c.d_Cb + S.c_off;
    h.M = T.n_c; h.N = 1; h.K = T.n_b;
    h.ars = 1; h.acs = std::max(T.n_c, 1); h.brs = 1; h.bcs = nbt; h.crs = 1; h.ccs = nct;
    dFrcT[s] = h;
    GemmDesc q{};
    q.A = c.d_modmem + M.Frc; q.B = c.d_Vc + S.c_off; q.C = c.d_Yb + S.b_off;
    q.M = T.n_b; q.N = 1; q.K = T.n_c;
    q.ars = std::max(T.n_c, 1); q.acs = 1; q.brs = 1; q.bcs = nct; q.crs = 1; q.ccs = nbt;
    dFrc[s] = q;
  }
  if (!c.d_gemm_F) {
    TRY(dalloc(c, c.d_gemm_F, hp.n_sub));
    TRY(dalloc(c, c.d_gemm_FrcT, hp.n_sub));
    TRY(dalloc(c, c.d_gemm_Frc, hp.n_sub));
  }
  CU(cudaMemcpy(c.d_gemm_F, dF.data(), dF.size() * sizeof(GemmDesc), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c.d_gemm_FrcT, dFrcT.data(), dFrcT.size() * sizeof(GemmDesc), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c.d_gemm_Frc, dFrc.data(), dFrc.size() * sizeof(GemmDesc), cudaMemcpyHostToDevice));
  if (hp.n_prob > 1 && c.d_gemm_coarse) {
    // per-problem coarse solves of a batch: V_p = Kbar_p^{-1} Vraw_p on the
    // (re)allocated corner buffers
    std::vector<GemmDesc> gc(hp.n_prob);
    const int np = hp.n_primal;
    for (int q = 0; q < hp.n_prob; ++q) {
      const int o = hp.prob_primal_off[q], npq = hp.prob_primal_off[q + 1] - o;
      GemmDesc g{};
      g.A = c.d_Kbar_inv + c.h_kbar_off[q]; g.B = c.d_Vraw + o; g.C = c.d_V + o;
      g.M = npq; g.N = 1; g.K = npq;
      g.ars = npq; g.acs = 1; g.brs = 1; g.bcs = np; g.crs = 1; g.ccs = np;
      gc[q] = g;
    }
    CU(cudaMemcpy(c.d_gemm_coarse, gc.data(), gc.size() * sizeof(GemmDesc), cudaMemcpyHostToDevice));
  }
  return FETI_OK;
}

// Block buffers of the dual operator for up to `m` columns.
feti_status ensure_blocks(Ctx& c, int m) {
  if (m <= c.blk_cap) return FETI_OK;
  const HostProblem& hp = c.hp;
  const int cap = std::max(m, 64);
  const int64_t nbt = hp.n_b_total, nct = std::max<int64_t>(c.n_c_total, 1);
  const int64_t np = std::max(hp.n_primal, 1);
  TRY(dalloc(c, c.d_Xb, (size_t)nbt * cap));
  TRY(dalloc(c, c.d_Yb, (size_t)nbt * cap));
  TRY(dalloc(c, c.d_Cb, (size_t)nct * cap));
  TRY(dalloc(c, c.d_Vc, (size_t)nct * cap));
  TRY(dalloc(c, c.d_Vraw, (size_t)np * cap));
  TRY(dalloc(c, c.d_V, (size_t)np * cap));
  if (c.n_coarse > 0 && hp.method == FETI_TFETI) {
    TRY(dalloc(c, c.d_ct1, (size_t)c.n_coarse * cap));
    TRY(dalloc(c, c.d_ct2, (size_t)c.n_coarse * cap));
  }
  if (c.d_Kbar_inv32) TRY(dalloc(c, c.d_coarse_part, (size_t)tc_coarse_scratch((int)np, (int)cap)));
  if (c.opt.precision != FETI_FP64) {
    const size_t eb = tc_elem_bytes(c.opt.precision);
    // the padding of the operand stays zero: the gather writes only the DOF slots
    TRY(dalloc_bytes(c, c.d_xb_hi, (size_t)c.nbp_total * cap * eb));
    CU(cudaMemsetAsync(c.d_xb_hi, 0, (size_t)c.nbp_total * cap * eb, c.stream));
    TRY(dalloc(c, c.d_Yb32, (size_t)nbt * cap));
    if (split_precision(c.opt.precision)) {
      TRY(dalloc_bytes(c, c.d_xb_lo, (size_t)c.nbp_total * cap * eb));
      CU(cudaMemsetAsync(c.d_xb_lo, 0, (size_t)c.nbp_total * cap * eb, c.stream));
    }
    c.xb_cap = cap;
  }
  c.blk_cap = cap;
  return build_block_descs(c);
}

feti_status ensure_split(Ctx& c, int64_t need) {
  if (need <= c.split_cap) return FETI_OK;
  TRY(dalloc(c, c.d_split, (size_t)need));
  c.split_cap = need;
  return FETI_OK;
}

// C (col-major M x N, ld ldc) = alpha * A^T B + beta * C with A (K x M) and
// B (K x N) column-major (ld lda, ldb): the Gram products of Algorithm 1.
feti_status gemm_tn(Ctx& c, const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                    int M, int N, int K, double alpha, double beta, int lower = 0) {
  if (M == 1 && N == 1 && alpha == 1.0 && beta == 0.0) {   // one direction: an inner product
    CU(dot(A, B, K, c.d_red, C, c.stream));
    return FETI_OK;
  }
  GemmDesc d{};
  d.A = A; d.B = B; d.C = C; d.M = M; d.N = N; d.K = K;
  d.ars = lda; d.acs = 1; d.brs = 1; d.bcs = ldb; d.crs = 1; d.ccs = ldc;
  d.tri = lower ? 1 : 0;
  const int splits = split_for(M, N, K, lower != 0);
  if (splits > 1) TRY(ensure_split(c, (int64_t)splits * M * N));
  // symmetric products: the algorithmic count is the lower triangle
  const double fl = lower ? (double)M * (M + 1.0) * K : -1.0;
  CU(dgemm_split(d, splits, c.d_split, alpha, beta, c.stream, fl));
  return FETI_OK;
}

// C (col-major M x N) = A[:, perm[0..K)] U with U upper triangular (K x N,
// column-major ld ldu), A column-major n x m.
feti_status gemm_perm_upper(Ctx& c, const double* A, int64_t lda, const int* perm, const double* U, int64_t ldu,
                            double* C, int64_t ldc, int M, int N, double alg_flops) {
  if (N == 1) {                                              // one direction: a scaled column
    CU(scale_col(M, A, lda, perm, U, C, c.stream));
    return FETI_OK;
  }
  GemmDesc d{};
  d.A = A; d.B = U; d.C = C; d.M = M; d.N = N; d.K = N;
  d.ars = 1; d.acs = lda; d.brs = 1; d.bcs = ldu; d.crs = 1; d.ccs = ldc;
  d.tri = 2;
  d.acol = perm;
  CU(dgemm_split(d, 1, nullptr, 1.0, 0.0, c.stream, alg_flops));
  return FETI_OK;
}

// C (col-major M x N) = alpha * A B + beta * C, A (M x K), B (K x N) column-major.
feti_status gemm_nn(Ctx& c, const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                    int M, int N, int K, double alpha, double beta, double alg_flops = -1.0) {
  if (N == 1 && K == 1) {                                    // one direction: a rank-one update
    CU(axpy_scalar(M, alpha, A, B, beta, C, c.stream));
    return FETI_OK;
  }
  GemmDesc d{};
  d.A = A; d.B = B; d.C = C; d.M = M; d.N = N; d.K = K;
  d.ars = 1; d.acs = lda; d.brs = 1; d.bcs = ldb; d.crs = 1; d.ccs = ldc;
  CU(dgemm_split(d, 1, nullptr, alpha, beta, c.stream, alg_flops));
  return FETI_OK;
}

// TFETI projector P X = X - G^T (G G^T)^{-1} G X, X column-major [n_lam x m].
// G = -R^T B^T is never read as a dense matrix here: G X is a per-subdomain
// reduction of the gathered block B^T X against the rigid modes at the
// interface, G^T t a per-multiplier combination of the modes at the row's
// two entries -- O(n_lambda m) traffic instead of O(n_coarse n_lambda).
feti_status project(Ctx& c, double* X, int64_t ldx, int m) {
  if (c.hp.method != FETI_TFETI) return FETI_OK;
  TRY(ensure_blocks(c, m));
  const int nco = c.n_coarse;
  // t1 = G X
  CU(gather_lam_to_b(c, X, ldx, m, c.d_Xb, c.stream));
  CU(tfeti_G_apply(c, c.d_Xb, m, c.d_ct1, c.stream));
  // t2 = (G G^T)^{-1} t1
  {
    GemmDesc d{};
    d.A = c.d_Kbar_inv; d.B = c.d_ct1; d.C = c.d_ct2; d.M = nco; d.N = m; d.K = nco;
    d.ars = nco; d.acs = 1; d.brs = 1; d.bcs = nco; d.crs = 1; d.ccs = nco;
    CU(dgemm_split(d, 1, nullptr, 1.0, 0.0, c.stream));
  }
  // X -= G^T t2
  CU(tfeti_Gt_sub(c, c.d_ct2, m, X, ldx, c.stream));
  return FETI_OK;
}

// Inverse of the coarse matrix in c.d_Kbar: one CTA for small ones, the
// blocked multi-CTA factorisation otherwise.
cudaError_t coarse_inverse(Ctx& c) {
  const int n = c.n_coarse;
  if (c.hp.n_prob > 1) {
    std::vector<DenseDesc> hd(c.hp.n_prob);
    for (int q = 0; q < c.hp.n_prob; ++q) hd[q].n = c.hp.prob_primal_off[q + 1] - c.hp.prob_primal_off[q];
    return dense_spd_inverse(c.d_dense_coarse_batch, hd.data(), c.hp.n_prob, c.d_status, c.stream);
  }
  if (n <= 128) {
    DenseDesc hd{};
    hd.n = n;
    return dense_spd_inverse(c.d_dense_coarse, &hd, 1, c.d_status, c.stream);
  }
  return dense_spd_inverse_blocked(c.d_Kbar, c.d_Kbar_L, c.d_Kbar_inv, n, c.d_coarse_work, c.d_status,
                                   c.d_dense_coarse, c.stream);
}

// Y = F X for m columns (device, column-major).
feti_status apply_dual(Ctx& c, const double* X, int64_t ldx, int m, double* Y, int64_t ldy) {
  TRY(ensure_blocks(c, m));
  CU(gather_lam_to_b(c, X, ldx, m, c.d_Xb, c.stream));
  // one column: matrix-vector kernels instead of padded GEMM tiles
  auto local = [&]() -> cudaError_t {
    return m == 1 ? batched_gemv(c, 0, c.d_Xb, c.d_Yb, 0.0, c.stream) : apply_local_F(c, c.d_Xb, c.d_Yb, m, 0.0, c.stream);
  };
  if (c.hp.method == FETI_FETIDP && c.hp.n_primal > 0) {
    CU(corner_reduce(c, c.d_Xb, m, c.d_Cb, c.d_Vraw, c.stream));
    CU(coarse_apply(c, c.d_Vraw, c.d_V, m, c.stream));
    CU(local());
    if (m == 1) CU(corner_expand_thin(c, c.d_V, m, c.d_Yb, c.stream));
    else CU(corner_expand(c, c.d_V, m, c.d_Vc, c.d_Yb, c.stream));
  } else {
    CU(local());
  }
  CU(scatter_b_to_lam(c, c.d_Yb, m, Y, ldy, c.stream));
  return FETI_OK;
}

// Y = F X with the local blocks on the tensor cores (TF32 / BF16 inputs,
// FP32 accumulation).  The corner reduction F_rc^T X runs on the tensor cores
// too (corner tiles of the same product kernel) and the coarse correction
// Kbar_cc^{-1} (F_rc^T X) is an FP32 product (the coarse matrix is factorized
// and inverted in FP64 at feti_factorize; only its application is rounded,
// like the local blocks').
feti_status apply_dual_lowp(Ctx& c, const double* X, int64_t ldx, int m, double* Y, int64_t ldy) {
  TRY(ensure_blocks(c, m));
  CU(tc_prepare_tiles(c, m));
  CU(tc_gather(c, X, ldx, m, c.stream));
  if (c.tc_aug) {
    // corner reduction, coarse solve, then the coarse correction rides in
    // the K-extension of the one tensor-core product
    CU(tc_corner_reduce(c, m, c.d_Vraw, c.stream));
    if (m > 1 && c.d_Kbar_inv32) CU(tc_coarse_apply(c, c.d_Vraw, c.d_V, m, c.stream));
    else CU(coarse_apply(c, c.d_Vraw, c.d_V, m, c.stream));
    CU(tc_put_v(c, c.d_V, m, c.stream));
  }
  const cudaError_t pe = tc_product(c, m, c.d_Yb32, c.stream);
  c.test_skip_chunk = -1;                          // the test hook acts on one product only
  CU(pe);
  CU(scatter_b_to_lam32(c, c.d_Yb32, m, Y, ldy, c.stream));
  return FETI_OK;
}

feti_status check_status(Ctx& c, const char* where) {
  int st = 0;
  CU(cudaMemcpy(&st, c.d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) {
    c.err = std::string(where) + ": non-positive pivot (";
    if (st >= 3000000) {
      c.err = std::string(where) + ": a tensor-core product timed out waiting for its copies or MMAs (subdomain " +
              std::to_string(st - 3000000) + ")";
      CU(cudaMemset(c.d_status, 0, sizeof(int)));
      return FETI_ETIMEOUT;
    }
    if (st >= 2000000) c.err += "dense factor, tag " + std::to_string(st - 2000000);
    else c.err += "banded factor of module " + std::to_string(st - 1000000);
    c.err += "); the stiffness is not positive definite (zero density with Emin = 0?)";
    CU(cudaMemset(c.d_status, 0, sizeof(int)));
    return FETI_EBREAKDOWN;
  }
  return FETI_OK;
}

// Host-side rigid modes at the b DOFs of a type: raw (same formula as the
// device's rbm()) and orthonormalised by modified Gram-Schmidt.
void type_rigid_modes(const HostProblem& hp, const StructType& T, std::vector<double>& raw,
                      std::vector<double>& hat) {
  const int nr = hp.n_rbm, dim = hp.dim;
  raw.assign((size_t)T.n_b * nr, 0.0);
  for (int k = 0; k < T.n_b; ++k) {
    const int ld = T.blist[k];
    int c[3];
    local_node_coords(hp, ld / dim, c);
    const int d = ld % dim;
    const double x = c[0], y = c[1], z = c[2];
    for (int q = 0; q < nr; ++q) {
      double v;
      if (dim == 2) v = q < 2 ? (d == q ? 1.0 : 0.0) : (d == 0 ? -y : x);
      else if (q < 3) v = d == q ? 1.0 : 0.0;
      else if (q == 3) v = d == 1 ? -z : (d == 2 ? y : 0.0);
      else if (q == 4) v = d == 0 ? z : (d == 2 ? -x : 0.0);
      else v = d == 0 ? -y : (d == 1 ? x : 0.0);
      raw[(size_t)k * nr + q] = v;
    }
  }
  hat = raw;
  for (int q = 0; q < nr; ++q) {
    for (int p = 0; p < q; ++p) {
      double dp = 0.0;
      for (int k = 0; k < T.n_b; ++k) dp += hat[(size_t)k * nr + p] * hat[(size_t)k * nr + q];
      for (int k = 0; k < T.n_b; ++k) hat[(size_t)k * nr + q] -= dp * hat[(size_t)k * nr + p];
    }
    double nn = 0.0;
    for (int k = 0; k < T.n_b; ++k) nn += hat[(size_t)k * nr + q] * hat[(size_t)k * nr + q];
    nn = std::sqrt(nn);
    for (int k = 0; k < T.n_b; ++k) hat[(size_t)k * nr + q] /= nn;
  }
}

}  // namespace

// ================================================================================
extern "C" {

feti_status feti_options_default(feti_options* opt) {
  if (!opt) return FETI_EINVAL;
  opt->method = FETI_FETIDP;
  opt->scaling = FETI_SCALING_K;
  opt->krylov = FETI_RRS;
  opt->precision = FETI_FP64;
  opt->max_iter = 500;
  opt->dedup_modules = 1;
  opt->tol = 1e-6;
  opt->rr_tol = 1e-10;
  opt->inner_tol = 0.0;                 // automatic (1e-2)
  opt->max_refine = 30;
  opt->precond = FETI_PRECOND_DIRICHLET;
  opt->primal = FETI_PRIMAL_CORNERS;
  opt->primal_jump = 10.0;
  opt->refine = FETI_REFINE_DUAL;
  return FETI_OK;
}

feti_status feti_create(feti_ctx** out, const feti_options* opt, void* stream) {
  if (!out) return FETI_EINVAL;
  *out = nullptr;
  feti_options o;
  feti_options_default(&o);
  if (opt) o = *opt;
  if ((o.method != FETI_TFETI && o.method != FETI_FETIDP) ||
      (o.scaling != FETI_SCALING_K && o.scaling != FETI_SCALING_MULT) ||
      (o.krylov < FETI_PCG || o.krylov > FETI_RRS) || o.max_iter < 0 || !(o.tol >= 0.0) || !(o.rr_tol >= 0.0))
    return FETI_EINVAL;
  if (o.precision < FETI_FP64 || o.precision > FETI_BF16X3) return FETI_EINVAL;
  if (o.precision != FETI_FP64 && !(o.inner_tol >= 0.0 && o.inner_tol < 1.0 && o.max_refine > 0)) return FETI_EINVAL;
  if (o.precond < FETI_PRECOND_DIRICHLET || o.precond > FETI_PRECOND_SUPERLUMPED) return FETI_EINVAL;
  if (o.primal != FETI_PRIMAL_CORNERS && o.primal != FETI_PRIMAL_EDGES && o.primal != FETI_PRIMAL_ADAPTIVE)
    return FETI_EINVAL;
  if (o.primal != FETI_PRIMAL_CORNERS && o.method != FETI_FETIDP) return FETI_EINVAL;
  if (o.primal != FETI_PRIMAL_CORNERS && o.precond != FETI_PRECOND_DIRICHLET) return FETI_ENOTSUP;
  if (o.primal == FETI_PRIMAL_ADAPTIVE && !(o.primal_jump >= 1.0)) return FETI_EINVAL;
  if (o.refine != FETI_REFINE_DUAL && o.refine != FETI_REFINE_PRIMAL) return FETI_EINVAL;
  feti_ctx* ctx = new (std::nothrow) feti_ctx;
  if (!ctx) return FETI_ENOMEM;
  Ctx& c = ctx->c;
  c.opt = o;
  c.stream = static_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&c.device) != cudaSuccess || cudaMallocHost(&c.h_pin, 64 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return FETI_ECUDA;
  }
  *out = ctx;
  return FETI_OK;
}

void feti_destroy(feti_ctx* ctx) {
  if (!ctx) return;
  if (ctx->c.cap_stream) cudaStreamDestroy(ctx->c.cap_stream);
  if (ctx->c.cap_event) cudaEventDestroy(ctx->c.cap_event);
  free_all(ctx->c);
  if (ctx->c.h_pin) cudaFreeHost(ctx->c.h_pin);
  delete ctx;
}

const char* feti_last_error(const feti_ctx* ctx) { return ctx ? ctx->c.err.c_str() : "null context"; }

feti_status feti_set_allocator(feti_ctx* ctx, const feti_allocator* a) {
  if (!ctx) return FETI_EINVAL;
  Ctx& c = ctx->c;
  c.err.clear();
  if (!c.allocs.empty() || c.d_tiles) {
    c.err = "feti_set_allocator: the context already holds device memory (install the allocator before set-up)";
    return FETI_ESTATE;
  }
  if (!a) {
    c.have_user_alloc = 0;
    c.user_alloc = feti_allocator{};
    return FETI_OK;
  }
  if (!a->alloc || !a->free) {
    c.err = "feti_set_allocator: null callback";
    return FETI_EINVAL;
  }
  c.user_alloc = *a;
  c.have_user_alloc = 1;
  return FETI_OK;
}

}  // extern "C"

// Set-up of one problem or of a batch of independent problems (merged into
// one description: every launch covers the whole batch).
static feti_status setup_impl(Ctx& c, const feti_problem* probs, int n) {
  c.err.clear();
  if (n < 1) { c.err = "n_problems must be >= 1"; return FETI_EINVAL; }
  for (int q = 0; q < n; ++q)
    if (!probs[q].rho || !probs[q].dirichlet || !probs[q].f) { c.err = "null problem array"; return FETI_EINVAL; }
  if (n > 1 && (c.opt.method != FETI_FETIDP || c.opt.krylov == FETI_FO || c.opt.precision != FETI_FP64)) {
    c.err = "batches of problems are solved with FETI-DP, PCG or the simultaneous variant, and FP64 block products";
    return FETI_ENOTSUP;
  }
  free_all(c);
  if (c.cap_stream) { cudaStreamDestroy(c.cap_stream); c.cap_stream = nullptr; }
  if (c.cap_event) { cudaEventDestroy(c.cap_event); c.cap_event = nullptr; }
  {
    Ctx fresh;
    fresh.opt = c.opt;
    fresh.stream = c.stream;
    fresh.device = c.device;
    fresh.h_pin = c.h_pin;
    fresh.user_alloc = c.user_alloc;
    fresh.have_user_alloc = c.have_user_alloc;
    c = std::move(fresh);
  }
  std::vector<HostProblem> parts(n);
  std::vector<double> rho_all;
  for (int q = 0; q < n; ++q) {
    const feti_problem* prob = &probs[q];
    if (prob->dim != 2 && prob->dim != 3) { c.err = "dim must be 2 or 3"; return FETI_EINVAL; }
    int64_t nel = 1;
    for (int a = 0; a < prob->dim && a < 3; ++a) nel *= (int64_t)prob->tiles[a] * prob->elems[a];
    std::vector<double> rho_h(nel);
    if (prob->on_device) CU(cudaMemcpy(rho_h.data(), prob->rho, nel * sizeof(double), cudaMemcpyDeviceToHost));
    else std::memcpy(rho_h.data(), prob->rho, nel * sizeof(double));
    for (double r : rho_h)
      if (!(r >= 0.0 && r <= 1.0)) { c.err = "densities must lie in [0, 1]"; return FETI_EINVAL; }
    std::string msg = build_host_problem(*prob, c.opt.method, c.opt.dedup_modules, rho_h.data(), parts[q],
                                         c.opt.primal, c.opt.primal_jump);
    if (!msg.empty()) { c.err = (n > 1 ? "problem " + std::to_string(q) + ": " : std::string()) + msg; return FETI_EINVAL; }
    rho_all.insert(rho_all.end(), rho_h.begin(), rho_h.end());
  }
  if (n == 1) {
    c.hp = std::move(parts[0]);
  } else {
    std::string msg = merge_host_problems(parts, c.hp);
    if (!msg.empty()) { c.err = msg; return FETI_EINVAL; }
  }
  HostProblem& hp = c.hp;
  // ---- problem arrays ----
  TRY(upload(c, c.d_rho, rho_all));
  TRY(dalloc(c, c.d_E, hp.n_elements));
  TRY(dalloc(c, c.d_fglob, hp.n_dofs));
  for (int q = 0; q < n; ++q)
    CU(cudaMemcpy(c.d_fglob + hp.prob_dof_off[q], probs[q].f,
                  (hp.prob_dof_off[q + 1] - hp.prob_dof_off[q]) * sizeof(double),
                  probs[q].on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
  c.h_k0.assign((size_t)(hp.dim == 2 ? 64 : 576), 0.0);
  element_stiffness_host(hp.dim, hp.nu, c.h_k0.data());
  TRY(upload(c, c.d_k0, c.h_k0));
  TRY(upload(c, c.d_dirichlet, hp.dirichlet));
  // ---- types ----
  c.h_types.resize(hp.types.size());
  c.max_nb = 1; c.max_nc = 1;
  for (size_t t = 0; t < hp.types.size(); ++t) {
    const StructType& T = hp.types[t];
    std::vector<int> ci(T.n_loc);
    for (int a = 0; a < T.n_loc; ++a) ci[a] = (T.cls[a] << 24) | std::max(T.idx[a], 0);
    DevType d{};
    d.n_loc = T.n_loc; d.n_i = T.n_i; d.n_b = T.n_b; d.n_c = T.n_c; d.bw = T.bw;
    for (int a = 0; a < 3; ++a) { d.e[a] = T.e[a]; d.ln[a] = T.ln[a]; }
    int *p1, *p2, *p3, *p4;
    TRY(upload(c, p1, ci));
    TRY(upload(c, p2, T.ilist));
    TRY(upload(c, p3, T.blist));
    TRY(upload(c, p4, T.clist));
    d.cls_idx = p1; d.ilist = p2; d.blist = p3; d.clist = p4;
    d.n_avg = (int)T.avg_c.size();
    if (d.n_avg > 0) {
      int *a1, *a2, *a3;
      TRY(upload(c, a1, T.avg_c));
      TRY(upload(c, a2, T.avg_off));
      TRY(upload(c, a3, T.avg_b));
      d.avg_c = a1; d.avg_off = a2; d.avg_b = a3;
      c.max_avg = std::max(c.max_avg, d.n_avg);
    }
    if (hp.n_rbm > 0) {
      std::vector<double> raw, hat;
      type_rigid_modes(hp, T, raw, hat);
      double *r1, *r2;
      TRY(upload(c, r1, raw));
      TRY(upload(c, r2, hat));
      d.Rraw = r1; d.Rhat = r2;
    }
    c.h_types[t] = d;
    c.max_nb = std::max(c.max_nb, T.n_b);
    c.max_nc = std::max(c.max_nc, T.n_c);
  }
  TRY(upload(c, c.d_types, c.h_types));
  // ---- modules: memory layout ----
  c.n_mod = (int)hp.module_rep.size();
  c.h_mods.resize(c.n_mod);
  int64_t off = 0;
  for (int m = 0; m < c.n_mod; ++m) {
    const StructType& T = hp.types[hp.module_type[m]];
    const int64_t W = T.bw + 1, nbc = T.n_bc();
    DevModule M{};
    M.type = hp.module_type[m];
    M.rep = hp.module_rep[m];
    M.lcol = off; off = align32(off + (int64_t)T.n_i * W);
    M.lrow = off; off = align32(off + (int64_t)T.n_i * W);
    M.rdiag = off; off = align32(off + T.n_i);
    M.Y = off; off = align32(off + (int64_t)T.n_i * nbc);
    M.S = off; off = align32(off + nbc * nbc);
    M.W = off; off = align32(off + nbc * nbc);
    M.Li = off; off = align32(off + (int64_t)T.n_b * T.n_b);
    M.F = off; off = align32(off + (int64_t)T.n_b * T.n_b);
    M.Frc = off; off = align32(off + (int64_t)T.n_b * T.n_c);
    M.Kb = off; off = align32(off + (int64_t)T.n_c * T.n_c);
    M.Rb = off; off = align32(off + (int64_t)T.n_b * hp.n_rbm);
    M.Kl = -1;
    if (c.opt.precond == FETI_PRECOND_LUMPED) { M.Kl = off; off = align32(off + (int64_t)T.n_b * T.n_b); }
    c.h_mods[m] = M;
  }
  c.modmem_len = off;
  TRY(dalloc(c, c.d_modmem, (size_t)off));
  TRY(upload(c, c.d_mods, c.h_mods));
  // ---- subdomains ----
  c.h_subs.resize(hp.n_sub);
  c.h_ioff.assign(hp.n_sub + 1, 0);
  std::vector<int64_t> coff(hp.n_sub);
  for (int s = 0; s < hp.n_sub; ++s) {
    const StructType& Ts = hp.types[hp.sub_type[s]];
    c.fl_F += 2.0 * Ts.n_b * (double)Ts.n_b;
    c.fl_FrcT += 2.0 * Ts.n_c * (double)Ts.n_b;
    c.fl_Frc += 2.0 * Ts.n_b * (double)Ts.n_c;
    DevSub S{};
    S.module = hp.sub_module[s];
    S.type = hp.sub_type[s];
    S.b_off = hp.b_off[s];
    S.c_off = hp.c_off.empty() ? 0 : hp.c_off[s];
    {
      const int q = hp.sub_prob[s];
      const int sl = s - hp.prob_sub_off[q];                  // index inside its problem
      const int t0 = hp.prob_nel[3 * q] / Ts.e[0], t1 = hp.prob_nel[3 * q + 1] / Ts.e[1];
      S.tile[0] = sl % t0;
      S.tile[1] = (sl / t0) % t1;
      S.tile[2] = sl / (t0 * t1);
      S.prob = q;
      S.loc_off = hp.loc_off[s];
      S.e_off = hp.prob_el_off[q];
      for (int a = 0; a < 3; ++a) S.nel[a] = hp.prob_nel[3 * q + a];
    }
    c.h_subs[s] = S;
    coff[s] = S.c_off;
    c.h_ioff[s + 1] = c.h_ioff[s] + align32(hp.types[S.type].n_i);
  }
  TRY(upload(c, c.d_subs, c.h_subs));
  TRY(upload(c, c.d_ioff, c.h_ioff));
  TRY(upload(c, c.d_c_off, coff));
  c.n_c_total = hp.c_off.empty() ? 0 : hp.c_off[hp.n_sub];
  // ---- maps ----
  TRY(upload(c, c.d_lam_b0, hp.lam_b0));
  TRY(upload(c, c.d_lam_b1, hp.lam_b1));
  TRY(upload(c, c.d_lam_s0, hp.lam_s0));
  TRY(upload(c, c.d_lam_s1, hp.lam_s1));
  TRY(upload(c, c.d_lam_group, hp.lam_group));
  TRY(upload(c, c.d_group_off, hp.group_off));
  TRY(upload(c, c.d_group_b, hp.group_b));
  TRY(upload(c, c.d_b2l_off, hp.b2l_off));
  TRY(upload(c, c.d_b2l_lam, hp.b2l_lam));
  TRY(upload(c, c.d_b2l_sign, hp.b2l_sign));

  TRY(upload(c, c.d_b_sub, hp.b_sub));
  {
    std::vector<int> lcol(hp.b_sub.size());
    for (size_t b = 0; b < lcol.size(); ++b) lcol[b] = hp.b_sub[b] - hp.prob_sub_off[hp.sub_prob[hp.b_sub[b]]];
    TRY(upload(c, c.d_b_lcol, lcol));
  }
  TRY(upload(c, c.d_c_glob, hp.c_glob));
  std::vector<int> csub(c.n_c_total);
  for (int s = 0; s < hp.n_sub; ++s)
    for (int64_t k = hp.c_off.empty() ? 0 : hp.c_off[s]; !hp.c_off.empty() && k < hp.c_off[s + 1]; ++k) csub[k] = s;
  TRY(upload(c, c.d_c_sub, csub));
  if (c.max_avg > 0) {
    std::vector<int> iota(std::max<int64_t>(c.n_c_total, 1));
    for (size_t k = 0; k < iota.size(); ++k) iota[k] = (int)k;
    TRY(upload(c, c.d_c_iota, iota));
    TRY(dalloc(c, c.d_ucl, (size_t)std::max<int64_t>(c.n_c_total, 1)));
  }
  TRY(upload(c, c.d_prim_off, hp.prim_off.empty() ? std::vector<int>{0} : hp.prim_off));
  TRY(upload(c, c.d_prim_src, hp.prim_src));
  TRY(upload(c, c.d_load_src, hp.load_src));
  TRY(upload(c, c.d_dof_copy_off, hp.dof_copy_off));
  TRY(upload(c, c.d_dof_copy, hp.dof_copy));
  // ---- vectors ----
  const int64_t nbt = hp.n_b_total, nl = hp.n_lam;
  TRY(dalloc(c, c.d_diagKb, nbt));
  TRY(dalloc(c, c.d_w0, nl));
  TRY(dalloc(c, c.d_w1, nl));
  TRY(dalloc(c, c.d_floc, (size_t)hp.n_loc_total));
  TRY(dalloc(c, c.d_h, c.h_ioff[hp.n_sub]));
  TRY(dalloc(c, c.d_t, c.h_ioff[hp.n_sub]));
  TRY(dalloc(c, c.d_ft, nbt + c.n_c_total));
  TRY(dalloc(c, c.d_pb0, nbt));
  TRY(dalloc(c, c.d_pb1, nbt));
  TRY(dalloc(c, c.d_pbh, nbt));
  c.n_coarse = hp.method == FETI_FETIDP ? hp.n_primal : hp.n_rbm * hp.n_sub;
  const int64_t nco = std::max(c.n_coarse, 1);
  // coarse blocks: one per problem (FETI-DP), one for TFETI
  c.h_kbar_off.assign(hp.n_prob + 1, 0);
  c.max_np = 0;
  std::vector<int> row_prob(std::max(hp.n_primal, 1), 0);
  for (int q = 0; q < hp.n_prob; ++q) {
    const int64_t npq = hp.method == FETI_FETIDP ? hp.prob_primal_off[q + 1] - hp.prob_primal_off[q] : nco;
    c.h_kbar_off[q + 1] = c.h_kbar_off[q] + npq * npq;
    c.max_np = std::max<int>(c.max_np, (int)npq);
    for (int r = hp.prob_primal_off[q]; r < hp.prob_primal_off[q + 1]; ++r) row_prob[r] = q;
  }
  const int64_t kb_len = std::max<int64_t>(c.h_kbar_off[hp.n_prob], 1);
  c.fl_coarse = hp.method == FETI_FETIDP ? 2.0 * (double)c.h_kbar_off[hp.n_prob] : 0.0;
  c.bytes_S = 0.0;
  c.bytes_apply1 = 0.0;
  for (int q = 0; q < (int)hp.module_type.size(); ++q) {
    const double nb = hp.types[hp.module_type[q]].n_b, nc = hp.types[hp.module_type[q]].n_c;
    c.bytes_S += 8.0 * nb * nb;
    c.bytes_apply1 += 8.0 * (nb * nb + (hp.method == FETI_FETIDP ? nb * nc : 0.0));
  }
  c.bytes_apply1 += 8.0 * ((hp.method == FETI_FETIDP ? (double)c.h_kbar_off[hp.n_prob] : 0.0) +
                           2.0 * hp.n_lam + 2.0 * hp.n_b_total);
  TRY(dalloc(c, c.d_Kbar, kb_len));
  TRY(dalloc(c, c.d_Kbar_L, kb_len));
  TRY(dalloc(c, c.d_Kbar_inv, kb_len));
  if (c.opt.precision != FETI_FP64 && hp.method == FETI_FETIDP && hp.n_prob == 1 && hp.n_primal > 0)
    TRY(dalloc(c, c.d_Kbar_inv32, kb_len));
  TRY(upload(c, c.d_kbar_off, c.h_kbar_off));
  TRY(upload(c, c.d_row_prob, row_prob));
  TRY(upload(c, c.d_prob_el_off, hp.prob_el_off));
  TRY(upload(c, c.d_prob_dof_off, hp.prob_dof_off));
  TRY(upload(c, c.d_prob_lam_off, hp.prob_lam_off));
  TRY(upload(c, c.d_prob_nel, hp.prob_nel));
  TRY(upload(c, c.d_prob_primal_off, hp.prob_primal_off));
  {
    std::vector<int> lam_prob(hp.n_lam);
    for (int q = 0; q < hp.n_prob; ++q)
      for (int64_t l = hp.prob_lam_off[q]; l < hp.prob_lam_off[q + 1]; ++l) lam_prob[l] = q;
    TRY(upload(c, c.d_lam_prob, lam_prob));
  }
  TRY(dalloc(c, c.d_fbar, std::max(hp.n_primal, 1)));
  TRY(dalloc(c, c.d_coarse_work, (size_t)128 * nco + (size_t)((nco + 63) / 64) * 4096));
  if (hp.method == FETI_TFETI) {
    TRY(dalloc(c, c.d_gwork, (size_t)kGgtCols * nl));
    TRY(dalloc(c, c.d_e, nco));
    TRY(dalloc(c, c.d_alpha, nco));
  }
  if (c.opt.precision != FETI_FP64) {
    // tensor-core operand layout: module rows in one arena, padded interface space
    std::vector<int> frow(c.n_mod);
    int64_t rows = 0;
    for (int q = 0; q < c.n_mod; ++q) {
      frow[q] = (int)rows;
      rows += c.h_types[c.h_mods[q].type].n_b;
    }
    c.tc_aug = (hp.method == FETI_FETIDP && hp.n_primal > 0 && c.max_nc <= 64) ? 1 : 0;
    if (hp.method == FETI_FETIDP && hp.n_primal > 0 && !c.tc_aug) {
      c.err = "precision form: more than 64 primal DOFs per subdomain";
      return FETI_ENOTSUP;
    }
    const int kc = tc_chunk(c.opt.precision);
    std::vector<int64_t> bpad(hp.n_sub);
    int64_t nbp = 0, kmax = kc;
    for (int s = 0; s < hp.n_sub; ++s) {
      const DevType& T = c.h_types[c.h_subs[s].type];
      bpad[s] = nbp;
      const int kx = tc_k_extent(T.n_b, T.n_c, c.tc_aug, kc);
      nbp += kx;
      kmax = std::max<int64_t>(kmax, kx);
    }
    if (rows >= (int64_t)1 << 31 || nbp >= (int64_t)1 << 31) {
      c.err = "precision form: interface space too large for 32-bit tensor coordinates";
      return FETI_ENOTSUP;
    }
    c.fa_pitch = kmax;
    c.fl_tc = 0.0;
    const int64_t parts = split_precision(c.opt.precision) ? 2 : 1;
    const int64_t eb = (int64_t)tc_elem_bytes(c.opt.precision);
    c.tc_bytes_col = 0;
    for (int s = 0; s < hp.n_sub; ++s) {
      const DevType& T = c.h_types[c.h_subs[s].type];
      const int ncx = c.tc_aug ? T.n_c : 0;
      c.fl_tc += 2.0 * T.n_b * (T.n_b + ncx);
      c.tc_bytes_col += (int64_t)(T.n_b + ncx) * eb * parts + (int64_t)T.n_b * 4;
    }
    c.tc_bytes_f = 0;
    for (int q = 0; q < c.n_mod; ++q) {
      const DevType& T = c.h_types[c.h_mods[q].type];
      c.tc_bytes_f += (int64_t)T.n_b * (T.n_b + (c.tc_aug ? T.n_c : 0)) * eb * parts;
    }
    // FETI-DP: a block of tile rows per module holding Frc_hat^T, for the corner
    // reduction on the tensor cores
    c.n_ctiles_rows = c.tc_aug ? 1 : 0;
    c.fcrow0 = (int)rows;
    if (c.tc_aug) rows += (int64_t)c.n_mod * tc_tile_rows();
    if (rows >= (int64_t)1 << 31) {
      c.err = "precision form: operand arena too large for 32-bit tensor coordinates";
      return FETI_ENOTSUP;
    }
    c.fa_rows = std::max<int64_t>(rows, 1);
    c.nbp_total = std::max<int64_t>(nbp, kc);
    TRY(upload(c, c.d_frow, frow));
    TRY(upload(c, c.d_bpad, bpad));
    {
      // the precision form's operand built from the multiplier side (ranges of
      // consecutive rows, the slots whose rows each range holds)
      std::vector<int64_t> pos_of_b(std::max<int64_t>(hp.n_b_total, 1));
      for (int64_t b = 0; b < hp.n_b_total; ++b) {
        const int s = hp.b_sub[b];
        pos_of_b[b] = bpad[s] + (b - hp.b_off[s]);
      }
      SpreadTables sp;
      const std::string msg = build_spread_tables(hp, pos_of_b, kSpreadRows, sp);
      if (!msg.empty()) { c.err = "precision form: " + msg; return FETI_ENOTSUP; }
      c.n_spread_ranges = (int)sp.row0.size() - 1;
      c.n_spread_slots = (int)sp.slot_pos.size();
      TRY(upload(c, c.d_sp_row0, sp.row0));
      TRY(upload(c, c.d_sp_slot_off, sp.slot_off));
      TRY(upload(c, c.d_sp_pos, sp.slot_pos));
      TRY(upload(c, c.d_sp_b, sp.slot_b));
      TRY(upload(c, c.d_sp_ent_off, sp.ent_off));
      TRY(upload(c, c.d_sp_ent, sp.ent));
      TRY(dalloc(c, c.d_sp_sd, std::max<size_t>(sp.slot_pos.size(), 1)));
    }
    const size_t fa_bytes = (size_t)(c.fa_rows * c.fa_pitch) * tc_elem_bytes(c.opt.precision);
    TRY(dalloc_bytes(c, c.d_fa_hi, fa_bytes));
    CU(cudaMemset(c.d_fa_hi, 0, fa_bytes));
    if (split_precision(c.opt.precision)) {
      TRY(dalloc_bytes(c, c.d_fa_lo, fa_bytes));
      CU(cudaMemset(c.d_fa_lo, 0, fa_bytes));
    }
    TRY(dalloc(c, c.d_fmem, (size_t)c.modmem_len));
    TRY(dalloc(c, c.d_sqrtDF, nbt));
    TRY(dalloc(c, c.d_sqrtDS, nbt));
    TRY(dalloc(c, c.d_rout, nl));
    TRY(dalloc(c, c.d_zout, nl));
    TRY(dalloc(c, c.d_dl, nl));           // the best refined multipliers so far
  }
  TRY(dalloc(c, c.d_d, nl));
  TRY(dalloc(c, c.d_lam0, nl));
  TRY(dalloc(c, c.d_lam, nl));
  TRY(dalloc(c, c.d_uloc, (size_t)hp.n_loc_total));
  TRY(dalloc(c, c.d_uglob, hp.n_dofs));
  TRY(dalloc(c, c.d_scalar, 64));
  TRY(dalloc(c, c.d_status, 4));
  TRY(dalloc(c, c.d_kdev, 4));
  TRY(dalloc(c, c.d_perm, 1024));
  TRY(dalloc(c, c.d_red, 1024));
  TRY(dalloc(c, c.d_bstate, (size_t)hp.n_prob * (6 + 2 * 16) + 16));
  TRY(dalloc(c, c.d_bflags, (size_t)hp.n_prob * 3 + 4));
  CU(cudaMemset(c.d_status, 0, 4 * sizeof(int)));
  // ---- per-module descriptors for the factorization ----
  {
    std::vector<GemmDesc> schur(c.n_mod), frc(c.n_mod), kb(c.n_mod);
    std::vector<DenseDesc> dd(c.n_mod);
    for (int m = 0; m < c.n_mod; ++m) {
      const DevModule& M = c.h_mods[m];
      const StructType& T = hp.types[M.type];
      const int nbc = T.n_bc();
      GemmDesc g{};   // S -= Y^T Y
      g.A = c.d_modmem + M.Y; g.B = c.d_modmem + M.Y; g.C = c.d_modmem + M.S;
      g.M = nbc; g.N = nbc; g.K = T.n_i;
      g.ars = 1; g.acs = nbc; g.brs = nbc; g.bcs = 1; g.crs = nbc; g.ccs = 1;
      schur[m] = g;
      GemmDesc f{};   // F_rc = L_bb^{-T} L_cb^T  (= S_bb^{-1} S_bc)
      f.A = c.d_modmem + M.Li; f.B = c.d_modmem + M.W + (int64_t)T.n_b * nbc; f.C = c.d_modmem + M.Frc;
      f.M = T.n_b; f.N = T.n_c; f.K = T.n_b;
      f.ars = 1; f.acs = T.n_b; f.brs = 1; f.bcs = nbc; f.crs = std::max(T.n_c, 1); f.ccs = 1;
      frc[m] = f;
      GemmDesc k{};   // Kb -= S_cb Frc
      k.A = c.d_modmem + M.S + (int64_t)T.n_b * nbc; k.B = c.d_modmem + M.Frc; k.C = c.d_modmem + M.Kb;
      k.M = T.n_c; k.N = T.n_c; k.K = T.n_b;
      k.ars = nbc; k.acs = 1; k.brs = std::max(T.n_c, 1); k.bcs = 1; k.crs = std::max(T.n_c, 1); k.ccs = 1;
      kb[m] = k;
      c.fl_schur += 2.0 * nbc * (double)nbc * T.n_i;
      c.fl_frcmake += 2.0 * T.n_b * (double)T.n_c * T.n_b;
      c.fl_kbmake += 2.0 * T.n_c * (double)T.n_c * T.n_b;
      DenseDesc q{};
      q.A = c.d_modmem + M.W; q.Linv = c.d_modmem + M.Li; q.out = c.d_modmem + M.F;
      q.n = T.n_b; q.ld = nbc; q.tag = m; q.n_full = nbc;
      dd[m] = q;
    }
    TRY(upload(c, c.d_gemm_schur, schur));
    TRY(upload(c, c.d_gemm_frcmake, frc));
    TRY(upload(c, c.d_gemm_kbmake, kb));
    TRY(upload(c, c.d_dense_mod, dd));
    std::vector<DenseDesc> dc(1);
    dc[0].A = c.d_Kbar; dc[0].Linv = c.d_Kbar_L; dc[0].out = c.d_Kbar_inv;
    dc[0].n = c.n_coarse; dc[0].ld = c.n_coarse; dc[0].tag = 999999; dc[0].n_full = c.n_coarse;
    TRY(upload(c, c.d_dense_coarse, dc));
    if (hp.n_prob > 1) {
      std::vector<DenseDesc> db(hp.n_prob);
      for (int q = 0; q < hp.n_prob; ++q) {
        const int npq = hp.prob_primal_off[q + 1] - hp.prob_primal_off[q];
        db[q].A = c.d_Kbar + c.h_kbar_off[q];
        db[q].Linv = c.d_Kbar_L + c.h_kbar_off[q];
        db[q].out = c.d_Kbar_inv + c.h_kbar_off[q];
        db[q].n = npq; db[q].ld = npq; db[q].tag = 900000 + q; db[q].n_full = npq;
      }
      TRY(upload(c, c.d_dense_coarse_batch, db));
      // the coarse-solve descriptors point at the block buffers: written by
      // build_block_descs whenever those are (re)allocated
      TRY(dalloc(c, c.d_gemm_coarse, (size_t)hp.n_prob));
    }
  }
  // direction-block buffers: one column per subdomain for the simultaneous
  // variant, a few for PCG / FO (grown on demand by feti_apply_dual)
  // (batches apply their direction blocks in column chunks of BATCH_CHUNK)
  TRY(ensure_blocks(c, hp.n_prob > 1 ? BATCH_CHUNK : c.opt.krylov == FETI_RRS ? std::max(64, hp.n_sub) : 64));
  TRY(sync_check(c));
  c.state = 1;
  return FETI_OK;
}

extern "C" {

feti_status feti_setup_subdomains(feti_ctx* ctx, const feti_problem* prob) {
  if (!ctx || !prob) return FETI_EINVAL;
  return setup_impl(ctx->c, prob, 1);
}

feti_status feti_setup_batch(feti_ctx* ctx, const feti_problem* probs, int n_problems) {
  if (!ctx || !probs) return FETI_EINVAL;
  return setup_impl(ctx->c, probs, n_problems);
}

feti_status feti_set_density(feti_ctx* ctx, const double* rho, int on_device) {
  if (!ctx || !rho) return FETI_EINVAL;
  Ctx& c = ctx->c;
  if (c.state < 1) { c.err = "feti_set_density before feti_setup_subdomains"; return FETI_ESTATE; }
  if (c.opt.dedup_modules && c.n_mod < c.hp.n_sub) {
    c.err = "feti_set_density needs a context created with dedup_modules = 0 (module sharing depends on rho)";
    return FETI_ENOTSUP;
  }
  CU(cudaMemcpyAsync(c.d_rho, rho, c.hp.n_elements * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c.stream));
  TRY(sync_check(c));
  c.state = 1;
  return FETI_OK;
}

}  // extern "C"

// The load-dependent part of Eqs. 7 / 12 for the current global load c.d_fglob
// (the matrix parts are factorized): f^s, h = L^{-1} f_i, f~ = f_bc - Y^T h;
// d = B K^# f (FETI-DP: d_r - F_rc Kbar_cc^{-1} fbar with fbar_c = sum_s B_c^sT
// (f~_c - F_rc,s^T f~_b)); TFETI: e = -R^T f and lambda_0 = G^T (G G^T)^{-1} e.
static feti_status load_rhs(Ctx& c) {
  const HostProblem& hp = c.hp;
  cudaStream_t st = c.stream;
  const bool dp = hp.method == FETI_FETIDP;
  CU(launch_load_gather(c, st));
  CU(launch_band_fwd_single(c, st));
  CU(launch_condense_load(c, st));
  if (c.max_avg > 0) CU(launch_edge_load(c, c.max_avg, st));      // f~ <- T^T f~
  const int64_t nl = hp.n_lam, nbt = hp.n_b_total;
  // d_r (FETI-DP) or d = B K^# f (TFETI, c = 0): x_b = F f~_b, scattered
  CU(batched_gemv(c, 0, c.d_ft, c.d_pb0, 0.0, st));
  CU(scatter_b_to_lam(c, c.d_pb0, 1, c.d_d, nl, st));
  CU(cudaMemsetAsync(c.d_lam0, 0, nl * sizeof(double), st));
  if (dp) {
    const int np = hp.n_primal;
    CU(cudaMemcpyAsync(c.d_Xb, c.d_ft, nbt * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CU(corner_reduce(c, c.d_Xb, 1, c.d_Cb, c.d_Vraw, st));
    CU(corner_gather_vec(c, c.d_ft + nbt, c.d_fbar, st));
    CU(axpby(np, -1.0, c.d_Vraw, 1.0, c.d_fbar, st));
    // d = d_r - F_rc Kbar^{-1} fbar
    CU(coarse_matvec(c, c.d_fbar, c.d_V, st));
    CU(cudaMemsetAsync(c.d_Yb, 0, nbt * sizeof(double), st));
    CU(corner_expand(c, c.d_V, 1, c.d_Vc, c.d_Yb, st));
    CU(scatter_b_to_lam(c, c.d_Yb, 1, c.d_lam, nl, st));
    CU(axpby(nl, -1.0, c.d_lam, 1.0, c.d_d, st));
  } else {
    const int nco = c.n_coarse;
    CU(tfeti_build_e(c, c.d_e, st));
    CU(gemv_dense(c.d_Kbar_inv, nco, nco, c.d_e, c.d_alpha, 0.0, st));
    // lambda_0 = G^T alpha: the G^T kernel subtracts, so from 0 it leaves -G^T alpha
    CU(tfeti_Gt_sub(c, c.d_alpha, 1, c.d_lam0, nl, st));
    CU(axpby(nl, -1.0, c.d_lam0, 0.0, c.d_lam0, st));
  }
  return FETI_OK;
}

extern "C" {

feti_status feti_factorize(feti_ctx* ctx) {
  if (!ctx) return FETI_EINVAL;
  Ctx& c = ctx->c;
  c.err.clear();
  if (c.state < 1) { c.err = "feti_factorize before feti_setup_subdomains"; return FETI_ESTATE; }
  const HostProblem& hp = c.hp;
  cudaStream_t st = c.stream;
  const bool dp = hp.method == FETI_FETIDP;
  PhaseScope phase(st, FETI_PHASE_FACTOR, 0.0);
  // local stiffness (Eqs. 1, 3)
  CU(launch_moduli(c, c.d_E, st));
  CU(cudaMemsetAsync(c.d_modmem, 0, c.modmem_len * sizeof(double), st));
  CU(launch_assemble_with(c, c.d_E, st));
  CU(launch_gather_diag_b(c, st));
  if (c.opt.precond == FETI_PRECOND_LUMPED) CU(launch_copy_kbb(c, st));   // K_bb before the Schur update
  CU(launch_scaling_weights(c, c.opt.scaling, st));
  // interior factor and Schur complement onto b + c
  CU(launch_band_chol(c, st));
  CU(launch_band_fwd_multi(c, st));
  int max_bc = 1;
  for (auto& t : hp.types) max_bc = std::max(max_bc, t.n_bc());
  CU(dgemm_batched(c.d_gemm_schur, c.n_mod, max_bc, max_bc, 0, -1.0, 1.0, st, c.fl_schur));
  if (c.max_avg > 0) CU(launch_edge_transform(c, max_bc, st));   // edge averages: S <- T^T S T
  // local dual block F_s = S_bb^{-1} (FETI-DP) or (S_b + Rhat Rhat^T)^{-1} (TFETI):
  // Cholesky of the whole b+c Schur complement with only the b columns
  // eliminated, so the corner block is Schur-complemented in the same
  // (stable) sweep instead of through the explicit inverse.
  CU(launch_copy_block(c, 0, st));
  if (!dp) CU(tfeti_add_rrt(c, st));
  {
    std::vector<DenseDesc> hd(c.n_mod);
    for (int m = 0; m < c.n_mod; ++m) {
      hd[m].n = hp.types[c.h_mods[m].type].n_b;
      hd[m].n_full = hp.types[c.h_mods[m].type].n_bc();
    }
    CU(dense_spd_inverse(c.d_dense_mod, hd.data(), c.n_mod, c.d_status, st));
  }
  TRY(sync_check(c));
  TRY(check_status(c, "subdomain factorization"));
  if (dp) {
    // the partial factorisation left Kbar_s = S_cc - S_cb S_bb^{-1} S_bc in the trailing block
    CU(dgemm_batched(c.d_gemm_frcmake, c.n_mod, c.max_nb, c.max_nc, 0, 1.0, 0.0, st, c.fl_frcmake));
    CU(launch_copy_block(c, 1, st));
  }
  if (c.opt.precision != FETI_FP64) CU(tc_prepare(c, st));
  if (hp.n_prob > 1 && c.gemv_cfg == 0) CU(autotune_gemv(c, st));   // batches: tune the matrix-vector shape
  if (dp) {
    // coarse matrix Kbar_cc (Eq. 12) and its inverse
    CU(coarse_assemble_batch(c, st));
    CU(coarse_inverse(c));
    if (c.d_Kbar_inv32) CU(tc_coarse_prepare(c, st));
  } else {
    // TFETI coarse space: G = -R^T B^T (applied, never stored) and G G^T
    TRY(ensure_blocks(c, kGgtCols));
    CU(tfeti_ggt(c, c.d_gwork, kGgtCols, c.d_ct1, c.d_ct2, c.d_Xb, c.d_Kbar, st));
    CU(coarse_inverse(c));
  }
  TRY(load_rhs(c));
  TRY(sync_check(c));
  TRY(check_status(c, "coarse factorization"));
  c.state = 2;
  c.have_solution = 0;
  return FETI_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- Algorithm 1
static feti_status ensure_krylov(Ctx& c, int mmax) {
  if (mmax <= c.kr_cap) return FETI_OK;
  const int64_t nl = c.hp.n_lam;
  TRY(dalloc(c, c.d_r, nl));
  TRY(dalloc(c, c.d_z, nl));
  TRY(dalloc(c, c.d_lamt, nl));
  TRY(dalloc(c, c.d_Wb, (size_t)nl * mmax));
  TRY(dalloc(c, c.d_Qb, (size_t)nl * mmax));
  TRY(dalloc(c, c.d_Delta, (size_t)mmax * mmax));
  TRY(dalloc(c, c.d_T, (size_t)mmax * mmax));
  TRY(dalloc(c, c.d_gamma, mmax));
  TRY(dalloc(c, c.d_rrwork, (size_t)rr_work_doubles(mmax)));
  c.kr_cap = mmax;
  return FETI_OK;
}

static feti_status read_scalar(Ctx& c, const double* d, double* out) {
  CU(cudaMemcpyAsync(c.h_pin, d, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  CU(cudaStreamSynchronize(c.stream));
  *out = c.h_pin[0];
  return FETI_OK;
}

// Algorithm 1 on F lambda~ = r_0 with r_0 already in c.d_r (projected);
// leaves lambda~ in c.d_lamt and the final residual in c.d_r.  lowp selects
// the tensor-core local products and the FP32 preconditioner blocks.
// eps_ref > 0 replaces the initial residual norm in the relative stopping test.
static feti_status krylov_core(Ctx& c, double tol, int max_iter, bool lowp, feti_stats& S, double eps_ref = -1.0) {
  const HostProblem& hp = c.hp;
  const int64_t nl = hp.n_lam;
  const bool multi = c.opt.krylov == FETI_RRS;
  const bool full = c.opt.krylov != FETI_PCG;
  const int m = multi ? hp.n_sub : 1;
  cudaStream_t st = c.stream;
  auto applyF = [&](const double* X, int mm, double* Y) {
    PhaseScope ph(st, FETI_PHASE_APPLY, mm * (c.fl_F + c.fl_FrcT + c.fl_Frc + c.fl_coarse));
    return lowp ? apply_dual_lowp(c, X, nl, mm, Y, nl) : apply_dual(c, X, nl, mm, Y, nl);
  };
  const double prec_bytes = c.bytes_S + 8.0 * (2.0 * nl + 2.0 * hp.n_b_total + (multi ? (double)nl * m : 0.0));
  auto precond = [&](double* Z, double* z) -> cudaError_t {
    PhaseScope ph(st, FETI_PHASE_PRECOND, prec_bytes);
    return lowp ? precond_apply_lowp(c, c.d_r, Z, nl, z, st) : precond_apply(c, c.d_r, Z, nl, z, st);
  };
  auto projectW = [&]() -> feti_status {
    if (hp.method != FETI_TFETI) return FETI_OK;
    PhaseScope ph(st, FETI_PHASE_PROJECT, 8.0 * (3.0 * (double)nl * m + 2.0 * (double)hp.n_b_total * m));
    return project(c, c.d_Wb, nl, m);
  };
  // Z_0, W_0 = P Z_0
  CU(precond(multi ? c.d_Wb : nullptr, c.d_z));
  if (!multi) CU(cudaMemcpyAsync(c.d_Wb, c.d_z, nl * sizeof(double), cudaMemcpyDeviceToDevice, st));
  TRY(projectW());
  CU(cudaMemsetAsync(c.d_lamt, 0, nl * sizeof(double), st));
  CU(dot(c.d_r, c.d_z, nl, c.d_red, c.d_scalar, st));
  double rz = 0.0;
  TRY(read_scalar(c, c.d_scalar, &rz));
  const double eps0 = eps_ref > 0.0 ? eps_ref : std::sqrt(std::max(rz, 0.0));
  double eps = std::sqrt(std::max(rz, 0.0));
  int it = 0;
  feti_status result = FETI_OK;
  c.hist_k.clear();
  while (eps > tol * eps0 && it < max_iter) {
    // Q = F W, Delta = Q^T W (symmetric: lower-triangular tiles suffice)
    TRY(applyF(c.d_Wb, m, c.d_Qb));
    int k = 0;
    {
      PhaseScope ph(st, FETI_PHASE_GRAM, (double)nl * m * (m + 1.0));
      TRY(gemm_tn(c, c.d_Qb, nl, c.d_Wb, nl, c.d_Delta, m, m, m, (int)nl, 1.0, 0.0, 1));
      // rank-revealing factorization and F-orthonormal transform: N^T [L~^{-T}; 0]
      // applied as (W with columns in pivot order) times the upper-triangular L~^{-T}
      CU(rr_cholesky(c.d_Delta, m, m, c.opt.rr_tol, c.d_rrwork, c.d_T, c.d_kdev, c.d_perm, st));
      CU(cudaMemcpyAsync(c.h_pin, c.d_kdev, sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    CU(cudaStreamSynchronize(st));
    std::memcpy(&k, c.h_pin, sizeof(int));
    S.last_rank = k;
    if (k <= 0) { result = FETI_EBREAKDOWN; c.err = "no independent search direction left"; break; }
    if ((int)c.hist_W.size() <= it) {
      double *w, *q;
      TRY(dalloc(c, w, (size_t)nl * m));
      TRY(dalloc(c, q, (size_t)nl * m));
      c.hist_W.push_back(w);
      c.hist_Q.push_back(q);
    }
    double* Wi = c.hist_W[it];
    double* Qi = c.hist_Q[it];
    c.hist_k.push_back(k);
    const double fl_T = (double)nl * k * (k + 1.0);   // 2 n nnz(U)
    // Inside a reduced-precision inner solve Q_i = F W_i is one more apply of
    // the k retained directions (tensor cores, a few ms) instead of the FP64
    // transform Q T (an n_lambda x k x k triangular product on the FP64 pipe).
    const bool q_by_apply = lowp && multi;
    {
      PhaseScope ph(st, FETI_PHASE_GRAM, (q_by_apply ? 1.0 : 2.0) * fl_T);
      TRY(gemm_perm_upper(c, c.d_Wb, nl, c.d_perm, c.d_T, m, Wi, nl, (int)nl, k, fl_T));
      if (!q_by_apply) TRY(gemm_perm_upper(c, c.d_Qb, nl, c.d_perm, c.d_T, m, Qi, nl, (int)nl, k, fl_T));
    }
    if (q_by_apply) {
      TRY(applyF(Wi, k, Qi));
      S.f_applies += k;
    }
    S.f_applies += m;
    // gamma = W^T r; lambda~ += W gamma; r -= P^T Q gamma
    {
      PhaseScope ph(st, FETI_PHASE_STEP, 8.0 * (double)nl * (3.0 * k + 4.0));
      CU(gemv_t(Wi, nl, nl, k, c.d_r, c.d_gamma, st));
      if (hp.method == FETI_TFETI) {
        CU(step_update(Wi, Qi, nl, nl, k, c.d_gamma, c.d_lamt, c.d_r, c.d_z, st));
        TRY(project(c, c.d_z, nl, 1));
        CU(axpby(nl, -1.0, c.d_z, 1.0, c.d_r, st));
      } else {
        CU(step_update(Wi, Qi, nl, nl, k, c.d_gamma, c.d_lamt, c.d_r, nullptr, st));
      }
    }
    // Z_{i+1}, W_{i+1} = P Z_{i+1}
    CU(precond(multi ? c.d_Wb : nullptr, c.d_z));
    if (!multi) CU(cudaMemcpyAsync(c.d_Wb, c.d_z, nl * sizeof(double), cudaMemcpyDeviceToDevice, st));
    TRY(projectW());
    // F-orthogonalise against the stored blocks, oldest first (modified Gram-Schmidt)
    {
      double fl_o = 0.0;
      for (int j = full ? 0 : it; j <= it; ++j) fl_o += 4.0 * (double)nl * c.hist_k[j] * m;
      PhaseScope ph(st, FETI_PHASE_ORTHO, fl_o);
      for (int j = full ? 0 : it; j <= it; ++j) {
        const int kj = c.hist_k[j];
        // Psi_j = Q_j^T W (FP64 inner products), then W -= W_j Psi_j: FP64, or
        // inside a reduced-precision inner solve an FP32 block update
        TRY(gemm_tn(c, c.hist_Q[j], nl, c.d_Wb, nl, c.d_Delta, kj, kj, m, (int)nl, 1.0, 0.0));
        if (lowp && m > 1) CU(sgemm_sub(nl, m, kj, c.hist_W[j], nl, c.d_Delta, kj, c.d_Wb, nl, st));
        else TRY(gemm_nn(c, c.hist_W[j], nl, c.d_Delta, kj, c.d_Wb, nl, (int)nl, m, kj, -1.0, 1.0));
      }
    }
    {
      PhaseScope ph(st, FETI_PHASE_STEP, 16.0 * (double)nl);
      CU(dot(c.d_r, c.d_z, nl, c.d_red, c.d_scalar, st));
    }
    TRY(read_scalar(c, c.d_scalar, &rz));
    ++it;
    eps = std::sqrt(std::max(rz, 0.0));
    if (!std::isfinite(rz)) { result = FETI_EBREAKDOWN; c.err = "NaN or Inf in the residual"; break; }
  }
  S.iterations += it;
  S.eps0 = eps0;
  S.eps = eps;
  S.converged = eps <= tol * eps0;
  return result;
}

// Device buffer of at least `need` elements: grown geometrically (the old
// buffer stays with the context until it is destroyed).
template <class T>
static feti_status grow(Ctx& c, T*& p, int64_t& cap, int64_t need) {
  if (need <= cap && p) return FETI_OK;
  const int64_t n = std::max<int64_t>(need, 2 * cap);
  TRY(dalloc(c, p, (size_t)n));
  cap = n;
  return FETI_OK;
}

// C_p = alpha A_p^T B_p + beta C_p for every entry of ops (split over K in
// fixed chunks, reduced in order).
static feti_status run_seg_tn(Ctx& c, const std::vector<SegTN>& ops, double alpha, double beta) {
  std::vector<GemmDesc> descs;
  std::vector<int64_t> coff;
  std::vector<SegRed> reds;
  int64_t plen = 0;
  int mm = 0, mn = 0;
  seg_tn_plan(ops, BATCH_KCHUNK, descs, coff, reds, &plen, &mm, &mn);
  if (descs.empty()) return FETI_OK;
  if (descs.size() > 65535 || reds.size() > 65535) { c.err = "batch too large for one launch"; return FETI_ENOTSUP; }
  TRY(grow(c, c.d_bk_split, c.bk_split_cap, plen));
  TRY(grow(c, c.d_bk_desc, c.bk_desc_cap, (int64_t)descs.size()));
  TRY(grow(c, c.d_bk_red, c.bk_red_cap, (int64_t)reds.size()));
  seg_tn_bind(descs, coff, c.d_bk_split);
  double fl = 0.0;
  for (const SegTN& o : ops) fl += 2.0 * o.M * (double)o.N * (double)o.K;
  CU(cudaMemcpyAsync(c.d_bk_desc, descs.data(), descs.size() * sizeof(GemmDesc), cudaMemcpyHostToDevice, c.stream));
  CU(cudaMemcpyAsync(c.d_bk_red, reds.data(), reds.size() * sizeof(SegRed), cudaMemcpyHostToDevice, c.stream));
  CU(seg_tn_run(c.d_bk_desc, (int)descs.size(), c.d_bk_red, (int)reds.size(), mm, mn, c.d_bk_split, alpha, beta, fl,
                c.stream));
  return FETI_OK;
}

// Batched C_p (+)= alpha A_p B_p over the descriptors in `descs` (one per row
// chunk of a problem), as one launch.
static feti_status run_row_chunks(Ctx& c, const std::vector<GemmDesc>& descs, double alpha, double beta) {
  if (descs.empty()) return FETI_OK;
  if (descs.size() > 65535) { c.err = "batch too large for one launch"; return FETI_ENOTSUP; }
  TRY(grow(c, c.d_bk_desc, c.bk_desc_cap, (int64_t)descs.size()));
  int mm = 0, mn = 0;
  double fl = 0.0;
  for (const GemmDesc& d : descs) {
    mm = std::max(mm, d.M);
    mn = std::max(mn, d.N);
    fl += d.tri == 2 ? (double)d.M * d.N * (d.N + 1.0) : 2.0 * d.M * (double)d.N * d.K;
  }
  CU(cudaMemcpyAsync(c.d_bk_desc, descs.data(), descs.size() * sizeof(GemmDesc), cudaMemcpyHostToDevice, c.stream));
  CU(dgemm_batched(c.d_bk_desc, (int)descs.size(), mm, mn, 0, alpha, beta, c.stream, fl));
  return FETI_OK;
}

// Algorithm 1 for every problem of a batch at once (FETI-DP, no projector).
// Problem p keeps its own block of m_p = N_s(p) directions, one per subdomain;
// the current blocks W, Q are stored stacked (all problems' multiplier rows,
// max_p m_p columns, problem p in its own rows and first m_p columns, so that
// one dual-operator apply covers the batch), the stored blocks W_i, Q_i packed
// per problem (n_lambda(p) x k_p each).  Every step is one launch over the
// problems still iterating: the Gram matrices (split-K, reduced in order),
// the rank-revealing factorizations, the F-orthonormal transforms, the step,
// the preconditioner and the modified Gram-Schmidt sweep over the stored
// blocks, oldest first.  Expects r_0 in c.d_r; leaves lambda~ in c.d_lamt.
static feti_status batch_rrs(Ctx& c, double tol, int max_iter, feti_stats& S) {
  const HostProblem& hp = c.hp;
  const int np = hp.n_prob;
  const int64_t nl = hp.n_lam;
  cudaStream_t st = c.stream;
  std::vector<int64_t> l0(np), nlp(np), doff(np), woff(np), moff(np);
  std::vector<int> mp(np);
  int M = 0;
  int64_t sm2 = 0, sw = 0, sm = 0;
  for (int p = 0; p < np; ++p) {
    l0[p] = hp.prob_lam_off[p];
    nlp[p] = hp.prob_lam_off[p + 1] - l0[p];
    mp[p] = hp.prob_sub_off[p + 1] - hp.prob_sub_off[p];
    M = std::max(M, mp[p]);
    doff[p] = sm2;
    woff[p] = sw;
    moff[p] = sm;
    sm2 += (int64_t)mp[p] * mp[p];
    sw += rr_work_doubles(mp[p]);
    sm += mp[p];
  }
  if (M > 1024) { c.err = "more than 1024 subdomains in one problem of the batch"; return FETI_ENOTSUP; }
  TRY(ensure_krylov(c, M));
  TRY(ensure_blocks(c, std::min(M, BATCH_CHUNK)));
  if (!c.d_bk_delta) {
    TRY(dalloc(c, c.d_bk_delta, (size_t)sm2));
    TRY(dalloc(c, c.d_bk_T, (size_t)sm2));
    TRY(dalloc(c, c.d_bk_work, (size_t)sw));
    TRY(dalloc(c, c.d_bk_gam, (size_t)sm));
    TRY(dalloc(c, c.d_bk_perm, (size_t)sm));
    TRY(dalloc(c, c.d_bk_k, (size_t)np));
    TRY(dalloc(c, c.d_bk_rz, (size_t)np));
    TRY(dalloc(c, c.d_bk_part, (size_t)np * 32));
    TRY(dalloc(c, c.d_bk_rr, (size_t)np));
    TRY(dalloc(c, c.d_bk_vec, (size_t)np));
  }
  double* W = c.d_Wb;
  double* Q = c.d_Qb;
  // local products per column chunk [j0, j0 + BATCH_CHUNK): subdomain s computes
  // only the columns its problem uses (min(N_s(p) - j0, chunk), possibly none)
  const int n_chunks = (M + BATCH_CHUNK - 1) / BATCH_CHUNK;
  {
    const int64_t nbt = hp.n_b_total;
    std::vector<GemmDesc> fc((size_t)n_chunks * hp.n_sub);
    for (int t = 0; t < n_chunks; ++t)
      for (int s2 = 0; s2 < hp.n_sub; ++s2) {
        const DevSub& Sd = c.h_subs[s2];
        const DevType& Td = c.h_types[Sd.type];
        GemmDesc g{};
        g.A = c.d_modmem + c.h_mods[Sd.module].F; g.B = c.d_Xb + Sd.b_off; g.C = c.d_Yb + Sd.b_off;
        g.M = Td.n_b; g.K = Td.n_b;
        g.N = std::max(0, std::min(BATCH_CHUNK, mp[hp.sub_prob[s2]] - t * BATCH_CHUNK));
        g.ars = Td.n_b; g.acs = 1; g.brs = 1; g.bcs = nbt; g.crs = 1; g.ccs = nbt;
        fc[(size_t)t * hp.n_sub + s2] = g;
      }
    TRY(grow(c, c.d_bk_fchunks, c.bk_fchunks_cap, (int64_t)fc.size()));
    CU(cudaMemcpy(c.d_bk_fchunks, fc.data(), fc.size() * sizeof(GemmDesc), cudaMemcpyHostToDevice));
  }
  struct ActiveF {
    Ctx& c;
    ~ActiveF() { c.gemm_F_active = nullptr; }
  } active_guard{c};
  auto read_rz = [&](std::vector<double>& rz) -> feti_status {
    CU(seg_dot2(c.d_prob_lam_off, np, c.d_r, c.d_z, nullptr, nullptr, c.d_bk_part, c.d_bk_rz, nullptr, st));
    CU(cudaMemcpyAsync(rz.data(), c.d_bk_rz, np * sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return FETI_OK;
  };
  // Z_0 (one column per subdomain, in its problem's columns), W_0 = Z_0
  CU(precond_apply_cols(c, c.d_r, W, nl, M, c.d_b_lcol, c.d_z, st));
  CU(cudaMemsetAsync(c.d_lamt, 0, nl * sizeof(double), st));
  std::vector<double> rz(np), eps0(np), eps(np);
  TRY(read_rz(rz));
  std::vector<int> active(np), iters(np, 0), conv(np), rank(np, 0), kk(np);
  std::vector<int64_t> fap(np, 0);
  for (int p = 0; p < np; ++p) {
    eps0[p] = eps[p] = std::sqrt(std::max(rz[p], 0.0));
    conv[p] = eps0[p] == 0.0;
    active[p] = eps0[p] > 0.0 && std::isfinite(eps0[p]);
  }
  std::vector<std::vector<int>> hk;          // hk[i][p]: columns of problem p in stored block i
  std::vector<std::vector<int64_t>> hoff;    // their offsets inside the packed block
  std::vector<SegTN> ops;
  std::vector<GemmDesc> rows;
  std::vector<RrDesc> rr;
  std::vector<SegVec> vec(np);
  feti_status result = FETI_OK;
  int it = 0;
  while (it < max_iter) {
    std::vector<int> act;
    int Mact = 0;
    for (int p = 0; p < np; ++p)
      if (active[p]) { act.push_back(p); Mact = std::max(Mact, mp[p]); }
    if (act.empty()) break;
    // Q = F W, BATCH_CHUNK columns at a time (the operator is block diagonal
    // over the problems, so one apply serves every problem's column j)
    {
      // the stacked apply computes all Mact columns of every subdomain (the
      // algorithmic count takes each problem's own m_p)
      double fl = 0.0;
      for (int p : act) fl += (double)mp[p] * mp[p] * (c.fl_F + c.fl_FrcT + c.fl_Frc + c.fl_coarse) / hp.n_sub;
      PhaseScope ph(st, FETI_PHASE_APPLY, fl);
      for (int j0 = 0; j0 < Mact; j0 += BATCH_CHUNK) {
        c.gemm_F_active = c.d_bk_fchunks + (int64_t)(j0 / BATCH_CHUNK) * hp.n_sub;
        TRY(apply_dual(c, W + (int64_t)j0 * nl, nl, std::min(BATCH_CHUNK, Mact - j0), Q + (int64_t)j0 * nl, nl));
      }
      c.gemm_F_active = nullptr;
    }
    {
      double fl = 0.0;
      for (int p : act) fl += (double)nlp[p] * mp[p] * (mp[p] + 1.0);
      PhaseScope ph(st, FETI_PHASE_GRAM, fl);
      // Delta_p = Q_p^T W_p (lower tiles)
      ops.clear();
      for (int p : act)
        ops.push_back(SegTN{Q + l0[p], nl, W + l0[p], nl, c.d_bk_delta + doff[p], mp[p], mp[p], mp[p], nlp[p], 1});
      TRY(run_seg_tn(c, ops, 1.0, 0.0));
      // rank-revealing factorizations
      rr.clear();
      for (int p : act)
        rr.push_back(RrDesc{c.d_bk_delta + doff[p], mp[p], mp[p], c.d_bk_work + woff[p], c.d_bk_T + doff[p],
                            c.d_bk_k + p, c.d_bk_perm + moff[p]});
      CU(cudaMemcpyAsync(c.d_bk_rr, rr.data(), rr.size() * sizeof(RrDesc), cudaMemcpyHostToDevice, st));
      CU(rr_cholesky_batched(c.d_bk_rr, (int)rr.size(), Mact, c.opt.rr_tol, st));
      CU(cudaMemcpyAsync(kk.data(), c.d_bk_k, np * sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    CU(cudaStreamSynchronize(st));
    // stored block `it`: the problems that kept at least one direction
    std::vector<int> ki(np, 0);
    std::vector<int64_t> oi(np, -1);
    int64_t tot = 0;
    int kmax = 0;
    for (int p : act) {
      if (kk[p] <= 0) {                       // no independent direction left: this problem stops
        active[p] = 0;
        result = FETI_EBREAKDOWN;
        c.err = "no independent search direction left in a problem of the batch";
        continue;
      }
      ki[p] = kk[p];
      rank[p] = kk[p];
      oi[p] = tot;
      tot += nlp[p] * kk[p];
      kmax = std::max(kmax, kk[p]);
      fap[p] += mp[p];
    }
    if (tot == 0) break;
    if ((int)c.bk_hW.size() <= it) {
      c.bk_hW.push_back(nullptr);
      c.bk_hQ.push_back(nullptr);
      c.bk_hcap.push_back(0);
    }
    if (c.bk_hcap[it] < tot) {
      int64_t cap = 0;
      TRY(grow(c, c.bk_hW[it], cap, tot));
      cap = 0;
      TRY(grow(c, c.bk_hQ[it], cap, tot));
      c.bk_hcap[it] = tot;
    }
    double* Wi = c.bk_hW[it];
    double* Qi = c.bk_hQ[it];
    hk.push_back(ki);
    hoff.push_back(oi);
    // W_i = W_p[:, perm_p] U_p and Q_i likewise (U_p upper triangular)
    auto transform_rows = [&](int64_t rt) {
      rows.clear();
      for (int pass = 0; pass < 2; ++pass)
        for (int p = 0; p < np; ++p) {
          if (ki[p] <= 0) continue;
          for (int64_t r0 = 0; r0 < nlp[p]; r0 += rt) {
            GemmDesc d{};
            d.A = (pass ? Q : W) + l0[p] + r0; d.ars = 1; d.acs = nl; d.acol = c.d_bk_perm + moff[p];
            d.B = c.d_bk_T + doff[p]; d.brs = 1; d.bcs = mp[p];
            d.C = (pass ? Qi : Wi) + oi[p] + r0; d.crs = 1; d.ccs = nlp[p];
            d.M = (int)std::min<int64_t>(rt, nlp[p] - r0); d.N = ki[p]; d.K = ki[p]; d.tri = 2;
            rows.push_back(d);
          }
        }
    };
    if (c.bk_rtile == 0) {
      // Autotune the row tile of the block updates on this batch's first
      // transform: every candidate computes the same rows in the same order
      // (only the split of the rows into work items differs), so the choice
      // changes the time, never the result.
      const int64_t cands[5] = {1024, 2048, 4096, 8192, 16384};
      cudaEvent_t e0, e1;
      CU(cudaEventCreate(&e0));
      CU(cudaEventCreate(&e1));
      float best = 1e30f;
      int64_t best_rt = BATCH_RCHUNK;
      feti_status tst = FETI_OK;
      for (int ci = 0; ci < 5 && tst == FETI_OK; ++ci) {
        transform_rows(cands[ci]);
        if (rows.size() > 65535) continue;
        float ts[3];
        for (int r = 0; r < 3 && tst == FETI_OK; ++r) {
          cudaEventRecord(e0, st);
          tst = run_row_chunks(c, rows, 1.0, 0.0);
          cudaEventRecord(e1, st);
          if (tst == FETI_OK && cudaEventSynchronize(e1) != cudaSuccess) {
            c.err = "batched Algorithm 1: row-tile autotuning failed";
            tst = FETI_ECUDA;
          }
          if (tst == FETI_OK) cudaEventElapsedTime(&ts[r], e0, e1);
        }
        if (tst != FETI_OK) break;
        std::sort(ts, ts + 3);
        if (ts[1] < best) { best = ts[1]; best_rt = cands[ci]; }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      TRY(tst);
      c.bk_rtile = best_rt;
    }
    transform_rows(c.bk_rtile);
    {
      double fl = 0.0;
      for (int p = 0; p < np; ++p) fl += 2.0 * nlp[p] * ki[p] * (ki[p] + 1.0);
      PhaseScope ph(st, FETI_PHASE_GRAM, fl);
      TRY(run_row_chunks(c, rows, 1.0, 0.0));
    }
    // gamma = W_i^T r ; lambda~ += W_i gamma ; r -= Q_i gamma
    for (int p = 0; p < np; ++p)
      vec[p] = SegVec{Wi + std::max<int64_t>(oi[p], 0), Qi + std::max<int64_t>(oi[p], 0), nlp[p], nlp[p], l0[p],
                      moff[p], ki[p]};
    {
      double by = 0.0;
      for (int p = 0; p < np; ++p) by += 8.0 * nlp[p] * (3.0 * ki[p] + 4.0);
      PhaseScope ph(st, FETI_PHASE_STEP, by);
      CU(cudaMemcpyAsync(c.d_bk_vec, vec.data(), np * sizeof(SegVec), cudaMemcpyHostToDevice, st));
      CU(gemv_t_seg(c.d_bk_vec, np, kmax, c.d_r, c.d_bk_gam, st));
      CU(step_seg(nl, c.d_lam_prob, c.d_bk_vec, c.d_bk_gam, c.d_lamt, c.d_r, st));
    }
    // Z_{i+1}, W_{i+1} = Z_{i+1}
    {
      PhaseScope ph(st, FETI_PHASE_PRECOND, c.bytes_S + 8.0 * (2.0 * nl + 2.0 * hp.n_b_total + (double)nl * M));
      CU(precond_apply_cols(c, c.d_r, W, nl, M, c.d_b_lcol, c.d_z, st));
    }
    // F-orthogonalise against the stored blocks, oldest first
    double fl_o = 0.0;
    for (int j = 0; j <= it; ++j)
      for (int p = 0; p < np; ++p)
        if (active[p] && hk[j][p] > 0) fl_o += 4.0 * nlp[p] * hk[j][p] * mp[p];
    std::unique_ptr<PhaseScope> ph_o(new PhaseScope(st, FETI_PHASE_ORTHO, fl_o));
    for (int j = 0; j <= it; ++j) {
      ops.clear();
      rows.clear();
      for (int p = 0; p < np; ++p) {
        if (!active[p]) continue;
        const int kj = hk[j][p];
        if (kj <= 0) continue;
        const double* Qj = c.bk_hQ[j] + hoff[j][p];
        const double* Wj = c.bk_hW[j] + hoff[j][p];
        double* Psi = c.d_bk_delta + doff[p];            // k_j x m_p, ld k_j
        ops.push_back(SegTN{Qj, nlp[p], W + l0[p], nl, Psi, kj, kj, mp[p], nlp[p], 0});
        for (int64_t r0 = 0; r0 < nlp[p]; r0 += c.bk_rtile) {
          GemmDesc d{};
          d.A = Wj + r0; d.ars = 1; d.acs = nlp[p];
          d.B = Psi; d.brs = 1; d.bcs = kj;
          d.C = W + l0[p] + r0; d.crs = 1; d.ccs = nl;
          d.M = (int)std::min<int64_t>(c.bk_rtile, nlp[p] - r0); d.N = mp[p]; d.K = kj;
          rows.push_back(d);
        }
      }
      TRY(run_seg_tn(c, ops, 1.0, 0.0));
      TRY(run_row_chunks(c, rows, -1.0, 1.0));
    }
    ph_o.reset();
    TRY(read_rz(rz));
    ++it;
    for (int p = 0; p < np; ++p) {
      if (ki[p] <= 0) continue;
      iters[p] += 1;
      eps[p] = std::sqrt(std::max(rz[p], 0.0));
      const bool fin = std::isfinite(rz[p]);
      conv[p] = fin && eps[p] <= tol * eps0[p];
      if (!fin || conv[p] || iters[p] >= max_iter) active[p] = 0;
    }
  }
  c.prob_stats.assign(np, feti_stats{});
  int maxit = 0;
  for (int p = 0; p < np; ++p) {
    feti_stats& P = c.prob_stats[p];
    P.iterations = iters[p];
    P.converged = conv[p];
    P.f_applies = fap[p];
    P.last_rank = rank[p];
    P.eps0 = eps0[p];
    P.eps = eps[p];
    maxit = std::max(maxit, iters[p]);
  }
  S.iterations = maxit;
  if (result == FETI_EBREAKDOWN) {
    // a problem that lost every direction is reported through its own stats;
    // the batch as a whole is judged by convergence
    c.err.clear();
    result = FETI_OK;
  }
  return result;
}

static feti_status apply_one(Ctx& c, const double* x, double* y) {
  return apply_dual(c, x, c.hp.n_lam, 1, y, c.hp.n_lam);
}

// Reference for the relative stopping test of a warm-started solve: the
// preconditioned residual norm sqrt(r^T z) at the method's own initial
// multiplier (lambda_0 = 0 for FETI-DP, G^T (G G^T)^{-1} e for TFETI), so that a
// good initial guess shortens the solve instead of tightening its target.
static feti_status cold_reference(Ctx& c, double* eps_ref) {
  const int64_t nl = c.hp.n_lam;
  cudaStream_t st = c.stream;
  TRY(apply_dual(c, c.d_lam0, nl, 1, c.d_r, nl));
  CU(axpby(nl, 1.0, c.d_d, -1.0, c.d_r, st));
  TRY(project(c, c.d_r, nl, 1));
  CU(precond_apply(c, c.d_r, nullptr, nl, c.d_z, st));
  CU(dot(c.d_r, c.d_z, nl, c.d_red, c.d_scalar, st));
  double rz = 0.0;
  TRY(read_scalar(c, c.d_scalar, &rz));
  *eps_ref = std::sqrt(std::max(rz, 0.0));
  return FETI_OK;
}

static feti_status recover_u(Ctx& c, const double* lam);

// FP64 refinement on the primal residual (the FETI_REFINE_PRIMAL reading of
// the precision form): r = f - K u element by element in FP64; each step
// solves K du = r with FETI and the reduced-precision operator (the dual
// problem of the load r, Algorithm 1 to inner_tol, default 1e-3), recovers du
// and adds it, u = sum of the du, lambda = sum of the multipliers; stops when
// ||r|| <= tol ||f|| (free DOFs), or at max_refine / max_iter.  The load is
// restored at the end; the recovery then returns the summed u.
static feti_status refine_primal(Ctx& c, feti_stats& S, feti_status& result) {
  const HostProblem& hp = c.hp;
  const int64_t nl = hp.n_lam, nd = hp.n_dofs;
  cudaStream_t st = c.stream;
  if (!c.d_f0) {
    TRY(dalloc(c, c.d_f0, nd));
    TRY(dalloc(c, c.d_uacc, nd));
    TRY(dalloc(c, c.d_lamacc, nl));
  }
  CU(cudaMemcpyAsync(c.d_f0, c.d_fglob, nd * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CU(cudaMemsetAsync(c.d_uacc, 0, nd * sizeof(double), st));
  CU(cudaMemsetAsync(c.d_lamacc, 0, nl * sizeof(double), st));
  if (!c.d_ubest) TRY(dalloc(c, c.d_ubest, nd));
  double fn2 = 0.0, rel = 1.0, best = 0.0;
  int outer = 0;
  for (;;) {
    CU(launch_residual(c, c.d_f0, outer == 0 ? nullptr : c.d_uacc, c.d_fglob, st));
    CU(dot(c.d_fglob, c.d_fglob, nd, c.d_red, c.d_scalar, st));
    double rn2 = 0.0;
    TRY(read_scalar(c, c.d_scalar, &rn2));
    if (outer == 0) fn2 = rn2;
    rel = fn2 > 0.0 ? std::sqrt(rn2 / fn2) : 0.0;
    // a correction that blew the residual up (a reduced-precision solve too
    // inaccurate for the problem) is undone: the best sums so far are kept and
    // the refinement stops unconverged
    if (outer > 0 && (!std::isfinite(rn2) || rel > 100.0 * best)) {
      CU(cudaMemcpyAsync(c.d_uacc, c.d_ubest, nd * sizeof(double), cudaMemcpyDeviceToDevice, st));
      CU(cudaMemcpyAsync(c.d_lamacc, c.d_dl, nl * sizeof(double), cudaMemcpyDeviceToDevice, st));
      c.err = std::isfinite(rn2) ? "the primal refinement diverged; the best solution is returned"
                                 : "NaN or Inf in the primal residual; the best solution is returned";
      if (!std::isfinite(rn2)) result = FETI_EBREAKDOWN;
      rel = best;
      break;
    }
    if (outer == 0 || rel < best) {
      best = rel;
      CU(cudaMemcpyAsync(c.d_ubest, c.d_uacc, nd * sizeof(double), cudaMemcpyDeviceToDevice, st));
      CU(cudaMemcpyAsync(c.d_dl, c.d_lamacc, nl * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    if (rel <= c.opt.tol || outer >= c.opt.max_refine || S.iterations >= c.opt.max_iter) break;
    // the dual problem of the load r, solved from its own lambda_0
    TRY(load_rhs(c));
    CU(cudaMemcpyAsync(c.d_lam, c.d_lam0, nl * sizeof(double), cudaMemcpyDeviceToDevice, st));
    TRY(apply_dual(c, c.d_lam, nl, 1, c.d_r, nl));
    CU(axpby(nl, 1.0, c.d_d, -1.0, c.d_r, st));
    TRY(project(c, c.d_r, nl, 1));
    feti_stats inner{};
    const int cap = std::min(c.opt.max_iter - S.iterations, 60);
    const double itol = c.opt.inner_tol > 0.0 ? c.opt.inner_tol : 1e-3;
    feti_status s2 = krylov_core(c, itol, cap, true, inner, -1.0);
    S.iterations += inner.iterations;
    S.f_applies += inner.f_applies + 1;
    S.last_rank = inner.last_rank;
    ++outer;
    if (s2 == FETI_EBREAKDOWN && inner.iterations > 0) c.err.clear();
    else if (s2 != FETI_OK && s2 != FETI_ENOTCONV) { result = s2; break; }
    CU(axpby(nl, 1.0, c.d_lamt, 1.0, c.d_lam, st));
    TRY(recover_u(c, c.d_lam));
    CU(axpby(nd, 1.0, c.d_uglob, 1.0, c.d_uacc, st));
    CU(axpby(nl, 1.0, c.d_lam, 1.0, c.d_lamacc, st));
  }
  // the loads of the corrections are the successive residuals, which do not
  // sum to f: u is the sum of the corrections (kept for the recovery), lambda
  // the sum of their multipliers
  CU(cudaMemcpyAsync(c.d_fglob, c.d_f0, nd * sizeof(double), cudaMemcpyDeviceToDevice, st));
  TRY(load_rhs(c));
  CU(cudaMemcpyAsync(c.d_lam, c.d_lamacc, nl * sizeof(double), cudaMemcpyDeviceToDevice, st));
  c.u_refined = 1;
  S.eps0 = 1.0;
  S.eps = rel;
  S.converged = rel <= c.opt.tol;
  S.refinements = outer;
  return FETI_OK;
}

static feti_status solve_impl(Ctx& c, double* lambda_inout, feti_stats* stats) {
  const HostProblem& hp = c.hp;
  const int64_t nl = hp.n_lam;
  const bool multi = c.opt.krylov == FETI_RRS;
  // directions per block: one per subdomain (of the largest problem of a
  // batch) for the simultaneous variant; batches apply them in column chunks
  int mmax = multi ? hp.n_sub : 1;
  if (hp.n_prob > 1) {
    mmax = 1;
    for (int p = 0; multi && p < hp.n_prob; ++p)
      mmax = std::max(mmax, hp.prob_sub_off[p + 1] - hp.prob_sub_off[p]);
  }
  if (mmax > 1024) { c.err = "more than 1024 subdomains per direction block"; return FETI_ENOTSUP; }
  TRY(ensure_krylov(c, mmax));
  // block buffers before any capture (a batch's PCG iteration is recorded as a graph)
  TRY(ensure_blocks(c, hp.n_prob == 1 ? mmax : 1));
  cudaStream_t st = c.stream;
  feti_stats S{};
  // lambda_0 (warm start or the method's own)
  CU(cudaMemcpyAsync(c.d_lam, lambda_inout ? lambda_inout : c.d_lam0, nl * sizeof(double),
                     cudaMemcpyDeviceToDevice, st));
  if (lambda_inout && hp.method == FETI_TFETI) {
    // keep G lambda = e: lambda = lambda_0 + P (lambda_in - lambda_0)
    CU(axpby(nl, -1.0, c.d_lam0, 1.0, c.d_lam, st));
    TRY(project(c, c.d_lam, nl, 1));
    CU(axpby(nl, 1.0, c.d_lam0, 1.0, c.d_lam, st));
  }
  feti_status result = FETI_OK;
  c.u_refined = 0;
  double eps_ref = -1.0;
  if (lambda_inout && hp.n_prob == 1) TRY(cold_reference(c, &eps_ref));
  if (hp.n_prob > 1) {
    // one solve per problem, advanced together: the simultaneous variant
    // (a block of directions per problem) or PCG (graph-captured iterations)
    TRY(apply_dual(c, c.d_lam, nl, 1, c.d_r, nl));
    CU(axpby(nl, 1.0, c.d_d, -1.0, c.d_r, st));
    int maxit = 0;
    if (multi) {
      TRY(batch_rrs(c, c.opt.tol, c.opt.max_iter, S));
      maxit = S.iterations;
    } else {
      CU(batch_pcg(c, st, c.opt.tol, c.opt.max_iter, &apply_one, &maxit));
    }
    CU(axpby(nl, 1.0, c.d_lamt, 1.0, c.d_lam, st));
    S.iterations = maxit;
    S.converged = 1;
    S.last_rank = 1;
    for (auto& ps : c.prob_stats) {
      S.converged = S.converged && ps.converged;
      S.f_applies += ps.f_applies;
      S.eps0 = std::max(S.eps0, ps.eps0);
      S.eps = std::max(S.eps, ps.eps);
    }
  } else if (c.opt.precision == FETI_FP64) {
    // r_0 = P^T (d - F lambda_0), then Algorithm 1; lambda = lambda_0 + lambda~
    TRY(apply_dual(c, c.d_lam, nl, 1, c.d_r, nl));
    CU(axpby(nl, 1.0, c.d_d, -1.0, c.d_r, st));
    TRY(project(c, c.d_r, nl, 1));
    result = krylov_core(c, c.opt.tol, c.opt.max_iter, false, S, eps_ref);
    CU(axpby(nl, 1.0, c.d_lamt, 1.0, c.d_lam, st));
  } else if (c.opt.refine == FETI_REFINE_PRIMAL) {
    TRY(refine_primal(c, S, result));
  } else {
    // FP64 iterative refinement on the dual residual: r = P^T (d - F lambda)
    // with the FP64 operator; each correction solves F dl = r with the
    // low-precision local products to inner_tol.
    double eps0 = -1.0, eps = 0.0, best = 0.0;
    int outer = 0;
    for (;;) {
      TRY(apply_dual(c, c.d_lam, nl, 1, c.d_rout, nl));
      CU(axpby(nl, 1.0, c.d_d, -1.0, c.d_rout, st));
      TRY(project(c, c.d_rout, nl, 1));
      CU(precond_apply(c, c.d_rout, nullptr, nl, c.d_zout, st));
      CU(dot(c.d_rout, c.d_zout, nl, c.d_red, c.d_scalar, st));
      double rz = 0.0;
      TRY(read_scalar(c, c.d_scalar, &rz));
      eps = std::sqrt(std::max(rz, 0.0));
      if (eps0 < 0.0) eps0 = eps_ref > 0.0 ? eps_ref : eps;
      S.f_applies += 1;
      // a correction that blew the FP64 residual up (a reduced-precision
      // operator too inaccurate for the problem) is undone: the best
      // multipliers so far are kept and the refinement stops unconverged
      const bool blown = outer > 0 && (!std::isfinite(rz) || eps > 100.0 * best);
      if (blown) {
        CU(cudaMemcpyAsync(c.d_lam, c.d_dl, nl * sizeof(double), cudaMemcpyDeviceToDevice, st));
        eps = best;
        c.err = std::isfinite(rz) ? "the refinement diverged; the best multipliers are returned"
                                  : "NaN or Inf in the refined residual; the best multipliers are returned";
        if (!std::isfinite(rz)) result = FETI_EBREAKDOWN;
        break;
      }
      if (!std::isfinite(rz)) { result = FETI_EBREAKDOWN; c.err = "NaN or Inf in the refined residual"; break; }
      if (outer == 0 || eps < best) {
        best = eps;
        CU(cudaMemcpyAsync(c.d_dl, c.d_lam, nl * sizeof(double), cudaMemcpyDeviceToDevice, st));
      }
      if (eps <= c.opt.tol * eps0 || outer >= c.opt.max_refine || S.iterations >= c.opt.max_iter) break;
      CU(cudaMemcpyAsync(c.d_r, c.d_rout, nl * sizeof(double), cudaMemcpyDeviceToDevice, st));
      feti_stats inner{};
      // each correction is capped (a stalled reduced-precision solve still
      // returns a useful correction; the FP64 outer loop decides convergence)
      const int cap = std::min(c.opt.max_iter - S.iterations, 30);
      // automatic inner tolerance: 1e-2 (measured best time-to-solve for both
      // reduced-precision products: each restart costs the orthogonalization
      // history, so long inner solves lose more than extra restarts)
      const double itol = c.opt.inner_tol > 0.0 ? c.opt.inner_tol : 1e-2;
      feti_status s2 = krylov_core(c, itol, cap, true, inner, -1.0);
      S.iterations += inner.iterations;
      S.f_applies += inner.f_applies;
      S.last_rank = inner.last_rank;
      ++outer;
      // a reduced-precision inner solve that loses every direction at the
      // rank test after some progress still returns a usable correction; the
      // FP64 outer loop decides.  Without progress the refinement cannot go on.
      if (s2 == FETI_EBREAKDOWN && inner.iterations > 0) {
        c.err.clear();
      } else if (s2 != FETI_OK && s2 != FETI_ENOTCONV) {
        result = s2;
        break;
      }
      CU(axpby(nl, 1.0, c.d_lamt, 1.0, c.d_lam, st));
    }
    S.eps0 = eps0;
    S.eps = eps;
    S.converged = eps <= c.opt.tol * eps0;
    S.refinements = outer;
  }
  if (lambda_inout) CU(cudaMemcpyAsync(lambda_inout, c.d_lam, nl * sizeof(double), cudaMemcpyDeviceToDevice, st));
  TRY(sync_check(c));
  TRY(check_status(c, "solve"));
  if (result == FETI_OK && !S.converged) {
    result = FETI_ENOTCONV;
    if (c.err.empty()) c.err = "max_iter reached";
  }
  c.last = S;
  if (stats) *stats = S;
  return result;
}

extern "C" {

feti_status feti_solve_dual(feti_ctx* ctx, double* lambda_inout, feti_stats* stats) {
  if (!ctx) return FETI_EINVAL;
  Ctx& c = ctx->c;
  c.err.clear();
  if (c.state < 2) { c.err = "feti_solve_dual before feti_factorize"; return FETI_ESTATE; }
  feti_status s = solve_impl(c, lambda_inout, stats);
  if (s == FETI_OK || s == FETI_ENOTCONV) {
    c.state = 3;
    c.have_solution = 1;
  }
  return s;
}

}  // extern "C"

// u (c.d_uglob) from the multipliers lam and the current load (Eq. 7 / Eq. 12
// back-substitution; TFETI: alpha = (G G^T)^{-1} G (d - F lambda) first).
static feti_status recover_u(Ctx& c, const double* lam) {
  const HostProblem& hp = c.hp;
  cudaStream_t st = c.stream;
  if (hp.method == FETI_FETIDP) {
    CU(recover_fetidp(c, lam, st));
  } else {
    const int64_t nl = hp.n_lam;
    const int nco = c.n_coarse;
    TRY(ensure_krylov(c, 1));
    TRY(apply_dual(c, lam, nl, 1, c.d_r, nl));
    CU(axpby(nl, 1.0, c.d_d, -1.0, c.d_r, st));
    TRY(ensure_blocks(c, 1));
    CU(gather_lam_to_b(c, c.d_r, nl, 1, c.d_Xb, st));
    CU(tfeti_G_apply(c, c.d_Xb, 1, c.d_ct1, st));
    CU(gemv_dense(c.d_Kbar_inv, nco, nco, c.d_ct1, c.d_alpha, 0.0, st));
    CU(recover_tfeti(c, lam, c.d_alpha, st));
  }
  CU(launch_gather_u(c, st));
  return FETI_OK;
}

extern "C" {

feti_status feti_recover_displacements(feti_ctx* ctx, double* u_out, int on_device, double* compliance_out) {
  if (!ctx) return FETI_EINVAL;
  Ctx& c = ctx->c;
  c.err.clear();
  if (c.state < 3 || !c.have_solution) { c.err = "feti_recover_displacements before feti_solve_dual"; return FETI_ESTATE; }
  const HostProblem& hp = c.hp;
  cudaStream_t st = c.stream;
  std::unique_ptr<PhaseScope> phase(new PhaseScope(st, FETI_PHASE_RECOVER, 0.0));
  if (c.u_refined) CU(cudaMemcpyAsync(c.d_uglob, c.d_uacc, hp.n_dofs * sizeof(double), cudaMemcpyDeviceToDevice, st));
  else TRY(recover_u(c, c.d_lam));
  phase.reset();
  if (u_out)
    CU(cudaMemcpyAsync(u_out, c.d_uglob, hp.n_dofs * sizeof(double),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  {
    // per-problem compliance f_p^T u_p
    const int np = hp.n_prob;
    double* part = c.d_bstate + 6 * np;
    double* comp = c.d_bstate;            // scratch (the PCG scalars are no longer needed)
    CU(seg_dot2(c.d_prob_dof_off, np, c.d_fglob, c.d_uglob, nullptr, nullptr, part, comp, nullptr, st));
    c.prob_compliance.assign(np, 0.0);
    CU(cudaMemcpyAsync(c.prob_compliance.data(), comp, np * sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (compliance_out) {
      double t = 0.0;
      for (double v : c.prob_compliance) t += v;
      *compliance_out = t;
    }
  }
  TRY(sync_check(c));
  c.state = 4;
  return FETI_OK;
}

feti_status feti_primal_residual(feti_ctx* ctx, const double* u, double* r, double* rel) {
  if (!ctx) return FETI_EINVAL;
  Ctx& c = ctx->c;
  c.err.clear();
  if (c.state < 2) { c.err = "feti_primal_residual before feti_factorize"; return FETI_ESTATE; }
  const int64_t nd = c.hp.n_dofs;
  cudaStream_t st = c.stream;
  double* out = r;
  if (!out) {
    if (!c.d_rres) TRY(dalloc(c, c.d_rres, nd));
    out = c.d_rres;
  }
  if (rel) {
    CU(launch_residual(c, c.d_fglob, nullptr, out, st));
    CU(dot(out, out, nd, c.d_red, c.d_scalar, st));
    double fn2 = 0.0;
    TRY(read_scalar(c, c.d_scalar, &fn2));
    CU(launch_residual(c, c.d_fglob, u, out, st));
    CU(dot(out, out, nd, c.d_red, c.d_scalar, st));
    double rn2 = 0.0;
    TRY(read_scalar(c, c.d_scalar, &rn2));
    *rel = fn2 > 0.0 ? std::sqrt(rn2 / fn2) : std::sqrt(rn2);
  } else {
    CU(launch_residual(c, c.d_fglob, u, out, st));
  }
  TRY(sync_check(c));
  return FETI_OK;
}

feti_status feti_compliance_grad(feti_ctx* ctx, double* dc_drho, int on_device) {
  if (!ctx || !dc_drho) return FETI_EINVAL;
  Ctx& c = ctx->c;
  c.err.clear();
  if (c.state < 4) { c.err = "feti_compliance_grad before feti_recover_displacements"; return FETI_ESTATE; }
  if (on_device) {
    CU(launch_grad(c, dc_drho, c.stream));
  } else {
    double* tmp;
    TRY(dalloc(c, tmp, c.hp.n_elements));
    CU(launch_grad(c, tmp, c.stream));
    CU(cudaMemcpyAsync(dc_drho, tmp, c.hp.n_elements * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  }
  TRY(sync_check(c));
  return FETI_OK;
}

feti_status feti_apply_dual(feti_ctx* ctx, const double* X, int ldx, int m, double* Y, int ldy) {
  if (!ctx || !X || !Y || m < 0) return FETI_EINVAL;
  Ctx& c = ctx->c;
  c.err.clear();
  if (c.state < 2) { c.err = "feti_apply_dual before feti_factorize"; return FETI_ESTATE; }
  if (ldx < c.hp.n_lam || ldy < c.hp.n_lam) { c.err = "leading dimension smaller than n_lambda"; return FETI_EINVAL; }
  if (m == 0) return FETI_OK;
  if (c.opt.precision != FETI_FP64) TRY(apply_dual_lowp(c, X, ldx, m, Y, ldy));
  else TRY(apply_dual(c, X, ldx, m, Y, ldy));
  TRY(sync_check(c));
  TRY(check_status(c, "feti_apply_dual"));
  return FETI_OK;
}

feti_status feti_test_skip_copy(feti_ctx* ctx, int chunk) {
  if (!ctx) return FETI_EINVAL;
  ctx->c.test_skip_chunk = chunk < 0 ? -1 : chunk;
  return FETI_OK;
}

feti_status feti_apply_precond(feti_ctx* ctx, const double* r, double* Z, int ldz, double* z) {
  if (!ctx || !r) return FETI_EINVAL;
  Ctx& c = ctx->c;
  c.err.clear();
  if (c.state < 2) { c.err = "feti_apply_precond before feti_factorize"; return FETI_ESTATE; }
  if (Z && ldz < c.hp.n_lam) { c.err = "ldz smaller than n_lambda"; return FETI_EINVAL; }
  CU(precond_apply(c, r, Z, ldz, z, c.stream));
  TRY(sync_check(c));
  return FETI_OK;
}

feti_status feti_query(const feti_ctx* ctx, int key, int64_t* value) {
  if (!ctx || !value) return FETI_EINVAL;
  const Ctx& c = ctx->c;
  if (key == FETI_Q_LAUNCHES) { *value = launches(); return FETI_OK; }
  if (c.state < 1) return FETI_ESTATE;
  const HostProblem& hp = c.hp;
  switch (key) {
    case FETI_Q_N_LAMBDA: *value = hp.n_lam; break;
    case FETI_Q_N_SUBDOMAINS: *value = hp.n_sub; break;
    case FETI_Q_N_PRIMAL: *value = hp.n_primal; break;
    case FETI_Q_N_MODULES: *value = c.n_mod; break;
    case FETI_Q_N_B_TOTAL: *value = hp.n_b_total; break;
    case FETI_Q_N_DOFS: *value = hp.n_dofs; break;
    case FETI_Q_N_ELEMENTS: *value = hp.n_elements; break;
    case FETI_Q_MAX_NB: *value = c.max_nb; break;
    case FETI_Q_DEVICE_BYTES: *value = (int64_t)c.device_bytes; break;
    case FETI_Q_N_RBM: *value = hp.n_rbm; break;
    case FETI_Q_LAUNCHES: *value = launches(); break;
    case FETI_Q_N_PROBLEMS: *value = hp.n_prob; break;
    case FETI_Q_GEMV_CONFIG: *value = c.gemv_cfg; break;
    case FETI_Q_BATCH_ROW_TILE: *value = c.bk_rtile; break;
    case FETI_Q_TC_BYTES_F: *value = c.tc_bytes_f; break;
    case FETI_Q_TC_BYTES_PER_COL: *value = c.tc_bytes_col; break;
    case FETI_Q_APPLY1_BYTES: *value = (int64_t)c.bytes_apply1; break;
    default: return FETI_EINVAL;
  }
  return FETI_OK;
}

feti_status feti_problem_result(const feti_ctx* ctx, int p, int64_t* dof_offset, int64_t* elem_offset,
                                int64_t* lambda_offset, feti_stats* stats, double* compliance) {
  if (!ctx) return FETI_EINVAL;
  const Ctx& c = ctx->c;
  if (c.state < 1) return FETI_ESTATE;
  const HostProblem& hp = c.hp;
  if (p < 0 || p >= hp.n_prob) return FETI_EINVAL;
  if (dof_offset) *dof_offset = hp.prob_dof_off[p];
  if (elem_offset) *elem_offset = hp.prob_el_off[p];
  if (lambda_offset) *lambda_offset = hp.prob_lam_off[p];
  if (stats) *stats = (hp.n_prob > 1 && (int)c.prob_stats.size() == hp.n_prob) ? c.prob_stats[p] : c.last;
  if (compliance) *compliance = (int)c.prob_compliance.size() > p ? c.prob_compliance[p] : 0.0;
  return FETI_OK;
}

feti_status feti_profile_begin(feti_ctx* ctx) {
  if (!ctx) return FETI_EINVAL;
  Ctx& c = ctx->c;
  if (c.prof) { c.err = "a profile is already active"; return FETI_ESTATE; }
  c.prof = new_gemm_profile();
  set_gemm_profile(static_cast<GemmProfile*>(c.prof));
  return FETI_OK;
}

feti_status feti_profile_end(feti_ctx* ctx, double* gemm_flops, double* gemm_ms, int64_t* gemm_launches) {
  if (!ctx) return FETI_EINVAL;
  Ctx& c = ctx->c;
  if (!c.prof) { c.err = "no active profile"; return FETI_ESTATE; }
  CU(cudaStreamSynchronize(c.stream));
  set_gemm_profile(nullptr);
  double f[2], t[2];
  int64_t n[2];
  finish_gemm_profile(static_cast<GemmProfile*>(c.prof), f, t, n, c.prof_ph_work, c.prof_ph_ms, c.prof_ph_count);
  c.prof = nullptr;
  c.prof_tc_flops = f[1];
  c.prof_tc_ms = t[1];
  c.prof_tc_launches = n[1];
  if (gemm_flops) *gemm_flops = f[0];
  if (gemm_ms) *gemm_ms = t[0];
  if (gemm_launches) *gemm_launches = n[0];
  return FETI_OK;
}

feti_status feti_profile_tensor(const feti_ctx* ctx, double* flops, double* ms, int64_t* launches) {
  if (!ctx) return FETI_EINVAL;
  const Ctx& c = ctx->c;
  if (flops) *flops = c.prof_tc_flops;
  if (ms) *ms = c.prof_tc_ms;
  if (launches) *launches = c.prof_tc_launches;
  return FETI_OK;
}

feti_status feti_profile_phases(const feti_ctx* ctx, double* work, double* ms, int64_t* count) {
  if (!ctx) return FETI_EINVAL;
  const Ctx& c = ctx->c;
  for (int q = 0; q < N_PHASES; ++q) {
    if (work) work[q] = c.prof_ph_work[q];
    if (ms) ms[q] = c.prof_ph_ms[q];
    if (count) count[q] = c.prof_ph_count[q];
  }
  return FETI_OK;
}

feti_status feti_lambda_layout(const feti_ctx* ctx, int32_t* out) {
  if (!ctx || !out) return FETI_EINVAL;
  const Ctx& c = ctx->c;
  if (c.state < 1) return FETI_ESTATE;
  const HostProblem& hp = c.hp;
  for (int64_t l = 0; l < hp.n_lam; ++l) {
    for (int t = 0; t < 2; ++t) {
      const int b = t == 0 ? hp.lam_b0[l] : hp.lam_b1[l];
      int32_t* o = out + 6 * l + 3 * t;
      if (b < 0) { o[0] = -1; o[1] = -1; o[2] = 0; continue; }
      const int s = hp.b_sub[b];
      const StructType& T = hp.types[hp.sub_type[s]];
      o[0] = s;
      o[1] = T.blist[b - hp.b_off[s]];
      o[2] = t == 0 ? hp.lam_s0[l] : hp.lam_s1[l];
    }
  }
  return FETI_OK;
}

feti_status feti_local_blocks(feti_ctx* ctx, int s, int* nb, int* nc, int32_t* bdofs, int32_t* cdofs, double* F,
                              double* Sout, double* Frc) {
  if (!ctx) return FETI_EINVAL;
  Ctx& c = ctx->c;
  if (c.state < 2) { c.err = "feti_local_blocks before feti_factorize"; return FETI_ESTATE; }
  if (s < 0 || s >= c.hp.n_sub) return FETI_EINVAL;
  const DevSub& S = c.h_subs[s];
  const DevModule& M = c.h_mods[S.module];
  const StructType& T = c.hp.types[S.type];
  if (nb) *nb = T.n_b;
  if (nc) *nc = T.n_c;
  if (bdofs) for (int k = 0; k < T.n_b; ++k) bdofs[k] = T.blist[k];
  if (cdofs) for (int k = 0; k < T.n_c; ++k) cdofs[k] = T.clist[k];
  const int nbc = T.n_bc();
  if (F) CU(cudaMemcpy(F, c.d_modmem + M.F, (size_t)T.n_b * T.n_b * sizeof(double), cudaMemcpyDeviceToHost));
  if (Sout)
    CU(cudaMemcpy2D(Sout, T.n_b * sizeof(double), c.d_modmem + M.S, nbc * sizeof(double), T.n_b * sizeof(double),
                    T.n_b, cudaMemcpyDeviceToHost));
  if (Frc && T.n_c > 0)
    CU(cudaMemcpy(Frc, c.d_modmem + M.Frc, (size_t)T.n_b * T.n_c * sizeof(double), cudaMemcpyDeviceToHost));
  return FETI_OK;
}

}  // extern "C"
