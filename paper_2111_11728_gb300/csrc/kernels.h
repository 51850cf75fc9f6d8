// Launchers of the device kernels (one namespace, several translation units).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "feti_internal.h"

namespace feti {

// Instrumentation: a process-wide count of kernel launches, and an optional
// CUDA-event profile of the FP64 GEMM launches (algorithmic flops, time).
void note_launches(int n);
int64_t launches();
struct GemmProfile;
void set_gemm_profile(GemmProfile* p);
GemmProfile* new_gemm_profile();
// Phases of the method, timed as regions (every launch inside, on the context
// stream) with their algorithmic work: flops for the FP64-pipe phases, bytes
// for the memory-bound ones (the numbering of include/feti.h).
constexpr int N_PHASES = 8;
constexpr int PHASE_KIND0 = 16;
// [2] each (GEMM, tensor) plus [N_PHASES] each per phase
void finish_gemm_profile(GemmProfile* p, double* flops, double* ms, int64_t* count, double* pwork, double* pms,
                         int64_t* pcount);
void prof_begin(cudaStream_t st, double flops, int kind);   // bracket launches (no-op without a profile; nests)
void prof_end(cudaStream_t st);
struct PhaseScope {                                          // one phase region
  PhaseScope(cudaStream_t st, int phase, double work);
  ~PhaseScope();
  PhaseScope(const PhaseScope&) = delete;
  PhaseScope& operator=(const PhaseScope&) = delete;
 private:
  cudaStream_t st_;
  bool on_;
};

// C = alpha * A B + beta * C with element (i,k) of A at A[i*ars + k*acs],
// (k,j) of B at B[k*brs + j*bcs] and (i,j) of C at C[i*crs + j*ccs].
//
// tri = 1: only tiles on or below the diagonal of C are computed (symmetric
//          products; the strictly upper part of C is left untouched).
// tri = 2: B is upper triangular (B(k, j) = 0 for k > j): each column tile
//          stops its K loop after its last column.
// acol (optional): column k of A is stored at A + acol[k] * acs.
struct GemmDesc {
  const double* A;
  const double* B;
  double* C;
  int M, N, K;
  int tri;
  int64_t ars, acs, brs, bcs, crs, ccs;
  const int* acol;
};

// Batched FP64 GEMM over n_batch descriptors living in device memory.
// n_override > 0 replaces every descriptor's N.  beta == 0 never reads C.
// alg_flops: the product's algorithmic flop count (for the profile only).
cudaError_t dgemm_batched(const GemmDesc* d_desc, int n_batch, int max_m, int max_n,
                          int n_override, double alpha, double beta, cudaStream_t st, double alg_flops = 0.0);

// One FP64 GEMM with a deterministic split over K: partial tiles go to
// `work` ([splits][M][N]) and are summed in a fixed order.
// alg_flops < 0 means 2 M N K.
cudaError_t dgemm_split(const GemmDesc& d, int splits, double* work, double alpha, double beta,
                        cudaStream_t st, double alg_flops = -1.0);

// Chooses a split count that fills the GPU for an M x N x K product.
int split_for(int M, int N, int K, bool lower);   // K splits of a Gram-type FP64 product (whole waves)

// ---- assembly (fem.cu) --------------------------------------------------------
void element_stiffness_host(int dim, double nu, double* k0);
cudaError_t launch_moduli(const Ctx& c, double* E, cudaStream_t st);
cudaError_t launch_assemble_with(const Ctx& c, const double* E, cudaStream_t st);
cudaError_t launch_gather_diag_b(const Ctx& c, cudaStream_t st);
cudaError_t launch_copy_kbb(const Ctx& c, cudaStream_t st);   // K_bb for the lumped preconditioner
cudaError_t launch_scaling_weights(const Ctx& c, int kind, cudaStream_t st);
cudaError_t launch_load_gather(const Ctx& c, cudaStream_t st);
cudaError_t launch_gather_u(const Ctx& c, cudaStream_t st);
cudaError_t launch_grad(const Ctx& c, double* out, cudaStream_t st);
// r = f - K u on the free DOFs (0 on the fixed ones), FP64, element by element
// (moduli of the last factorization); u null: r = free part of f
cudaError_t launch_residual(const Ctx& c, const double* f, const double* u, double* r, cudaStream_t st);

// ---- factorization (factor.cu) ------------------------------------------------
cudaError_t launch_band_chol(const Ctx& c, cudaStream_t st);
cudaError_t launch_band_fwd_multi(const Ctx& c, cudaStream_t st);
// Dense SPD matrices listed as (pointer, n, ld) triples in device memory:
// Cholesky in place (lower), then explicit inverse into `out` via L^{-T} L^{-1}.
// With n_full > n the Cholesky eliminates only the leading n columns of the
// n_full x n_full matrix: the trailing block is left holding the Schur
// complement of the leading block (lower triangle), rows n.. of the first n
// columns hold L_21.
struct DenseDesc {
  double* A;      // n_full x n_full row-major with leading dimension ld (overwritten by L)
  double* Linv;   // n x n row-major scratch for L^{-1} of the leading block
  double* out;    // n x n row-major result (leading block)^{-1}
  int n, ld;
  int tag;        // reported in the status word on failure
  int n_full;     // 0 or n: plain Cholesky of the n x n matrix
};
cudaError_t dense_spd_inverse(const DenseDesc* d_desc, const DenseDesc* h_desc, int count, int* d_status,
                              cudaStream_t st);
// 0: W = S (the whole b+c Schur complement); 1: Kb = symmetrised trailing block of W
// One large SPD matrix (the coarse problem): blocked multi-CTA Cholesky, L^{-1}
// and out = L^{-T} L^{-1} through the FP64 GEMM.  X receives L^{-1}; the
// device descriptor must describe (Linv = X, out, n).
cudaError_t dense_spd_inverse_blocked(double* A, double* X, double* out, int n, double* work, int* status,
                                      const DenseDesc* d_desc_for_ltl, cudaStream_t st);
cudaError_t launch_copy_block(const Ctx& c, int which, cudaStream_t st);
cudaError_t launch_coarse_assemble_impl(const Ctx& c, const int* d_c_sub, const int64_t* d_c_off, double* K,
                                        cudaStream_t st);
cudaError_t launch_band_fwd_single(const Ctx& c, cudaStream_t st);   // h = L^{-1} f_i
// ---- edge averages (edges.cu): change of basis on the averaged edges ------------
cudaError_t launch_edge_transform(const Ctx& c, int max_bc, cudaStream_t st);   // S <- T^T S T per module
cudaError_t launch_edge_load(const Ctx& c, int max_avg, cudaStream_t st);       // f~ <- T^T f~ per subdomain
// nodal values: xb (b slots, in place) and ucl (c slots) from the transformed ones
cudaError_t launch_edge_unmap(const Ctx& c, const double* uc, double* xb, double* ucl, cudaStream_t st);
cudaError_t launch_condense_load(const Ctx& c, cudaStream_t st);     // f~ = f_bc - Y^T h

// ---- dual operator pieces (dual.cu) -------------------------------------------
// Xb[b + j*nbt] = sum over the rows l of b of sign * X[l + j*ldx]  (B^T X in b space)
cudaError_t gather_lam_to_b(const Ctx& c, const double* X, int64_t ldx, int m, double* Xb, cudaStream_t st);
// Y[l + j*ldy] = sum over the entries (b, sign) of row l of sign * Yb[b + j*nbt]  (B Yb)
cudaError_t scatter_b_to_lam(const Ctx& c, const double* Yb, int m, double* Y, int64_t ldy, cudaStream_t st);
// Y_b(s) = F_s X_b(s) for every subdomain (batched over subdomains)
cudaError_t apply_local_F(Ctx& c, const double* Xb, double* Yb, int m, double beta, cudaStream_t st);
// Vraw[g + j*np] = sum over corner copies of (F_rc,s^T X_b(s))[k, j]
cudaError_t corner_reduce(Ctx& c, const double* Xb, int m, double* Cb, double* Vraw, cudaStream_t st);
// out[g] = sum over the corner copies of g of src[c_off(s) + k]  (B_c^T applied to a c-space vector)
cudaError_t corner_gather_vec(const Ctx& c, const double* src, double* out, cudaStream_t st);
// Yb(s) += F_rc,s V[c_glob(s), :]
cudaError_t corner_expand(Ctx& c, const double* V, int m, double* Vc, double* Yb, cudaStream_t st);
// weighted gather / preconditioner scatter
cudaError_t precond_apply(Ctx& c, const double* r, double* Z, int64_t ldz, double* z, cudaStream_t st);
// the same with Z's column of b-space entry b given by bcol[b]; ncols columns of Z are cleared
cudaError_t precond_apply_cols(Ctx& c, const double* r, double* Z, int64_t ldz, int ncols, const int* bcol,
                               double* z, cudaStream_t st);
cudaError_t precond_apply_scratch(const Ctx& c, const double* r, double* Z, int64_t ldz, double* z, double* rb,
                                  double* zb, cudaStream_t st);
cudaError_t batched_gemv_F(Ctx& c, const double* xb, double* yb, cudaStream_t st);   // y_b = F_s x_b
// y_b = A_s x_b (+ beta y_b), A_s = F_s (which 0) or S_bb (which 1)
cudaError_t batched_gemv(const Ctx& c, int which, const double* xb, double* yb, double beta, cudaStream_t st);
// picks the fastest launch shape of batched_gemv on this problem (stored in c.gemv_cfg)
cudaError_t autotune_gemv(Ctx& c, cudaStream_t st);

// ---- Krylov helpers (krylov.cu) ------------------------------------------------
// Rank-revealing pivoted Cholesky of Delta (m x m, column-major ld; only its
// lower triangle is read): writes U = L~^{-T} (k x k upper triangular,
// column-major ld m) into T, the pivot order into d_perm[0..m) and k into
// *d_k, so that W N^T [L~^{-T}; 0] = W[:, perm[0..k)] U.  work: rr_work_doubles(m).
cudaError_t rr_cholesky(const double* Delta, int m, int ld, double rr_tol, double* work, double* T,
                        int* d_k, int* d_perm, cudaStream_t st);
// The same for n independent matrices (m <= 1024 each), one descriptor per
// matrix in device memory; work holds rr_work_doubles(m) doubles per matrix.
struct RrDesc {
  const double* Delta;
  int m, ld;
  double* work;
  double* T;
  int* k;
  int* perm;
};
cudaError_t rr_cholesky_batched(const RrDesc* d_desc, int n, int max_m, double rr_tol, cudaStream_t st);
int64_t rr_work_doubles(int m);   // work buffer of the rank-revealing factorization per matrix
// lam_t += W g ; then r -= Q g, or qout = Q g when qout is not null
// (W, Q column-major n x k with leading dimension ld)
cudaError_t step_update(const double* W, const double* Q, int64_t ld, int64_t n, int k, const double* g,
                        double* lam_t, double* r, double* qout, cudaStream_t st);
// out[0] = x . y (deterministic two-pass reduction; work has >= 1024 doubles)
cudaError_t dot(const double* x, const double* y, int64_t n, double* work, double* out, cudaStream_t st);
// y = a*x + b*y
cudaError_t axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st);
// C[i] = A[i + perm[0] * lda] * U[0] for i < n (one-direction transform)
cudaError_t scale_col(int64_t n, const double* A, int64_t lda, const int* perm, const double* U, double* C,
                      cudaStream_t st);
// C[i] = alpha * A[i] * b[0] + beta * C[i] for i < n (beta == 0 never reads C)
cudaError_t axpy_scalar(int64_t n, double alpha, const double* A, const double* b, double beta, double* C,
                        cudaStream_t st);
// out[j] = W[:, j] . r for j < k
cudaError_t gemv_t(const double* W, int64_t ld, int64_t n, int k, const double* r, double* out, cudaStream_t st);
// y = A x (+ beta y), A row-major n x n with leading dimension ld
cudaError_t gemv_dense(const double* A, int n, int ld, const double* x, double* y, double beta, cudaStream_t st);

// ---- internal device memory (api.cu): the caller's allocator if installed,
// otherwise stream-ordered allocation on the context stream
cudaError_t dev_alloc(Ctx& c, void** p, size_t bytes);
void dev_free(Ctx& c, void* p, size_t bytes);

// ---- precision form: FP32 block update C -= A B of FP64 blocks (lowp_blas.cu)
cudaError_t sgemm_sub(int64_t n, int m, int k, const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                      int64_t ldc, cudaStream_t st);

// ---- precision form (tc_apply.cu) -------------------------------------------------
size_t tc_apply_smem_bytes(int passes);
int tc_tile_rows();                     // rows of one tensor-core tile (and of a module's corner block)
cudaError_t tc_prepare(const Ctx& c, cudaStream_t st);   // Fhat, Shat (FP32) and sqrt-diagonals
// Yb = D^{1/2} Fhat D^{1/2} B^T X (tcgen05 kind::tf32); rows >= n_b untouched
// Multiplier rows per range of the precision form's operand construction.
constexpr int kSpreadRows = 128;
cudaError_t tc_gather(const Ctx& c, const double* X, int64_t ldx, int m, cudaStream_t st);
cudaError_t tc_corner_reduce(const Ctx& c, int m, double* Vraw, cudaStream_t st);
cudaError_t tc_put_v(const Ctx& c, const double* V, int m, cudaStream_t st);
cudaError_t tc_coarse_prepare(const Ctx& c, cudaStream_t st);   // FP32 copy of Kbar_cc^{-1}
int64_t tc_coarse_scratch(int n, int cap);   // floats of the FP32 coarse product's scratch
cudaError_t tc_coarse_apply(const Ctx& c, const double* Vraw, double* V, int m, cudaStream_t st);
cudaError_t tc_prepare_tiles(Ctx& c, int m);   // work list of the persistent product for m directions
cudaError_t tc_product(const Ctx& c, int m, float* Yb, cudaStream_t st);
cudaError_t scatter_b_to_lam32(const Ctx& c, const float* Yb, int m, double* Y, int64_t ldy, cudaStream_t st);
int tc_k_extent(int nb, int nc, int aug, int kc);
int tc_chunk(int precision);            // K chunk of the operand format: 32 (TF32) or 64 (BF16)
size_t tc_elem_bytes(int precision);    // 4 (TF32) or 2 (BF16)
cudaError_t corner_assemble(const Ctx& c, int m, double* Vraw, cudaStream_t st);
cudaError_t lowp_gemv_S(const Ctx& c, const double* xb, float* xh, double* yb, cudaStream_t st);
// Yb(s) += F_rc,s V[c_glob(s), :] with a thin kernel (no tile padding)
cudaError_t corner_expand_thin(Ctx& c, const double* V, int m, double* Yb, cudaStream_t st);
cudaError_t precond_apply_lowp(Ctx& c, const double* r, double* Z, int64_t ldz, double* z, cudaStream_t st);

// ---- coarse problem over one or many problems (dual.cu) --------------------------
cudaError_t coarse_assemble_batch(const Ctx& c, cudaStream_t st);
cudaError_t coarse_matvec(const Ctx& c, const double* x, double* y, cudaStream_t st);
cudaError_t coarse_apply(const Ctx& c, const double* Vraw, double* V, int m, cudaStream_t st);

// ---- batching form (batch.cu) -----------------------------------------------------
// out0[p] = a0.b0 and out1[p] = a1.b1 over each problem's index range off[p]..off[p+1)
cudaError_t seg_dot2(const int64_t* d_off, int n_prob, const double* a0, const double* b0, const double* a1,
                     const double* b1, double* part, double* out0, double* out1, cudaStream_t st);
cudaError_t batch_pcg(Ctx& c, cudaStream_t user, double tol, int max_iter,
                      feti_status (*apply)(Ctx&, const double*, double*), int* total_iters);

// Segmented products of the batched Algorithm 1: for every problem p of a
// batch, C_p = alpha A_p^T B_p + beta C_p with A_p (K x M), B_p (K x N)
// column-major (ld lda, ldb) and C_p column-major (ld ldc).  The K range is cut
// into chunks of at most kchunk rows, each chunk one entry of a batched GEMM
// into a partial buffer; k_seg_reduce sums the chunks in order
// (bit-reproducible).  tri = 1: only the lower tiles of C_p are formed.
struct SegTN {
  const double* A;
  int64_t lda;
  const double* B;
  int64_t ldb;
  double* C;
  int64_t ldc;
  int M, N;
  int64_t K;
  int tri;
};
struct SegRed {
  double* C;
  int64_t crs, ccs;
  int M, N, nz, tri;
  int64_t poff;
};
// Plans the chunk descriptors (their C is bound to a partial buffer of
// *partial_len doubles by seg_tn_bind) and the reductions.
void seg_tn_plan(const std::vector<SegTN>& ops, int64_t kchunk, std::vector<GemmDesc>& descs,
                 std::vector<int64_t>& coff, std::vector<SegRed>& reds, int64_t* partial_len, int* max_m,
                 int* max_n);
void seg_tn_bind(std::vector<GemmDesc>& descs, const std::vector<int64_t>& coff, double* partial);
cudaError_t seg_tn_run(const GemmDesc* d_desc, int n_desc, const SegRed* d_red, int n_red, int max_m, int max_n,
                       const double* partial, double alpha, double beta, double flops, cudaStream_t st);
// A problem's current block in packed storage: W, Q (n x k, leading dimension
// ld) for the multiplier rows l0 .. l0 + n, step lengths at g[goff ..]
struct SegVec {
  const double* W;
  const double* Q;
  int64_t ld, n, l0, goff;
  int k;
};
// out[goff_p + j] = W_p[:, j] . r[l0_p ..] for j < k_p
cudaError_t gemv_t_seg(const SegVec* d_v, int n_prob, int max_k, const double* r, double* out, cudaStream_t st);
// lam_t += W_p g_p and r -= Q_p g_p on every problem's rows (k_p = 0: untouched)
cudaError_t step_seg(int64_t nl, const int* d_lam_prob, const SegVec* d_v, const double* g, double* lam_t,
                     double* r, cudaStream_t st);

// ---- recovery (recover.cu) ------------------------------------------------------
cudaError_t recover_fetidp(Ctx& c, const double* lam, cudaStream_t st);
// TFETI: u^s = K^#(f^s - B^sT lambda) + R^s alpha_s
cudaError_t recover_tfeti(Ctx& c, const double* lam, const double* alpha, cudaStream_t st);

// ---- TFETI (tfeti.cu) -------------------------------------------------------------
cudaError_t tfeti_add_rrt(const Ctx& c, cudaStream_t st);                 // W += Rhat Rhat^T per module
cudaError_t tfeti_ggt(const Ctx& c, double* W, int ldw, double* t1, double* t2, double* Xb, double* Kbar,
                      cudaStream_t st);   // G G^T through the sparse G, ldw coarse columns at a time
cudaError_t tfeti_build_e(const Ctx& c, double* e, cudaStream_t st);      // e = -R^T f
// t = G X from the gathered block Xb = B^T X (no dense G); X -= G^T t
cudaError_t tfeti_G_apply(const Ctx& c, const double* Xb, int m, double* t, cudaStream_t st);
cudaError_t tfeti_Gt_sub(const Ctx& c, const double* t, int m, double* X, int64_t ldx, cudaStream_t st);

}  // namespace feti
