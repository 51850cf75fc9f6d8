/*
 * feti.h - C ABI of the GB300 FETI dual-operator library.
 *
 * The library solves the linear-elastic state problem K u = f (Eq. 2 of
 * "Comparison of FETI-based domain decomposition methods for topology
 * optimization problems", Medricky, Doskar, Pultarova, Zeman) on a regular
 * grid of subdomains (modules) with Total FETI (Section 2.1) or FETI-DP
 * (Section 2.2), k-scaling or multiplicity scaling (Section 3.1), and plain
 * PCG, full orthogonalization (Section 3.2) or rank-revealing Simultaneous
 * FETI (Section 3.3, Algorithm 1).  Every step of the computation runs in
 * CUDA kernels on the device of the stream given to feti_create.
 *
 * Conventions used by every entry point
 * -------------------------------------
 * - Mesh: tiles[d] subdomains per axis, each of elems[d] unit elements
 *   (Q4 bilinear quads in 2D, plane stress, unit thickness; H8 trilinear
 *   hexahedra in 3D).  Global elements and nodes are numbered
 *   lexicographically, x fastest; DOF = dim * node + direction.
 * - Subdomain s is the tile with lexicographic index s; its local nodes
 *   are numbered lexicographically inside the tile; local DOF
 *   = dim * local_node + direction.
 * - All floating-point data are IEEE double (FP64) unless stated.
 * - "Device pointer" means memory of the context's CUDA device; "host
 *   pointer" means ordinary CPU memory.  Where a call accepts both, the
 *   on_device flag of the problem (or the argument) says which.
 * - Ownership: the caller owns every buffer it passes; the library copies
 *   what it needs during the call (or, for device outputs, writes into the
 *   caller's memory on the context stream).  The library owns the context
 *   and all internal device memory, released by feti_destroy.  That memory is
 *   taken from the caller's allocator when one is installed with
 *   feti_set_allocator (e.g. a framework's caching allocator), otherwise
 *   stream-ordered (cudaMallocAsync / cudaFreeAsync) on the context stream.
 * - Errors: no entry point aborts or exits.  A non-OK status leaves a
 *   human-readable message in feti_last_error(ctx).  FETI_ESTATE means the
 *   call order setup -> factorize -> solve -> recover was not respected.
 * - Asynchrony: device outputs are complete when the call returns (every
 *   call synchronises the context stream before returning).
 */
#ifndef FETI_GB300_H
#define FETI_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct feti_ctx feti_ctx;

typedef enum {
  FETI_OK = 0,
  FETI_EINVAL = 1,      /* bad argument (null pointer, size, option value) */
  FETI_ENOMEM = 2,      /* device allocation failed */
  FETI_ESTATE = 3,      /* call order violated */
  FETI_ENOTCONV = 4,    /* max_iter reached: outputs valid but unconverged */
  FETI_EBREAKDOWN = 5,  /* NaN/Inf or no independent search direction left */
  FETI_ECUDA = 6,       /* a CUDA runtime call or kernel launch failed */
  FETI_ENOTSUP = 7,     /* option combination not implemented */
  FETI_ETIMEOUT = 8     /* a bounded device-side wait (tensor-core pipeline) expired; the
                           context stays usable, the results of that call are not */
} feti_status;

enum { FETI_TFETI = 0, FETI_FETIDP = 1 };                 /* Sections 2.1 / 2.2 */
enum { FETI_SCALING_K = 0, FETI_SCALING_MULT = 1 };       /* Eq. 15 / multiplicity */
enum { FETI_PCG = 0, FETI_FO = 1, FETI_RRS = 2 };         /* Sections 3.2, 3.3 */
enum { FETI_FP64 = 0, FETI_TF32 = 1, FETI_TF32X3 = 2, FETI_BF16 = 3, FETI_BF16X3 = 4 };  /* block products */
enum { FETI_PRECOND_DIRICHLET = 0, FETI_PRECOND_LUMPED = 1, FETI_PRECOND_SUPERLUMPED = 2 };
enum { FETI_PRIMAL_CORNERS = 0, FETI_PRIMAL_EDGES = 1, FETI_PRIMAL_ADAPTIVE = 2 };
enum { FETI_REFINE_DUAL = 0, FETI_REFINE_PRIMAL = 1 };   /* reduced precision: the FP64 outer residual */
                                               /* FETI-DP primal set (Section 2.2; richer and adaptive
                                                  sets: Section 5, future work) */

typedef struct {
  int method;          /* FETI_TFETI or FETI_FETIDP */
  int scaling;         /* FETI_SCALING_K or FETI_SCALING_MULT */
  int krylov;          /* FETI_PCG, FETI_FO or FETI_RRS */
  int precision;       /* FETI_FP64 (default), FETI_TF32, FETI_TF32X3, FETI_BF16, FETI_BF16X3: the
                          dense F_s (and F_rc) block products on the tensor cores with FP32
                          accumulation -- one TF32 / BF16 pass, or the three-pass split
                          (hi*hi + hi*lo + lo*hi) -- and FP32 S_s blocks, inside FP64 iterative
                          refinement on the dual residual; factorizations, coarse problem, Gram
                          and orthogonalization stay FP64 */
  int max_iter;        /* Krylov iteration cap (default 500) */
  int dedup_modules;   /* 1: factorize identical modules once (Section 1) */
  double tol;          /* relative tolerance on sqrt(r^T z) (default 1e-6) */
  double rr_tol;       /* rank-revealing cutoff on the remaining/initial pivot ratio (1e-10) */
  double inner_tol;    /* FETI_TF32 / FETI_TF32X3: relative tolerance of each low-precision inner
                          solve; 0 (default) picks 1e-2.
                          Each inner solve is also capped at 30 iterations */
  int max_refine;      /* reduced precision: cap on the FP64 refinement steps (30) */
  int precond;         /* local block of the preconditioner (Section 3): FETI_PRECOND_DIRICHLET
                          (default; the interface Schur complement S_s of Eq. 13), FETI_PRECOND_LUMPED
                          (the interface stiffness block K_bb: no interior solve) or
                          FETI_PRECOND_SUPERLUMPED (diag K_bb) */
  int primal;          /* FETI-DP primal set: FETI_PRIMAL_CORNERS (default; the DOFs at the vertices
                          of the tile grid) or FETI_PRIMAL_EDGES (also one average per component over
                          the interior nodes of every tile-grid edge shared by two or more
                          subdomains -- 3D: tile edges, 2D: tile sides -- whose nodes are all free in
                          that component; introduced by a change of basis on each edge, with the
                          Dirichlet preconditioner only) or FETI_PRIMAL_ADAPTIVE (the same averages
                          only on the edges across which the stiffness jumps: on some interior node
                          of the edge the sharers' diagonal stiffness entries -- the quantities
                          k-scaling weighs -- differ by a factor >= primal_jump; chosen from the
                          densities given at set-up).  TFETI: must be FETI_PRIMAL_CORNERS */
  double primal_jump;  /* FETI_PRIMAL_ADAPTIVE: the jump ratio that selects an edge (default 10; >= 1) */
  int refine;          /* reduced precision, one problem: the residual the FP64 outer loop refines on.
                          FETI_REFINE_DUAL (default): r = P^T (d - F lambda) with the FP64 operator,
                          each correction a reduced-precision solve of F dl = r (inner_tol, default
                          1e-2); convergence as in FP64 (sqrt(r^T z) <= tol * initial).
                          FETI_REFINE_PRIMAL: r = f - K u element by element in FP64, each correction
                          a reduced-precision FETI solve of K du = r (its own dual problem, inner_tol
                          default 1e-3); converged when ||r|| <= tol ||f|| over the free DOFs (stats
                          eps0 = 1, eps = that ratio).  feti_recover_displacements then returns the
                          sum of the du; lambda_inout is output only and receives the sum of the
                          corrections' multipliers (each for its own residual load: not the
                          multipliers of f in general) */
} feti_options;

typedef struct {
  int dim;                       /* 2 or 3 */
  int tiles[3];                  /* subdomains per axis (unused axes: 1) */
  int elems[3];                  /* elements per subdomain per axis */
  double E0, Emin, nu, p;        /* SIMP parameters of Eq. 1 and Poisson ratio */
  const double* rho;             /* [n_elements] element densities */
  const unsigned char* dirichlet;/* [n_nodes*dim] 1 = DOF fixed to zero */
  const double* f;               /* [n_nodes*dim] global nodal load */
  int on_device;                 /* rho and f are device pointers (dirichlet is always host) */
} feti_problem;

typedef struct {
  int iterations;       /* Krylov iterations performed */
  int converged;        /* 1 if sqrt(r^T z) <= tol * initial value */
  int f_applies;        /* dual-operator columns applied (sum of retained ranks) */
  int last_rank;        /* retained directions in the last iteration */
  double eps0, eps;     /* initial and final sqrt(r^T z) (FP64 operator) */
  int refinements;      /* FETI_TF32: FP64 refinement steps taken (0 for FETI_FP64) */
} feti_stats;

/* Caller-supplied device allocator for a context's internal memory.
 * alloc(user, bytes, stream) returns device memory of the context's device
 * usable on `stream` (the context stream), or NULL on failure (the library then
 * returns FETI_ENOMEM); free(user, ptr, bytes, stream) releases a pointer that
 * alloc returned, with the same byte count.  The library frees every pointer
 * it was given, at the latest in feti_destroy, after synchronising the stream.
 * The callbacks are called from the thread that calls the library. */
typedef struct {
  void* (*alloc)(void* user, size_t bytes, void* stream);
  void (*free)(void* user, void* ptr, size_t bytes, void* stream);
  void* user;
} feti_allocator;

/* Fill *opt with the defaults listed above.  Never fails for non-null opt. */
feti_status feti_options_default(feti_options* opt);

/* Create a context bound to the current CUDA device and to `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * context (owned by the library until feti_destroy). */
feti_status feti_create(feti_ctx** out, const feti_options* opt, void* stream);

/* Install (a != NULL, both callbacks set) or remove (a == NULL: back to
 * cudaMallocAsync on the context stream) the allocator of the context's
 * internal device memory.  Allowed only while the context holds no device
 * memory -- after feti_create, before feti_setup_subdomains / feti_setup_batch
 * (FETI_ESTATE otherwise); FETI_EINVAL for a null callback.  Not part of the
 * paper's method: the ownership rule of the boundary. */
feti_status feti_set_allocator(feti_ctx* ctx, const feti_allocator* a);

/* Tear the mesh into subdomains and build every index map on the host
 * (Eqs. 4-5 for TFETI; Eqs. 8-10 and the corner primal set for FETI-DP;
 * pair-wise redundant multipliers at DOFs shared by more than two subdomains,
 * Section 3.1), then copy the maps and the problem data to the device.
 * May be called again to replace the problem (resets the call order).
 * Errors: FETI_EINVAL for inconsistent sizes or null pointers. */
feti_status feti_setup_subdomains(feti_ctx* ctx, const feti_problem* prob);

/* Set up a batch of n_problems independent state problems of uneven size in
 * one context (the batching form; the paper solves one problem at a time).
 * Every kernel launch then covers all problems; the problems keep their own
 * multipliers, primal DOFs and coarse problems, and feti_solve_dual runs one
 * PCG per problem with all per-problem scalars on the device, replaying a
 * CUDA graph of one iteration.  Requires FETI_FETIDP, FETI_PCG and FETI_FP64,
 * and equal E0, Emin, nu, p and dim across the batch (FETI_ENOTSUP / EINVAL
 * otherwise).  Vectors of the batch (lambda, u, rho, dc/drho) are the
 * problems' vectors concatenated in input order; feti_problem_result gives
 * each problem's offsets and statistics. */
feti_status feti_setup_batch(feti_ctx* ctx, const feti_problem* probs, int n_problems);

/* Per-problem results of a batch (or of a single problem, p = 0): offsets of
 * problem p in the concatenated DOF, element and multiplier vectors, its
 * Krylov statistics and, after feti_recover_displacements, its compliance
 * f_p^T u_p.  Each output pointer may be NULL. */
feti_status feti_problem_result(const feti_ctx* ctx, int p, int64_t* dof_offset, int64_t* elem_offset,
                                int64_t* lambda_offset, feti_stats* stats, double* compliance);

/* Replace the element densities (same mesh, same boundary conditions):
 * `rho` has n_elements entries, host or device per on_device.  Requires a
 * new feti_factorize before the next solve.  (Used by the SIMP loop,
 * Section 1.) */
feti_status feti_set_density(feti_ctx* ctx, const double* rho, int on_device);

/* Assemble the SIMP-weighted subdomain stiffness (Eqs. 1, 3), factorise its
 * interior block (banded Cholesky), form the Schur complement onto the
 * interface and corner DOFs, and from it the dense local dual blocks:
 * FETI-DP: F_s = [K_rr^{-1}]_bb, F_rc,s, local Kbar_cc (Eq. 12) and the
 * Dirichlet-preconditioner Schur complement S_s (Eq. 13); TFETI: a
 * generalised inverse of K_s on the interface (Section 2.1) and S_s.
 * Then the coarse problem (Kbar_cc for FETI-DP, G G^T for TFETI), the
 * scaling weights (Eq. 15) and the right-hand sides of Eq. 7 / Eq. 12.
 * All in FP64 on the device. */
feti_status feti_factorize(feti_ctx* ctx);

/* Run the Krylov solver (Algorithm 1 or its PCG/FO special cases) on the
 * dual problem.  lambda_inout: NULL, or a DEVICE array [n_lambda] used as the
 * initial multiplier (warm start) and overwritten with the result.  The
 * relative stopping test sqrt(r^T z) <= tol * eps0 takes eps0 at the method's
 * own initial multiplier (0 for FETI-DP, G^T (G G^T)^{-1} e for TFETI) also
 * when a warm start is given, so a good initial guess shortens the solve
 * (single problems; a batch measures each problem from its own start).
 * stats may be NULL.  Returns FETI_ENOTCONV if max_iter was reached (results
 * still valid) and FETI_EBREAKDOWN if no direction survived the rank test. */
feti_status feti_solve_dual(feti_ctx* ctx, double* lambda_inout, feti_stats* stats);

/* Recover the global displacement from the last solve: FETI-DP from the
 * second rows of Eq. 12 and Eq. 11; TFETI from u = K^+(f - B^T lambda) + R alpha
 * (Section 2.1).  u_out: [n_nodes*dim], device pointer if on_device != 0 else
 * host; a node shared by several subdomains gets the mean of its copies and
 * fixed DOFs are exactly zero.  compliance_out (host, may be NULL): f^T u. */
feti_status feti_recover_displacements(feti_ctx* ctx, double* u_out, int on_device,
                                       double* compliance_out);

/* SIMP compliance sensitivity from the recovered displacement (self-adjoint,
 * Section 1): dc/drho_e = -p rho_e^(p-1) (E0 - Emin) u_e^T k0 u_e.
 * dc_drho: [n_elements], device if on_device else host. */
feti_status feti_compliance_grad(feti_ctx* ctx, double* dc_drho, int on_device);

/* The dual operator on a block of directions (the hot path of Algorithm 1):
 * Y = F X with F the TFETI F of Eq. 7 or the condensed FETI-DP operator
 * F_rr + F_rc Kbar_cc^{-1} F_rc^T of Eq. 12, with the local blocks in the
 * context's precision (FETI_TF32: tensor-core products of the diagonally
 * scaled blocks).  X, Y: DEVICE column-major
 * [n_lambda x m] with leading dimensions ldx, ldy >= n_lambda.  Requires
 * feti_factorize. */
feti_status feti_apply_dual(feti_ctx* ctx, const double* X, int ldx, int m, double* Y, int ldy);

/* Test hook of the failure path (not part of the method).  The next
 * tensor-core product of ctx that runs in the one-tile-per-CTA kernel (the
 * FETI_TF32 and FETI_TF32X3 precisions) skips, in its first tile only, the
 * copy of K chunk `chunk` (0-based) and every later one, so that the MMA
 * lane's bounded wait (1 s) for it runs out: that product records the
 * time-out, frees its tensor memory and returns, and the call that launched it
 * returns FETI_ETIMEOUT; the context stays usable.  The hook is used by one
 * product and then cleared; chunk < 0 clears it.  No copy is left in flight. */
feti_status feti_test_skip_copy(feti_ctx* ctx, int chunk);

/* The block Dirichlet preconditioner of Algorithm 1: column s of Z is
 * B~^s S^s B~^sT r (Eq. 13 with the scaled B~ of Section 3.1), z = Z 1.
 * r: DEVICE [n_lambda]; Z: DEVICE column-major [n_lambda x n_subdomains] with
 * ldz >= n_lambda (may be NULL); z: DEVICE [n_lambda] (may be NULL). */
feti_status feti_apply_precond(feti_ctx* ctx, const double* r, double* Z, int ldz, double* z);

/* Allocation-free variant of feti_apply_precond (the paper has no
 * counterpart: this is a deployment aid).  Same arguments, same result.
 * It is meant for callers that cannot let the library call cudaMalloc while
 * they run -- e.g. code under a fixed device-memory budget or one that must
 * not bypass its own device allocator.  The two interface-space work vectors
 * live in a static device array of 4 MiB that every GPU loading the library
 * holds until the process exits; problems whose interface space has more
 * than 262144 entries (FETI_Q_N_B_TOTAL) are rejected with FETI_EINVAL.
 * All calls share that array: calls whose kernels overlap on the GPU race,
 * so serialise them.  The first call on a device looks up the array's device
 * address; make that first call before any stream capture.  That address
 * belongs to the device's primary context: after cudaDeviceReset the process
 * must not call this entry point on that device again.  Problems too large
 * for the array are rejected as soon as they are set up (before any device
 * work).  No CUDA or other allocation is made by this call. */
feti_status feti_apply_precond_noalloc(feti_ctx* ctx, const double* r, double* Z, int ldz, double* z);

/* r = f - K u over the free DOFs (0 on the fixed ones) in FP64, element by
 * element (Eq. 2 with the element moduli of Eq. 1 from the densities of the
 * last feti_factorize), for the whole set-up problem or batch.  u: device
 * [n_dofs] (NULL: u = 0); r: device [n_dofs] or NULL (internal scratch);
 * rel: host, receives ||r|| / ||f|| over the free DOFs (||r|| if that f is
 * zero), or NULL.  Errors: FETI_ESTATE before feti_factorize. */
feti_status feti_primal_residual(feti_ctx* ctx, const double* u, double* r, double* rel);

/* Integer facts about the set-up problem; key is one of FETI_Q_*. */
enum {
  FETI_Q_N_LAMBDA = 0, FETI_Q_N_SUBDOMAINS = 1, FETI_Q_N_PRIMAL = 2, FETI_Q_N_MODULES = 3,
  FETI_Q_N_B_TOTAL = 4, FETI_Q_N_DOFS = 5, FETI_Q_N_ELEMENTS = 6, FETI_Q_MAX_NB = 7,
  FETI_Q_DEVICE_BYTES = 8, FETI_Q_N_RBM = 9,
  FETI_Q_LAUNCHES = 10,  /* process-wide count of kernels this library has launched (any ctx state) */
  FETI_Q_N_PROBLEMS = 11,
  FETI_Q_GEMV_CONFIG = 12,  /* autotuned launch shape of the per-subdomain matrix-vector kernel (batches):
                              warps per CTA + 100 if vector loads; 0 = default */
  FETI_Q_TC_BYTES_F = 13,      /* reduced precision: bytes of the tensor-core product's stationary operand
                                  (every module's scaled blocks, all parts), read once per apply */
  FETI_Q_TC_BYTES_PER_COL = 14, /* reduced precision: bytes the product moves per direction: the
                                   gathered operand in (all parts) and the FP32 interface result out */
  FETI_Q_APPLY1_BYTES = 15,    /* FP64: algorithmic bytes of a one-direction dual-operator apply (PCG):
                                  every distinct module's F_s and F_rc read once, the coarse inverse
                                  (FETI-DP), the multiplier and interface vectors in and out */
  FETI_Q_BATCH_ROW_TILE = 16   /* batches, Algorithm 1: multiplier rows per work item of the block
                                  updates (W T, Q T, W -= W_j Psi_j), autotuned on the first batched
                                  solve by timing 1024..16384 (the split of the rows into work items
                                  changes the time, not the result); 0 before it */
};
feti_status feti_query(const feti_ctx* ctx, int key, int64_t* value);

/* Instrumentation (not part of the method): between feti_profile_begin and
 * feti_profile_end every FP64 GEMM launch of this process is bracketed by
 * CUDA events on its stream.  feti_profile_end synchronises the context
 * stream and returns (each pointer may be NULL) the summed algorithmic flops
 * of those products (2 M N K, or the structural count where a factor is
 * triangular), their summed device time in milliseconds, and the number of
 * profiled launches.  One profile may be active per process. */
feti_status feti_profile_begin(feti_ctx* ctx);
feti_status feti_profile_end(feti_ctx* ctx, double* gemm_flops, double* gemm_ms, int64_t* gemm_launches);

/* The tensor-core local products (FETI_TF32 / FETI_TF32X3) bracketed during
 * the last completed profile of this context: their summed algorithmic flops
 * (2 n_b (n_b + n_c) per subdomain and column, the corner coupling included
 * for FETI-DP; the split product's three passes count once), device time in
 * milliseconds and launch count.  Each pointer may be NULL. */
feti_status feti_profile_tensor(const feti_ctx* ctx, double* flops, double* ms, int64_t* launches);

/* Phases of the last completed profile (instrumentation): each phase region is
 * bracketed by CUDA events on the context stream (every launch inside counts),
 * with its algorithmic work -- flops for the FP64-pipe phases, bytes for the
 * memory-bound ones.  Arrays of FETI_N_PHASES entries, indexed by the enum:
 *   APPLY    dual-operator block apply Q = F W (Eq. 12; flops: sum_s 2 n_b^2 m plus
 *            the corner coupling 4 n_b n_c m and the coarse solve 2 n_c^2 m)
 *   PRECOND  preconditioner Z (Eq. 13; bytes: the distinct local blocks once, the
 *            residual and interface vectors, the dense Z of the simultaneous variant)
 *   PROJECT  TFETI projector (bytes: the block read for G X and read and written for
 *            the G^T update, its interface copy written and read)
 *   GRAM     Gram matrix, rank-revealing factorization and F-orthonormal transform
 *            (Algorithm 1; flops n_lambda m (m + 1) + 2 n_lambda k (k + 1))
 *   STEP     step length, multiplier and residual update, residual norm (bytes)
 *   ORTHO    full orthogonalization against the stored blocks (flops sum_j 4 n_lambda k_j m)
 *   FACTOR   local factorizations and coarse problem (time only: work 0)
 *   RECOVER  primal recovery (time only) */
enum { FETI_PHASE_APPLY = 0, FETI_PHASE_PRECOND = 1, FETI_PHASE_PROJECT = 2, FETI_PHASE_GRAM = 3,
       FETI_PHASE_STEP = 4, FETI_PHASE_ORTHO = 5, FETI_PHASE_FACTOR = 6, FETI_PHASE_RECOVER = 7,
       FETI_N_PHASES = 8 };
feti_status feti_profile_phases(const feti_ctx* ctx, double* work, double* ms, int64_t* count);

/* Layout of the multipliers, for comparing lambda-space vectors with an
 * independent implementation: for each multiplier l, out[6*l .. 6*l+5] =
 * (s1, local_dof1, sign1, s2, local_dof2, sign2); a single-subdomain
 * (Dirichlet) row has s2 = -1.  out: host [6 * n_lambda]. */
feti_status feti_lambda_layout(const feti_ctx* ctx, int32_t* out);

/* Dense local blocks of subdomain s after feti_factorize, for parity checks:
 * bdofs/cdofs (host int32 [n_b] / [n_c], may be NULL) receive the local DOF
 * ids of the interface / corner DOFs in the library's order; F [n_b*n_b],
 * S [n_b*n_b], Frc [n_b*n_c] (FETI-DP) receive F_s, S_s, F_rc,s row-major
 * (host, each may be NULL); nb, nc (host) receive the sizes. */
feti_status feti_local_blocks(feti_ctx* ctx, int s, int* nb, int* nc, int32_t* bdofs, int32_t* cdofs,
                              double* F, double* S, double* Frc);

/* The last error message of ctx (never NULL; "" if none). */
const char* feti_last_error(const feti_ctx* ctx);

/* Release the context and all of its device memory.  Accepts NULL. */
void feti_destroy(feti_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* FETI_GB300_H */
