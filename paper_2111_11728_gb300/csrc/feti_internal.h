// Internal declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/feti.h"

namespace feti {

// ---------------------------------------------------------------------------
// Host-side description of the torn problem (built by setup.cpp).
// ---------------------------------------------------------------------------

// Local DOF classes.  FETI-DP: interior (i), interface (b), corner primal (c),
// fixed and eliminated (x).  TFETI: i and b only (b = every DOF a row of B touches).
enum DofClass : int { CLS_I = 0, CLS_B = 1, CLS_C = 2, CLS_X = 3 };

// Subdomains with the same boundary situation share one DOF classification.
struct StructType {
  int e[3] = {1, 1, 1};          // elements per axis of the tile (its problem's elems)
  int ln[3] = {1, 1, 1};         // local nodes per axis
  int n_loc = 0;                 // local DOFs
  std::vector<int> cls;          // [n_loc] DofClass
  std::vector<int> idx;          // [n_loc] position inside its class list
  std::vector<int> ilist, blist, clist;   // local DOF ids per class (i, b, c order)
  int n_i = 0, n_b = 0, n_c = 0;
  int bw = 0;                    // half-bandwidth of K_ii in i-order
  // edge averages (FETI-DP, richer primal set): average a sits in c slot
  // avg_c[a]; the b slots of the other nodes of its edge are
  // avg_b[avg_off[a] .. avg_off[a + 1])
  std::vector<int> avg_c, avg_off, avg_b;
  int n_bc() const { return n_b + n_c; }
};

struct HostProblem {
  // mesh
  int dim = 2;
  int tiles[3] = {1, 1, 1}, elems[3] = {1, 1, 1};
  int nel[3] = {1, 1, 1}, nnod[3] = {1, 1, 1}, lnod[3] = {1, 1, 1};
  int64_t n_nodes = 0, n_elements = 0, n_dofs = 0;
  int n_sub = 0, n_loc_nodes = 0, n_loc_dofs = 0, n_loc_elems = 0;
  double E0 = 1, Emin = 0, nu = 0.3, p = 3;
  int method = FETI_FETIDP;

  // structure types and modules
  std::vector<StructType> types;
  std::vector<int> sub_type;     // [n_sub]
  std::vector<int> sub_module;   // [n_sub]
  std::vector<int> module_rep;   // [n_mod] representative subdomain
  std::vector<int> module_type;  // [n_mod]

  // interface (b) space: global b index = b_off[s] + position in the type's blist
  std::vector<int64_t> b_off;    // [n_sub + 1]
  int64_t n_b_total = 0;
  std::vector<int> b_sub;        // [n_b_total] owning subdomain

  // multipliers: each row has one or two (global b, sign) entries
  int64_t n_lam = 0;
  std::vector<int> lam_b0, lam_b1;        // [n_lam] global b indices (lam_b1 = -1 for one-entry rows)
  std::vector<signed char> lam_s0, lam_s1;
  std::vector<int> lam_group;             // [n_lam] sharing group (all copies of the DOF)
  std::vector<int> group_off, group_b;    // CSR over groups -> global b of every copy
  std::vector<int> b2l_off, b2l_lam;      // CSR global b -> multiplier rows
  std::vector<signed char> b2l_sign;

  // primal (FETI-DP corners)
  int n_primal = 0;
  std::vector<int64_t> c_off;             // [n_sub + 1] offset into c_glob
  std::vector<int> c_glob;                // primal index of each local corner DOF
  std::vector<int> prim_off, prim_src;    // CSR primal -> (c_off[s] + k) contributors

  // loads and output gather
  std::vector<int64_t> load_src;          // [n_sub * n_loc_dofs] global DOF feeding the local load, or -1
  std::vector<int64_t> dof_copy_off;      // [n_dofs + 1] CSR global DOF -> local copies
  std::vector<int64_t> dof_copy;          // s * n_loc_dofs + local dof
  std::vector<unsigned char> dirichlet;   // [n_dofs]

  // rigid-body modes (TFETI): n_rbm per subdomain
  int n_rbm = 0;

  // per-subdomain placement (a batch concatenates independent problems)
  std::vector<int64_t> loc_off;           // [n_sub + 1] offset of each subdomain's local vectors
  std::vector<int> sub_prob;              // [n_sub] problem of each subdomain
  int64_t n_loc_total = 0;
  // per-problem ranges (one entry for a single problem)
  int n_prob = 1;
  std::vector<int64_t> prob_dof_off, prob_el_off, prob_lam_off;   // [n_prob + 1]
  std::vector<int> prob_sub_off, prob_primal_off;                  // [n_prob + 1]
  std::vector<int> prob_nel;                                       // [3 * n_prob]
};

// Concatenate independently built problems into one description (offsets
// shifted; each problem keeps its own types, modules, multipliers, primal
// DOFs).  All parts must share dim and method.
std::string merge_host_problems(std::vector<HostProblem>& parts, HostProblem& out);

// The multiplier rows cut into ranges of at most max_rows consecutive rows,
// never between two rows of one interface DOF; per range the DOFs ("slots")
// whose rows it holds -- those with one row first, then those with several,
// each by position -- with their operand position pos_of_b[b], the DOF b and
// its rows as offsets in the range (~offset for a row entering with sign -1),
// in the DOF's row order.  DOFs without rows get no slot.
struct SpreadTables {
  std::vector<int> row0;        // [n_ranges + 1] first row of each range
  std::vector<int> slot_off;    // [n_ranges + 1] slots of range r: [slot_off[r], slot_off[r + 1])
  std::vector<int> slot_pos, slot_b;
  std::vector<int> ent_off;     // [n_slots + 1]
  std::vector<short> ent;
};
std::string build_spread_tables(const HostProblem& hp, const std::vector<int64_t>& pos_of_b, int max_rows,
                                SpreadTables& out);

// Builds the host description; returns an error message or "".  edge_mode:
// 0 corners only, 1 every shared tile-grid edge averaged, 2 only the edges
// across which the sharers' diagonal stiffness jumps by >= jump_ratio.
std::string build_host_problem(const feti_problem& prob, int method, int dedup,
                               const double* rho_host, HostProblem& hp, int edge_mode = 0,
                               double jump_ratio = 10.0);

// Local node (lexicographic in the tile) -> tile-local integer coordinates.
inline void local_node_coords(const HostProblem& hp, int ln, int c[3]) {
  c[0] = ln % hp.lnod[0];
  int r = ln / hp.lnod[0];
  c[1] = r % hp.lnod[1];
  c[2] = r / hp.lnod[1];
}

// ---------------------------------------------------------------------------
// Device-side data.
// ---------------------------------------------------------------------------

// Per-structure-type device info.
struct DevType {
  int n_loc, n_i, n_b, n_c, bw;
  int n_avg;                     // edge averages (0: corners only)
  int e[3];                      // elements per axis of the tile
  int ln[3];                     // local nodes per axis
  const int* cls_idx;            // [n_loc] (cls << 24) | idx
  const int* ilist;              // [n_i]
  const int* blist;              // [n_b]
  const int* clist;              // [n_c]
  const double* Rraw;            // [n_b x n_rbm] rigid modes at the b DOFs (TFETI)
  const double* Rhat;            // [n_b x n_rbm] orthonormal basis of their span (TFETI)
  const int* avg_c;              // [n_avg] c slot of each edge average
  const int* avg_off;            // [n_avg + 1]
  const int* avg_b;              // b slots of the edges' other nodes
};

// Per-module offsets into the module arrays (in doubles).
struct DevModule {
  int type;
  int rep;                       // representative subdomain
  int64_t lcol, lrow, rdiag;     // band factor (column and row form), reciprocal diagonal
  int64_t Y;                     // [n_i x n_bc] row-major: L^{-1} K_{i,bc}
  int64_t S;                     // [n_bc x n_bc] row-major Schur complement onto b+c
  int64_t W;                     // [n_b x n_b] Cholesky factor of S_bb (work)
  int64_t Li;                    // [n_b x n_b] its inverse (work)
  int64_t F;                     // [n_b x n_b] row-major local dual block
  int64_t Frc;                   // [n_b x n_c] row-major (FETI-DP)
  int64_t Kb;                    // [n_c x n_c] local Kbar_cc (FETI-DP)
  int64_t Rb;                    // [n_b x n_rbm] orthonormal rigid modes on b (TFETI)
  int64_t Kl;                    // [n_b x n_b] row-major K_bb (lumped preconditioner; -1 if unused)
};

// Per-subdomain device info.
struct DevSub {
  int module;
  int type;
  int64_t b_off;                 // into the global b space
  int64_t c_off;                 // into c_glob
  int tile[3];                   // tile coordinates inside its problem
  int prob;                      // problem index
  int64_t loc_off;               // into the local vectors (loads, displacements)
  int64_t e_off;                 // element offset of its problem
  int nel[3];                    // global element grid of its problem
  int pad2;
};

struct GemmDesc;
struct DenseDesc;
struct RrDesc;
struct SegVec;
struct SegRed;

struct Ctx {
  feti_options opt{};
  cudaStream_t stream = nullptr;
  std::string err;
  int state = 0;                 // 0 created, 1 set up, 2 factorized, 3 solved, 4 recovered
  int device = 0;
  HostProblem hp;
  std::vector<void*> allocs;     // every device allocation (freed at destroy)
  std::vector<size_t> alloc_bytes;   // their sizes
  feti_allocator user_alloc{};   // caller's allocator (feti_set_allocator), if installed
  int have_user_alloc = 0;
  size_t device_bytes = 0;
  double* h_pin = nullptr;       // pinned host scalars

  // problem data
  double* d_rho = nullptr;       // [n_elements]
  double* d_E = nullptr;         // [n_elements] SIMP moduli
  double* d_fglob = nullptr;     // [n_dofs]
  double* d_k0 = nullptr;        // element stiffness for E = 1
  std::vector<double> h_k0;
  // types / modules / subdomains
  DevType* d_types = nullptr;
  DevModule* d_mods = nullptr;
  DevSub* d_subs = nullptr;
  std::vector<DevType> h_types;
  std::vector<DevModule> h_mods;
  std::vector<DevSub> h_subs;
  int n_mod = 0, max_nb = 1, max_nc = 1;
  // algorithmic flops of the batched products (per column where they scale with m)
  double fl_F = 0, fl_FrcT = 0, fl_Frc = 0, fl_schur = 0, fl_frcmake = 0, fl_kbmake = 0;
  double fl_coarse = 0;          // flops of one coarse solve column (FETI-DP: sum_p 2 n_c(p)^2)
  double bytes_S = 0;            // the distinct preconditioner blocks S_bb, in bytes
  double bytes_apply1 = 0;       // algorithmic bytes of a one-direction FP64 apply
  void* prof = nullptr;          // active GEMM profile (GemmProfile*)
  double* d_modmem = nullptr;    // module arrays
  int64_t modmem_len = 0;
  // maps
  int *d_lam_b0 = nullptr, *d_lam_b1 = nullptr, *d_lam_group = nullptr;
  signed char *d_lam_s0 = nullptr, *d_lam_s1 = nullptr;
  int *d_group_off = nullptr, *d_group_b = nullptr;
  int *d_b2l_off = nullptr, *d_b2l_lam = nullptr;
  // precision form, operand built from the multiplier side: ranges of consecutive
  // rows (d_sp_row0), the operand slots whose rows lie in each range
  // (d_sp_slot_off: position, interface DOF, FP32 sqrt(D)) and each slot's rows
  // relative to its range (d_sp_ent_off; ~rel for a row entering with sign -1)
  int *d_sp_row0 = nullptr, *d_sp_slot_off = nullptr, *d_sp_pos = nullptr, *d_sp_b = nullptr;
  int* d_sp_ent_off = nullptr;
  short* d_sp_ent = nullptr;
  float* d_sp_sd = nullptr;
  int n_spread_ranges = 0, n_spread_slots = 0;
  signed char* d_b2l_sign = nullptr;
  int* d_b_sub = nullptr;
  int* d_c_glob = nullptr;
  int* d_c_sub = nullptr;
  int64_t* d_c_off = nullptr;    // [n_sub] c offsets
  int *d_prim_off = nullptr, *d_prim_src = nullptr;
  int64_t* d_load_src = nullptr;
  int64_t *d_dof_copy_off = nullptr, *d_dof_copy = nullptr;
  unsigned char* d_dirichlet = nullptr;
  // per-b data
  double* d_diagKb = nullptr;    // [n_b_total] diagonal stiffness of each b copy
  double* d_w0 = nullptr;        // [n_lam] scaling weight of entry 0
  double* d_w1 = nullptr;        // [n_lam] scaling weight of entry 1
  // per-subdomain vectors
  double* d_floc = nullptr;      // [n_sub * n_loc_dofs] local loads
  double* d_h = nullptr;         // [sum n_i] L^{-1} f_i per subdomain
  double* d_t = nullptr;         // [sum n_i] recovery work
  int64_t* d_ioff = nullptr;     // [n_sub + 1] offsets of per-subdomain i-vectors
  std::vector<int64_t> h_ioff;
  double* d_ft = nullptr;        // [n_b_total + n_c_total] condensed loads f~ (b part, then c part)
  int64_t n_c_total = 0;
  // coarse
  double* d_Kbar = nullptr;      // [n_coarse^2]
  double* d_Kbar_L = nullptr;    // [n_coarse^2] inverse Cholesky factor (work)
  double* d_Kbar_inv = nullptr;  // [n_coarse^2] explicit inverse
  float* d_Kbar_inv32 = nullptr; // precision form, one problem: FP32 copy of the inverse
  float* d_coarse_part = nullptr;   // its split-K partials and FP32 right-hand sides (tc_coarse_scratch)
  double* d_coarse_work = nullptr;   // blocked coarse factorisation work
  // precision form (FETI_TF32)
  float* d_fmem = nullptr;       // FP32 copies at the module offsets: Shat at M.W
  void* d_fa_hi = nullptr;       // [fa_rows x fa_pitch] Fhat rows of every module (TF32 or BF16), zero padded
  void* d_fa_lo = nullptr;       // same layout: rounding of the remainder (split products)
  int64_t fa_pitch = 0, fa_rows = 0;
  int* d_frow = nullptr;         // [n_mod] first arena row of each module
  int64_t nbp_total = 0;         // interface space with each subdomain padded to the format's chunk
  int64_t* d_bpad = nullptr;     // [n_sub] padded offsets
  void *d_xb_hi = nullptr, *d_xb_lo = nullptr;    // [m x nbp_total] gathered scaled directions
  float* d_Yb32 = nullptr;       // [m x n_b_total] output of the tensor-core product (FP32)
  int xb_cap = 0;
  int tc_aug = 0;                // FETI-DP corner coupling appended to the operands (K-extension)
  int4* d_tiles = nullptr;       // persistent tensor-core kernel: (subdomain, row tile, column tile)
  int64_t tiles_cap = 0;
  int n_tiles = 0, tiles_ncb = 0, n_sm = 0;
  int n_ctiles = 0;              // corner tiles after the n_tiles product tiles in d_tiles
  int fcrow0 = 0;                // first arena row of the corner blocks (128 rows per module)
  int n_ctiles_rows = 0;         // 1 when the arena carries corner blocks
  double fl_tc = 0.0;            // algorithmic flops of the tensor-core product per column
  int test_skip_chunk = -1;      // test hook: K chunk whose copy the next TF32 product's first tile skips
  int64_t tc_bytes_f = 0;        // algorithmic bytes: scaled blocks (read once per apply)
  int64_t tc_bytes_col = 0;      // algorithmic bytes per column: operand in + FP32 result out
  double prof_tc_flops = 0.0, prof_tc_ms = 0.0;   // tensor-core products of the last profile
  double prof_ph_work[8] = {}, prof_ph_ms[8] = {};  // phases of the last profile
  int64_t prof_ph_count[8] = {};
  int64_t prof_tc_launches = 0;
  double* d_sqrtDF = nullptr;    // [n_b_total] sqrt(diag F_s)
  double* d_sqrtDS = nullptr;    // [n_b_total] sqrt(diag S_s)
  double *d_rout = nullptr, *d_zout = nullptr, *d_dl = nullptr;   // refinement vectors
  double *d_f0 = nullptr, *d_uacc = nullptr, *d_lamacc = nullptr;  // primal refinement: load, sums
  double* d_ubest = nullptr;                                       // the best summed u so far
  double* d_rres = nullptr;                                        // primal residual scratch [n_dofs]
  int u_refined = 0;             // the last solve refined on the primal residual: u = d_uacc
  // per-problem tables (device)
  int64_t *d_prob_el_off = nullptr, *d_prob_dof_off = nullptr, *d_prob_lam_off = nullptr;
  int *d_prob_nel = nullptr, *d_prob_primal_off = nullptr;
  int64_t* d_kbar_off = nullptr;     // [n_prob + 1] offsets of the per-problem coarse blocks
  std::vector<int64_t> h_kbar_off;
  int* d_row_prob = nullptr;         // [n_primal] problem of each primal row
  int* d_lam_prob = nullptr;         // [n_lam] problem of each multiplier
  GemmDesc* d_gemm_coarse = nullptr; // per-problem coarse GEMMs (batches)
  DenseDesc* d_dense_coarse_batch = nullptr;
  int max_np = 0;
  int64_t bk_rtile = 0;             // autotuned row tile of the batched Algorithm 1's block updates (0: not yet)
  int gemv_cfg = 0;                  // autotuned launch shape of the per-subdomain GEMV (0: default)
  float gemv_ms = 0.f;
  // batched PCG state
  cudaStream_t cap_stream = nullptr;  // private stream for graph capture
  cudaEvent_t cap_event = nullptr;
  double* d_bstate = nullptr;        // per-problem scalars
  int* d_bflags = nullptr;           // per-problem activity / iteration / convergence
  std::vector<feti_stats> prob_stats;
  std::vector<double> prob_compliance;
  double* d_fbar = nullptr;      // [n_primal]
  int n_coarse = 0;
  double* d_gwork = nullptr;     // TFETI: [n_lam x 64] work block for forming G G^T
  double* d_e = nullptr;         // TFETI: e = -R^T f
  double* d_alpha = nullptr;     // TFETI: rigid-body amplitudes
  double *d_ct1 = nullptr, *d_ct2 = nullptr;   // [n_coarse x blk] projector work
  // dual right-hand side and solution
  double* d_d = nullptr;         // [n_lam]
  double* d_lam0 = nullptr;      // [n_lam]
  double* d_lam = nullptr;       // [n_lam]
  double* d_uloc = nullptr;      // [n_sub * n_loc_dofs]
  double* d_uglob = nullptr;     // [n_dofs]
  int have_solution = 0;
  // scratch
  double* d_scalar = nullptr;    // small device scalars
  int* d_status = nullptr;       // device status word
  int* d_kdev = nullptr;         // rank from the rank-revealing factorization
  int* d_perm = nullptr;         // its pivot order
  double* d_red = nullptr;       // reduction partials (>= 1024)
  // block buffers for the dual operator
  int blk_cap = 0;
  double *d_Xb = nullptr, *d_Yb = nullptr, *d_Cb = nullptr, *d_Vraw = nullptr, *d_V = nullptr, *d_Vc = nullptr;
  double *d_pb0 = nullptr, *d_pb1 = nullptr;   // [n_b_total] vectors
  float* d_pbh = nullptr;                      // [n_b_total] FP32 scratch (precision form)
  // GEMM descriptors (device)
  GemmDesc *d_gemm_F = nullptr, *d_gemm_FrcT = nullptr, *d_gemm_Frc = nullptr;
  GemmDesc *d_gemm_schur = nullptr, *d_gemm_frcmake = nullptr, *d_gemm_kbmake = nullptr;
  DenseDesc *d_dense_mod = nullptr, *d_dense_coarse = nullptr;
  // Krylov buffers
  int kr_cap = 0;
  double *d_r = nullptr, *d_z = nullptr, *d_lamt = nullptr, *d_Wb = nullptr, *d_Qb = nullptr, *d_Wn = nullptr;
  double *d_Delta = nullptr, *d_T = nullptr, *d_gamma = nullptr, *d_rrwork = nullptr, *d_split = nullptr;
  int64_t split_cap = 0;
  std::vector<double*> hist_W, hist_Q;
  std::vector<int> hist_k;
  // edge averages (richer FETI-DP primal set)
  int max_avg = 0;                         // most edge averages in one type (0: corners only)
  int* d_c_iota = nullptr;                 // [n_c_total] identity map of the c space
  double* d_ucl = nullptr;                 // [n_c_total] nodal values at the c slots (recovery)
  // batched Algorithm 1 (a block of directions per problem of a batch)
  int* d_b_lcol = nullptr;                 // [n_b_total] subdomain index inside its problem
  double *d_bk_delta = nullptr, *d_bk_T = nullptr, *d_bk_work = nullptr, *d_bk_gam = nullptr;
  double *d_bk_rz = nullptr, *d_bk_part = nullptr, *d_bk_split = nullptr;
  int *d_bk_perm = nullptr, *d_bk_k = nullptr;
  RrDesc* d_bk_rr = nullptr;
  SegVec* d_bk_vec = nullptr;
  GemmDesc* d_bk_desc = nullptr;
  SegRed* d_bk_red = nullptr;
  int64_t bk_split_cap = 0, bk_desc_cap = 0, bk_red_cap = 0;
  GemmDesc* d_bk_fchunks = nullptr;        // local F_s products per column chunk, N capped per subdomain
  int64_t bk_fchunks_cap = 0;
  const GemmDesc* gemm_F_active = nullptr; // when set, the local products use these descriptors
  std::vector<double*> bk_hW, bk_hQ;       // packed history blocks (one per iteration)
  std::vector<int64_t> bk_hcap;
  feti_stats last{};
};

// error helpers
#define FETI_CUDA_TRY(ctx, expr)                                                     \
  do {                                                                               \
    cudaError_t _e = (expr);                                                         \
    if (_e != cudaSuccess) {                                                         \
      (ctx)->err = std::string(#expr) + ": " + cudaGetErrorString(_e);              \
      return FETI_ECUDA;                                                             \
    }                                                                                \
  } while (0)

}  // namespace feti
