// Finite-element kernels: SIMP moduli (Eq. 1), deterministic gather-form
// assembly of each module's stiffness (Eq. 3) straight into the blocks the
// factorization needs, k-scaling weights (Eq. 15), load split, output gather
// and the SIMP compliance sensitivity.
//
// Element-local node order used on the device: node a sits at offset
// (a & 1, (a >> 1) & 1, (a >> 2) & 1) inside the unit element; element DOF
// = dim * a + direction.
#include <algorithm>
#include <cmath>

#include "kernels.h"

namespace feti {

namespace {

struct MeshArgs {
  int dim;
  int e[3];      // elements per subdomain per axis
  int ln[3];     // local nodes per axis
  int nel[3];    // global elements per axis
  int nnod[3];   // global nodes per axis
};

MeshArgs mesh_args(const HostProblem& hp) {
  MeshArgs m;
  m.dim = hp.dim;
  for (int a = 0; a < 3; ++a) {
    m.e[a] = a < hp.dim ? hp.elems[a] : 1;
    m.ln[a] = hp.lnod[a];
    m.nel[a] = hp.nel[a];
    m.nnod[a] = hp.nnod[a];
  }
  return m;
}

__global__ void k_moduli(const double* __restrict__ rho, int64_t n, double E0, double Emin, double p,
                         double* __restrict__ E) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) E[i] = Emin + pow(rho[i], p) * (E0 - Emin);
}

// One thread per local DOF a of one module: row a of K^s, summed over the
// elements that contain both end nodes (no atomics, fixed order), routed to
// the K_ii band (lower part), Y = K_{i,bc} or S = K_{bc,bc}.
__global__ void k_assemble(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                           const DevSub* __restrict__ subs, const double* __restrict__ E,
                           const double* __restrict__ k0, double* __restrict__ mem, MeshArgs g) {
  const DevModule M = mods[blockIdx.y];
  const DevType T = types[M.type];
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= T.n_loc) return;
  const int ca = T.cls_idx[a];
  const int cla = ca >> 24, ia = ca & 0xffffff;
  if (cla == CLS_X) return;
  const DevSub S = subs[M.rep];
  const int dim = g.dim, nen = 1 << dim, nek = nen * dim;
  const int na = a / dim, da = a % dim;
  const int c0 = na % T.ln[0], c1 = (na / T.ln[0]) % T.ln[1], c2 = na / (T.ln[0] * T.ln[1]);
  const int nb = T.n_b, nbc = T.n_b + T.n_c, W = T.bw + 1;
  double* Lcol = mem + M.lcol;
  double* Y = mem + M.Y;
  double* Sm = mem + M.S;
  const int zlo = dim == 3 ? -1 : 0, zhi = dim == 3 ? 1 : 0;
  for (int dz = zlo; dz <= zhi; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int q0 = c0 + dx, q1 = c1 + dy, q2 = c2 + dz;
        if (q0 < 0 || q0 > T.e[0] || q1 < 0 || q1 > T.e[1]) continue;
        if (dim == 3 && (q2 < 0 || q2 > T.e[2])) continue;
        const int nbn = q0 + T.ln[0] * (q1 + T.ln[1] * q2);
        for (int db = 0; db < dim; ++db) {
          const int b = nbn * dim + db;
          const int cb = T.cls_idx[b];
          const int clb = cb >> 24, ib = cb & 0xffffff;
          if (clb == CLS_X) continue;
          if (cla == CLS_I && clb == CLS_I && ib > ia) continue;   // upper band: not stored
          if (cla != CLS_I && clb == CLS_I) continue;             // stored by the i-row as Y
          double v = 0.0;
          // elements containing node a: origin = c - o, o in {0,1}^dim
          for (int o = 0; o < nen; ++o) {
            const int o0 = o & 1, o1 = (o >> 1) & 1, o2 = (o >> 2) & 1;
            const int e0 = c0 - o0, e1 = c1 - o1, e2 = c2 - o2;
            if (e0 < 0 || e0 >= T.e[0] || e1 < 0 || e1 >= T.e[1]) continue;
            if (dim == 3 && (e2 < 0 || e2 >= T.e[2])) continue;
            const int p0 = q0 - e0, p1 = q1 - e1, p2 = q2 - e2;
            if (p0 < 0 || p0 > 1 || p1 < 0 || p1 > 1) continue;
            if (dim == 3 && (p2 < 0 || p2 > 1)) continue;
            const int lb = p0 | (p1 << 1) | (p2 << 2);
            const int64_t ge0 = (int64_t)S.tile[0] * T.e[0] + e0;
            const int64_t ge1 = (int64_t)S.tile[1] * T.e[1] + e1;
            const int64_t ge2 = dim == 3 ? (int64_t)S.tile[2] * T.e[2] + e2 : 0;
            const double Ee = E[S.e_off + ge0 + S.nel[0] * (ge1 + (int64_t)S.nel[1] * ge2)];
            v = fma(Ee, k0[(o * dim + da) * nek + lb * dim + db], v);
          }
          if (cla == CLS_I && clb == CLS_I) {
            Lcol[(int64_t)ib * W + (ia - ib)] = v;
          } else if (cla == CLS_I) {
            const int j = clb == CLS_B ? ib : nb + ib;
            Y[(int64_t)ia * nbc + j] = v;
          } else {
            const int r = cla == CLS_B ? ia : nb + ia;
            const int j = clb == CLS_B ? ib : nb + ib;
            Sm[(int64_t)r * nbc + j] = v;
          }
        }
      }
}

// diagKb[b_off[s] + k] = K^s_bb(k, k) (read before the Schur update)
__global__ void k_diag_b(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                         const DevSub* __restrict__ subs, const double* __restrict__ mem,
                         double* __restrict__ diagKb) {
  const DevSub S = subs[blockIdx.y];
  const DevModule M = mods[S.module];
  const DevType T = types[S.type];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= T.n_b) return;
  const int nbc = T.n_b + T.n_c;
  diagKb[S.b_off + k] = mem[M.S + (int64_t)k * nbc + k];
}

// Kl = K_bb, the interface block of the assembled local stiffness (held in
// the S slot until the Schur update): the lumped preconditioner's block.
__global__ void k_copy_kbb(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                           double* __restrict__ mem) {
  const DevModule M = mods[blockIdx.y];
  const DevType T = types[M.type];
  const int n = T.n_b, nbc = T.n_b + T.n_c;
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    mem[M.Kl + e] = mem[M.S + (int64_t)i * nbc + j];
  }
}

// Eq. (15) with summed denominators (k-scaling) or 1/multiplicity.
__global__ void k_weights(int64_t n_lam, const int* __restrict__ b0, const int* __restrict__ b1,
                          const int* __restrict__ grp, const int* __restrict__ goff,
                          const int* __restrict__ gb, const double* __restrict__ diagKb, int kind,
                          double* __restrict__ w0, double* __restrict__ w1) {
  int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= n_lam) return;
  if (b1[l] < 0) { w0[l] = 1.0; w1[l] = 0.0; return; }
  const int g = grp[l];
  if (kind == FETI_SCALING_MULT) {
    const double w = 1.0 / (double)(goff[g + 1] - goff[g]);
    w0[l] = w; w1[l] = w;
    return;
  }
  double den = 0.0;
  for (int q = goff[g]; q < goff[g + 1]; ++q) den += diagKb[gb[q]];
  w0[l] = diagKb[b1[l]] / den;
  w1[l] = diagKb[b0[l]] / den;
}

__global__ void k_load_gather(const int64_t* __restrict__ src, int64_t n, const double* __restrict__ f,
                              double* __restrict__ floc) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t q = src[i];
  floc[i] = q >= 0 ? f[q] : 0.0;
}

// Global u: mean of the subdomain copies, fixed DOFs exactly zero.
__global__ void k_gather_u(int64_t n_dofs, const int64_t* __restrict__ off, const int64_t* __restrict__ cp,
                           const unsigned char* __restrict__ fixed, const double* __restrict__ uloc,
                           double* __restrict__ u) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= n_dofs) return;
  if (fixed[q]) { u[q] = 0.0; return; }
  double s = 0.0;
  const int64_t b = off[q], e = off[q + 1];
  for (int64_t t = b; t < e; ++t) s += uloc[cp[t]];
  u[q] = e > b + 1 ? s / (double)(e - b) : s;
}

// dc/drho_e = -p rho_e^(p-1) (E0 - Emin) u_e^T k0 u_e; elements of all
// problems of a batch are numbered consecutively (problem tables el_off,
// dof_off, nel).
__global__ void k_grad(int dim, int n_prob, const int64_t* __restrict__ el_off, const int64_t* __restrict__ dof_off,
                       const int* __restrict__ pnel, const double* __restrict__ rho, const double* __restrict__ u,
                       const double* __restrict__ k0, double E0, double Emin, double p,
                       double* __restrict__ out) {
  const int64_t ge = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (ge >= el_off[n_prob]) return;
  int lo = 0, hi = n_prob;                       // problem containing element ge
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (el_off[mid] <= ge) lo = mid; else hi = mid;
  }
  const int nel0 = pnel[3 * lo], nel1 = pnel[3 * lo + 1];
  const int64_t e = ge - el_off[lo];
  const int nen = 1 << dim, nek = nen * dim;
  const int64_t x = e % nel0, y = (e / nel0) % nel1, z = e / ((int64_t)nel0 * nel1);
  const int64_t nn0 = nel0 + 1, nn1 = nel1 + 1;
  const double* up = u + dof_off[lo];
  double ue[24];
  for (int a = 0; a < nen; ++a) {
    const int64_t nx = x + (a & 1), ny = y + ((a >> 1) & 1), nz = z + ((a >> 2) & 1);
    const int64_t node = nx + nn0 * (ny + nn1 * nz);
    for (int d = 0; d < dim; ++d) ue[a * dim + d] = up[node * dim + d];
  }
  double en = 0.0;
  for (int i = 0; i < nek; ++i) {
    double t = 0.0;
    for (int j = 0; j < nek; ++j) t = fma(k0[i * nek + j], ue[j], t);
    en = fma(ue[i], t, en);
  }
  out[ge] = -p * pow(rho[ge], p - 1.0) * (E0 - Emin) * en;
}

// r = f - K u element by element (Eq. 2 with the SIMP moduli E_e of Eq. 1),
// one thread per global DOF: the DOF's row of every element around its node,
// the elements taken in a fixed order (x, then y, then z offset), so that the
// sum is deterministic; fixed DOFs get r = 0 (u null: u = 0).  Problems of a batch are
// numbered consecutively (tables dof_off, el_off, nel).
__global__ void k_residual(int dim, int n_prob, const int64_t* __restrict__ dof_off,
                           const int64_t* __restrict__ el_off, const int* __restrict__ pnel,
                           const double* __restrict__ E, const double* __restrict__ k0,
                           const unsigned char* __restrict__ dirichlet, const double* __restrict__ f,
                           const double* __restrict__ u, double* __restrict__ r) {
  const int64_t gq = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gq >= dof_off[n_prob]) return;
  int lo = 0, hi = n_prob;                       // problem containing DOF gq
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (dof_off[mid] <= gq) lo = mid; else hi = mid;
  }
  if (dirichlet[gq]) { r[gq] = 0.0; return; }
  if (!u) { r[gq] = f[gq]; return; }            // u = 0: the free part of f
  const int nel0 = pnel[3 * lo], nel1 = pnel[3 * lo + 1], nel2 = dim == 3 ? pnel[3 * lo + 2] : 1;
  const int64_t q = gq - dof_off[lo];
  const int64_t node = q / dim;
  const int comp = (int)(q % dim);
  const int64_t nn0 = nel0 + 1, nn1 = nel1 + 1;
  const int64_t nx = node % nn0, ny = (node / nn0) % nn1, nz = node / (nn0 * nn1);
  const int nen = 1 << dim, nek = nen * dim;
  const double* up = u + dof_off[lo];
  const double* Ep = E + el_off[lo];
  double acc = f[gq];
  for (int o = 0; o < nen; ++o) {                // element at (nx, ny, nz) minus offset o
    const int64_t ex = nx - (o & 1), ey = ny - ((o >> 1) & 1), ez = nz - ((o >> 2) & 1);
    if (ex < 0 || ey < 0 || ez < 0 || ex >= nel0 || ey >= nel1 || ez >= nel2) continue;
    const int ln = o;                            // the node's local index in that element
    const int row = ln * dim + comp;
    double s = 0.0;
    for (int a = 0; a < nen; ++a) {
      const int64_t an = (ex + (a & 1)) + nn0 * ((ey + ((a >> 1) & 1)) + nn1 * (ez + ((a >> 2) & 1)));
      for (int d = 0; d < dim; ++d) s = fma(k0[row * nek + a * dim + d], up[an * dim + d], s);
    }
    acc = fma(-Ep[ex + (int64_t)nel0 * (ey + (int64_t)nel1 * ez)], s, acc);
  }
  r[gq] = acc;
}

}  // namespace

// Reference element stiffness for E = 1 (plane stress in 2D), by 2-point
// Gauss quadrature per axis, which integrates the multilinear unit element
// exactly.  Device element-node order (see the file header).
void element_stiffness_host(int dim, double nu, double* k0) {
  const int nen = 1 << dim, nek = nen * dim;
  double D[6][6] = {};
  int nv;
  if (dim == 2) {
    nv = 3;
    const double c = 1.0 / (1.0 - nu * nu);
    D[0][0] = c; D[0][1] = c * nu; D[1][0] = c * nu; D[1][1] = c; D[2][2] = c * 0.5 * (1.0 - nu);
  } else {
    nv = 6;
    const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = 0.5 / (1.0 + nu);
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) D[i][j] = lam;
      D[i][i] += 2.0 * mu;
      D[3 + i][3 + i] = mu;
    }
  }
  for (int i = 0; i < nek * nek; ++i) k0[i] = 0.0;
  const double gp[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
  const int nq = dim == 2 ? 4 : 8;
  for (int q = 0; q < nq; ++q) {
    const double xi[3] = {gp[q & 1], gp[(q >> 1) & 1], gp[(q >> 2) & 1]};
    const double w = dim == 2 ? 0.25 : 0.125;
    double G[8][3];
    for (int a = 0; a < nen; ++a) {
      const int off[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
      double f[3], df[3];
      for (int d = 0; d < dim; ++d) {
        f[d] = off[d] ? xi[d] : 1.0 - xi[d];
        df[d] = off[d] ? 1.0 : -1.0;
      }
      for (int d = 0; d < dim; ++d) {
        double v = df[d];
        for (int e = 0; e < dim; ++e) if (e != d) v *= f[e];
        G[a][d] = v;
      }
    }
    double B[6][24] = {};
    for (int a = 0; a < nen; ++a) {
      if (dim == 2) {
        B[0][2 * a] = G[a][0];
        B[1][2 * a + 1] = G[a][1];
        B[2][2 * a] = G[a][1]; B[2][2 * a + 1] = G[a][0];
      } else {
        B[0][3 * a] = G[a][0];
        B[1][3 * a + 1] = G[a][1];
        B[2][3 * a + 2] = G[a][2];
        B[3][3 * a + 1] = G[a][2]; B[3][3 * a + 2] = G[a][1];
        B[4][3 * a] = G[a][2]; B[4][3 * a + 2] = G[a][0];
        B[5][3 * a] = G[a][1]; B[5][3 * a + 1] = G[a][0];
      }
    }
    for (int i = 0; i < nek; ++i)
      for (int j = 0; j < nek; ++j) {
        double s = 0.0;
        for (int r = 0; r < nv; ++r)
          for (int t = 0; t < nv; ++t) s += B[r][i] * D[r][t] * B[t][j];
        k0[i * nek + j] += w * s;
      }
  }
  for (int i = 0; i < nek; ++i)
    for (int j = i + 1; j < nek; ++j) {
      const double v = 0.5 * (k0[i * nek + j] + k0[j * nek + i]);
      k0[i * nek + j] = v; k0[j * nek + i] = v;
    }
}

cudaError_t launch_moduli(const Ctx& c, double* E, cudaStream_t st) {
  const int64_t n = c.hp.n_elements;
  k_moduli<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c.d_rho, n, c.hp.E0, c.hp.Emin, c.hp.p, E);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_assemble_with(const Ctx& c, const double* E, cudaStream_t st) {
  int maxn = 0;
  for (auto& t : c.h_types) maxn = std::max(maxn, t.n_loc);
  dim3 grid((maxn + 127) / 128, c.n_mod);
  (void)mesh_args;
  k_assemble<<<grid, 128, 0, st>>>(c.d_types, c.d_mods, c.d_subs, E, c.d_k0, c.d_modmem, mesh_args(c.hp));
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gather_diag_b(const Ctx& c, cudaStream_t st) {
  int maxb = 1;
  for (auto& t : c.h_types) maxb = std::max(maxb, t.n_b);
  dim3 grid((maxb + 127) / 128, c.hp.n_sub);
  k_diag_b<<<grid, 128, 0, st>>>(c.d_types, c.d_mods, c.d_subs, c.d_modmem, c.d_diagKb);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_copy_kbb(const Ctx& c, cudaStream_t st) {
  k_copy_kbb<<<dim3(32, c.n_mod), 256, 0, st>>>(c.d_types, c.d_mods, c.d_modmem);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_scaling_weights(const Ctx& c, int kind, cudaStream_t st) {
  const int64_t n = c.hp.n_lam;
  k_weights<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, c.d_lam_b0, c.d_lam_b1, c.d_lam_group, c.d_group_off,
                                                         c.d_group_b, c.d_diagKb, kind, c.d_w0, c.d_w1);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_load_gather(const Ctx& c, cudaStream_t st) {
  const int64_t n = c.hp.n_loc_total;
  k_load_gather<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c.d_load_src, n, c.d_fglob, c.d_floc);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gather_u(const Ctx& c, cudaStream_t st) {
  const int64_t n = c.hp.n_dofs;
  k_gather_u<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, c.d_dof_copy_off, c.d_dof_copy, c.d_dirichlet,
                                                          c.d_uloc, c.d_uglob);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_residual(const Ctx& c, const double* f, const double* u, double* r, cudaStream_t st) {
  const int64_t n = c.hp.n_dofs;
  k_residual<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c.hp.dim, c.hp.n_prob, c.d_prob_dof_off, c.d_prob_el_off,
                                                          c.d_prob_nel, c.d_E, c.d_k0, c.d_dirichlet, f, u, r);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_grad(const Ctx& c, double* out, cudaStream_t st) {
  const int64_t n = c.hp.n_elements;
  k_grad<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c.hp.dim, c.hp.n_prob, c.d_prob_el_off, c.d_prob_dof_off,
                                                      c.d_prob_nel, c.d_rho, c.d_uglob, c.d_k0, c.hp.E0, c.hp.Emin,
                                                      c.hp.p, out);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace feti
