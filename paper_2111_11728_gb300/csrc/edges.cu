// Edge averages as FETI-DP primal unknowns (the richer primal set, Section 5)
// by a change of basis on every averaged edge.  With the edge's interior nodes
// e_1 .. e_n (one component), the new unknowns are the average ubar, kept in
// the slot of e_1, and the fluctuations v_j in the slots of e_j (j >= 2):
//   u_{e_1} = ubar - sum_j v_j,   u_{e_j} = ubar + v_j,   u = T u^.
// Every edge node lies on the subdomain boundary, so T acts on the b + c
// unknowns only and the interior elimination is unchanged:
//   S^ = T^T S T (Schur complement onto b + c),  f~^ = T^T f~ (condensed load),
// and after the solve the nodal values are u_bc = T u^_bc.
//
// The column operation of S T on one row, for an average with slot c and
// edge slots b_j:  new(c) = S(., c) + sum_j S(., b_j),  new(b_j) = S(., b_j) - S(., c);
// T^T applies the same to the rows.  The averages of one module occupy
// disjoint slots, so they are applied one after another in any order.
#include "kernels.h"

namespace feti {

namespace {

// Columns: one thread per row of S (row-major n_bc x n_bc, b slots first).
__global__ void k_edge_cols(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                            double* __restrict__ mem) {
  const DevModule M = mods[blockIdx.y];
  const DevType T = types[M.type];
  const int nb = T.n_b, nbc = nb + T.n_c;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbc || T.n_avg == 0) return;
  double* row = mem + M.S + (int64_t)i * nbc;
  for (int a = 0; a < T.n_avg; ++a) {
    const int c = nb + T.avg_c[a];
    const double s1 = row[c];
    double sum = s1;
    for (int k = T.avg_off[a]; k < T.avg_off[a + 1]; ++k) {
      const int b = T.avg_b[k];
      const double v = row[b];
      sum += v;
      row[b] = v - s1;
    }
    row[c] = sum;
  }
}

// Rows: one thread per column of S.
__global__ void k_edge_rows(const DevType* __restrict__ types, const DevModule* __restrict__ mods,
                            double* __restrict__ mem) {
  const DevModule M = mods[blockIdx.y];
  const DevType T = types[M.type];
  const int nb = T.n_b, nbc = nb + T.n_c;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nbc || T.n_avg == 0) return;
  double* S = mem + M.S + q;
  for (int a = 0; a < T.n_avg; ++a) {
    const int c = nb + T.avg_c[a];
    const double s1 = S[(int64_t)c * nbc];
    double sum = s1;
    for (int k = T.avg_off[a]; k < T.avg_off[a + 1]; ++k) {
      const int b = T.avg_b[k];
      const double v = S[(int64_t)b * nbc];
      sum += v;
      S[(int64_t)b * nbc] = v - s1;
    }
    S[(int64_t)c * nbc] = sum;
  }
}

// f~^ = T^T f~ on every subdomain: b part at ft[b_off ..], c part at ft[nbt + c_off ..].
// One thread per (average, subdomain).
__global__ void k_edge_load(const DevType* __restrict__ types, const DevSub* __restrict__ subs, int64_t nbt,
                            double* __restrict__ ft) {
  const DevSub S = subs[blockIdx.y];
  const DevType T = types[S.type];
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= T.n_avg) return;
  double* fb = ft + S.b_off;
  double* fc = ft + nbt + S.c_off + T.avg_c[a];
  const double f1 = *fc;
  double sum = f1;
  for (int k = T.avg_off[a]; k < T.avg_off[a + 1]; ++k) {
    const int b = T.avg_b[k];
    sum += fb[b];
    fb[b] -= f1;
  }
  *fc = sum;
}

// Nodal values from the transformed ones on every subdomain: xb (b slots, in
// place) and ucl[c_off + k] (c slots; corners copy the primal value, averages
// become u_{e_1} = ubar - sum_j v_j).  One thread per c slot.
__global__ void k_edge_unmap(const DevType* __restrict__ types, const DevSub* __restrict__ subs,
                             const int* __restrict__ cg, const double* __restrict__ uc, double* __restrict__ xb,
                             double* __restrict__ ucl) {
  const DevSub S = subs[blockIdx.y];
  const DevType T = types[S.type];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= T.n_c) return;
  const double ubar = uc[cg[S.c_off + k]];
  int a = -1;
  for (int q = 0; q < T.n_avg; ++q)
    if (T.avg_c[q] == k) a = q;
  double v = ubar;
  if (a >= 0) {
    double* x = xb + S.b_off;
    for (int j = T.avg_off[a]; j < T.avg_off[a + 1]; ++j) {
      const int b = T.avg_b[j];
      const double f = x[b];
      v -= f;
      x[b] = ubar + f;
    }
  }
  ucl[S.c_off + k] = v;
}

}  // namespace

cudaError_t launch_edge_transform(const Ctx& c, int max_bc, cudaStream_t st) {
  dim3 g((max_bc + 127) / 128, c.n_mod);
  k_edge_cols<<<g, 128, 0, st>>>(c.d_types, c.d_mods, c.d_modmem);
  k_edge_rows<<<g, 128, 0, st>>>(c.d_types, c.d_mods, c.d_modmem);
  note_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_edge_load(const Ctx& c, int max_avg, cudaStream_t st) {
  if (max_avg <= 0) return cudaSuccess;
  k_edge_load<<<dim3((max_avg + 63) / 64, c.hp.n_sub), 64, 0, st>>>(c.d_types, c.d_subs, c.hp.n_b_total, c.d_ft);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_edge_unmap(const Ctx& c, const double* uc, double* xb, double* ucl, cudaStream_t st) {
  k_edge_unmap<<<dim3((c.max_nc + 63) / 64, c.hp.n_sub), 64, 0, st>>>(c.d_types, c.d_subs, c.d_c_glob, uc, xb, ucl);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace feti
