// The batching form: one PCG per problem of a batch (FETI-DP, k-scaling), all
// problems advanced by the same launches.  Every per-problem scalar (step
// lengths, conjugation coefficients, residual norms, convergence flags) lives
// on the device, so one iteration is a fixed sequence of kernels that is
// captured once as a CUDA graph and replayed; the host reads only the
// problems' activity flags between replay chunks.
//
// PCG here is Algorithm 1 with the single direction w = P Z 1 conjugated
// against the previous direction only (the "plain" variant of Sections 3.2-3.3),
// with unnormalised directions: gamma = (w.r)/(w.Fw), w <- z - ((Fw).z/(w.Fw)) w.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "kernels.h"

namespace feti {

namespace {

constexpr int SEG_CHUNKS = 16;
constexpr int SEG_THREADS = 256;

// part[(p * SEG_CHUNKS + chunk) * 2 + {0, 1}] = partial a0.b0 and a1.b1 over
// chunk `chunk` of problem p's index range [off[p], off[p+1]).
__global__ void k_seg_dot2(const int64_t* __restrict__ off, const double* __restrict__ a0,
                           const double* __restrict__ b0, const double* __restrict__ a1,
                           const double* __restrict__ b1, double* __restrict__ part) {
  const int p = blockIdx.y, chunk = blockIdx.x;
  const int64_t lo = off[p], n = off[p + 1] - lo;
  const int64_t c0 = lo + n * chunk / SEG_CHUNKS, c1 = lo + n * (chunk + 1) / SEG_CHUNKS;
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
    s0 = fma(a0[i], b0[i], s0);
    if (a1) s1 = fma(a1[i], b1[i], s1);
  }
  __shared__ double r0[SEG_THREADS / 32], r1[SEG_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) { r0[threadIdx.x >> 5] = s0; r1[threadIdx.x >> 5] = s1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w = 0; w < SEG_THREADS / 32; ++w) { t0 += r0[w]; t1 += r1[w]; }
    part[((int64_t)p * SEG_CHUNKS + chunk) * 2] = t0;
    part[((int64_t)p * SEG_CHUNKS + chunk) * 2 + 1] = t1;
  }
}

__global__ void k_seg_finish(int n_prob, const double* __restrict__ part, double* __restrict__ out0,
                             double* __restrict__ out1) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_prob) return;
  double t0 = 0.0, t1 = 0.0;
  for (int ch = 0; ch < SEG_CHUNKS; ++ch) {
    t0 += part[((int64_t)p * SEG_CHUNKS + ch) * 2];
    t1 += part[((int64_t)p * SEG_CHUNKS + ch) * 2 + 1];
  }
  out0[p] = t0;
  if (out1) out1[p] = t1;
}

// lam_t += gamma_p w ; r -= gamma_p q  (gamma_p = (w.r)/(w.Fw)) for active problems
__global__ void k_cg_update(int64_t n, const int* __restrict__ lam_prob, const int* __restrict__ active,
                            const double* __restrict__ wq, const double* __restrict__ wr,
                            const double* __restrict__ w, const double* __restrict__ q, double* __restrict__ lam_t,
                            double* __restrict__ r) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= n) return;
  const int p = lam_prob[l];
  if (!active[p]) return;
  const double g = wr[p] / wq[p];
  lam_t[l] = fma(g, w[l], lam_t[l]);
  r[l] = fma(-g, q[l], r[l]);
}

// w <- z - ((Fw).z / (w.Fw)) w for active problems
__global__ void k_cg_dir(int64_t n, const int* __restrict__ lam_prob, const int* __restrict__ active,
                         const double* __restrict__ wq, const double* __restrict__ qz, const double* __restrict__ z,
                         double* __restrict__ w) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= n) return;
  const int p = lam_prob[l];
  if (!active[p]) return;
  w[l] = fma(-(qz[p] / wq[p]), w[l], z[l]);
}

// convergence bookkeeping per problem
__global__ void k_cg_check(int n_prob, double tol, int max_iter, const double* __restrict__ rz,
                           const double* __restrict__ eps0, int* __restrict__ active, int* __restrict__ iters,
                           int* __restrict__ conv, double* __restrict__ eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_prob || !active[p]) return;
  iters[p] += 1;
  const double e = sqrt(fmax(rz[p], 0.0));
  eps[p] = e;
  const bool fin = isfinite(rz[p]);
  conv[p] = fin && e <= tol * eps0[p];
  if (!fin || conv[p] || iters[p] >= max_iter) active[p] = 0;
}

__global__ void k_cg_init(int n_prob, const double* __restrict__ rz, double* __restrict__ eps0,
                          int* __restrict__ active, int* __restrict__ iters, int* __restrict__ conv,
                          double* __restrict__ eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_prob) return;
  const double e = sqrt(fmax(rz[p], 0.0));
  eps0[p] = e;
  eps[p] = e;
  iters[p] = 0;
  conv[p] = e == 0.0;
  active[p] = e > 0.0 && isfinite(e);
}

// Sum of the split-K partial products of one segmented product:
// C_p(i, j) = alpha * sum_z P_p,z(i, j) + beta * C_p(i, j), chunks in order.
__global__ void k_seg_reduce(const SegRed* __restrict__ reds, const double* __restrict__ partial, double alpha,
                             double beta) {
  const SegRed R = reds[blockIdx.y];
  const int64_t total = (int64_t)R.M * R.N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % R.M), j = (int)(e / R.M);
    if (R.tri && (j / 64) * 64 > (i / 64) * 64 + 63) continue;   // tile never computed
    double s = 0.0;
    for (int z = 0; z < R.nz; ++z) s += partial[R.poff + (int64_t)z * total + e];
    double* cp = R.C + (int64_t)i * R.crs + (int64_t)j * R.ccs;
    double v = alpha * s;
    if (beta != 0.0) v = fma(beta, *cp, v);
    *cp = v;
  }
}

// out_p[j] = A_p[:, j] . r_p for j < k_p  (grid: x = column, y = problem)
__global__ void k_gemv_t_seg(const SegVec* __restrict__ v, const double* __restrict__ r, double* __restrict__ out) {
  const SegVec V = v[blockIdx.y];
  const int j = blockIdx.x;
  if (j >= V.k) return;
  const double* a = V.W + (int64_t)j * V.ld;
  const double* rp = r + V.l0;
  double acc = 0.0;
  for (int64_t l = threadIdx.x; l < V.n; l += blockDim.x) acc = fma(a[l], rp[l], acc);
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    out[V.goff + j] = s;
  }
}

// lam_t += W_p g_p ; r -= Q_p g_p on the rows of every problem with a block
// (k_p > 0); one thread per multiplier row.
__global__ void k_step_seg(int64_t nl, const int* __restrict__ lam_prob, const SegVec* __restrict__ v,
                           const double* __restrict__ g, double* __restrict__ lam_t, double* __restrict__ r) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= nl) return;
  const SegVec V = v[lam_prob[l]];
  if (V.k <= 0) return;
  const int64_t row = l - V.l0;
  const double* gp = g + V.goff;
  double aw = 0.0, aq = 0.0;
  for (int j = 0; j < V.k; ++j) {
    const double gj = gp[j];
    aw = fma(V.W[row + (int64_t)j * V.ld], gj, aw);
    aq = fma(V.Q[row + (int64_t)j * V.ld], gj, aq);
  }
  lam_t[l] += aw;
  r[l] -= aq;
}

}  // namespace

cudaError_t seg_dot2(const int64_t* d_off, int n_prob, const double* a0, const double* b0, const double* a1,
                     const double* b1, double* part, double* out0, double* out1, cudaStream_t st) {
  k_seg_dot2<<<dim3(SEG_CHUNKS, n_prob), SEG_THREADS, 0, st>>>(d_off, a0, b0, a1, b1, part);
  k_seg_finish<<<(n_prob + 127) / 128, 128, 0, st>>>(n_prob, part, out0, out1);
  note_launches(2);
  return cudaGetLastError();
}

// The batched PCG.  Expects r_0 in c.d_r; leaves lambda~ in c.d_lamt and the
// per-problem results in the host vectors of c.  apply / precond are the
// library's own one-column operators, launched on `st`.
cudaError_t batch_pcg(Ctx& c, cudaStream_t user, double tol, int max_iter,
                      feti_status (*apply)(Ctx&, const double*, double*), int* total_iters) {
  const HostProblem& hp = c.hp;
  const int np = hp.n_prob;
  const int64_t nl = hp.n_lam;
  cudaError_t e;
  // private non-blocking stream for capture (the caller's stream may be the legacy one)
  if (!c.cap_stream) {
    if ((e = cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&c.cap_event, cudaEventDisableTiming)) != cudaSuccess) return e;
  }
  cudaStream_t st = c.cap_stream;
  if ((e = cudaEventRecord(c.cap_event, user)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(st, c.cap_event, 0)) != cudaSuccess) return e;
  cudaStream_t saved = c.stream;
  c.stream = st;
  double* w = c.d_Wb;
  double* q = c.d_Qb;
  double* S = c.d_bstate;              // per-problem scalars
  double *wq = S, *wr = S + np, *qz = S + 2 * np, *rz = S + 3 * np, *eps0 = S + 4 * np, *eps = S + 5 * np;
  double* part = S + 6 * np;
  int *active = c.d_bflags, *iters = c.d_bflags + np, *conv = c.d_bflags + 2 * np;
  const unsigned gl = (unsigned)((nl + 255) / 256), gp = (unsigned)((np + 127) / 128);
  auto fail = [&](cudaError_t err) { c.stream = saved; return err; };
  // initial direction and residual norms
  if ((e = precond_apply(c, c.d_r, nullptr, nl, c.d_z, st)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpyAsync(w, c.d_z, nl * sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return fail(e);
  if ((e = cudaMemsetAsync(c.d_lamt, 0, nl * sizeof(double), st)) != cudaSuccess) return fail(e);
  if ((e = seg_dot2(c.d_prob_lam_off, np, c.d_r, c.d_z, nullptr, nullptr, part, rz, nullptr, st)) != cudaSuccess)
    return fail(e);
  k_cg_init<<<gp, 128, 0, st>>>(np, rz, eps0, active, iters, conv, eps);
  note_launches(1);
  // capture one iteration
  const int64_t l0 = launches();
  cudaGraph_t graph = nullptr;
  if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed)) != cudaSuccess) return fail(e);
  feti_status fs = apply(c, w, q);
  cudaError_t ce = cudaGetLastError();
  if (fs == FETI_OK && ce == cudaSuccess) ce = seg_dot2(c.d_prob_lam_off, np, w, q, w, c.d_r, part, wq, wr, st);
  if (ce == cudaSuccess) {
    k_cg_update<<<gl, 256, 0, st>>>(nl, c.d_lam_prob, active, wq, wr, w, q, c.d_lamt, c.d_r);
    note_launches(1);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) ce = precond_apply(c, c.d_r, nullptr, nl, c.d_z, st);
  if (ce == cudaSuccess) ce = seg_dot2(c.d_prob_lam_off, np, q, c.d_z, c.d_r, c.d_z, part, qz, rz, st);
  if (ce == cudaSuccess) {
    k_cg_dir<<<gl, 256, 0, st>>>(nl, c.d_lam_prob, active, wq, qz, c.d_z, w);
    k_cg_check<<<gp, 128, 0, st>>>(np, tol, max_iter, rz, eps0, active, iters, conv, eps);
    note_launches(2);
    ce = cudaGetLastError();
  }
  cudaError_t ee = cudaStreamEndCapture(st, &graph);
  if (fs != FETI_OK) { if (graph) cudaGraphDestroy(graph); return fail(cudaErrorUnknown); }
  if (ce != cudaSuccess || ee != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return fail(ce != cudaSuccess ? ce : ee); }
  const int64_t per_iter = launches() - l0;
  cudaGraphExec_t exec = nullptr;
  if ((e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess) { cudaGraphDestroy(graph); return fail(e); }
  // replay in chunks; between chunks read the activity flags
  const int chunk = 8;
  int done_iters = 0;
  std::vector<int> flags(np);
  while (done_iters < max_iter) {
    for (int k = 0; k < chunk; ++k) {
      if ((e = cudaGraphLaunch(exec, st)) != cudaSuccess) break;
      note_launches((int)per_iter);
    }
    if (e != cudaSuccess) break;
    done_iters += chunk;
    if ((e = cudaMemcpyAsync(flags.data(), active, np * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
    bool any = false;
    for (int v : flags) any = any || v != 0;
    if (!any) break;
  }
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  c.stream = saved;
  if (e != cudaSuccess) return e;
  // results per problem
  std::vector<int> it(np), cv(np);
  std::vector<double> e0(np), e1(np);
  if ((e = cudaMemcpy(it.data(), iters, np * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) return e;
  if ((e = cudaMemcpy(cv.data(), conv, np * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) return e;
  if ((e = cudaMemcpy(e0.data(), eps0, np * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess) return e;
  if ((e = cudaMemcpy(e1.data(), eps, np * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess) return e;
  c.prob_stats.assign(np, feti_stats{});
  int maxit = 0;
  for (int p = 0; p < np; ++p) {
    feti_stats& s = c.prob_stats[p];
    s.iterations = it[p];
    s.converged = cv[p];
    s.f_applies = it[p];
    s.last_rank = 1;
    s.eps0 = e0[p];
    s.eps = e1[p];
    maxit = std::max(maxit, it[p]);
  }
  *total_iters = maxit;
  // make the caller's stream wait for the private one
  if ((e = cudaEventRecord(c.cap_event, st)) != cudaSuccess) return e;
  return cudaStreamWaitEvent(user, c.cap_event, 0);
}

// ---- segmented products of the batched Algorithm 1 ----------------------------

void seg_tn_plan(const std::vector<SegTN>& ops, int64_t kchunk, std::vector<GemmDesc>& descs,
                 std::vector<int64_t>& coff, std::vector<SegRed>& reds, int64_t* partial_len, int* max_m,
                 int* max_n) {
  descs.clear();
  coff.clear();
  reds.clear();
  int64_t poff = 0;
  *max_m = 0;
  *max_n = 0;
  for (const SegTN& o : ops) {
    if (o.M <= 0 || o.N <= 0) continue;
    const int nz = (int)std::max<int64_t>(1, (o.K + kchunk - 1) / kchunk);
    SegRed R{};
    R.C = o.C; R.crs = 1; R.ccs = o.ldc; R.M = o.M; R.N = o.N; R.nz = nz; R.tri = o.tri; R.poff = poff;
    reds.push_back(R);
    for (int z = 0; z < nz; ++z) {
      const int64_t k0 = o.K * z / nz, k1 = o.K * (z + 1) / nz;
      GemmDesc d{};
      // (A^T)(i, k) = A[k + i*lda]; B(k, j) = B[k + j*ldb]
      d.A = o.A + k0; d.ars = o.lda; d.acs = 1;
      d.B = o.B + k0; d.brs = 1; d.bcs = o.ldb;
      d.C = nullptr;                                   // bound to the partial buffer by seg_tn_bind
      d.crs = 1; d.ccs = o.M;
      d.M = o.M; d.N = o.N; d.K = (int)(k1 - k0); d.tri = o.tri;
      descs.push_back(d);
      coff.push_back(poff + (int64_t)z * o.M * o.N);
    }
    poff += (int64_t)nz * o.M * o.N;
    *max_m = std::max(*max_m, o.M);
    *max_n = std::max(*max_n, o.N);
  }
  *partial_len = poff;
}

void seg_tn_bind(std::vector<GemmDesc>& descs, const std::vector<int64_t>& coff, double* partial) {
  for (size_t i = 0; i < descs.size(); ++i) descs[i].C = partial + coff[i];
}

cudaError_t seg_tn_run(const GemmDesc* d_desc, int n_desc, const SegRed* d_red, int n_red, int max_m, int max_n,
                       const double* partial, double alpha, double beta, double flops, cudaStream_t st) {
  if (n_desc <= 0) return cudaSuccess;
  cudaError_t e = dgemm_batched(d_desc, n_desc, max_m, max_n, 0, 1.0, 0.0, st, flops);
  if (e != cudaSuccess) return e;
  k_seg_reduce<<<dim3(64, n_red), 256, 0, st>>>(d_red, partial, alpha, beta);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t gemv_t_seg(const SegVec* d_v, int n_prob, int max_k, const double* r, double* out, cudaStream_t st) {
  if (max_k <= 0 || n_prob <= 0) return cudaSuccess;
  k_gemv_t_seg<<<dim3(max_k, n_prob), 256, 0, st>>>(d_v, r, out);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t step_seg(int64_t nl, const int* d_lam_prob, const SegVec* d_v, const double* g, double* lam_t,
                     double* r, cudaStream_t st) {
  k_step_seg<<<(unsigned)((nl + 255) / 256), 256, 0, st>>>(nl, d_lam_prob, d_v, g, lam_t, r);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace feti
