// FP64 GEMM kernels.  On GB300 the FP64 pipe retires about two DFMA per clock
// per SM, so these products are bound by that pipe, not by memory: a 64x64
// register-blocked tile with 16-deep shared-memory staging feeds it with
// enough independent DFMAs per thread (16 accumulators) and keeps global
// traffic far below the HBM roofline.  The split-K variant writes partial
// tiles to scratch and reduces them in a fixed order (bit-reproducible).
#include <algorithm>
#include <atomic>
#include <vector>

#include "kernels.h"

namespace feti {

struct GemmProfile {
  std::vector<cudaEvent_t> ev;     // start/stop pairs
  std::vector<double> flops;       // algorithmic flops (bytes for the memory-bound phases)
  std::vector<int> kind;           // 0: FP64 GEMM, 1: tensor-core local product, PHASE_KIND0 + p: phase p
  std::vector<int> open;           // pairs opened by prof_begin, not yet closed
};

namespace {
std::atomic<int64_t> g_launches{0};
GemmProfile* g_prof = nullptr;

struct ProfScope {
  cudaStream_t st;
  bool on;
  ProfScope(cudaStream_t s, double fl, int kind = 0) : st(s), on(g_prof != nullptr) {
    if (!on) return;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    g_prof->ev.push_back(a);
    g_prof->ev.push_back(b);
    g_prof->flops.push_back(fl);
    g_prof->kind.push_back(kind);
    cudaEventRecord(a, st);
  }
  ~ProfScope() {
    if (on) cudaEventRecord(g_prof->ev.back(), st);
  }
};
}  // namespace

void prof_begin(cudaStream_t st, double flops, int kind) {
  if (!g_prof) return;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  g_prof->ev.push_back(a);
  g_prof->ev.push_back(b);
  g_prof->flops.push_back(flops);
  g_prof->kind.push_back(kind);
  g_prof->open.push_back((int)g_prof->flops.size() - 1);
  cudaEventRecord(a, st);
}

void prof_end(cudaStream_t st) {
  if (!g_prof || g_prof->open.empty()) return;
  const int i = g_prof->open.back();
  g_prof->open.pop_back();
  cudaEventRecord(g_prof->ev[2 * i + 1], st);
}

PhaseScope::PhaseScope(cudaStream_t st, int phase, double work) : st_(st), on_(g_prof != nullptr) {
  if (on_) prof_begin(st, work, PHASE_KIND0 + phase);
}

PhaseScope::~PhaseScope() {
  if (on_) prof_end(st_);
}

void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches() { return g_launches.load(std::memory_order_relaxed); }
void set_gemm_profile(GemmProfile* p) { g_prof = p; }

GemmProfile* new_gemm_profile() { return new GemmProfile(); }

// Sums of the profiled durations (ms), flops and launches per kind (0: FP64
// GEMM, 1: tensor-core product) and per phase; releases the events.
void finish_gemm_profile(GemmProfile* p, double* flops, double* ms, int64_t* count, double* pwork, double* pms,
                         int64_t* pcount) {
  for (int k = 0; k < 2; ++k) { flops[k] = 0.0; ms[k] = 0.0; count[k] = 0; }
  for (int k = 0; k < N_PHASES; ++k) { pwork[k] = 0.0; pms[k] = 0.0; pcount[k] = 0; }
  for (size_t i = 0; i < p->flops.size(); ++i) {
    float x = 0.f;
    cudaEventElapsedTime(&x, p->ev[2 * i], p->ev[2 * i + 1]);
    cudaEventDestroy(p->ev[2 * i]);
    cudaEventDestroy(p->ev[2 * i + 1]);
    if (p->kind[i] >= PHASE_KIND0) {
      const int q = p->kind[i] - PHASE_KIND0;
      if (q >= 0 && q < N_PHASES) { pwork[q] += p->flops[i]; pms[q] += x; pcount[q] += 1; }
      continue;
    }
    const int k = p->kind[i] ? 1 : 0;
    flops[k] += p->flops[i];
    ms[k] += x;
    count[k] += 1;
  }
  delete p;
}

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__device__ __forceinline__ void load_tile_A(const GemmDesc& d, int row0, int k0, int k1,
                                            double (*As)[BM + 1], int tid) {
  // As[k][i] = A(row0 + i, k0 + k); choose the thread order that walks the
  // contiguous dimension of A.
  if (d.acol) {
#pragma unroll
    for (int e = tid; e < BM * BK; e += NT) {
      int i = e % BM, k = e / BM;
      int gi = row0 + i, gk = k0 + k;
      As[k][i] = (gi < d.M && gk < k1) ? d.A[(int64_t)gi * d.ars + (int64_t)d.acol[gk] * d.acs] : 0.0;
    }
  } else if (d.ars == 1) {
#pragma unroll
    for (int e = tid; e < BM * BK; e += NT) {
      int i = e % BM, k = e / BM;
      int gi = row0 + i, gk = k0 + k;
      As[k][i] = (gi < d.M && gk < k1) ? d.A[gi + (int64_t)gk * d.acs] : 0.0;
    }
  } else {
#pragma unroll
    for (int e = tid; e < BM * BK; e += NT) {
      int k = e % BK, i = e / BK;
      int gi = row0 + i, gk = k0 + k;
      As[k][i] = (gi < d.M && gk < k1) ? d.A[(int64_t)gi * d.ars + (int64_t)gk * d.acs] : 0.0;
    }
  }
}

__device__ __forceinline__ void load_tile_B(const GemmDesc& d, int col0, int k0, int k1, int N,
                                            double (*Bs)[BN + 1], int tid) {
  if (d.bcs == 1) {
#pragma unroll
    for (int e = tid; e < BN * BK; e += NT) {
      int j = e % BN, k = e / BN;
      int gj = col0 + j, gk = k0 + k;
      Bs[k][j] = (gj < N && gk < k1) ? d.B[(int64_t)gk * d.brs + gj] : 0.0;
    }
  } else {
#pragma unroll
    for (int e = tid; e < BN * BK; e += NT) {
      int k = e % BK, j = e / BK;
      int gj = col0 + j, gk = k0 + k;
      Bs[k][j] = (gj < N && gk < k1) ? d.B[(int64_t)gk * d.brs + (int64_t)gj * d.bcs] : 0.0;
    }
  }
}

// grid: x = tile index (m-major), y = batch entry, z = K split
__global__ void __launch_bounds__(NT) dgemm_kernel(const GemmDesc* __restrict__ descs, GemmDesc single,
                                                   int use_single, int n_override, double alpha,
                                                   double beta, double* __restrict__ partial, int splits) {
  const GemmDesc d = use_single ? single : descs[blockIdx.y];
  const int N = n_override > 0 ? n_override : d.N;
  const int tiles_m = (d.M + BM - 1) / BM;
  const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
  const int row0 = tm * BM, col0 = tn * BN;
  if (row0 >= d.M || col0 >= N) return;
  if (d.tri == 1 && col0 > row0 + BM - 1) return;          // strictly above the diagonal
  int kchunk = (d.K + splits - 1) / splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  const int kb = blockIdx.z * kchunk;
  int ke = min(d.K, kb + kchunk);
  if (d.tri == 2) ke = min(ke, col0 + BN);                  // B upper triangular

  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

  for (int k0 = kb; k0 < ke; k0 += BK) {
    load_tile_A(d, row0, k0, ke, As, tid);
    load_tile_B(d, col0, k0, ke, N, Bs, tid);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[k][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }

  if (splits == 1) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      int gi = row0 + ty + 16 * a;
      if (gi >= d.M) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        int gj = col0 + tx + 16 * b;
        if (gj >= N) continue;
        double* cp = d.C + (int64_t)gi * d.crs + (int64_t)gj * d.ccs;
        double v = alpha * acc[a][b];
        if (beta != 0.0) v = fma(beta, *cp, v);
        *cp = v;
      }
    }
  } else {
    double* P = partial + (int64_t)blockIdx.z * d.M * N;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      int gi = row0 + ty + 16 * a;
      if (gi >= d.M) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        int gj = col0 + tx + 16 * b;
        if (gj >= N) continue;
        P[(int64_t)gi * N + gj] = acc[a][b];
      }
    }
  }
}

__global__ void split_reduce_kernel(GemmDesc d, const double* __restrict__ partial, int splits,
                                    double alpha, double beta) {
  int64_t total = (int64_t)d.M * d.N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int gi = (int)(e / d.N), gj = (int)(e % d.N);
    if (d.tri == 1 && (gj / BN) * BN > (gi / BM) * BM + BM - 1) continue;   // tile never computed
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += partial[(int64_t)z * total + e];
    double* cp = d.C + (int64_t)gi * d.crs + (int64_t)gj * d.ccs;
    double v = alpha * s;
    if (beta != 0.0) v = fma(beta, *cp, v);
    *cp = v;
  }
}

}  // namespace

cudaError_t dgemm_batched(const GemmDesc* d_desc, int n_batch, int max_m, int max_n, int n_override,
                          double alpha, double beta, cudaStream_t st, double alg_flops) {
  if (n_batch <= 0 || max_m <= 0 || max_n <= 0) return cudaSuccess;
  if (n_override > 0) max_n = n_override;
  int tiles = ((max_m + BM - 1) / BM) * ((max_n + BN - 1) / BN);
  GemmDesc dummy{};
  dim3 grid(tiles, n_batch, 1);
  ProfScope ps(st, alg_flops);
  dgemm_kernel<<<grid, NT, 0, st>>>(d_desc, dummy, 0, n_override, alpha, beta, nullptr, 1);
  note_launches(1);
  return cudaGetLastError();
}

// K splits of an M x N product (lower: only the tiles on or below the
// diagonal run) chosen to fill whole waves: the split count with the best ratio
// of working CTAs to the resident slots of the waves they occupy (the device's
// SMs times dgemm_kernel's occupancy), the smallest such count on ties, at
// least 64 of K per split.  A grid one CTA past a wave would otherwise run a
// whole extra wave.
int split_for(int M, int N, int K, bool lower) {
  static int slots = 0;
  if (slots <= 0) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dgemm_kernel, NT, 0);
    cudaGetLastError();
    slots = std::max(1, sms) * std::max(1, occ);
  }
  const int tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
  int64_t tiles = (int64_t)tm * tn;
  if (lower) {
    tiles = 0;
    for (int i = 0; i < tm; ++i)
      for (int j = 0; j < tn; ++j)
        if (j * BN <= i * BM + BM - 1) ++tiles;
  }
  if (tiles <= 0) return 1;
  const int maxs = std::max(1, std::min(64, (K + 4 * BK - 1) / (4 * BK)));   // keep >= 64 of K per split
  int best = 1;
  double best_eff = -1.0;
  for (int sp = 1; sp <= maxs; ++sp) {
    const int64_t work = tiles * sp;
    const int64_t waves = (work + slots - 1) / slots;
    const double eff = (double)work / (double)(waves * slots);
    if (eff > best_eff + 1e-12) { best_eff = eff; best = sp; }
  }
  return best;
}

cudaError_t dgemm_split(const GemmDesc& d, int splits, double* work, double alpha, double beta,
                        cudaStream_t st, double alg_flops) {
  if (d.M <= 0 || d.N <= 0) return cudaSuccess;
  if (alg_flops < 0.0) alg_flops = 2.0 * d.M * (double)d.N * d.K;
  int tiles = ((d.M + BM - 1) / BM) * ((d.N + BN - 1) / BN);
  if (splits <= 1 || d.K <= BK) {
    dim3 grid(tiles, 1, 1);
    ProfScope ps(st, alg_flops);
    dgemm_kernel<<<grid, NT, 0, st>>>(nullptr, d, 1, 0, alpha, beta, nullptr, 1);
    note_launches(1);
    return cudaGetLastError();
  }
  dim3 grid(tiles, 1, splits);
  {
    ProfScope ps(st, alg_flops);
    dgemm_kernel<<<grid, NT, 0, st>>>(nullptr, d, 1, 0, 1.0, 0.0, work, splits);
  }
  int64_t total = (int64_t)d.M * d.N;
  int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
  split_reduce_kernel<<<blocks, 256, 0, st>>>(d, work, splits, alpha, beta);
  note_launches(2);
  return cudaGetLastError();
}

}  // namespace feti
