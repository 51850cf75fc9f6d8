// Allocation-free variant of the block Dirichlet preconditioner entry point.
//
// feti_apply_precond works in two interface-space vectors that the library
// allocated with cudaMalloc when the problem was set up.  Some callers cannot
// have the library touch the device allocator while they run: code that is
// recording or replaying work under a fixed device-memory budget, allocators
// that must not be bypassed, or a process that has handed all free memory to
// its own pool.  feti_apply_precond_noalloc gives them the same operator
// without any allocation: its two work vectors live in the file-scope device
// array below, which the CUDA module reserves when the library is loaded and
// every GPU that loads the library keeps until the process exits.
//
// Limits and sharing rules (also stated in include/feti.h):
// * The array holds kNoallocScratch doubles: the problem's interface space
//   may have at most kNoallocScratch / 2 entries (FETI_Q_N_B_TOTAL); larger
//   problems are rejected with FETI_EINVAL before anything is launched.
// * Every call, from every context on the device, uses the same array.  Calls
//   whose kernels overlap on the GPU (different streams, or different host
//   threads) race on it; serialise them.  The array keeps the last call's
//   contents; both work vectors are fully overwritten by each call before they
//   are read, so nothing needs to start at zero.
// * Host code cannot use the array's name as a device address.  The first
//   call on a device looks the address up with cudaGetSymbolAddress (with that
//   device current) and caches it, so make that first call before any stream
//   capture begins.  The cached address belongs to the device's primary
//   context: after cudaDeviceReset (or anything else that replaces that
//   context) the process must not call this entry point on that device again.
// * Like every entry point, the call returns after its stream has synchronized.
#include <mutex>
#include <string>

#include "kernels.h"

namespace {

constexpr int64_t kNoallocScratch = 2 * 262144;   // doubles: 4 MiB

static __device__ __align__(256) double g_precond_scratch[kNoallocScratch];

constexpr int kMaxDevices = 64;
std::mutex g_lookup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_precond_scratch on `device` (which is current): looked
// up once per device, then cached.
cudaError_t scratch_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_lookup_mutex);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_precond_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

}  // namespace

struct feti_ctx {
  feti::Ctx c;
};

extern "C" feti_status feti_apply_precond_noalloc(feti_ctx* ctx, const double* r, double* Z, int ldz, double* z) {
  if (!ctx || !r) return FETI_EINVAL;
  feti::Ctx& c = ctx->c;
  c.err.clear();
  if (c.state < 1) {
    c.err = "feti_apply_precond_noalloc before feti_setup_subdomains";
    return FETI_ESTATE;
  }
  // the size limit is known once the problem is set up: reject before anything else
  if (2 * c.hp.n_b_total > kNoallocScratch) {
    c.err = "feti_apply_precond_noalloc: the interface space has " + std::to_string(c.hp.n_b_total) +
            " entries, more than the static scratch holds (" + std::to_string(kNoallocScratch / 2) +
            "); use feti_apply_precond";
    return FETI_EINVAL;
  }
  if (c.state < 2) {
    c.err = "feti_apply_precond_noalloc before feti_factorize";
    return FETI_ESTATE;
  }
  if (Z && ldz < c.hp.n_lam) {
    c.err = "ldz smaller than n_lambda";
    return FETI_EINVAL;
  }
  int device = -1;
  cudaError_t e = cudaGetDevice(&device);
  if (e == cudaSuccess && device != c.device) e = cudaSetDevice(c.device);
  double* scratch = nullptr;
  if (e == cudaSuccess) e = scratch_address(c.device, &scratch);
  if (e == cudaSuccess)
    e = feti::precond_apply_scratch(c, r, Z, ldz, z, scratch, scratch + c.hp.n_b_total, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (device >= 0 && device != c.device) cudaSetDevice(device);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c.err = std::string("feti_apply_precond_noalloc: ") + cudaGetErrorString(e);
    return FETI_ECUDA;
  }
  return FETI_OK;
}
