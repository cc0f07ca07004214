// Orthogonalisation for callers that cannot allocate device memory.
//
// stab_orthogonalize needs a handle, and a handle owns device workspace that
// stab_create obtains with cudaMalloc.  Some host programs cannot make that
// call: their device memory is owned by another framework's pool, or they run
// under a fixed device-memory budget reserved up front.  This entry point
// performs the same CGS2 step with its reduction scratch in a file-scope
// device array instead, so it allocates nothing.
//
// Limits: at most kMaxK basis vectors and kMaxN unknowns.  The array
// (about 1.3 MB) lives on every device that loads the library until the
// process exits.  All calls share it: calls whose GPU work overlaps (on two
// streams, or from two host threads) race on it and must be serialised by the
// caller.  The first call on a device looks up the array's device address
// with that device current; make that first call before any stream capture.
// That address is kept until the process exits, so a device reset
// (cudaDeviceReset) after the first call is not supported.
#include <mutex>

#include "internal.cuh"

void stab_set_global_error(const char* msg);

namespace {

constexpr int kMaxK = 128;                 // basis vectors
constexpr long long kMaxN = 1LL << 28;     // unknowns
constexpr int kMaxRedBlocks = 608;         // dot-product reduction blocks (152 x 4)
constexpr int kMaxNormBlocks = 1024;       // norm reduction blocks
constexpr size_t kPartial = (size_t)kMaxRedBlocks * kMaxK;
constexpr size_t kElems = kPartial + 2 * kMaxK + kMaxNormBlocks / 2 + 1;

// Device-side scratch: dot-product partials, the two h vectors, norm
// partials, the norm.  Host code must not use this name as an address.
static __device__ __align__(256) double2 g_noalloc_scratch[kElems];

std::mutex g_mu;
double2* g_dev_ptr[128] = {nullptr};

// The device address of the scratch on the current device (set up once per device).
cudaError_t scratch_ptr(double2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_dev_ptr[dev] = (double2*)p;
  }
  *out = g_dev_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" stab_status stab_orthogonalize_noalloc(const void* V, int k, long long n, void* w, double* hcoef,
                                                  double* norm, void* stream) {
  if (k < 0 || k > kMaxK || n < 1 || n > kMaxN) {
    stab_set_global_error("stab_orthogonalize_noalloc: need 0 <= k <= 128 basis vectors and 1 <= n <= 2^28 unknowns");
    return STAB_ERR_INVALID_ARG;
  }
  if ((k > 0 && !V) || !w) {
    stab_set_global_error("stab_orthogonalize_noalloc: null V or w");
    return STAB_ERR_INVALID_ARG;
  }
  double2* base = nullptr;
  cudaError_t e = scratch_ptr(&base);
  if (e != cudaSuccess) {
    stab_set_global_error(cudaGetErrorString(e));
    return STAB_ERR_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double2* partial = base;
  double2* dh = base + kPartial;
  double* norm_partial = (double*)(dh + 2 * kMaxK);
  double* dnorm = norm_partial + kMaxNormBlocks;
  long long nb = (n + 1023) / 1024;
  if (nb > kMaxNormBlocks) nb = kMaxNormBlocks;
  e = kry_cgs2_stream(st, (const double2*)V, k, n, (double2*)w, dh, dnorm, partial, norm_partial, (int)nb);
  if (e == cudaSuccess && hcoef && k > 0) e = cudaMemcpyAsync(hcoef, dh, sizeof(double2) * k, cudaMemcpyDeviceToHost, st);
  double nv = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nv, dnorm, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    stab_set_global_error(cudaGetErrorString(e));
    return STAB_ERR_CUDA;
  }
  if (norm) *norm = nv;
  return STAB_OK;
}
