// nn_residual_noalloc: the FP64 residual s = ||I - A X||_F / N without any device allocation.
//
// Some callers cannot allocate device memory: real-time or embedded services that forbid any
// allocation after start-up (an allocation can block or fail at an arbitrary moment), and
// plug-ins whose host framework owns and budgets all device memory and hands them only the
// operands, with no allocator and no workspace to draw on. This entry point serves them. Its
// scratch (the N x N residual matrix, the per-block partial sums and the result scalar) lives
// in one file-scope __device__ array of fixed size, so the caller passes only the inputs A
// and X and receives s on the host.
//
// Limits and sharing:
// * N <= NN_RESIDUAL_NOALLOC_MAX_N (1440): the array holds 16 MiB, and every GPU that loads
//   libnn keeps it reserved until the process exits. Larger N is rejected with
//   NN_ERR_TOO_LARGE before any device work.
// * One array per device, shared by every call on that device: calls whose work overlaps on
//   the GPU (different streams, or host threads without ordering) race on it. Each call
//   overwrites all the scratch it reads (R, every partial, the scalar), so no state carries
//   over from the previous call and nothing needs clearing.
// * The first call on a device resolves the array's device address with
//   cudaGetSymbolAddress (in host code the symbol names a host-side stand-in, not device
//   memory) and keeps it for the device's context; a call after cudaDeviceReset, which ends
//   that context, resolves it again. Make the first call on each device before any stream
//   capture on that device.
#include <cuda.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace nn {
namespace {

constexpr size_t kNoallocScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_residual_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};
unsigned long long g_noalloc_ctx[kMaxDevices] = {};  // context the address belongs to

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique id of the current device's context (0 if the driver cannot tell): a device reset
// ends the context, and the id of the next one differs, so a cached address is re-resolved.
unsigned long long current_ctx_id() {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
    (void)cudaGetLastError();
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_cur == nullptr || get_id == nullptr || get_cur(&ctx) != CUDA_SUCCESS || ctx == nullptr ||
      get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of g_residual_scratch on the current device: resolved at the first call on
// the device (the set-up step), again only when the device's context has changed.
int noalloc_scratch(void** out) {
  int dev = 0;
  NN_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return NN_ERR_UNSUPPORTED;
  // (0 when this thread has no current context yet: the set-up below makes it current)
  const unsigned long long ctx = current_ctx_id();
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr || ctx == 0 || g_noalloc_ctx[dev] != ctx) {
    void* p = nullptr;
    NN_CUDA_TRY(cudaGetSymbolAddress(&p, g_residual_scratch));
    if (p == nullptr) return NN_ERR_CUDA;
    g_noalloc_ptr[dev] = p;
    g_noalloc_ctx[dev] = current_ctx_id();
  }
  *out = g_noalloc_ptr[dev];
  return NN_OK;
}

}  // namespace
}  // namespace nn

using namespace nn;

extern "C" int nn_residual_noalloc(const double* A, int64_t lda, const double* X, int64_t ldx, int64_t n,
                                   double* rms_frob, void* stream) {
  if (A == nullptr || X == nullptr || rms_frob == nullptr || n < 1 || lda < n || ldx < n) return NN_ERR_ARG;
  if (n > NN_RESIDUAL_NOALLOC_MAX_N) return NN_ERR_TOO_LARGE;
  void* base = nullptr;
  NN_TRY(noalloc_scratch(&base));
  const int ni = int(n);
  Carver c(base, kNoallocScratchBytes);
  double* R = c.take<double>(size_t(n) * size_t(n));
  const int parts = gemm_simt_partials<double>(ni, ni);
  double* partial = c.take<double>(size_t(parts));
  double* scal = c.take<double>(1);
  if (!c.ok) return NN_ERR_TOO_LARGE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  NN_TRY(gemm_simt<double>(st, ni, ni, ni, A, lda, X, ldx, R, n, EPI_RESIDUAL, nullptr, 0, ni, partial));
  NN_TRY(reduce_rms(st, partial, parts, 1.0 / double(n), scal));
  NN_CUDA_TRY(cudaMemcpyAsync(rms_frob, scal, sizeof(double), cudaMemcpyDeviceToHost, st));
  NN_CUDA_TRY(cudaStreamSynchronize(st));
  return NN_OK;
}
