// nn_residual_noalloc: the FP64 residual s = ||I - A X||_F / N without any device allocation.
//
// Some callers cannot allocate device memory: code that runs inside a CUDA graph being
// captured, where an allocation would break the capture; real-time or embedded services
// that forbid allocation after start-up; and hosts whose device memory is owned and
// budgeted by another framework that hands out only the operands. This entry point serves
// them. Its scratch (the N x N residual matrix, the per-block partial sums and the result
// scalar) lives in one file-scope __device__ array of fixed size, so the caller passes
// only the inputs A and X and receives s on the host.
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
//   cudaGetSymbolAddress (host code cannot use the symbol itself as a pointer). Make that
//   first call before any stream capture on the device.
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

// Device address of g_residual_scratch on the current device (resolved once per device).
int noalloc_scratch(void** out) {
  int dev = 0;
  NN_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return NN_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    NN_CUDA_TRY(cudaGetSymbolAddress(&p, g_residual_scratch));
    if (p == nullptr) return NN_ERR_CUDA;
    g_noalloc_ptr[dev] = p;
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
