// General (non-Hermitian, real or complex) linear systems through the normal equations
// (Corollary 3): A x = B  ->  x = (A^H A)^-1 A^H B. W = A^H A is Hermitian positive definite,
// the NN runs on W from X_0 = Theta I with Theta = 1 / Tr(W) (Eq. (trace)), and the solution is
// X_k A^H B, the right-form counterpart of Eq. (nnlinearsystem).
//
// Complex systems run on the real embedding of size m = 2n,
//     z -> [[Re z, -Im z], [Im z, Re z]],
// which maps complex matrix products, sums and the conjugate transpose onto real ones
// (A^H -> A-hat^T), so A-hat^T A-hat is the embedding of A^H A and the real NN iterates on it
// are the embeddings of the complex iterates (the trace doubles, so Theta = 2 / Tr(W-hat)).
// The right-hand sides embed as the stacked [Re B; Im B] (the first block column of the
// embedding of B). The embedding's residual sqrt(2) ||R_k||_F / (2n) is the complex
// ||R_k||_F / n divided by sqrt(2); the stop test and the reported history use the complex one.
//
// All steps run on the device: one tiled kernel writes A-hat (complex only) and A-hat^T; W is
// formed by the FP64 CUDA-core GEMM, or by the emulated FP64 product for NN_F64_EMU; C = A-hat^T
// B-hat and Y = X C (n x nrhs) use the CUDA-core GEMM; the inversion of W is the dense NN of
// nn_invert with the caller's options.
#include <math.h>
#include <string.h>

#include "common.cuh"
#include "kernels.h"

namespace nn {
namespace {

constexpr int NT = 32;  // transpose tile

// Writes the real form A-hat (m x m, row-major, ld m; only for complex input) and its transpose
// A-hat^T (m x m, ld m) from A (real: n x n FP64, lda; complex: n x n interleaved complex128,
// lda in complex elements). m = n (real) or 2n (complex).
__global__ void normal_operands_kernel(const double* __restrict__ A, int n, int64_t lda, int is_complex, int m,
                                       double* __restrict__ Ahat, double* __restrict__ AhatT) {
  __shared__ double tile[NT][NT + 1];
  const int bi = blockIdx.y * NT, bj = blockIdx.x * NT;
  // load A-hat[bi + ty][bj + tx]
  for (int ty = threadIdx.y; ty < NT; ty += blockDim.y) {
    const int i = bi + ty, j = bj + threadIdx.x;
    double v = 0.0;
    if (i < m && j < m) {
      if (!is_complex) {
        v = A[int64_t(i) * lda + j];
      } else {
        const int ii = i < n ? i : i - n, jj = j < n ? j : j - n;
        const double re = A[2 * (int64_t(ii) * lda + jj)];
        const double im = A[2 * (int64_t(ii) * lda + jj) + 1];
        const bool top = i < n, left = j < n;
        v = (top == left) ? re : (top ? -im : im);
        Ahat[int64_t(i) * m + j] = v;
      }
    }
    tile[ty][threadIdx.x] = v;
  }
  __syncthreads();
  // A-hat^T[bj + ty][bi + tx] = A-hat[bi + tx][bj + ty]
  for (int ty = threadIdx.y; ty < NT; ty += blockDim.y) {
    const int r = bj + ty, c = bi + threadIdx.x;
    if (r < m && c < m) AhatT[int64_t(r) * m + c] = tile[threadIdx.x][ty];
  }
}

// B-hat (m x nrhs, ld nrhs) = B (real) or [Re B; Im B] (complex, interleaved, ldb in complex elements)
__global__ void stack_rhs_kernel(const double* __restrict__ B, int n, int64_t ldb, int nrhs, int is_complex,
                                 double* __restrict__ Bh) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int m = is_complex ? 2 * n : n;
  if (e >= int64_t(m) * nrhs) return;
  const int i = int(e / nrhs), c = int(e % nrhs);
  if (!is_complex)
    Bh[e] = B[int64_t(i) * ldb + c];
  else
    Bh[e] = i < n ? B[2 * (int64_t(i) * ldb + c)] : B[2 * (int64_t(i - n) * ldb + c) + 1];
}

// X (real: n x nrhs, ldx; complex: interleaved) from Y (m x nrhs, ld nrhs)
__global__ void unstack_kernel(const double* __restrict__ Y, int n, int nrhs, int is_complex, double* __restrict__ X,
                               int64_t ldx) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= int64_t(n) * nrhs) return;
  const int i = int(e / nrhs), c = int(e % nrhs);
  if (!is_complex) {
    X[int64_t(i) * ldx + c] = Y[e];
  } else {
    X[2 * (int64_t(i) * ldx + c)] = Y[e];
    X[2 * (int64_t(i) * ldx + c) + 1] = Y[int64_t(i + n) * nrhs + c];
  }
}

// X0_ii *= factor (X0 diagonal)
__global__ void scale_diag_kernel(double* X0, int m, double factor) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) X0[int64_t(i) * m + i] *= factor;
}

struct NormalWs {
  double* Ahat;   // complex only
  double* AhatT;
  double* W;
  double* X0;
  double* Xw;
  double* Bh;
  double* C;
  double* Y;
  double* scratch;
  int* err;
};

void carve_normal(Carver& c, int64_t m, int64_t nrhs, bool is_complex, NormalWs& w) {
  const size_t mm = size_t(m) * size_t(m), mr = size_t(m) * size_t(nrhs);
  w.Ahat = is_complex ? c.take<double>(mm) : nullptr;
  w.AhatT = c.take<double>(mm);
  w.W = c.take<double>(mm);
  w.X0 = c.take<double>(mm);
  w.Xw = c.take<double>(mm);
  w.Bh = c.take<double>(mr);
  w.C = c.take<double>(mr);
  w.Y = c.take<double>(mr);
  w.scratch = c.take<double>(8);
  w.err = c.take<int>(8);
}

size_t outer_bytes(int64_t m, int64_t nrhs, bool is_complex) {
  Carver c(nullptr, 0);
  NormalWs w;
  carve_normal(c, m, nrhs, is_complex, w);
  return align_up(c.used, 256);
}

}  // namespace
}  // namespace nn

using namespace nn;

extern "C" {

size_t nn_normal_workspace_bytes(int64_t n, int64_t nrhs, int is_complex, int dtype) {
  if (n < 1 || nrhs < 1 || nrhs > (int64_t(1) << 20) || (is_complex != 0 && is_complex != 1)) return 0;
  const int64_t m = is_complex ? 2 * n : n;
  const size_t inner = nn_workspace_bytes(m, dtype);
  if (inner == 0) return 0;
  return inner + outer_bytes(m, nrhs, is_complex != 0);
}

int nn_solve_normal(const void* A, int64_t n, int64_t lda, int is_complex, const void* B, int64_t ldb, int64_t nrhs,
                    const nn_opts* opts, void* X, int64_t ldx, nn_result* res, void* workspace, size_t ws_bytes,
                    void* stream) {
  if (res == nullptr) return NN_ERR_ARG;
  memset(res, 0, sizeof(*res));
  res->status = NN_ERR_ARG;
  if (A == nullptr || B == nullptr || X == nullptr || opts == nullptr) return NN_ERR_ARG;
  if (is_complex != 0 && is_complex != 1) return NN_ERR_ARG;
  if (n < 1 || nrhs < 1 || lda < n || ldb < nrhs || ldx < nrhs) return NN_ERR_ARG;
  const int64_t m = is_complex ? 2 * n : n;
  NN_TRY(check_opts(opts, m));
  const size_t need = nn_normal_workspace_bytes(n, nrhs, is_complex, opts->dtype);
  if (need == 0) return NN_ERR_ARG;
  if (workspace == nullptr || ws_bytes < need) return NN_ERR_OOM_BUDGET;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t inner = nn_workspace_bytes(m, opts->dtype);
  Carver c(static_cast<char*>(workspace) + inner, ws_bytes - inner);
  NormalWs w;
  carve_normal(c, m, nrhs, is_complex != 0, w);
  if (!c.ok) return NN_ERR_OOM_BUDGET;
  const int mi = int(m), ni = int(n), ri = int(nrhs);
  const double* Ad = static_cast<const double*>(A);

  // A-hat (complex) and A-hat^T
  {
    const dim3 block(NT, 8);
    const dim3 grid(unsigned((m + NT - 1) / NT), unsigned((m + NT - 1) / NT));
    normal_operands_kernel<<<grid, block, 0, st>>>(Ad, ni, lda, is_complex, mi, w.Ahat, w.AhatT);
    NN_CUDA_TRY(cudaGetLastError());
  }
  const double* Ahat = is_complex ? w.Ahat : Ad;
  const int64_t ld_hat = is_complex ? m : lda;
  // W = A-hat^T A-hat, X_0 = I / Tr(W)
  if (opts->dtype == NN_F64_EMU) {
    // the inversion's workspace is idle until invert_device: lend it to the emulated product
    NN_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    NN_TRY(gemm_f64_emu(st, mi, w.AhatT, m, Ahat, ld_hat, w.W, m, EPI_COPY, nullptr, 0, 0, nullptr, nullptr, workspace,
                        inner, w.err));
  } else {
    NN_TRY(gemm_simt<double>(st, mi, mi, mi, w.AhatT, m, Ahat, ld_hat, w.W, m, EPI_COPY, nullptr, 0, 0, nullptr));
  }
  NN_TRY(precond_fill(st, w.W, m, mi, NN_PC_TRACE, 0.0, w.X0, m, w.scratch, nullptr));
  if (is_complex) {
    // The embedding doubles the trace (Tr W-hat = 2 Re Tr W): Theta = 1 / Tr(A^H A) = 2 / Tr(W-hat).
    scale_diag_kernel<<<unsigned((m + 255) / 256), 256, 0, st>>>(w.X0, mi, 2.0);
    NN_CUDA_TRY(cudaGetLastError());
  }
  // B-hat and C = A-hat^T B-hat (independent of the inversion)
  {
    const int64_t cnt = m * nrhs;
    stack_rhs_kernel<<<unsigned((cnt + 255) / 256), 256, 0, st>>>(static_cast<const double*>(B), ni, ldb, ri,
                                                                   is_complex, w.Bh);
    NN_CUDA_TRY(cudaGetLastError());
  }
  NN_TRY(gemm_simt<double>(st, mi, ri, mi, w.AhatT, m, w.Bh, nrhs, w.C, nrhs, EPI_COPY, nullptr, 0, 0, nullptr));
  // X_k ~ W^-1 by the dense NN (the caller's depth, tolerance, nest cap and precision)
  // Complex: the embedding's s_k is the complex residual / sqrt(2), so the stop test runs on
  // tol / sqrt(2) and the reported history is scaled back to the complex ||R_k||_F / n.
  nn_opts o = *opts;
  o.x0_scalar = 0.0;  // X_0 of W is built here, whatever the caller asserted about its own
  const double rs = is_complex ? sqrt(2.0) : 1.0;
  if (is_complex && o.tol > 0) o.tol /= rs;
  const int s = invert_device(w.W, m, m, w.X0, m, &o, w.Xw, m, res, workspace, inner, st);
  if (s == NN_ERR_CUDA || s == NN_ERR_ARG || s == NN_ERR_UNSUPPORTED || s == NN_ERR_OOM_BUDGET ||
      s == NN_ERR_TIMEOUT)
    return s;
  if (is_complex) {
    for (int k = 0; k <= res->nests && k < NN_MAX_HISTORY; ++k) res->history[k] *= rs;
    res->residual *= rs;
  }
  // Y = X_k C, then back to the caller's layout
  NN_TRY(gemm_simt<double>(st, mi, ri, mi, w.Xw, m, w.C, nrhs, w.Y, nrhs, EPI_COPY, nullptr, 0, 0, nullptr));
  {
    const int64_t cnt = n * nrhs;
    unstack_kernel<<<unsigned((cnt + 255) / 256), 256, 0, st>>>(w.Y, ni, ri, is_complex, static_cast<double*>(X),
                                                                ldx);
    NN_CUDA_TRY(cudaGetLastError());
  }
  res->launches += 5;
  res->flops += 2.0 * double(m) * double(m) * double(m) + 4.0 * double(m) * double(m) * double(nrhs);
  NN_CUDA_TRY(cudaStreamSynchronize(st));
  if (opts->dtype == NN_F64_EMU) {
    int e = DEV_OK;
    NN_CUDA_TRY(cudaMemcpy(&e, w.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e != DEV_OK) {
      res->status = NN_ERR_TIMEOUT;
      return NN_ERR_TIMEOUT;
    }
  }
  res->status = s;
  return s;
}

}  // extern "C"
