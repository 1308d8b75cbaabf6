// Sparse NN chain: the explicit product form applied to right-hand sides through a CSR
// matrix (Corollary 1, Eq. (NNexplicit); Corollary 6; Algorithm 2), with the Jacobi start
// phi^(0) = D^-1:
//     X = D^-1 prod_{j=0}^{k-1} ( sum_{n=0}^{L} P^{n (L+1)^j} ) B,     P = I - A D^-1.
// D^-1 is folded into the stored values once (A' = A D^-1, so P v = v - A' v), and the chain
// runs as (L+1)^k - 1 sparse products. Each product is HBM-bound: the kernel streams a
// contiguous slice of (val, col) into shared memory with coalesced streaming loads (one block =
// 256 consecutive rows), then each thread reduces its own row; the x gathers hit L2 and use
// plain global loads (the read-only path is the texture pipeline, four requests per cycle).
//
// Fused variants: the last product of each block of (L+1)^j products adds its result into
// the factor accumulator (acc_out = acc_in + y, element-wise), and the last block of a factor
// skips writing y; the residual variant computes r = b - A' z with sum(r^2) partials.
#include <math.h>
#include <string.h>

#include "common.cuh"
#include "kernels.h"

namespace nn {
namespace {

constexpr int SP_ROWS = 256;   // rows per block = threads per block
constexpr int SP_CHUNK = 2048; // nonzeros staged per pass
constexpr int SP_MAXR = 4;     // right-hand sides per launch

enum : int { SP_Y = 0, SP_Y_ACC = 1, SP_ACC = 2, SP_RESID = 3 };

template <typename T>
__global__ void __launch_bounds__(SP_ROWS)
spmv_p_kernel(int n, const int* __restrict__ row_ptr, const int* __restrict__ col, const T* __restrict__ val,
              const T* __restrict__ v, int64_t ldv, T* __restrict__ y, int64_t ldy, const T* acc_in, T* acc_out,
              int64_t ld_acc, const T* __restrict__ b, int64_t ldb, int nrhs, int mode, double* __restrict__ partial) {
  __shared__ T sval[SP_CHUNK];
  __shared__ int scol[SP_CHUNK];
  __shared__ double red[2][SP_ROWS / 32];
  const int tid = threadIdx.x;
  const int r0 = blockIdx.x * SP_ROWS;
  const int r1 = min(r0 + SP_ROWS, n);
  const int row = r0 + tid;
  const int e_begin = row_ptr[r0];
  const int e_end = row_ptr[r1];
  const int my_b = row < n ? row_ptr[row] : 0;
  const int my_e = row < n ? row_ptr[row + 1] : 0;
  T sum[SP_MAXR];
#pragma unroll
  for (int r = 0; r < SP_MAXR; ++r) sum[r] = T(0);

  constexpr int PER = SP_CHUNK / SP_ROWS;
  for (int base = e_begin; base < e_end; base += SP_CHUNK) {
    const int cnt = min(SP_CHUNK, e_end - base);
    // Issue every load of the slice before any shared-memory store, so each thread has PER
    // independent requests in flight; the matrix streams through (evict-first) and leaves
    // L2 to the vector, which the gathers below reuse across rows.
    T vv[PER];
    int cc[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int i = tid + q * SP_ROWS;
      if (i < cnt) {
        vv[q] = __ldcs(val + base + i);
        cc[q] = __ldcs(col + base + i);
      }
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int i = tid + q * SP_ROWS;
      if (i < cnt) {
        sval[i] = vv[q];
        scol[i] = cc[q];
      }
    }
    __syncthreads();
    const int lo = max(my_b, base), hi = min(my_e, base + cnt);
    int e = lo;
    // four gathers in flight per step
    for (; e + 4 <= hi; e += 4) {
      const T a0 = sval[e - base], a1 = sval[e + 1 - base], a2 = sval[e + 2 - base], a3 = sval[e + 3 - base];
      const int c0 = scol[e - base], c1 = scol[e + 1 - base], c2 = scol[e + 2 - base], c3 = scol[e + 3 - base];
#pragma unroll
      for (int r = 0; r < SP_MAXR; ++r) {
        if (r < nrhs) {
          const T* vr = v + r * ldv;
          // plain cached global loads (ld.global.ca): the non-coherent path goes through the
          // texture pipeline, which accepts only four threads' requests per cycle
          const T x0 = __ldca(vr + c0), x1 = __ldca(vr + c1), x2 = __ldca(vr + c2), x3 = __ldca(vr + c3);
          sum[r] = fma(a0, x0, sum[r]);
          sum[r] = fma(a1, x1, sum[r]);
          sum[r] = fma(a2, x2, sum[r]);
          sum[r] = fma(a3, x3, sum[r]);
        }
      }
    }
    for (; e < hi; ++e) {
      const T a = sval[e - base];
      const int c = scol[e - base];
#pragma unroll
      for (int r = 0; r < SP_MAXR; ++r)
        if (r < nrhs) sum[r] = fma(a, __ldca(v + c + r * ldv), sum[r]);
    }
    __syncthreads();
  }

  double ss_r = 0.0, ss_b = 0.0;
  if (row < n) {
#pragma unroll
    for (int r = 0; r < SP_MAXR; ++r) {
      if (r >= nrhs) break;
      if (mode == SP_RESID) {
        const T bi = b[row + r * ldb];
        const T ri = bi - sum[r];
        ss_r = fma(double(ri), double(ri), ss_r);
        ss_b = fma(double(bi), double(bi), ss_b);
      } else {
        const T yi = __ldca(v + row + r * ldv) - sum[r];
        if (mode != SP_ACC) y[row + r * ldy] = yi;
        if (mode != SP_Y) acc_out[row + r * ld_acc] = acc_in[row + r * ld_acc] + yi;
      }
    }
  }
  if (mode == SP_RESID) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ss_r += __shfl_down_sync(0xffffffffu, ss_r, o);
      ss_b += __shfl_down_sync(0xffffffffu, ss_b, o);
    }
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = ss_r;
      red[1][tid >> 5] = ss_b;
    }
    __syncthreads();
    if (tid == 0) {
      double a = 0, c = 0;
      for (int w = 0; w < SP_ROWS / 32; ++w) {
        a += red[0][w];
        c += red[1][w];
      }
      partial[2 * blockIdx.x] = a;
      partial[2 * blockIdx.x + 1] = c;
    }
  }
}

// dinv[i] = 1 / A_ii; flags a missing or zero diagonal in *err.
template <typename T>
__global__ void diag_inv_kernel(int n, const int* __restrict__ row_ptr, const int* __restrict__ col,
                                const T* __restrict__ val, T* __restrict__ dinv, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T d = T(0);
  for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
    if (col[e] == i) d += val[e];
  if (d == T(0)) {
    atomicExch(err, DEV_BAD_ARG);
    dinv[i] = T(0);
  } else {
    dinv[i] = T(1) / d;
  }
}

// A' = A D^-1 (column scaling).
template <typename T>
__global__ void scale_cols_kernel(int64_t nnz, const int* __restrict__ col, const T* __restrict__ val,
                                  const T* __restrict__ dinv, T* __restrict__ out) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e < nnz) out[e] = val[e] * dinv[col[e]];
}

// dst(n x nrhs, ldd) = src(n x nrhs, lds) [* dinv if given]
template <typename T>
__global__ void copy_cols_kernel(int n, int nrhs, const T* __restrict__ src, int64_t lds, T* __restrict__ dst,
                                 int64_t ldd, const T* __restrict__ dinv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (i >= n || r >= nrhs) return;
  T v = src[i + r * lds];
  if (dinv) v *= dinv[i];
  dst[i + r * ldd] = v;
}

struct CsrWs {
  void* dinv;
  void* vals;
  void* z[2];
  void* u[2];
  double* partial;
  double* scal;
  int* err;
};

template <typename T>
void carve_csr(Carver& c, int64_t n, int64_t nnz, int64_t nrhs, CsrWs& w) {
  const size_t vec = size_t(n) * size_t(nrhs);
  w.dinv = c.take<T>(size_t(n));
  w.vals = c.take<T>(size_t(nnz));
  w.z[0] = c.take<T>(vec);
  w.z[1] = c.take<T>(vec);
  w.u[0] = c.take<T>(vec);
  w.u[1] = c.take<T>(vec);
  const int64_t slices = (nrhs + SP_MAXR - 1) / SP_MAXR;
  w.partial = c.take<double>(size_t(2 * slices * ((n + SP_ROWS - 1) / SP_ROWS)));
  w.scal = c.take<double>(8);
  w.err = c.take<int>(8);
}

template <typename T>
int spmv(cudaStream_t st, int n, const int* rp, const int* col, const T* vals, const T* v, T* y, const T* acc_in,
         T* acc_out, const T* b, int64_t ldb, int nrhs, int mode, double* partial) {
  const int blocks = (n + SP_ROWS - 1) / SP_ROWS;
  for (int r0 = 0; r0 < nrhs; r0 += SP_MAXR) {
    const int nr = nrhs - r0 < SP_MAXR ? nrhs - r0 : SP_MAXR;
    const int64_t off = int64_t(r0) * n;
    // residual partials of slice r0/SP_MAXR follow those of the previous slices
    double* part = partial ? partial + int64_t(2) * blocks * (r0 / SP_MAXR) : nullptr;
    spmv_p_kernel<T><<<blocks, SP_ROWS, 0, st>>>(n, rp, col, vals, v + off, n, y ? y + off : nullptr, n,
                                                 acc_in ? acc_in + off : nullptr, acc_out ? acc_out + off : nullptr, n,
                                                 b ? b + int64_t(r0) * ldb : nullptr, ldb, nr, mode, part);
    NN_CUDA_TRY(cudaGetLastError());
  }
  return NN_OK;
}

__global__ void reduce_pair_kernel(const double* __restrict__ partial, int count, double* out) {
  __shared__ double a[256], c[256];
  double x = 0, y = 0;
  for (int i = threadIdx.x; i < count; i += 256) {
    x += partial[2 * i];
    y += partial[2 * i + 1];
  }
  a[threadIdx.x] = x;
  c[threadIdx.x] = y;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      a[threadIdx.x] += a[threadIdx.x + w];
      c[threadIdx.x] += c[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = c[0] > 0 ? sqrt(a[0] / c[0]) : sqrt(a[0]);
}

template <typename T>
int solve_csr(const int* rp, const int* col, const T* val, int64_t n64, int64_t nnz, const T* B, int64_t ldb,
              int64_t nrhs64, int depth, int nests, double tol, T* X, int64_t ldx, nn_result* res, void* ws,
              size_t ws_bytes, cudaStream_t st) {
  const int n = int(n64), nrhs = int(nrhs64);
  Carver c(ws, ws_bytes);
  CsrWs w;
  carve_csr<T>(c, n64, nnz, nrhs64, w);
  if (!c.ok) return NN_ERR_OOM_BUDGET;
  T* dinv = static_cast<T*>(w.dinv);
  T* vals = static_cast<T*>(w.vals);
  T* z = static_cast<T*>(w.z[0]);
  T* znew = static_cast<T*>(w.z[1]);
  T* u[2] = {static_cast<T*>(w.u[0]), static_cast<T*>(w.u[1])};
  const int blocks = (n + SP_ROWS - 1) / SP_ROWS;
  const int64_t vec = int64_t(n) * nrhs;

  NN_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  diag_inv_kernel<T><<<(n + 255) / 256, 256, 0, st>>>(n, rp, col, val, dinv, w.err);
  NN_CUDA_TRY(cudaGetLastError());
  scale_cols_kernel<T><<<unsigned((nnz + 255) / 256), 256, 0, st>>>(nnz, col, val, dinv, vals);
  NN_CUDA_TRY(cudaGetLastError());
  copy_cols_kernel<T><<<dim3((n + 255) / 256, nrhs), 256, 0, st>>>(n, nrhs, B, ldb, z, n, nullptr);
  NN_CUDA_TRY(cudaGetLastError());
  res->launches += 3;
  int dev_err = 0;
  NN_CUDA_TRY(cudaMemcpyAsync(&dev_err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  NN_CUDA_TRY(cudaStreamSynchronize(st));
  if (dev_err != DEV_OK) return NN_ERR_ARG;

  auto residual = [&](const T* zz, double* out) -> int {
    // r = B - A X = B - A' z (since A X = A D^-1 z); relative Frobenius norm.
    NN_TRY(spmv<T>(st, n, rp, col, vals, zz, nullptr, nullptr, nullptr, B, ldb, nrhs, SP_RESID, w.partial));
    const int slices = (nrhs + SP_MAXR - 1) / SP_MAXR;
    reduce_pair_kernel<<<1, 256, 0, st>>>(w.partial, blocks * slices, w.scal);
    NN_CUDA_TRY(cudaGetLastError());
    res->launches += 1 + slices;
    res->flops += 2.0 * double(nnz) * nrhs;
    NN_CUDA_TRY(cudaMemcpyAsync(out, w.scal, sizeof(double), cudaMemcpyDeviceToHost, st));
    NN_CUDA_TRY(cudaStreamSynchronize(st));
    return NN_OK;
  };

  int applied = 0;
  res->status = NN_OK;
  for (int j = 0; j < nests; ++j) {
    long long t = 1;
    for (int q = 0; q < j; ++q) t *= (depth + 1);
    const T* src = z;
    int ping = 0;
    for (int blk = 1; blk <= depth; ++blk) {
      for (long long s = 1; s <= t; ++s) {
        const bool last_of_block = (s == t);
        const bool last_of_factor = last_of_block && (blk == depth);
        T* dst = u[ping];
        int mode = SP_Y;
        const T* acc_in = nullptr;
        T* acc_out = nullptr;
        if (last_of_block) {
          mode = last_of_factor ? SP_ACC : SP_Y_ACC;
          acc_in = (blk == 1) ? z : znew;
          acc_out = znew;
        }
        NN_TRY(spmv<T>(st, n, rp, col, vals, src, mode == SP_ACC ? nullptr : dst, acc_in, acc_out, nullptr, 0, nrhs,
                       mode, nullptr));
        res->launches += (nrhs + SP_MAXR - 1) / SP_MAXR;
        res->flops += 2.0 * double(nnz) * nrhs;
        src = dst;
        ping ^= 1;
      }
    }
    // znew = z + sum of the L blocks: swap
    T* tmp = z;
    z = znew;
    znew = tmp;
    applied = j + 1;
    if (tol > 0 || j == nests - 1) {
      double rel = 0;
      NN_TRY(residual(z, &rel));
      res->history[j] = rel;
      res->residual = rel;
      if (!isfinite(rel)) {
        res->status = NN_ERR_DIVERGED;
        break;
      }
      if (tol > 0 && rel < tol) break;
      if (j >= 1 && rel >= 1.0 && tol > 0 && rel > res->history[j - 1]) {
        res->status = NN_ERR_DIVERGED;
        break;
      }
    }
  }
  res->nests = applied;
  if (nests == 0) {
    // X = D^-1 B: still report its residual
    double rel = 0;
    NN_TRY(residual(z, &rel));
    res->history[0] = rel;
    res->residual = rel;
  }
  if (res->status == NN_OK && tol > 0 && !(res->residual < tol)) res->status = NN_ERR_NOT_CONVERGED;
  copy_cols_kernel<T><<<dim3((n + 255) / 256, nrhs), 256, 0, st>>>(n, nrhs, z, n, X, ldx, dinv);
  NN_CUDA_TRY(cudaGetLastError());
  res->launches += 1;
  NN_CUDA_TRY(cudaStreamSynchronize(st));
  (void)vec;
  return res->status;
}

}  // namespace
}  // namespace nn

using namespace nn;

extern "C" {

size_t nn_csr_workspace_bytes(int64_t n, int64_t nnz, int64_t nrhs, int dtype) {
  if (n < 1 || nnz < n || nrhs < 1 || n > (int64_t(1) << 30) || nnz > (int64_t(1) << 31) - 1) return 0;
  if (dtype != NN_F64 && dtype != NN_F32) return 0;
  Carver c(nullptr, 0);
  CsrWs w;
  if (dtype == NN_F64)
    carve_csr<double>(c, n, nnz, nrhs, w);
  else
    carve_csr<float>(c, n, nnz, nrhs, w);
  return align_up(c.used, 256);
}

int nn_solve_csr(const int32_t* row_ptr, const int32_t* col, const void* val, int64_t n, int64_t nnz, int dtype,
                 const void* B, int64_t ldb, int64_t nrhs, int depth, int nests, double tol, void* X, int64_t ldx,
                 nn_result* res, void* workspace, size_t ws_bytes, void* stream) {
  if (res == nullptr) return NN_ERR_ARG;
  memset(res, 0, sizeof(*res));
  res->status = NN_ERR_ARG;
  if (row_ptr == nullptr || col == nullptr || val == nullptr || B == nullptr || X == nullptr) return NN_ERR_ARG;
  if (depth < 1 || nests < 0 || nests > NN_MAX_HISTORY - 1 || ldb < n || ldx < n || isnan(tol)) return NN_ERR_ARG;
  // (L+1)^nests - 1 sparse products must stay countable
  double total = pow(double(depth + 1), double(nests));
  if (total > 4.0e9) return NN_ERR_ARG;
  const size_t need = nn_csr_workspace_bytes(n, nnz, nrhs, dtype);
  if (need == 0) return NN_ERR_ARG;
  if (workspace == nullptr || ws_bytes < need) {
    res->status = NN_ERR_OOM_BUDGET;
    return NN_ERR_OOM_BUDGET;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int s;
  if (dtype == NN_F64)
    s = solve_csr<double>(row_ptr, col, static_cast<const double*>(val), n, nnz, static_cast<const double*>(B), ldb,
                          nrhs, depth, nests, tol, static_cast<double*>(X), ldx, res, workspace, ws_bytes, st);
  else
    s = solve_csr<float>(row_ptr, col, static_cast<const float*>(val), n, nnz, static_cast<const float*>(B), ldb, nrhs,
                         depth, nests, tol, static_cast<float*>(X), ldx, res, workspace, ws_bytes, st);
  res->status = s;
  return s;
}

}  // extern "C"
