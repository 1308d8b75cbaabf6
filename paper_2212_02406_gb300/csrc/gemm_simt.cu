// CUDA-core GEMM for the FP64 and FP32 nest chains, with the NN epilogues fused:
//   EPI_COPY      C = A B
//   EPI_RESIDUAL  C = I_n - A B            (R_k = I - A X_k; I restricted to rows/cols < n_id)
//   EPI_ADD       C = D + A B              (Horner T = R + R T, update X_{k+1} = X_k + X_k T)
// and, when `partial` is given, one FP64 partial of sum(C_ij^2) per thread block (a fixed
// block order, so the reduced ||C||_F is deterministic).
//
// Row-major operands with leading dimensions; M, N, K arbitrary (ragged edges are guarded).
// FP64 uses 64x64 tiles (4x4 per thread), FP32 128x128 tiles (8x8 per thread), 256 threads.
#include "common.cuh"
#include "kernels.h"

namespace nn {

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
gemm_simt_kernel(int M, int N, int K, const T* __restrict__ A, int64_t lda, const T* __restrict__ B, int64_t ldb,
                 T* __restrict__ C, int64_t ldc, int mode, const T* __restrict__ D, int64_t ldd, int n_id,
                 double* __restrict__ partial) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int TX = BN / TN;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN];
  __shared__ double red[32];

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int e = tid; e < BM * BK; e += NT) {
      int r = e / BK, c = e % BK;
      int gr = m0 + r, gc = k0 + c;
      As[c][r] = (gr < M && gc < K) ? A[(int64_t)gr * lda + gc] : T(0);
    }
#pragma unroll
    for (int e = tid; e < BK * BN; e += NT) {
      int r = e / BN, c = e % BN;
      int gr = k0 + r, gc = n0 + c;
      Bs[r][c] = (gr < K && gc < N) ? B[(int64_t)gr * ldb + gc] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[k][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[k][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

  double ss = 0.0;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int gr = m0 + ty * TM + i;
    if (gr >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int gc = n0 + tx * TN + j;
      if (gc >= N) continue;
      T v = acc[i][j];
      if (mode == EPI_RESIDUAL) {
        v = ((gr == gc && gr < n_id) ? T(1) : T(0)) - v;
      } else if (mode == EPI_ADD) {
        v = D[(int64_t)gr * ldd + gc] + v;
      }
      C[(int64_t)gr * ldc + gc] = v;
      double dv = static_cast<double>(v);
      ss = fma(dv, dv, ss);
    }
  }
  if (partial != nullptr) {
    // warp reduce, then across warps (fixed order)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
    if ((tid & 31) == 0) red[tid >> 5] = ss;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < NT / 32; ++w) t += red[w];
      partial[blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
  }
}

template <typename T>
struct SimtCfg;
template <>
struct SimtCfg<double> {
  static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
};
template <>
struct SimtCfg<float> {
  static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
};

template <typename T>
int gemm_simt_partials(int M, int N) {
  using C = SimtCfg<T>;
  return ((N + C::BN - 1) / C::BN) * ((M + C::BM - 1) / C::BM);
}

template <typename T>
int gemm_simt(cudaStream_t st, int M, int N, int K, const T* A, int64_t lda, const T* B, int64_t ldb, T* Cm,
              int64_t ldc, int mode, const T* D, int64_t ldd, int n_id, double* partial) {
  using C = SimtCfg<T>;
  if (M <= 0 || N <= 0) return NN_OK;
  dim3 grid((N + C::BN - 1) / C::BN, (M + C::BM - 1) / C::BM);
  dim3 block((C::BM / C::TM) * (C::BN / C::TN));
  gemm_simt_kernel<T, C::BM, C::BN, C::BK, C::TM, C::TN>
      <<<grid, block, 0, st>>>(M, N, K, A, lda, B, ldb, Cm, ldc, mode, D, ldd, n_id, partial);
  NN_CUDA_TRY(cudaGetLastError());
  return NN_OK;
}

template int gemm_simt<double>(cudaStream_t, int, int, int, const double*, int64_t, const double*, int64_t, double*,
                               int64_t, int, const double*, int64_t, int, double*);
template int gemm_simt<float>(cudaStream_t, int, int, int, const float*, int64_t, const float*, int64_t, float*,
                              int64_t, int, const float*, int64_t, int, double*);
template int gemm_simt_partials<double>(int, int);
template int gemm_simt_partials<float>(int, int);

}  // namespace nn
