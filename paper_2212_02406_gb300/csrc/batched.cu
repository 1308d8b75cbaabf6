// Batched NN inversion of many small complex matrices (massive-MIMO Gram matrices,
// U x U with U <= 64) in one persistent kernel.
//
// Each matrix runs the right-multiplied NN loop of the dense path (Theorem, Eq.
// (nestedneumann); L = 1 Newton, L = 2 Chebyshev as in Corollary 4) entirely in shared
// memory, from the damped Jacobi start X_0 = diag(A)^-1 / (1 + damping U) (a diagonal Theta,
// Appendix 1), for a fixed number of nests:
//     k = 0..nests:  R = I - A X_k, s_k = ||R||_F / U;  stop if diverged or k = nests;
//                    T = R, L-1 times T = R + R T;  X_{k+1} = X_k + X_k T.
// Divergence (s_k non-finite, or s_k >= 1 and s_k > s_{k-1}) freezes X at X_k, as the dense
// path does.
//
// Scheduling: the host plan (nn_batched_plan) sorts the matrices by size, largest first,
// and cuts them into work items of G equal-size matrices; the grid is one CTA (256 threads)
// per SM, and each CTA pulls items from a global counter. Inside a CTA, G thread groups run
// G matrices in lock-step (same U, same barriers). Two tile configurations exist per size:
//   cfg 0: 8 x 8 threads per matrix, each computing a ceil(U/8)^2 tile of every product;
//   cfg 1: 16 x 16 threads per matrix, tile ceil(U/16)^2, one matrix per CTA.
// The plan takes a per-size configuration table, which the autotuner fills.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace nn {
namespace {

constexpr int BT_THREADS = 256;
constexpr int BT_MAX_U = 64;
constexpr int BT_BUFS = 5;                  // A, X, R, T, W
constexpr int BT_SMEM = 200 * 1024;         // dynamic shared memory per CTA
constexpr int PLAN_HDR = 2;                 // [n_items, count]

enum : int { BM_RESID = 0, BM_ADD = 1 };

// out = (mode RESID) I - P Q  or  (mode ADD) D + P Q, for a U x U complex group tile.
// Thread (ti, tj) of the TG x TG group owns rows ti + a TG and columns tj + b TG.
// UC > 0 fixes U = UC = T * TG at compile time (no bounds tests, static addressing, unrolled
// k loop); UC = 0 handles any U <= T * TG.
template <int TG, int T, int UC>
__device__ __forceinline__ float group_gemm(int U_rt, int ti, int tj, const float2* __restrict__ P,
                                            const float2* __restrict__ Q, float2* __restrict__ out,
                                            const float2* __restrict__ D, int mode) {
  const int U = UC > 0 ? UC : U_rt;
  constexpr bool exact = UC > 0 && UC == T * TG;
  float2 acc[T][T];
#pragma unroll
  for (int a = 0; a < T; ++a)
#pragma unroll
    for (int b = 0; b < T; ++b) acc[a][b] = make_float2(0.f, 0.f);
  if (exact && (UC % 2) == 0) {
    // P[i, k] and P[i, k + 1] arrive in one 16-byte load (two k steps per P load), which cuts
    // the shared-memory wavefronts of the P operand in half; same FMA order as below.
#pragma unroll 4
    for (int k = 0; k < UC; k += 2) {
      float4 pa2[T];
#pragma unroll
      for (int a = 0; a < T; ++a) pa2[a] = *reinterpret_cast<const float4*>(P + (ti + a * TG) * UC + k);
      float2 q0[T], q1[T];
#pragma unroll
      for (int b = 0; b < T; ++b) {
        q0[b] = Q[k * UC + tj + b * TG];
        q1[b] = Q[(k + 1) * UC + tj + b * TG];
      }
#pragma unroll
      for (int a = 0; a < T; ++a)
#pragma unroll
        for (int b = 0; b < T; ++b) {
          acc[a][b].x = fmaf(pa2[a].x, q0[b].x, acc[a][b].x);
          acc[a][b].x = fmaf(-pa2[a].y, q0[b].y, acc[a][b].x);
          acc[a][b].y = fmaf(pa2[a].x, q0[b].y, acc[a][b].y);
          acc[a][b].y = fmaf(pa2[a].y, q0[b].x, acc[a][b].y);
        }
#pragma unroll
      for (int a = 0; a < T; ++a)
#pragma unroll
        for (int b = 0; b < T; ++b) {
          acc[a][b].x = fmaf(pa2[a].z, q1[b].x, acc[a][b].x);
          acc[a][b].x = fmaf(-pa2[a].w, q1[b].y, acc[a][b].x);
          acc[a][b].y = fmaf(pa2[a].z, q1[b].y, acc[a][b].y);
          acc[a][b].y = fmaf(pa2[a].w, q1[b].x, acc[a][b].y);
        }
    }
  } else {
#pragma unroll(UC > 0 ? 8 : 1)
  for (int k = 0; k < U; ++k) {
    float2 pa[T], qb[T];
#pragma unroll
    for (int a = 0; a < T; ++a) {
      const int i = ti + a * TG;
      pa[a] = (exact || i < U) ? P[i * U + k] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int b = 0; b < T; ++b) {
      const int j = tj + b * TG;
      qb[b] = (exact || j < U) ? Q[k * U + j] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int a = 0; a < T; ++a)
#pragma unroll
      for (int b = 0; b < T; ++b) {
        acc[a][b].x = fmaf(pa[a].x, qb[b].x, acc[a][b].x);
        acc[a][b].x = fmaf(-pa[a].y, qb[b].y, acc[a][b].x);
        acc[a][b].y = fmaf(pa[a].x, qb[b].y, acc[a][b].y);
        acc[a][b].y = fmaf(pa[a].y, qb[b].x, acc[a][b].y);
      }
  }
  }
  float ss = 0.f;
#pragma unroll
  for (int a = 0; a < T; ++a) {
    const int i = ti + a * TG;
    if (!exact && i >= U) continue;
#pragma unroll
    for (int b = 0; b < T; ++b) {
      const int j = tj + b * TG;
      if (!exact && j >= U) continue;
      float2 v;
      if (mode == BM_RESID) {
        v = make_float2((i == j ? 1.f : 0.f) - acc[a][b].x, -acc[a][b].y);
        ss = fmaf(v.x, v.x, fmaf(v.y, v.y, ss));
      } else {
        const float2 d = D[i * U + j];
        v = make_float2(d.x + acc[a][b].x, d.y + acc[a][b].y);
      }
      out[i * U + j] = v;
    }
  }
  return ss;
}

struct BatchedParams {
  const float2* A;
  const int64_t* offsets;
  const int32_t* sizes;
  const int32_t* plan;
  int depth;
  int nests;
  float damping;
  float2* X;
  float* residual;
  int32_t* status;
  int* queue;
};

// Sum over the threads of one group (nthr = TG*TG threads, whole warps), result in red_out[g].
__device__ __forceinline__ void group_sum(float v, int g, int lt, int nthr, float* red_warp, float* red_out) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red_warp[threadIdx.x >> 5] = v;
  __syncthreads();
  if (lt == 0) {
    float t = 0.f;
    const int w0 = (g * nthr) >> 5, nw = nthr >> 5;
    for (int w = 0; w < nw; ++w) t += red_warp[w0 + w];
    red_out[g] = t;
  }
  __syncthreads();
}

template <int TG, int T, int UC>
__device__ void process_item(const BatchedParams& p, int U, int start, int cnt, float2* smem, float* red_warp,
                             float* red_grp) {
  constexpr int NTHR = TG * TG;
  const int groups = BT_THREADS / NTHR;
  const int g = threadIdx.x / NTHR;
  const int lt = threadIdx.x % NTHR;
  const int ti = lt / TG, tj = lt % TG;
  const bool active = g < groups && g < cnt;
  const int uu = U * U;
  const int b = active ? p.plan[PLAN_HDR + start + g] : -1;
  float2* base = smem + size_t(g < groups ? g : 0) * BT_BUFS * uu;
  float2* Ab = base;
  float2* Xb = base + uu;
  float2* Rb = base + 2 * uu;
  float2* Tb = base + 3 * uu;
  float2* Wb = base + 4 * uu;
  const int64_t off = active ? p.offsets[b] : 0;

  if (active) {
    for (int e = lt; e < uu; e += NTHR) Ab[e] = p.A[off + e];
  }
  __syncthreads();
  if (active) {
    const float c = 1.f / (1.f + p.damping * float(U));
    for (int e = lt; e < uu; e += NTHR) {
      const int i = e / U, j = e % U;
      float2 v = make_float2(0.f, 0.f);
      if (i == j) {
        const float2 a = Ab[i * U + i];
        const float den = a.x * a.x + a.y * a.y;
        v = make_float2(c * a.x / den, -c * a.y / den);
      }
      Xb[e] = v;
    }
  }
  __syncthreads();

  bool frozen = !active;
  float s_prev = 0.f, s_last = 0.f;
  int st = NN_OK;
  for (int k = 0; k <= p.nests; ++k) {
    float ss = 0.f;
    if (!frozen) ss = group_gemm<TG, T, UC>(U, ti, tj, Ab, Xb, Rb, nullptr, BM_RESID);
    group_sum(ss, g < groups ? g : 0, lt, NTHR, red_warp, red_grp);
    if (!frozen) {
      const float s = sqrtf(red_grp[g]) / float(U);
      s_last = s;
      if (!isfinite(s) || (k >= 1 && s >= 1.f && s > s_prev)) {
        st = NN_ERR_DIVERGED;
        frozen = true;
      }
      s_prev = s;
    }
    if (k == p.nests) break;
    // Horner: T_1 = R, T_{j+1} = R + R T_j; then X_{k+1} = X_k + X_k T.
    float2* t_cur = Rb;
    for (int j = 1; j < p.depth; ++j) {
      float2* dst = (t_cur == Tb) ? Wb : Tb;
      if (!frozen) group_gemm<TG, T, UC>(U, ti, tj, Rb, t_cur, dst, Rb, BM_ADD);
      __syncthreads();
      t_cur = dst;
    }
    float2* xdst = (t_cur == Wb) ? Tb : Wb;
    if (!frozen) group_gemm<TG, T, UC>(U, ti, tj, Xb, t_cur, xdst, Xb, BM_ADD);
    __syncthreads();
    if (!frozen) {
      // the old X buffer becomes free: keep five distinct buffers for the next nest
      float2* tmp = Xb;
      Xb = xdst;
      if (xdst == Wb)
        Wb = tmp;
      else
        Tb = tmp;
    }
  }
  if (active) {
    for (int e = lt; e < uu; e += NTHR) p.X[off + e] = Xb[e];
    if (lt == 0) {
      p.residual[b] = s_last;
      p.status[b] = st;
    }
  }
  __syncthreads();
}

template <int TG>
__device__ void dispatch_tile(const BatchedParams& p, int U, int start, int cnt, float2* smem, float* rw, float* rg) {
  // sizes with a compile-time path: the massive-MIMO user counts
  if (TG == 8) {
    switch (U) {
      case 8: process_item<TG, 1, 8>(p, U, start, cnt, smem, rw, rg); return;
      case 16: process_item<TG, 2, 16>(p, U, start, cnt, smem, rw, rg); return;
      case 24: process_item<TG, 3, 24>(p, U, start, cnt, smem, rw, rg); return;
      case 32: process_item<TG, 4, 32>(p, U, start, cnt, smem, rw, rg); return;
      default: break;
    }
  } else {
    switch (U) {
      case 16: process_item<TG, 1, 16>(p, U, start, cnt, smem, rw, rg); return;
      case 32: process_item<TG, 2, 32>(p, U, start, cnt, smem, rw, rg); return;
      case 48: process_item<TG, 3, 48>(p, U, start, cnt, smem, rw, rg); return;
      case 64: process_item<TG, 4, 64>(p, U, start, cnt, smem, rw, rg); return;
      default: break;
    }
  }
  const int t = (U + TG - 1) / TG;
  switch (t) {
    case 1: process_item<TG, 1, 0>(p, U, start, cnt, smem, rw, rg); break;
    case 2: process_item<TG, 2, 0>(p, U, start, cnt, smem, rw, rg); break;
    case 3: process_item<TG, 3, 0>(p, U, start, cnt, smem, rw, rg); break;
    case 4: process_item<TG, 4, 0>(p, U, start, cnt, smem, rw, rg); break;
    case 5: if (TG == 8) process_item<TG, 5, 0>(p, U, start, cnt, smem, rw, rg); break;
    case 6: if (TG == 8) process_item<TG, 6, 0>(p, U, start, cnt, smem, rw, rg); break;
    case 7: if (TG == 8) process_item<TG, 7, 0>(p, U, start, cnt, smem, rw, rg); break;
    case 8: if (TG == 8) process_item<TG, 8, 0>(p, U, start, cnt, smem, rw, rg); break;
    default: break;
  }
}

__global__ void __launch_bounds__(BT_THREADS, 1) batched_nn_kernel(const BatchedParams p) {
  extern __shared__ float2 smem[];
  __shared__ float red_warp[BT_THREADS / 32];
  __shared__ float red_grp[BT_THREADS / 32];
  __shared__ int item;
  const int n_items = p.plan[0];
  const int count = p.plan[1];
  const int32_t* items = p.plan + PLAN_HDR + count;
  while (true) {
    if (threadIdx.x == 0) item = atomicAdd(p.queue, 1);
    __syncthreads();
    const int it = item;
    __syncthreads();
    if (it >= n_items) break;
    const int U = items[4 * it + 0];
    const int start = items[4 * it + 1];
    const int cnt = items[4 * it + 2];
    const int cfg = items[4 * it + 3];
    if (cfg == 0)
      dispatch_tile<8>(p, U, start, cnt, smem, red_warp, red_grp);
    else
      dispatch_tile<16>(p, U, start, cnt, smem, red_warp, red_grp);
  }
}

int g_bt_sms = 0;
bool g_bt_init = false;

int bt_init() {
  if (g_bt_init) return NN_OK;
  int dev = 0;
  NN_CUDA_TRY(cudaGetDevice(&dev));
  NN_CUDA_TRY(cudaDeviceGetAttribute(&g_bt_sms, cudaDevAttrMultiProcessorCount, dev));
  NN_CUDA_TRY(cudaFuncSetAttribute(batched_nn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, BT_SMEM));
  g_bt_init = true;
  return NN_OK;
}

// Matrices per work item for (U, cfg): thread groups available and shared memory.
int group_count(int U, int cfg) {
  const int by_threads = cfg == 0 ? BT_THREADS / 64 : 1;
  const int per = BT_BUFS * U * U * int(sizeof(float2));
  int by_smem = BT_SMEM / per;
  return std::max(1, std::min(by_threads, by_smem));
}

}  // namespace
}  // namespace nn

using namespace nn;

extern "C" {

int64_t nn_batched_plan_size(int64_t count) {
  if (count < 1) return 0;
  return PLAN_HDR + count + 4 * count;
}

int nn_batched_plan(const int32_t* sizes_host, int64_t count, const int32_t* cfg_by_u, int32_t* plan_host) {
  if (sizes_host == nullptr || plan_host == nullptr || count < 1 || count > (int64_t(1) << 30)) return NN_ERR_ARG;
  std::vector<int32_t> order(static_cast<size_t>(count));
  for (int64_t i = 0; i < count; ++i) {
    if (sizes_host[i] < 1 || sizes_host[i] > BT_MAX_U) return NN_ERR_ARG;
    order[size_t(i)] = int32_t(i);
  }
  // Largest matrices first (longest-processing-time order); ties keep index order.
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return sizes_host[a] > sizes_host[b]; });
  plan_host[1] = int32_t(count);
  for (int64_t i = 0; i < count; ++i) plan_host[PLAN_HDR + i] = order[size_t(i)];
  int32_t* items = plan_host + PLAN_HDR + count;
  int64_t n_items = 0;
  int64_t pos = 0;
  while (pos < count) {
    const int U = sizes_host[order[size_t(pos)]];
    int cfg = (cfg_by_u != nullptr && cfg_by_u[U] >= 0) ? cfg_by_u[U] : (U <= 32 ? 0 : 1);
    if (cfg != 0 && cfg != 1) return NN_ERR_ARG;
    if (cfg == 1 && (U + 15) / 16 > 4) cfg = 0;
    if (cfg == 0 && (U + 7) / 8 > 8) return NN_ERR_ARG;
    const int gmax = group_count(U, cfg);
    int cnt = 0;
    while (pos + cnt < count && cnt < gmax && sizes_host[order[size_t(pos + cnt)]] == U) ++cnt;
    items[4 * n_items + 0] = U;
    items[4 * n_items + 1] = int32_t(pos);
    items[4 * n_items + 2] = cnt;
    items[4 * n_items + 3] = cfg;
    ++n_items;
    pos += cnt;
  }
  plan_host[0] = int32_t(n_items);
  return NN_OK;
}

size_t nn_batched_workspace_bytes(int64_t count) {
  if (count < 1) return 0;
  return 256;
}

int nn_invert_batched_c64(const void* A, const int64_t* offsets, const int32_t* sizes, int64_t count,
                          const int32_t* plan, int depth, int nests, double damping, void* X, float* residual,
                          int32_t* status, void* workspace, size_t ws_bytes, void* stream) {
  if (A == nullptr || offsets == nullptr || sizes == nullptr || plan == nullptr || X == nullptr ||
      residual == nullptr || status == nullptr || count < 1)
    return NN_ERR_ARG;
  if (depth < 1 || depth > 16 || nests < 0 || nests > NN_MAX_HISTORY - 1 || !(damping >= 0)) return NN_ERR_ARG;
  if (workspace == nullptr || ws_bytes < nn_batched_workspace_bytes(count)) return NN_ERR_OOM_BUDGET;
  NN_TRY(bt_init());
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  BatchedParams p;
  p.A = static_cast<const float2*>(A);
  p.offsets = offsets;
  p.sizes = sizes;
  p.plan = plan;
  p.depth = depth;
  p.nests = nests;
  p.damping = float(damping);
  p.X = static_cast<float2*>(X);
  p.residual = residual;
  p.status = status;
  p.queue = static_cast<int*>(workspace);
  NN_CUDA_TRY(cudaMemsetAsync(p.queue, 0, sizeof(int), st));
  batched_nn_kernel<<<g_bt_sms, BT_THREADS, BT_SMEM, st>>>(p);
  NN_CUDA_TRY(cudaGetLastError());
  return NN_OK;
}

}  // extern "C"
