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
// and cuts them into work items of G equal-size matrices. Inside a CTA, G thread groups run
// G matrices in lock-step (same U, same barriers). Two tile configurations exist per size:
//   cfg 0: 8 x 8 threads per matrix, each computing a ceil(U/8)^2 tile of every product;
//   cfg 1: 16 x 16 threads per matrix, tile ceil(U/16)^2, one matrix per CTA.
// The plan takes a per-size configuration table, which the autotuner fills. Items fall into
// tile classes (tensor cores; or CUDA cores with a given (threads per matrix, tile, exact U)),
// and each class has its own persistent kernel, compiled alone so that the CUDA-core ones fit
// 128 registers and run two 256-thread CTAs per SM. The classes' kernels are chained with
// programmatic dependent launch: the next class's CTAs take the SM slots that the previous
// class frees at its tail. Each kernel pulls the items of its class from its own counter.
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
constexpr int BT_SMEM = 200 * 1024;         // dynamic shared memory of a tensor-core CTA
// CUDA-core items: two CTAs per SM at depth <= 2 (three buffers per matrix), one at depth >= 3
// (four buffers, 4/3 of the same shared memory), so a plan sized for the first fits both.
constexpr int BT_SMEM_SIMT = 112 * 1024;
constexpr int BT_SMEM_SIMT_DEEP = BT_SMEM_SIMT / 3 * 4;
// Tile classes: 0 = tensor-core items; 1..16 = CUDA-core items, ordered by cost: 16x16 threads
// then 8x8, tile 4 down to 1, exact U (= tile * threads per side) before other sizes.
constexpr int BT_NCLS = NN_BATCHED_KERNELS;
constexpr int PLAN_HDR = 3 + BT_NCLS + 1;   // [n_items, count, n_tc, class_first[BT_NCLS + 1]]
constexpr int BT_QUEUE_ERR = 32;            // workspace: int counters [0, BT_NCLS), error word here

static_assert(BT_NCLS <= BT_QUEUE_ERR && (BT_QUEUE_ERR + 1) * 4 <= 256, "counters fit the workspace");

__host__ __device__ constexpr int bt_class(int cfg, int U) {
  return cfg == 2 ? 0
                  : 1 + (cfg == 0 ? 8 : 0) + (4 - (U + (cfg == 0 ? 7 : 15)) / (cfg == 0 ? 8 : 16)) * 2 +
                        (U % (cfg == 0 ? 8 : 16) == 0 ? 0 : 1);
}

enum : int { BM_RESID = 0, BM_ADD = 1 };

// acc = P Q for this thread's part of a U x U complex group tile: thread (ti, tj) of the
// TG x TG group owns rows ti + a TG and columns tj + b TG. UC > 0 fixes U = UC = T * TG at
// compile time (no bounds tests, static addressing); UC = 0 handles any U <= T * TG.
template <int TG, int T, int UC>
__device__ __forceinline__ void group_acc(int U_rt, int ti, int tj, const float2* P, const float2* Q,
                                          float2 (&acc)[T][T]) {
  const int U = UC > 0 ? UC : U_rt;
  constexpr bool exact = UC > 0 && UC == T * TG;
#pragma unroll
  for (int a = 0; a < T; ++a)
#pragma unroll
    for (int b = 0; b < T; ++b) acc[a][b] = make_float2(0.f, 0.f);
  if (exact && (UC % 2) == 0) {
    // P[i, k] and P[i, k + 1] arrive in one 16-byte load (two k steps per P load), which cuts
    // the shared-memory wavefronts of the P operand in half; same FMA order as below.
#pragma unroll 2
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
#pragma unroll(UC > 0 ? 2 : 1)
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
}

// out = (mode RESID) I - acc  or  (mode ADD) D + acc on this thread's elements; returns the
// thread's sum of |out|^2 (residual mode). out may be D or an operand of the product as long as
// every thread of the CTA has finished the product (a barrier between group_acc and this).
template <int TG, int T, int UC>
__device__ __forceinline__ float group_store(int U_rt, int ti, int tj, const float2 (&acc)[T][T], float2* out,
                                             const float2* D, int mode) {
  const int U = UC > 0 ? UC : U_rt;
  constexpr bool exact = UC > 0 && UC == T * TG;
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
  int* err;     // device error word of the tensor-core path's bounded waits
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

// One product of the nest: acc = P Q, an optional CTA barrier (when out aliases P, Q or D), then
// out = mode(acc). Every thread of the CTA calls it (frozen groups skip the arithmetic).
template <int TG, int T, int UC>
__device__ __forceinline__ float group_product(int U, int ti, int tj, const float2* P, const float2* Q,
                                               float2* out, const float2* D, int mode, bool barrier, bool frozen) {
  float2 acc[T][T];
  if (!frozen) group_acc<TG, T, UC>(U, ti, tj, P, Q, acc);
  if (barrier) __syncthreads();
  return frozen ? 0.f : group_store<TG, T, UC>(U, ti, tj, acc, out, D, mode);
}

// Buffers per matrix: A, X, R, and T for depth >= 3. Products whose output overwrites one of
// their own operands (T in place of R at depth 2, T <- R + R T, X <- X + X T) accumulate in
// registers, wait at a CTA barrier, then store.
__host__ __device__ constexpr int bt_buffers(int depth) { return depth >= 3 ? 4 : 3; }

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
  float2* base = smem + size_t(g < groups ? g : 0) * bt_buffers(p.depth) * uu;
  float2* Ab = base;
  float2* Xb = base + uu;
  float2* Rb = base + 2 * uu;
  float2* Tb = p.depth >= 3 ? base + 3 * uu : Rb;
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
    const float ss = group_product<TG, T, UC>(U, ti, tj, Ab, Xb, Rb, nullptr, BM_RESID, false, frozen);
    group_sum(ss, g < groups ? g : 0, lt, NTHR, red_warp, red_grp);  // includes CTA barriers
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
    // Horner: T_1 = R, T_{j+1} = R + R T_j (depth 2: T_2 replaces R in place); then
    // X_{k+1} = X_k + X_k T in place.
    const float2* t_cur = Rb;
    for (int j = 1; j < p.depth; ++j) {
      group_product<TG, T, UC>(U, ti, tj, Rb, t_cur, Tb, Rb, BM_ADD, true, frozen);
      __syncthreads();
      t_cur = Tb;
    }
    group_product<TG, T, UC>(U, ti, tj, Xb, t_cur, Xb, Xb, BM_ADD, true, frozen);
    __syncthreads();
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

// ---- tensor-core path (plan configuration 2; U in {16, 32, 48, 64}) ------------------------
//
// One matrix per CTA at a time, every iterate kept on chip:
//   * masters (A, X, R, T, W) live in TMEM as the real form [Re; Im] of each U x U complex matrix:
//     lane i < U holds row i's real parts, lane U + i its imaginary parts, columns 0..U-1;
//   * a complex product C = P Q runs as one real MMA on the embedding
//         [Cr; Ci] (2U x U) = [[Pr, -Pi], [Pi, Pr]] (2U x 2U) . [Qr; Qi] (2U x U),
//     i.e. M = 128 (2U rows used), N = U, K = 2U, with no redundant work. Its left operand is
//     built from P's master rows, its right operand (K-major: row j = column j of [Qr; Qi]) is
//     exactly the transpose of Q's master (lane k, column j -> row j, k);
//   * operands are split into three BF16 pieces (x = p0 + p1 + p2, each the BF16 rounding of the
//     remainder) and written to shared memory in the SWIZZLE_128B K-major layout; six piece
//     products (the pairs with i + j <= 2, smallest first) accumulate in FP32 in TMEM, which
//     matches an FP32 product to about 2^-24 relative;
//   * the epilogue reads the accumulator, applies I - C or D + C in FP32 and writes the result
//     master back to TMEM; the residual's sum of squares is reduced across the CTA.
namespace btc {
constexpr int M = 128;                         // MMA rows (2U used)
constexpr int KP = 128;                        // K capacity (2U used): two 64-wide k-blocks
constexpr int NP = 64;                         // B-operand rows capacity (U used)
constexpr int A_PIECE = M * KP * 2;            // 32 KB
constexpr int B_PIECE = NP * KP * 2;           // 16 KB
constexpr int OPS_BYTES = 3 * A_PIECE + 3 * B_PIECE;
constexpr uint32_t ACC = 0, MA = 64, MX = 128, MR = 192, MT = 256, MW = 320;
constexpr uint32_t TMEM_COLS = 512;
static_assert(OPS_BYTES + 1024 <= BT_SMEM, "operand pieces fit the dynamic shared memory");
}  // namespace btc

// Shared-memory matrix descriptor of a K-major SWIZZLE_128B tile (8-row atoms 1024 B apart).
__device__ __forceinline__ uint64_t bt_sw128_desc(uint32_t saddr) {
  return uint64_t((saddr & 0x3FFFFu) >> 4) | (uint64_t(1) << 16) | (uint64_t(1024 >> 4) << 32) |
         (uint64_t(1) << 46) | (uint64_t(2) << 61);
}

// Byte offset of element (r, k) in a K-major SWIZZLE_128B operand of `rows` rows and 64-wide
// k-blocks: 16-byte chunk c of row r sits at chunk c ^ (r mod 8) of its 128-byte line.
__device__ __forceinline__ uint32_t bt_sw128_offset(int r, int k, int rows) {
  const int kb = k >> 6, c = (k & 63) >> 3, e = k & 7;
  return uint32_t(kb * rows * 128 + (r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4) + (e << 1));
}

__device__ __forceinline__ void split3(float x, __nv_bfloat16& p0, __nv_bfloat16& p1, __nv_bfloat16& p2) {
  p0 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(p0);
  p1 = __float2bfloat16_rn(r1);
  p2 = __float2bfloat16_rn(r1 - __bfloat162float(p1));
}

// Left operand [[Pr, -Pi], [Pi, Pr]] pieces from master P; warp (q, h) owns lanes 32q.. and
// columns 32h.. of the master.
template <int U>
__device__ __forceinline__ void bt_build_left(uint32_t tmem, uint32_t cP, uint8_t* ops, int q, int h, int l) {
  if (h * 32 >= U) return;
  uint32_t raw[32];
  tmem_ld_32x32b_x32(tmem + (uint32_t(q * 32) << 16) + cP + uint32_t(h * 32), raw);
  tmem_ld_wait();
  if (l >= 2 * U) return;
  const bool re = l < U;
  const int i = re ? l : l - U;
  // destination 1: row i at K = (re ? 0 : U) + column, sign (re ? + : -); destination 2: row
  // U + i at K = (re ? U : 0) + column, sign +
  const int rows[2] = {i, U + i};
  const int kbase[2] = {re ? 0 : U, re ? U : 0};
  const float sgn[2] = {re ? 1.0f : -1.0f, 1.0f};
#pragma unroll
  for (int d = 0; d < 2; ++d) {
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
      const int j0 = h * 32 + ch * 8;
      if (j0 >= U) break;
      uint32_t pk[3][4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        __nv_bfloat16 a0, a1, a2, b0, b1, b2;
        split3(sgn[d] * __uint_as_float(raw[ch * 8 + 2 * e]), a0, a1, a2);
        split3(sgn[d] * __uint_as_float(raw[ch * 8 + 2 * e + 1]), b0, b1, b2);
        pk[0][e] = uint32_t(__bfloat16_as_ushort(a0)) | (uint32_t(__bfloat16_as_ushort(b0)) << 16);
        pk[1][e] = uint32_t(__bfloat16_as_ushort(a1)) | (uint32_t(__bfloat16_as_ushort(b1)) << 16);
        pk[2][e] = uint32_t(__bfloat16_as_ushort(a2)) | (uint32_t(__bfloat16_as_ushort(b2)) << 16);
      }
      const uint32_t off = bt_sw128_offset(rows[d], kbase[d] + j0, btc::M);
#pragma unroll
      for (int pc = 0; pc < 3; ++pc)
        *reinterpret_cast<uint4*>(ops + pc * btc::A_PIECE + off) = make_uint4(pk[pc][0], pk[pc][1], pk[pc][2], pk[pc][3]);
    }
  }
}

// Right operand pieces: row j, column k = master Q (lane k, column j), k < 2U, j < U. Even lanes
// store the pair (k, k + 1) received from the odd neighbour.
template <int U>
__device__ __forceinline__ void bt_build_right(uint32_t tmem, uint32_t cQ, uint8_t* ops, int q, int h, int l) {
  if (h * 32 >= U) return;
  uint32_t raw[32];
  tmem_ld_32x32b_x32(tmem + (uint32_t(q * 32) << 16) + cQ + uint32_t(h * 32), raw);
  tmem_ld_wait();
  uint8_t* bops = ops + 3 * btc::A_PIECE;
  const bool store = (l & 1) == 0 && l < 2 * U;
#pragma unroll
  for (int t = 0; t < 32; ++t) {
    const float v = __uint_as_float(raw[t]);
    const float w = __shfl_down_sync(0xffffffffu, v, 1);
    const int j = h * 32 + t;
    if (store && j < U) {
      __nv_bfloat16 a0, a1, a2, b0, b1, b2;
      split3(v, a0, a1, a2);
      split3(w, b0, b1, b2);
      const uint32_t off = bt_sw128_offset(j, l, btc::NP);
      *reinterpret_cast<uint32_t*>(bops + off) =
          uint32_t(__bfloat16_as_ushort(a0)) | (uint32_t(__bfloat16_as_ushort(b0)) << 16);
      *reinterpret_cast<uint32_t*>(bops + btc::B_PIECE + off) =
          uint32_t(__bfloat16_as_ushort(a1)) | (uint32_t(__bfloat16_as_ushort(b1)) << 16);
      *reinterpret_cast<uint32_t*>(bops + 2 * btc::B_PIECE + off) =
          uint32_t(__bfloat16_as_ushort(a2)) | (uint32_t(__bfloat16_as_ushort(b2)) << 16);
    }
  }
}

// out = mode(P Q) for masters at TMEM columns cP, cQ, cD (addend), cOut; returns this thread's
// sum of squares of the result (residual mode). false if the MMA wait timed out.
template <int U>
__device__ bool bt_product(uint32_t tmem, uint8_t* ops, uint64_t* bar, uint32_t& phase, volatile int* abort_flag,
                           int* err, uint32_t cP, uint32_t cQ, uint32_t cD, uint32_t cOut, int mode, float* ss) {
  const int w = int(threadIdx.x >> 5), q = w & 3, h = w >> 2, l = q * 32 + int(threadIdx.x & 31);
  bt_build_left<U>(tmem, cP, ops, q, h, l);
  bt_build_right<U>(tmem, cQ, ops, q, h, l);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    tc_fence_after();
    constexpr uint32_t idesc =
        (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(U >> 3) << 17) | (uint32_t(btc::M >> 4) << 24);
    const uint32_t base = smem_u32(ops);
    // piece pairs (a, b), smallest terms first: (2,0) (1,1) (0,2) (1,0) (0,1) (0,0)
    uint32_t acc = 0;
#pragma unroll 1
    for (int pp = 0; pp < 6; ++pp) {
      const int pa = pp == 0 ? 2 : (pp == 1 || pp == 3) ? 1 : 0;
      const int pb = pp == 2 ? 2 : (pp == 1 || pp == 4) ? 1 : 0;
      const uint32_t a0 = base + uint32_t(pa * btc::A_PIECE);
      const uint32_t b0 = base + uint32_t(3 * btc::A_PIECE + pb * btc::B_PIECE);
#pragma unroll 1
      for (int st = 0; st < U / 8; ++st) {
        const int kb = st >> 2, kk = st & 3;
        const uint64_t ad = bt_sw128_desc(a0 + uint32_t(kb * btc::M * 128)) + uint64_t(2 * kk);
        const uint64_t bd = bt_sw128_desc(b0 + uint32_t(kb * btc::NP * 128)) + uint64_t(2 * kk);
        tc_mma_bf16(tmem + btc::ACC, ad, bd, idesc, acc);
        acc = 1;
      }
    }
    tc_commit(bar);
  }
  // every thread learns the same outcome (a timed-out wait in any thread aborts the item)
  const bool ok = __syncthreads_and(mbar_wait(bar, phase, abort_flag, err) ? 1 : 0) != 0;
  phase ^= 1u;
  tc_fence_after();
  if (!ok) return false;
  // epilogue: warp (q, h) owns accumulator lanes 32q.. and columns 32h..
  float local = 0.f;
  if (h * 32 < U) {
    uint32_t c[32], d[32];
    const uint32_t lane_off = uint32_t(q * 32) << 16;
    tmem_ld_32x32b_x32(tmem + lane_off + btc::ACC + uint32_t(h * 32), c);
    if (mode == BM_ADD) tmem_ld_32x32b_x32(tmem + lane_off + cD + uint32_t(h * 32), d);
    tmem_ld_wait();
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      const int j = h * 32 + t;
      const float cv = __uint_as_float(c[t]);
      float v;
      if (mode == BM_RESID) {
        v = ((l < U && j == l) ? 1.f : 0.f) - cv;
        if (l < 2 * U && j < U) local = fmaf(v, v, local);
      } else {
        v = __uint_as_float(d[t]) + cv;
      }
      c[t] = __float_as_uint(v);
    }
    tmem_st_32x32b_x32(tmem + lane_off + cOut + uint32_t(h * 32), c);
    tmem_st_wait();
  }
  *ss = local;
  tc_fence_before();
  __syncthreads();
  return true;
}

// Sum over the CTA (256 threads); result broadcast to every thread.
__device__ __forceinline__ float bt_block_sum(float v, float* red_warp) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red_warp[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  for (int w = 0; w < BT_THREADS / 32; ++w) t += red_warp[w];
  __syncthreads();
  return t;
}

template <int U>
__device__ void process_item_tc(const BatchedParams& p, int start, uint8_t* ops, uint32_t tmem, uint64_t* bar,
                                uint32_t& phase, volatile int* abort_flag, float* red_warp) {
  const int w = int(threadIdx.x >> 5), q = w & 3, h = w >> 2, l = q * 32 + int(threadIdx.x & 31);
  const int b = p.plan[PLAN_HDR + start];
  const int64_t off = p.offsets[b];
  const float2* A = p.A + off;
  // masters A and X_0 = c diag(A)^-1 (damped Jacobi) in their real forms
  if (h * 32 < U) {
    uint32_t va[32], vx[32];
    const bool valid_row = l < 2 * U;
    const bool re = l < U;
    const int i = re ? l : l - U;
    float2 aii = make_float2(1.f, 0.f);
    if (valid_row) aii = A[i * U + i];
    const float cdamp = 1.f / (1.f + p.damping * float(U));
    const float den = aii.x * aii.x + aii.y * aii.y;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      const int j = h * 32 + t;
      float av = 0.f, xv = 0.f;
      if (valid_row && j < U) {
        const float2 a = A[i * U + j];
        av = re ? a.x : a.y;
        if (j == i) xv = re ? cdamp * aii.x / den : -cdamp * aii.y / den;
      }
      va[t] = __float_as_uint(av);
      vx[t] = __float_as_uint(xv);
    }
    const uint32_t lane_off = uint32_t(q * 32) << 16;
    tmem_st_32x32b_x32(tmem + lane_off + btc::MA + uint32_t(h * 32), va);
    tmem_st_32x32b_x32(tmem + lane_off + btc::MX + uint32_t(h * 32), vx);
    tmem_st_wait();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  bool frozen = false, timed_out = false;
  float s_prev = 0.f, s_last = 0.f;
  int st = NN_OK;
  uint32_t cX = btc::MX;
  for (int k = 0; k <= p.nests; ++k) {
    if (!frozen) {
      float ss = 0.f;
      if (!bt_product<U>(tmem, ops, bar, phase, abort_flag, p.err, btc::MA, cX, 0, btc::MR, BM_RESID, &ss)) {
        timed_out = true;
        break;
      }
      const float s = sqrtf(bt_block_sum(ss, red_warp)) / float(U);
      s_last = s;
      if (!isfinite(s) || (k >= 1 && s >= 1.f && s > s_prev)) {
        st = NN_ERR_DIVERGED;
        frozen = true;
      }
      s_prev = s;
    }
    if (k == p.nests || frozen) break;
    // Horner: T_1 = R, T_{j+1} = R + R T_j (T, W alternate); X_{k+1} = X_k + X_k T
    uint32_t t_cur = btc::MR;
    bool ok = true;
    for (int j = 1; j < p.depth && ok; ++j) {
      const uint32_t dst = (t_cur == btc::MT) ? btc::MW : btc::MT;
      float unused = 0.f;
      ok = bt_product<U>(tmem, ops, bar, phase, abort_flag, p.err, btc::MR, t_cur, btc::MR, dst, BM_ADD, &unused);
      t_cur = dst;
    }
    float unused = 0.f;
    if (!ok || !bt_product<U>(tmem, ops, bar, phase, abort_flag, p.err, cX, t_cur, cX, cX, BM_ADD, &unused)) {
      timed_out = true;
      break;
    }
  }
  if (timed_out) st = NN_ERR_TIMEOUT;
  // X (complex, row-major) from the X master; 2U is a multiple of 32, so the test is warp-uniform
  if (h * 32 < U && q * 32 < 2 * U) {
    uint32_t vx[32];
    tmem_ld_32x32b_x32(tmem + (uint32_t(q * 32) << 16) + cX + uint32_t(h * 32), vx);
    tmem_ld_wait();
    const bool re = l < U;
    const int i = re ? l : l - U;
    float* Xf = reinterpret_cast<float*>(p.X + off);
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      const int j = h * 32 + t;
      if (j < U) Xf[2 * (i * U + j) + (re ? 0 : 1)] = __uint_as_float(vx[t]);
    }
  }
  if (threadIdx.x == 0) {
    p.residual[b] = s_last;
    p.status[b] = st;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

__device__ void dispatch_tc(const BatchedParams& p, int U, int start, uint8_t* ops, uint32_t tmem, uint64_t* bar,
                            uint32_t& phase, volatile int* abort_flag, float* red_warp) {
  switch (U) {
    case 16: process_item_tc<16>(p, start, ops, tmem, bar, phase, abort_flag, red_warp); break;
    case 32: process_item_tc<32>(p, start, ops, tmem, bar, phase, abort_flag, red_warp); break;
    case 48: process_item_tc<48>(p, start, ops, tmem, bar, phase, abort_flag, red_warp); break;
    default: process_item_tc<64>(p, start, ops, tmem, bar, phase, abort_flag, red_warp); break;
  }
}

__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// Waits for the previous kernel of the chain to complete, so that each kernel's completion
// implies its predecessors' (stream order for whatever follows the last one).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// The tensor-core items (class 0): one CTA per SM, 512 TMEM columns.
__global__ void __launch_bounds__(BT_THREADS, 1) batched_tc_kernel(const BatchedParams p) {
  extern __shared__ float2 smem[];
  __shared__ float red_warp[BT_THREADS / 32];
  __shared__ int item;
  __shared__ __align__(8) uint64_t tc_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_word;
  pdl_launch_dependents();
  const int count = p.plan[1];
  const int first = p.plan[3], last = p.plan[4];
  const int32_t* items = p.plan + PLAN_HDR + count;
  if (first < last) {
    // operand pieces at a 1024-aligned offset of the dynamic shared memory, one mbarrier for
    // MMA completion
    uint8_t* ops = reinterpret_cast<uint8_t*>(smem);
    ops += (1024u - (smem_u32(ops) & 1023u)) & 1023u;
    if (threadIdx.x == 0) {
      mbar_init(&tc_bar, 1);
      abort_word = 0;
      mbar_fence_init();
    }
    if (threadIdx.x < 32) tmem_alloc(&tmem_slot, btc::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    uint32_t phase = 0;
    while (true) {
      if (threadIdx.x == 0) item = first + atomicAdd(p.queue, 1);
      __syncthreads();
      const int it = item;
      __syncthreads();
      if (it >= last) break;
      dispatch_tc(p, items[4 * it + 0], items[4 * it + 1], ops, tmem, &tc_bar, phase, &abort_word, red_warp);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(tmem, btc::TMEM_COLS);
  }
  pdl_wait();
}

// The CUDA-core items of one class (TG x TG threads per matrix, T x T tile, UC = exact U or
// 0): two CTAs per SM at depth <= 2.
template <int TG, int T, int UC>
__global__ void __launch_bounds__(BT_THREADS, 2) batched_simt_kernel(const BatchedParams p, int cls) {
  extern __shared__ float2 smem[];
  __shared__ float red_warp[BT_THREADS / 32];
  __shared__ float red_grp[BT_THREADS / 32];
  __shared__ int item;
  pdl_launch_dependents();
  const int count = p.plan[1];
  const int first = p.plan[3 + cls], last = p.plan[3 + cls + 1];
  const int32_t* items = p.plan + PLAN_HDR + count;
  if (first < last) {
    while (true) {
      if (threadIdx.x == 0) item = first + atomicAdd(p.queue + cls, 1);
      __syncthreads();
      const int it = item;
      __syncthreads();
      if (it >= last) break;
      process_item<TG, T, UC>(p, items[4 * it + 0], items[4 * it + 1], items[4 * it + 2], smem, red_warp, red_grp);
    }
  }
  pdl_wait();
}

using SimtKernel = void (*)(const BatchedParams, int);

// Kernel of each CUDA-core class, in class order (bt_class).
const SimtKernel kSimtKernels[BT_NCLS - 1] = {
    batched_simt_kernel<16, 4, 64>, batched_simt_kernel<16, 4, 0>, batched_simt_kernel<16, 3, 48>,
    batched_simt_kernel<16, 3, 0>,  batched_simt_kernel<16, 2, 32>, batched_simt_kernel<16, 2, 0>,
    batched_simt_kernel<16, 1, 16>, batched_simt_kernel<16, 1, 0>,  batched_simt_kernel<8, 4, 32>,
    batched_simt_kernel<8, 4, 0>,   batched_simt_kernel<8, 3, 24>,  batched_simt_kernel<8, 3, 0>,
    batched_simt_kernel<8, 2, 16>,  batched_simt_kernel<8, 2, 0>,   batched_simt_kernel<8, 1, 8>,
    batched_simt_kernel<8, 1, 0>};

int g_bt_sms = 0;
bool g_bt_init = false;

int bt_init() {
  if (g_bt_init) return NN_OK;
  int dev = 0;
  NN_CUDA_TRY(cudaGetDevice(&dev));
  NN_CUDA_TRY(cudaDeviceGetAttribute(&g_bt_sms, cudaDevAttrMultiProcessorCount, dev));
  NN_CUDA_TRY(cudaFuncSetAttribute(batched_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, BT_SMEM));
  for (SimtKernel k : kSimtKernels)
    NN_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, BT_SMEM_SIMT_DEEP));
  g_bt_init = true;
  return NN_OK;
}

// Matrices per work item for (U, cfg): thread groups available and shared memory.
int group_count(int U, int cfg) {
  if (cfg == 2) return 1;
  const int by_threads = cfg == 0 ? BT_THREADS / 64 : 1;
  const int per = bt_buffers(2) * U * U * int(sizeof(float2));
  int by_smem = BT_SMEM_SIMT / per;
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
    if (cfg < 0 || cfg > 2) return NN_ERR_ARG;
    if (cfg == 2 && (U % 16 != 0 || U > 64)) cfg = U <= 32 ? 0 : 1;
    if (cfg == 0 && (U + 7) / 8 > 4) cfg = 1;  // 8 x 8 threads with up to 4 x 4 elements each
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
  // items grouped by class (each class's kernel takes [class_first[c], class_first[c + 1])),
  // each class still largest first
  std::vector<int32_t> tmp(items, items + 4 * n_items);
  int64_t w = 0;
  int32_t* class_first = plan_host + 3;
  for (int c = 0; c < BT_NCLS; ++c) {
    class_first[c] = int32_t(w);
    for (int64_t it = 0; it < n_items; ++it)
      if (bt_class(tmp[size_t(4 * it + 3)], tmp[size_t(4 * it)]) == c) {
        for (int f = 0; f < 4; ++f) items[4 * w + f] = tmp[size_t(4 * it + f)];
        ++w;
      }
  }
  class_first[BT_NCLS] = int32_t(w);
  plan_host[0] = int32_t(n_items);
  plan_host[2] = class_first[1];
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
  p.err = static_cast<int*>(workspace) + BT_QUEUE_ERR;
  NN_CUDA_TRY(cudaMemsetAsync(p.queue, 0, nn_batched_workspace_bytes(count), st));
  batched_tc_kernel<<<g_bt_sms, BT_THREADS, BT_SMEM, st>>>(p);
  NN_CUDA_TRY(cudaGetLastError());
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(depth <= 2 ? 2 * g_bt_sms : g_bt_sms));
  cfg.blockDim = dim3(BT_THREADS);
  cfg.dynamicSmemBytes = size_t(depth <= 2 ? BT_SMEM_SIMT : BT_SMEM_SIMT_DEEP);
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  for (int c = 1; c < BT_NCLS; ++c) NN_CUDA_TRY(cudaLaunchKernelEx(&cfg, kSimtKernels[c - 1], p, c));
  return NN_OK;
}

}  // extern "C"
