// Batched NN inversion of many small complex matrices (massive-MIMO Gram matrices,
// U x U with U <= 64) in persistent kernels.
//
// Each matrix runs the right-multiplied NN loop of the dense path (Theorem, Eq.
// (nestedneumann); L = 1 Newton, L = 2 Chebyshev as in Corollary 4) entirely on chip (shared
// memory, or TMEM on the tensor-core path), from the damped Jacobi start
// X_0 = diag(A)^-1 / (1 + damping U) (a diagonal Theta, Appendix 1), for a fixed number of
// nests:
//     k = 0..nests:  R = I - A X_k, s_k = ||R||_F / U;  stop if diverged or k = nests;
//                    T = R, L-1 times T = R + R T;  X_{k+1} = X_k + X_k T.
// Divergence (s_k non-finite, or s_k >= 1 and s_k > s_{k-1}) freezes X at X_k, as the dense
// path does.
//
// Scheduling: the host plan (nn_batched_plan) sorts the matrices by size, largest first,
// and cuts them into work items of equal-size matrices, each with a configuration taken from a
// per-size table (the autotuner fills it):
//   cfg 0: CUDA cores, 8 x 8 threads per matrix, each computing a ceil(U/8)^2 tile of every
//          product, up to four matrices per CTA in lock-step;
//   cfg 1: CUDA cores, 16 x 16 threads per matrix, tile ceil(U/16)^2, one matrix per CTA;
//   cfg 2: tensor cores, U in {48, 64} (see the tensor-core notes below);
//   cfg 3: CUDA cores, one warp per matrix, U in {8, 16, 24, 32}.
// Items fall into tile classes, and each class has its own persistent kernel, compiled alone
// so that the CTA-wide CUDA-core ones fit 128 registers and run two 256-thread CTAs per SM.
// Only the classes that hold items are launched, chained with programmatic dependent launch:
// the next class's CTAs take the SM slots that the previous class frees at its tail. Each
// kernel pulls the items of its class from its own counter.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace nn {
namespace {

constexpr int BT_THREADS = 256;
constexpr int BT_MAX_U = 64;
constexpr int BT_SMEM = 193 * 1024;         // dynamic shared memory of a tensor-core CTA
// CUDA-core items: two CTAs per SM at depth <= 2 (three buffers per matrix), one at depth >= 3
// (four buffers, 4/3 of the same shared memory), so a plan sized for the first fits both.
constexpr int BT_SMEM_SIMT = 112 * 1024;
constexpr int BT_SMEM_SIMT_DEEP = BT_SMEM_SIMT / 3 * 4;
// Tile classes: 0, 1 = tensor-core items of U = 64, 48; 2..17 = CUDA-core items, ordered by
// cost: 16x16 threads then 8x8, tile 4 down to 1, exact U (= tile * threads per side) first;
// 18..21 = warp-per-matrix CUDA-core items of U = 32, 24, 16, 8.
constexpr int BT_NCLS = NN_BATCHED_KERNELS;
constexpr int PLAN_HDR = 3 + BT_NCLS + 1;   // [n_items, count, n_tc, class_first[BT_NCLS + 1]]
constexpr int BT_QUEUE_ERR = 32;            // workspace: int counters [0, BT_NCLS), error word here

static_assert(BT_NCLS <= BT_QUEUE_ERR && (BT_QUEUE_ERR + 1) * 4 <= 256, "counters fit the workspace");

__host__ __device__ constexpr int bt_class(int cfg, int U) {
  return cfg == 3   ? 18 + (4 - U / 8)
         : cfg == 2 ? (U == 64 ? 0 : 1)
                    : 2 + (cfg == 0 ? 8 : 0) + (4 - (U + (cfg == 0 ? 7 : 15)) / (cfg == 0 ? 8 : 16)) * 2 +
                        (U % (cfg == 0 ? 8 : 16) == 0 ? 0 : 1);
}

enum : int { BM_RESID = 0, BM_ADD = 1 };

// Row pitch (complex elements) of the shared-memory tiles of the CUDA-core classes. An exact
// class (U a multiple of TG) pads its rows to the smallest pitch with pitch % 16 in {4, 12}:
// the four rows that one warp of an 8 x 8 group touches then start 8 banks apart, so the
// 16-byte loads of P (four rows, one k pair) take one wavefront instead of four and the
// 8-byte stores of the epilogue (four rows of eight elements) two instead of four; the two
// rows of a 16 x 16 group's warp fall in different banks as well. Other classes keep pitch U.
__host__ __device__ constexpr int bt_pad_pitch(int U) {
  return U % 16 <= 4 ? U - U % 16 + 4 : (U % 16 <= 12 ? U - U % 16 + 12 : U - U % 16 + 20);
}
__host__ __device__ constexpr int bt_simt_pitch(int U, int TG) { return U % TG == 0 ? bt_pad_pitch(U) : U; }

// acc = P Q for this thread's part of a U x U complex group tile: thread (ti, tj) of the
// TG x TG group owns rows ti + a TG and columns tj + b TG. UC > 0 fixes U = UC = T * TG at
// compile time (no bounds tests, static addressing); UC = 0 handles any U <= T * TG.
template <int TG, int T, int UC>
__device__ __forceinline__ void group_acc(int U_rt, int ti, int tj, const float2* P, const float2* Q,
                                          float2 (&acc)[T][T]) {
  const int U = UC > 0 ? UC : U_rt;
  constexpr bool exact = UC > 0 && UC == T * TG;
  const int ld = exact ? bt_pad_pitch(UC) : U;
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
      for (int a = 0; a < T; ++a) pa2[a] = *reinterpret_cast<const float4*>(P + (ti + a * TG) * ld + k);
      float2 q0[T], q1[T];
#pragma unroll
      for (int b = 0; b < T; ++b) {
        q0[b] = Q[k * ld + tj + b * TG];
        q1[b] = Q[(k + 1) * ld + tj + b * TG];
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
      pa[a] = (exact || i < U) ? P[i * ld + k] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int b = 0; b < T; ++b) {
      const int j = tj + b * TG;
      qb[b] = (exact || j < U) ? Q[k * ld + j] : make_float2(0.f, 0.f);
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
  const int ld = exact ? bt_pad_pitch(UC) : U;
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
        const float2 d = D[i * ld + j];
        v = make_float2(d.x + acc[a][b].x, d.y + acc[a][b].y);
      }
      out[i * ld + j] = v;
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
  int withhold;  // failure-detection test hook: each CTA's MMA warp withholds its first commit
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
  if (UC > 0) U = UC;  // exact classes: compile-time size (static addressing and divisions)
  const int groups = BT_THREADS / NTHR;
  const int g = threadIdx.x / NTHR;
  const int lt = threadIdx.x % NTHR;
  const int ti = lt / TG, tj = lt % TG;
  const bool active = g < groups && g < cnt;
  const int uu = U * U;
  // tiles are U x ld (ld = bt_simt_pitch); element e of the matrix (row-major) sits at
  // (e / U) * ld + e % U
  const int ld = UC > 0 && UC == T * TG ? bt_pad_pitch(UC) : U;
  const int tile = U * ld;
  const int b = active ? p.plan[PLAN_HDR + start + g] : -1;
  float2* base = smem + size_t(g < groups ? g : 0) * bt_buffers(p.depth) * tile;
  float2* Ab = base;
  float2* Xb = base + tile;
  float2* Rb = base + 2 * tile;
  float2* Tb = p.depth >= 3 ? base + 3 * tile : Rb;
  const int64_t off = active ? p.offsets[b] : 0;

  if (active) {
    for (int e = lt; e < uu; e += NTHR) Ab[(e / U) * ld + e % U] = p.A[off + e];
  }
  __syncthreads();
  if (active) {
    const float c = 1.f / (1.f + p.damping * float(U));
    for (int e = lt; e < uu; e += NTHR) {
      const int i = e / U, j = e % U;
      float2 v = make_float2(0.f, 0.f);
      if (i == j) {
        const float2 a = Ab[i * ld + i];
        const float den = a.x * a.x + a.y * a.y;
        v = make_float2(c * a.x / den, -c * a.y / den);
      }
      Xb[i * ld + j] = v;
    }
  }
  __syncthreads();

  bool frozen = !active;
  float s_prev = 0.f, s_last = 0.f;
  int st = NN_OK;
  // X_0 is diagonal, so with at least one nest the first nest's residual R_0 = I - A X_0 (a
  // column scaling) and update X_1 = X_0 (I + T) (a row scaling) are element-wise; x0 is
  // recomputed from A's diagonal exactly as X_0 was, so X is never read while it is rewritten.
  const float cdamp = 1.f / (1.f + p.damping * float(U));
  for (int k = 0; k <= p.nests; ++k) {
    const bool diag0 = k == 0;
    float ss = 0.f;
    if (diag0) {
      if (!frozen) {
        for (int e = lt; e < uu; e += NTHR) {
          const int i = e / U, j = e % U;
          const float2 a = Ab[i * ld + j];
          const float2 xj = Xb[j * ld + j];
          const float2 r = make_float2((i == j ? 1.f : 0.f) - (a.x * xj.x - a.y * xj.y), -(a.x * xj.y + a.y * xj.x));
          Rb[i * ld + j] = r;
          ss = fmaf(r.x, r.x, fmaf(r.y, r.y, ss));
        }
      }
    } else {
      ss = group_product<TG, T, UC>(U, ti, tj, Ab, Xb, Rb, nullptr, BM_RESID, false, frozen);
    }
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
    if (diag0) {
      if (!frozen) {
        for (int e = lt; e < uu; e += NTHR) {
          const int i = e / U, j = e % U;
          const float2 a = Ab[i * ld + i];
          const float den = a.x * a.x + a.y * a.y;
          const float2 xi = make_float2(cdamp * a.x / den, -cdamp * a.y / den);
          const float2 te = t_cur[i * ld + j];
          const float2 t = make_float2(te.x + (i == j ? 1.f : 0.f), te.y);
          Xb[i * ld + j] = make_float2(xi.x * t.x - xi.y * t.y, xi.x * t.y + xi.y * t.x);
        }
      }
    } else {
      group_product<TG, T, UC>(U, ti, tj, Xb, t_cur, Xb, Xb, BM_ADD, true, frozen);
    }
    __syncthreads();
  }
  if (active) {
    for (int e = lt; e < uu; e += NTHR) p.X[off + e] = Xb[(e / U) * ld + e % U];
    if (lt == 0) {
      p.residual[b] = s_last;
      p.status[b] = st;
    }
  }
  __syncthreads();
}

// ---- tensor-core path (plan configuration 2; U in {48, 64}) --------------------------------
//
// Two matrices per CTA, every iterate kept on chip:
//   * masters (X, R; T at depth >= 3) live in TMEM as the real form [Re; Im] of each U x U
//     complex matrix: adjacent lanes hold row i's real and imaginary parts, columns 0..U-1
//     (tc_lane_row gives the row of each lane); each of the two slots owns 256 columns (X, R,
//     a 2U-column accumulator);
//   * a complex product C = P Q is one real MMA chain
//         D (2U x 2U) = [Pr; Pi] (2U x U) . [Qr | Qi] (U x 2U)
//           = [[Pr Qr, Pr Qi], [Pi Qr, Pi Qi]],   Cr = Pr Qr - Pi Qi,  Ci = Pi Qr + Pr Qi,
//     i.e. M = 128 (2U rows used, in the lanes' order), N = 2U, K = U. The left operand's rows
//     are P's master lanes (K-major); the right operand is MN-major, its row k being master row
//     k of Q (real part at N < U, imaginary part at N >= U), so each lane stages its own values.
//     A's left operand is split once per matrix and kept in shared memory (one copy per slot);
//   * operands are split into three BF16 pieces (x = p0 + p1 + p2, each the BF16 rounding of the
//     remainder) and written in SWIZZLE_128B layouts; the six piece products with
//     i + j <= 2 (smallest first) accumulate in FP32 in TMEM, which matches an FP32 product to
//     about 2^-24 relative;
//   * epilogue: the real-part lane of a row needs Pi Qi and the imaginary-part lane Pr Qi, each
//     the other lane's own cross term, exchanged with one lane shuffle; then I - C or D + C is
//     applied in FP32 and written to the result master, and the residual's sum of squares is
//     reduced across the workers;
//   * the two slots alternate: 16 worker warps stage one slot's product and hand it to a 17th
//     warp that only issues its MMA chain; while the tensor core runs it, the workers finish
//     the other slot's previous product, then stage that slot's next product once the MMAs
//     (which read the single staging buffers) have completed;
//   * an 18th warp claims each slot's next matrix ahead of time (the item queue's atomic and the
//     plan's dependent reads) and pulls it toward L2, handing it over through a mailbox in
//     shared memory; the workers read a new matrix in coalesced row segments.
namespace btc {
constexpr int M = 128;                         // MMA rows (2U used)
constexpr int WARPS = 16;                      // warp (q, h): lane quadrant q, column block h (U / 4 columns)
constexpr int THREADS = 32 * WARPS;            // worker threads; one more warp issues the MMAs
constexpr int PIECE = 128 * 128;               // one piece: 128 rows x 64 BF16 (one SW128 k-block)
constexpr int OPND = 3 * PIECE;                // an operand's three pieces: 48 KB
constexpr int A_CACHE = 0;                     // the slots' left operands of A: 2 x 48 KB
constexpr int L_STAGE = 2 * OPND;              // staged left operand
constexpr int B_STAGE = 3 * OPND;              // staged right operand
constexpr int OPS_BYTES = 4 * OPND;
constexpr int BLOCK = THREADS + 64;            // workers, the MMA warp, the claimer warp
constexpr uint32_t SLOT_COLS = 256;            // TMEM columns per slot
constexpr uint32_t MX = 0, MR = 64, ACC = 128;
constexpr uint32_t MT = 256;                   // T master (depth >= 3: one slot only)
constexpr uint32_t TMEM_COLS = 512;
static_assert(OPS_BYTES + 1024 <= BT_SMEM, "operands fit the dynamic shared memory");
static_assert(PIECE % 1024 == 0, "swizzle atoms stay aligned");
}  // namespace btc

// Named barriers of the tensor-core kernel: the btc::THREADS worker threads synchronise among
// themselves on barrier 1; a staged product is handed to the MMA warp on barrier 2 (the workers
// arrive without waiting, the MMA warp waits), so the MMA warp, which stalls while the tensor
// core drains its queue, never holds the workers up.
__device__ __forceinline__ void tc_wsync() { asm volatile("bar.sync 1, %0;" ::"n"(btc::THREADS) : "memory"); }
__device__ __forceinline__ bool tc_wsync_and(bool v) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbar.red.and.pred po, 1, %2, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(out)
      : "r"(v ? 1u : 0u), "n"(btc::THREADS)
      : "memory");
  return out != 0;
}
__device__ __forceinline__ void tc_handoff_arrive() {
  asm volatile("bar.arrive 2, %0;" ::"n"(btc::THREADS + 32) : "memory");
}
__device__ __forceinline__ void tc_handoff_wait() { asm volatile("bar.sync 2, %0;" ::"n"(btc::THREADS + 32) : "memory"); }

// The master columns one worker warp owns: the four warps of a lane quadrant split the U
// columns evenly (CW = U / 4: 16 for U = 64, 12 for U = 48), so every worker warp carries data.
template <int U>
struct TcCols {
  static_assert(U == 48 || U == 64, "tensor-core sizes");
  static constexpr int CW = U / 4;
};

// TMEM access of a warp's 32 lanes x n consecutive columns, n = 4, 8, 12 or 16.
template <int n>
__device__ __forceinline__ void tmem_ld_n(uint32_t taddr, uint32_t (&r)[n]) {
  static_assert(n == 4 || n == 8 || n == 12 || n == 16, "widths");
  if constexpr (n == 16) {
    tmem_ld_32x32b_x16(taddr, r);
  } else {
    if constexpr (n >= 8)
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                   : "r"(taddr)
                   : "memory");
    if constexpr (n == 4 || n == 12)
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                   : "=r"(r[n - 4]), "=r"(r[n - 3]), "=r"(r[n - 2]), "=r"(r[n - 1])
                   : "r"(taddr + uint32_t(n - 4))
                   : "memory");
  }
}
template <int n>
__device__ __forceinline__ void tmem_st_n(uint32_t taddr, const uint32_t (&r)[n]) {
  static_assert(n == 4 || n == 8 || n == 12 || n == 16, "widths");
  if constexpr (n == 16) {
    tmem_st_32x32b_x16(taddr, r);
  } else {
    if constexpr (n >= 8)
      asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
                   "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                   : "memory");
    if constexpr (n == 4 || n == 12)
      asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr + uint32_t(n - 4)),
                   "r"(r[n - 4]), "r"(r[n - 3]), "r"(r[n - 2]), "r"(r[n - 1])
                   : "memory");
  }
}

// Shared-memory matrix descriptor of a K-major SWIZZLE_128B tile (8-row atoms 1024 B apart).
__device__ __forceinline__ uint64_t bt_sw128_desc(uint32_t saddr) {
  return uint64_t((saddr & 0x3FFFFu) >> 4) | (uint64_t(1) << 16) | (uint64_t(1024 >> 4) << 32) |
         (uint64_t(1) << 46) | (uint64_t(2) << 61);
}

// Byte offset of element (r, kk), kk < 64, in one k-block of a K-major SWIZZLE_128B operand:
// 16-byte chunk c of row r sits at chunk c ^ (r mod 8) of its 128-byte line.
__device__ __forceinline__ uint32_t bt_sw128_offset(int r, int kk) {
  return uint32_t((r >> 3) * 1024 + (r & 7) * 128 + (((kk >> 3) ^ (r & 7)) << 4) + ((kk & 7) << 1));
}

// The right operand B = [Qr | Qi] (K = U rows, N = 2U columns) is staged MN-major: B's row k is
// master row k of Q (its real part in columns 0..U-1, its imaginary part in U..2U-1), so each lane
// writes its own master values with no transposition. SWIZZLE_128B MN-major atoms hold 8 rows (K)
// x 64 elements (N); atoms along N sit BT_MN_LBO apart (the leading byte offset), along K
// BT_MN_SBO apart (the stride byte offset), so one piece (K <= 64, N <= 128) spans 16 KB. Were
// the two offsets read the other way round, every access would still stay inside the piece.
constexpr uint32_t BT_MN_LBO = 1024, BT_MN_SBO = 2048;
__device__ __forceinline__ uint64_t bt_sw128_mn_desc(uint32_t saddr) {
  return uint64_t((saddr & 0x3FFFFu) >> 4) | (uint64_t(BT_MN_LBO >> 4) << 16) | (uint64_t(BT_MN_SBO >> 4) << 32) |
         (uint64_t(1) << 46) | (uint64_t(2) << 61);
}
// Byte offset of element (k, n) of an MN-major SWIZZLE_128B operand: 16-byte chunk c of a row's
// 64-element span sits at chunk c ^ (k mod 8).
__device__ __forceinline__ uint32_t bt_mn_offset(int k, int n) {
  return uint32_t((k >> 3) * int(BT_MN_SBO) + (n >> 6) * int(BT_MN_LBO) + (k & 7) * 128 +
                  ((((n >> 3) & 7) ^ (k & 7)) << 4) + ((n & 7) << 1));
}

// Three BF16 pieces of the pair (a, b) (a in the low halves): each piece is the BF16 rounding
// of what the previous pieces leave (the remainders are exact in FP32).
__device__ __forceinline__ void split3x2(float a, float b, uint32_t& w0, uint32_t& w1, uint32_t& w2) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  w0 = *reinterpret_cast<uint32_t*>(&v);
  a -= __uint_as_float(w0 << 16);
  b -= __uint_as_float(w0 & 0xffff0000u);
  v = __floats2bfloat162_rn(a, b);
  w1 = *reinterpret_cast<uint32_t*>(&v);
  a -= __uint_as_float(w1 << 16);
  b -= __uint_as_float(w1 & 0xffff0000u);
  v = __floats2bfloat162_rn(a, b);
  w2 = *reinterpret_cast<uint32_t*>(&v);
}

// Row of the real form held by master lane l: row i's real part (im = false) in lane 2i, its
// imaginary part in lane 2i + 1, so that the two parts of a row sit in one warp and the epilogue
// combines the cross terms with a lane shuffle. Returns false for the padding lanes >= 2U.
template <int U>
__device__ __forceinline__ bool tc_lane_row(int l, int& i, bool& im) {
  static_assert(U == 48 || U == 64, "tensor-core sizes");
  im = (l & 1) != 0;
  i = l >> 1;
  return l < 2 * U;
}

// Splits G consecutive values v[0..G-1] (FP32 bits) into three BF16 pieces and stores piece pc
// at dst + pc PIECE + off (and, DUAL, at dst2 + pc PIECE + off2): one 16-byte store a piece for
// G = 8, one 8-byte store for G = 4.
template <int G, bool DUAL>
__device__ __forceinline__ void tc_put_group(const uint32_t (&v)[G], uint8_t* dst, uint32_t off, uint8_t* dst2,
                                             uint32_t off2) {
  static_assert(G == 4 || G == 8, "groups of 4 or 8 values");
  uint32_t w[3][G / 2];
#pragma unroll
  for (int e = 0; e < G / 2; ++e)
    split3x2(__uint_as_float(v[2 * e]), __uint_as_float(v[2 * e + 1]), w[0][e], w[1][e], w[2][e]);
#pragma unroll
  for (int pc = 0; pc < 3; ++pc) {
    if constexpr (G == 8) {
      const uint4 x = make_uint4(w[pc][0], w[pc][1], w[pc][2], w[pc][3]);
      *reinterpret_cast<uint4*>(dst + pc * btc::PIECE + off) = x;
      if constexpr (DUAL) *reinterpret_cast<uint4*>(dst2 + pc * btc::PIECE + off2) = x;
    } else {
      const uint2 x = make_uint2(w[pc][0], w[pc][1]);
      *reinterpret_cast<uint2*>(dst + pc * btc::PIECE + off) = x;
      if constexpr (DUAL) *reinterpret_cast<uint2*>(dst2 + pc * btc::PIECE + off2) = x;
    }
  }
}

// v = r[8 g .. 8 g + 7] for 16-column blocks (g a compile-time constant after unrolling).
__device__ __forceinline__ void tc_take8(const uint32_t (&r)[16], int g, uint32_t (&v)[8]) {
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    uint32_t x = r[e];
    x = g == 1 ? r[8 + e] : x;
    v[e] = x;
  }
}

// Calls f(width, first) for the store groups of this warp's CW master columns, as compile-time
// constants: 8-value groups (16-byte stores) at multiples of 8 and, for 12-column blocks, one
// 4-value group (8-byte stores) at the odd multiple of 4: h even (8 at 0, 4 at 8), h odd (4 at
// 0, 8 at 4). Fewer, wider stores than 4-value groups, and the 16-byte ones are free of bank
// conflicts (8-lane phases: eight rows of distinct swizzle phases, or a row's two part lanes).
template <int U, typename F>
__device__ __forceinline__ void tc_for_groups(int h, F&& f) {
  using I0 = std::integral_constant<int, 0>;
  using I4 = std::integral_constant<int, 4>;
  using I8 = std::integral_constant<int, 8>;
  static_assert(TcCols<U>::CW == 12, "16-column blocks use plain 8-value groups");
  {
    if (h & 1) {
      f(I4(), I0());
      f(I8(), I4());
    } else {
      f(I8(), I0());
      f(I4(), I8());
    }
  }
}

// N position of column j of Qi in the right operand, minus U: for U = 64 the 32-column halves
// are swapped (j ^ 32), which puts the real- and imaginary-part chunks that the two lanes of a
// row store at the same time into different swizzle phases (no bank conflicts); for U = 48 the
// imaginary-part lanes take their chunks in the other order instead.
template <int U>
__device__ __forceinline__ int tc_imag_col(int j) {
  return U == 64 ? (j ^ 32) : j;
}

// Stages one product: the right operand [Qr | Qi] (MN-major, see above) from master Q and, unless
// the product is the residual (whose left operand is A's cached pieces), the left operand
// [Pr; Pi] (K-major, operand row = master lane) from master P. Warp (q, h) owns lanes 32q.. and
// master columns h CW..: lane (i, part) holds row i of one part of each master, which is B's
// row i at N = h CW.. (real part) or U + tc_imag_col(h CW..) (imaginary part). When P and Q
// are the same master (the first Horner product, T_1 = R), each value is split once for both.
template <int U>
__device__ __forceinline__ void tc_stage(uint32_t tmem, bool left, uint32_t cP, uint32_t cQ, uint8_t* ldst,
                                         uint8_t* bdst, int q, int h, int l) {
  constexpr int CW = TcCols<U>::CW;
  const uint32_t lane_off = uint32_t(q * 32) << 16;
  const bool same = left && cP == cQ;
  int i;
  bool im;
  const bool valid = tc_lane_row<U>(l, i, im);
  uint32_t r[CW];
  // the right operand (and, for P = Q, the left one from the same pieces), then the left one
  tmem_ld_n<CW>(tmem + lane_off + cQ + uint32_t(h * CW), r);
  tmem_ld_wait();
  if constexpr (CW == 16) {
    if (valid) {
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const int j0 = h * CW + 8 * g;  // master columns j0 .. j0 + 7
        uint32_t v[8];
        tc_take8(r, g, v);
        const uint32_t boff = bt_mn_offset(i, im ? U + tc_imag_col<U>(j0) : j0);
        if (same)
          tc_put_group<8, true>(v, bdst, boff, ldst, bt_sw128_offset(l, j0));
        else
          tc_put_group<8, false>(v, bdst, boff, nullptr, 0);
      }
    }
  } else if (valid) {
    tc_for_groups<U>(h, [&](auto width, auto first) {
      constexpr int W = decltype(width)::value, S = decltype(first)::value;
      const int j0 = h * CW + S;  // master columns j0 .. j0 + W - 1
      uint32_t v[W];
#pragma unroll
      for (int e = 0; e < W; ++e) v[e] = r[S + e];
      const uint32_t boff = bt_mn_offset(i, im ? U + tc_imag_col<U>(j0) : j0);
      if (same)
        tc_put_group<W, true>(v, bdst, boff, ldst, bt_sw128_offset(l, j0));
      else
        tc_put_group<W, false>(v, bdst, boff, nullptr, 0);
    });
  }
  if (left && !same) {
    tmem_ld_n<CW>(tmem + lane_off + cP + uint32_t(h * CW), r);
    tmem_ld_wait();
    if constexpr (CW == 16) {
      if (valid) {
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          uint32_t v[8];
          tc_take8(r, g, v);
          tc_put_group<8, false>(v, ldst, bt_sw128_offset(l, h * CW + 8 * g), nullptr, 0);
        }
      }
    } else if (valid) {
      tc_for_groups<U>(h, [&](auto width, auto first) {
        constexpr int W = decltype(width)::value, S = decltype(first)::value;
        uint32_t v[W];
#pragma unroll
        for (int e = 0; e < W; ++e) v[e] = r[S + e];
        tc_put_group<W, false>(v, ldst, bt_sw128_offset(l, h * CW + S), nullptr, 0);
      });
    }
  }
}

// One thread: the MMA chain D = L B^T (K = U) into d_tmem, piece pairs (a, b) smallest terms
// first: (2,0) (1,1) (0,2) (1,0) (0,1) (0,0).
template <int U>
__device__ __forceinline__ void tc_issue(uint32_t d_tmem, uint32_t l_saddr, uint32_t b_saddr) {
  constexpr uint32_t idesc =
      (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t((2 * U) >> 3) << 17) | (uint32_t(btc::M >> 4) << 24);
  // bit 16: B is MN-major; a K = 16 step advances A by 32 bytes within its 128-byte lines and
  // B by two 8-row K-atoms
  constexpr uint32_t idesc_b = idesc | (1u << 16);
  constexpr uint64_t b_step = (2 * BT_MN_SBO) >> 4;
  const uint64_t ld = bt_sw128_desc(l_saddr);
  const uint64_t bd = bt_sw128_mn_desc(b_saddr);
#pragma unroll
  for (int pp = 0; pp < 6; ++pp) {
    const int pa = pp == 0 ? 2 : (pp == 1 || pp == 3) ? 1 : 0;
    const int pb = pp == 2 ? 2 : (pp == 1 || pp == 4) ? 1 : 0;
#pragma unroll
    for (int st = 0; st < U / 16; ++st)
      tc_mma_bf16(d_tmem, ld + uint64_t((pa * btc::PIECE) >> 4) + uint64_t(2 * st),
                  bd + uint64_t((pb * btc::PIECE) >> 4) + b_step * uint64_t(st), idesc_b, (pp | st) != 0 ? 1u : 0u);
  }
}

// Columns col .. col + W - 1 of the epilogue below (W = 8 or 4).
template <int U, int W>
__device__ __forceinline__ void tc_epilogue_part(uint32_t tmem, uint32_t lane_off, uint32_t cAcc, uint32_t cD,
                                                 uint32_t cOut, int mode, uint32_t col, int i, bool re, bool valid,
                                                 float& local) {
  // cross terms: the real-part lane needs Pi Qi (Cr = Pr Qr - Pi Qi) and the imaginary-part
  // lane Pr Qi (Ci = Pi Qr + Pr Qi): each is the other lane's own cross term (lanes l, l ^ 1)
  uint32_t dd[W], dx[W], dm[W];
  tmem_ld_n<W>(tmem + lane_off + cAcc + col, dd);
  tmem_ld_n<W>(tmem + lane_off + cAcc + uint32_t(U + tc_imag_col<U>(int(col))), dx);
  if (mode == BM_ADD) tmem_ld_n<W>(tmem + lane_off + cD + col, dm);
  tmem_ld_wait();
  const float sgn = re ? -1.f : 1.f;
#pragma unroll
  for (int t = 0; t < W; ++t) {
    const float x = __shfl_xor_sync(0xffffffffu, __uint_as_float(dx[t]), 1);
    const int j = int(col) + t;
    const float cv = fmaf(sgn, x, __uint_as_float(dd[t]));
    float v;
    if (mode == BM_RESID) {
      v = ((re && j == i) ? 1.f : 0.f) - cv;
      if (valid) local = fmaf(v, v, local);
    } else {
      v = __uint_as_float(dm[t]) + cv;
    }
    dd[t] = __float_as_uint(v);
  }
  tmem_st_n<W>(tmem + lane_off + cOut + col, dd);
}

// out = mode(C) from the accumulator D of a product (see above) on this warp's 32 x CW block
// of the real form; returns this thread's sum of squares of the result (residual mode, valid
// lanes only). Every lane of the warp calls it (shuffles); padding lanes (rows >= U) carry no
// data and feed only padding rows of later products (the residual sum skips them).
template <int U>
__device__ __forceinline__ float tc_epilogue(uint32_t tmem, uint32_t cAcc, uint32_t cD, uint32_t cOut, int mode,
                                             int q, int h, int l) {
  constexpr int CW = TcCols<U>::CW;
  int i;
  bool im;
  const bool valid = tc_lane_row<U>(l, i, im);
  const uint32_t lane_off = uint32_t(q * 32) << 16;
  float local = 0.f;
  const uint32_t col0 = uint32_t(h * CW);
#pragma unroll
  for (int ph = 0; ph < CW / 8; ++ph)
    tc_epilogue_part<U, 8>(tmem, lane_off, cAcc, cD, cOut, mode, col0 + uint32_t(8 * ph), i, !im, valid, local);
  if constexpr (CW % 8 != 0)
    tc_epilogue_part<U, CW % 8>(tmem, lane_off, cAcc, cD, cOut, mode, col0 + uint32_t(CW - CW % 8), i, !im, valid,
                                local);
  tmem_st_wait();
  return local;
}

// Sum over the worker threads; result broadcast to each of them.
__device__ __forceinline__ float bt_block_sum(float v, float* red_warp) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red_warp[threadIdx.x >> 5] = v;
  tc_wsync();
  float t = 0.f;
  for (int w = 0; w < btc::WARPS; ++w) t += red_warp[w];
  tc_wsync();
  return t;
}

// The claimer warp hands the workers their next item through a one-entry mailbox in shared
// memory: full = 1 once it has claimed an item (it, its matrix index b and offset off; b = -1
// for it >= last) and pulled the item's matrix toward L2; the workers set full = 0 once they have
// taken it. exit = 1 (set by the workers) ends the claimer.
struct TcMailbox {
  long long off;
  int full, it, b, exit;
};
__device__ __forceinline__ int ld_acquire_shared(const int* a) {
  int v;
  asm volatile("ld.acquire.cta.shared.b32 %0, [%1];" : "=r"(v) : "r"(smem_u32(a)) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_shared(int* a, int v) {
  asm volatile("st.release.cta.shared.b32 [%0], %1;" ::"r"(smem_u32(a)), "r"(v) : "memory");
}
// Bounded wait (one thread) for a full mailbox; false (a timeout recorded as by mbar_wait) if it
// stayed empty past the wait limit or another role gave up.
__device__ __forceinline__ bool tc_wait_full(TcMailbox* mb, int* abort_word, int* err) {
  if (ld_acquire_shared(&mb->full)) return true;
  const unsigned long long t0 = global_ns();
  uint32_t spins = 0;
  while (true) {
    if (ld_acquire_shared(&mb->full)) return true;
    if ((++spins & 15u) == 0) {
      if (*reinterpret_cast<volatile int*>(abort_word)) return false;
      if (global_ns() - t0 > kWaitLimitNs) {
        *reinterpret_cast<volatile int*>(abort_word) = 1;
        atomicExch(err, DEV_TIMEOUT);
        return false;
      }
    }
    __nanosleep(32);
  }
}

// The claimer warp: claims the next item of this class whenever the mailbox is empty and
// prefetches its matrix into L2 (one prefetch per 128-byte line, every address inside the
// matrix), so that the dependent reads of the plan and most of the matrix's global latency stay
// off the workers' path. Items it claims are always delivered (the workers take every full
// mailbox). Returns when the workers set exit, or (recording a timeout) when nothing empties the
// mailbox within the wait limit.
template <int U>
__device__ __forceinline__ void tc_claimer(const BatchedParams& p, int cls, int first, int last,
                                           const int32_t* items, TcMailbox* mb, int* abort_word) {
  const int lane = int(threadIdx.x & 31);
  while (true) {
    int state = 0;  // 0: empty (claim), 1: exit, 2: gave up
    if (lane == 0) {
      unsigned long long t0 = 0;
      uint32_t spins = 0;
      while (true) {
        if (*reinterpret_cast<volatile int*>(&mb->exit)) {
          state = 1;
          break;
        }
        if (ld_acquire_shared(&mb->full) == 0) break;
        if (spins++ == 0) t0 = global_ns();
        if ((spins & 15u) == 0) {
          if (*reinterpret_cast<volatile int*>(abort_word)) {
            state = 2;
            break;
          }
          if (global_ns() - t0 > kWaitLimitNs) {
            *reinterpret_cast<volatile int*>(abort_word) = 1;
            atomicExch(p.err, DEV_TIMEOUT);
            state = 2;
            break;
          }
        }
        __nanosleep(1024);
      }
    }
    state = __shfl_sync(0xffffffffu, state, 0);
    if (state == 1) return;
    if (state == 2) {
      // the workers learn of it through abort_word; wait (bounded) for their exit
      if (lane == 0) {
        const unsigned long long t0 = global_ns();
        while (!*reinterpret_cast<volatile int*>(&mb->exit) && global_ns() - t0 < kWaitLimitNs) __nanosleep(1024);
      }
      __syncwarp();
      return;
    }
    int it = 0, b = -1;
    long long off = 0;
    if (lane == 0) {
      it = first + atomicAdd(p.queue + cls, 1);
      if (it < last) {
        b = p.plan[PLAN_HDR + items[4 * it + 1]];
        off = p.offsets[b];
      }
    }
    it = __shfl_sync(0xffffffffu, it, 0);
    b = __shfl_sync(0xffffffffu, b, 0);
    off = __shfl_sync(0xffffffffu, off, 0);
    if (b >= 0) {
      constexpr int bytes = U * U * int(sizeof(float2));
      const char* base = reinterpret_cast<const char*>(p.A + off);
      for (int k = lane * 128; k <= bytes; k += 32 * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(base + (k < bytes ? k : bytes - 1)));
    }
    __syncwarp();
    if (lane == 0) {
      mb->it = it;
      mb->b = b;
      mb->off = off;
      st_release_shared(&mb->full, 1);
    }
    __syncwarp();
  }
}

// A new matrix into a slot, straight from global memory (the claimer pulled it toward L2) into
// registers: lane (i, part) reads its part of A[i][h CW .. h CW + CW - 1] (the row's two lanes
// together read whole complex values) and takes the other part from its partner lane where a
// complex product needs it. The real-part lane of row j in its diagonal block (warp h = j / CW)
// forms x0[j] = c / A[j][j] (damped Jacobi, c = 1 / (1 + damping U)) into x0s; after a worker
// barrier X_0 goes to the X master at column cX (padding lanes zero) and the pieces of A's left
// operand [Ar; Ai] to the slot's cache area (free: its previous matrix is done). Every worker
// thread calls it (shuffles).
// first_nest: X_0 is diagonal, so the first nest's residual R_0 = I - A X_0 is the column
// scaling R_0[i][j] = delta_ij - A[i][j] x0[j]; it is formed here in FP32 (R_0 into the R master
// at column cR; depth 1 (one_step): X_1 = X_0 (I + R_0), the row scaling x0[i] (delta_ij +
// R_0[i][j]), into the X master instead of X_0). Returns this thread's sum of squares of R_0
// (valid lanes and columns).
template <int U>
__device__ __forceinline__ float tc_load_matrix(const float2* A, float damping, uint8_t* acache, uint32_t tmem,
                                                uint32_t cX, uint32_t cR, float2* x0s, bool first_nest, bool one_step,
                                                int q, int h, int l) {
  constexpr int CW = TcCols<U>::CW, SP = CW + 1;
  int i;
  bool im;
  const bool valid_row = tc_lane_row<U>(l, i, im);
  const bool re = !im;
  // the warp's 16 x CW block of A (rows 16q.., columns h CW..) in coalesced row segments (a
  // half-warp reads one row's CW values), turned to the lanes' layout through a scratch block in
  // the slot's cache area (rows padded to CW + 1 complex values: no bank conflicts either way)
  float av[CW];
  {
    static_assert(btc::WARPS * 16 * SP * 8 <= btc::OPND, "scratch blocks fit the cache area");
    float2* sc = reinterpret_cast<float2*>(acache) + (threadIdx.x >> 5) * (16 * SP);
    const int lw = int(threadIdx.x & 31), c = lw & 15;
    float2 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int r = q * 16 + 2 * k + (lw >> 4);
      v[k] = (r < U && c < CW) ? __ldg(A + size_t(r) * U + h * CW + c) : make_float2(0.f, 0.f);
    }
    if (c < CW) {
#pragma unroll
      for (int k = 0; k < 8; ++k) sc[(2 * k + (lw >> 4)) * SP + c] = v[k];
    }
    __syncwarp();
    const float* own = reinterpret_cast<const float*>(sc + (lw >> 1) * SP) + (im ? 1 : 0);
#pragma unroll
    for (int t = 0; t < CW; ++t) av[t] = own[2 * t];
    if (valid_row && re && i / CW == h) {
      const float2 d = sc[(lw >> 1) * SP + (i - h * CW)];
      const float r = (1.f / (1.f + damping * float(U))) / (d.x * d.x + d.y * d.y);
      x0s[i] = make_float2(d.x * r, -d.y * r);
    }
  }
  // (after this barrier every warp has read its scratch block: the pieces may overwrite it)
  tc_wsync();
  // the diagonal lanes' division (and its slow path) can leave the warp diverged past the
  // barrier; every shuffle of the loops below would then run once per half of the warp
  __syncwarp();
  const uint32_t lane_off = uint32_t(q * 32) << 16;
  const float2 xi = valid_row ? x0s[i] : make_float2(0.f, 0.f);
  float local = 0.f;
  // the X master (X_0, or X_1 at depth 1 with the first nest element-wise) and R_0 to TMEM, in
  // parts of 8 and CW - 8 columns
  auto part = [&](auto width, int c0) {
    constexpr int W = decltype(width)::value;
    uint32_t vx[W], vr[W];
#pragma unroll
    for (int t = 0; t < W; ++t) {
      const int j = h * CW + c0 + t;
      const float mine = av[c0 + t];
      const float other = __shfl_xor_sync(0xffffffffu, mine, 1);
      float xv = 0.f, rv = 0.f;
      if (valid_row) {
        if (j == i) xv = re ? xi.x : xi.y;
        if (first_nest) {
          const float ar = re ? mine : other, ai = re ? other : mine;
          const float2 xj = x0s[j];
          const float d = (re && j == i) ? 1.f : 0.f;
          rv = re ? d - (ar * xj.x - ai * xj.y) : -(ar * xj.y + ai * xj.x);
          local = fmaf(rv, rv, local);
        }
      }
      vx[t] = __float_as_uint(xv);
      vr[t] = __float_as_uint(rv);
    }
    if (first_nest && one_step) {
      // X_1[i][j] = x0[i] (delta_ij + R_0[i][j]); the row's other part from the partner lane
#pragma unroll
      for (int t = 0; t < W; ++t) {
        const int j = h * CW + c0 + t;
        const float mine = __uint_as_float(vr[t]) + ((re && j == i) ? 1.f : 0.f);
        const float other = __shfl_xor_sync(0xffffffffu, mine, 1);
        const float pr = re ? mine : other, pi = re ? other : mine;
        const float xv = re ? xi.x * pr - xi.y * pi : xi.x * pi + xi.y * pr;
        vx[t] = __float_as_uint(valid_row ? xv : 0.f);
      }
    }
    const uint32_t col = uint32_t(h * CW + c0);
    tmem_st_n<W>(tmem + lane_off + cX + col, vx);
    if (first_nest) tmem_st_n<W>(tmem + lane_off + cR + col, vr);
  };
  part(std::integral_constant<int, 8>(), 0);
  part(std::integral_constant<int, CW - 8>(), 8);
  // the pieces of A's left operand
  if (valid_row) {
    uint32_t ab[CW];
#pragma unroll
    for (int t = 0; t < CW; ++t) ab[t] = __float_as_uint(av[t]);
    if constexpr (CW == 16) {
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        uint32_t v[8];
        tc_take8(ab, g, v);
        tc_put_group<8, false>(v, acache, bt_sw128_offset(l, h * CW + 8 * g), nullptr, 0);
      }
    } else {
      tc_for_groups<U>(h, [&](auto width, auto first) {
        constexpr int W = decltype(width)::value, S = decltype(first)::value;
        uint32_t v[W];
#pragma unroll
        for (int e = 0; e < W; ++e) v[e] = ab[S + e];
        tc_put_group<W, false>(v, acache, bt_sw128_offset(l, h * CW + S), nullptr, 0);
      });
    }
  }
  tmem_st_wait();
  return local;
}

// X_1 = X_0 (I + T) for a diagonal X_0 (the first nest's update): the row scaling
// x0[i] (delta_ij + T[i][j]) from the T master at column cT into the X master at column cX.
// Every lane of the warp calls it (shuffles).
template <int U>
__device__ __forceinline__ void tc_diag_update(uint32_t tmem, uint32_t cT, uint32_t cX, const float2* x0s, int q,
                                               int h, int l) {
  constexpr int CW = TcCols<U>::CW;
  int i;
  bool im;
  const bool valid = tc_lane_row<U>(l, i, im);
  const bool re = !im;
  const float2 xi = valid ? x0s[i] : make_float2(0.f, 0.f);
  const uint32_t lane_off = uint32_t(q * 32) << 16;
  uint32_t tv[CW];
  tmem_ld_n<CW>(tmem + lane_off + cT + uint32_t(h * CW), tv);
  tmem_ld_wait();
#pragma unroll
  for (int t = 0; t < CW; ++t) {
    const int j = h * CW + t;
    const float own = __uint_as_float(tv[t]) + ((re && j == i) ? 1.f : 0.f);
    const float other = __shfl_xor_sync(0xffffffffu, own, 1);
    const float pr = re ? own : other, pi = re ? other : own;
    const float xv = re ? xi.x * pr - xi.y * pi : xi.x * pi + xi.y * pr;
    tv[t] = __float_as_uint(valid ? xv : 0.f);
  }
  tmem_st_n<CW>(tmem + lane_off + cX + uint32_t(h * CW), tv);
  tmem_st_wait();
}

// X (complex, row-major) from the X master at column cX, through the slot's cache area (free:
// its matrix is done; rows padded to 2U + 1 floats) so that the global writes are coalesced.
// Every worker thread calls it.
template <int U>
__device__ __forceinline__ void tc_store_x(float2* X, uint32_t tmem, uint32_t cX, uint8_t* acache, int q, int h,
                                           int l) {
  constexpr int CW = TcCols<U>::CW, XP = 2 * U + 1;
  float* xs = reinterpret_cast<float*>(acache);
  {
    uint32_t vx[CW];
    tmem_ld_n<CW>(tmem + (uint32_t(q * 32) << 16) + cX + uint32_t(h * CW), vx);
    tmem_ld_wait();
    int i;
    bool im;
    if (tc_lane_row<U>(l, i, im)) {
      const bool re = !im;
#pragma unroll
      for (int t = 0; t < CW; ++t) xs[i * XP + 2 * (h * CW + t) + (re ? 0 : 1)] = __uint_as_float(vx[t]);
    }
  }
  tc_wsync();
  float* dst = reinterpret_cast<float*>(X);
#pragma unroll 4
  for (int k = 0; k < 2 * U * U / btc::THREADS; ++k) {
    const int e = threadIdx.x + k * btc::THREADS;
    dst[e] = xs[(e / (2 * U)) * XP + e % (2 * U)];
  }
  tc_wsync();
}

// Slot state (identical in every thread: all updates are CTA-uniform). The slot's last two
// residuals live in shared memory (slot_s[s] = (s_prev, s_last), written by thread 0 after a
// worker barrier), which keeps the loop's registers down.
struct TcSlot {
  int b;          // matrix index, -1 = empty
  int k, j;       // nest, product within the nest (0 = residual, 1..L-1 Horner, L = update)
  int diag;       // the first nest runs element-wise (R_0 formed at load, X_1 by row scaling)
};

// Masters of the product that a slot at state (k, j) runs next (the residual's left operand is
// A's cached pieces).
struct TcProd {
  uint32_t cP, cQ, cD, cOut;
  int mode;
};

__device__ __forceinline__ TcProd tc_product(const TcSlot& s, uint32_t sb, int depth) {
  TcProd r;
  if (s.j == 0) {
    r = {0u, sb + btc::MX, 0u, sb + btc::MR, BM_RESID};
  } else if (s.j < depth) {
    // Horner T_{j+1} = R + R T_j; at depth 2 it replaces R in place
    r = {sb + btc::MR, s.j == 1 ? sb + btc::MR : btc::MT, sb + btc::MR, depth == 2 ? sb + btc::MR : btc::MT, BM_ADD};
  } else {
    r = {sb + btc::MX, depth <= 2 ? sb + btc::MR : btc::MT, sb + btc::MX, sb + btc::MX, BM_ADD};
  }
  return r;
}

__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// Waits for the previous kernel of the chain to complete, so that each kernel's completion
// implies its predecessors' (stream order for whatever follows the last one).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// The tensor-core items of size U (classes 0 and 1): one CTA per SM, 512 TMEM columns, two
// slots at depth <= 2 (one at depth >= 3, whose T master takes the second slot's columns);
// btc::THREADS worker threads stage, finish and move matrices, one more warp issues the MMAs
// and another claims the next items.
struct TcCmd {
  uint32_t d_tmem, l_saddr, b_saddr;
  int exit;
};

// The worker threads of batched_tc_kernel: pull matrices, stage products, hand them to the MMA
// warp, finish them; see the tensor-core notes above.
template <int U>
__device__ __forceinline__ void batched_tc_work(const BatchedParams& p, int cls, int first, int last,
                                                const int32_t* items, uint8_t* ops, uint32_t ops_s, uint32_t tmem,
                                                uint64_t* mma_bar, int* abort_word, int* item_sh, float* red_warp,
                                                TcCmd* cmd, float2 (*x0s)[64], TcMailbox* mb, long long* slot_off,
                                                float2* slot_s) {
  const int w = int(threadIdx.x >> 5), q = w & 3, h = w >> 2, l = q * 32 + int(threadIdx.x & 31);
  const int nslots = p.depth <= 2 ? 2 : 1;
  TcSlot sl0 = {-1, 0, 0, 0}, sl1 = sl0;  // two named slots: no local memory
  // With at least one nest the first nest's residual and update are element-wise (X_0 is
  // diagonal); with none the residual of X_0 runs as a product.
  const bool first_nest = p.nests >= 1;
  uint32_t phase = 0;
  bool outstanding = false;
  bool ok = true;

  // the claimer's next item into slot s, or the slot left empty (no item left, or the wait for
  // the mailbox ran out: ok = false)
  auto fetch = [&](int s) {
    if (threadIdx.x == 0) {
      const bool got = tc_wait_full(mb, abort_word, p.err);
      item_sh[0] = got ? mb->it : -1;
      item_sh[1] = mb->b;
      if (got) {
        if (mb->b >= 0) slot_off[s] = mb->off;
        st_release_shared(&mb->full, 0);  // taken: the claimer claims the next one
      }
    }
    __syncwarp();
    tc_wsync();
    const int it = item_sh[0], b = item_sh[1];
    if (it < 0) ok = false;
    TcSlot t = {-1, 0, 0, 0};
    if (it >= 0 && b >= 0) {
      t.b = b;
      const uint32_t sb = uint32_t(s) * btc::SLOT_COLS;
      const float ss = tc_load_matrix<U>(p.A + slot_off[s], p.damping, ops + btc::A_CACHE + s * btc::OPND, tmem,
                                         sb + btc::MX, sb + btc::MR, x0s[s], first_nest, p.depth == 1, q, h, l);
      float s0 = 0.f;
      if (first_nest) {
        s0 = sqrtf(bt_block_sum(ss, red_warp)) / float(U);
        if (isfinite(s0)) {
          // nest 0's residual is done; next: its first Horner product, or (depth 1, X_1 already
          // formed) nest 1's residual
          t.diag = 1;
          if (p.depth == 1) {
            t.k = 1;
            t.j = 0;
          } else {
            t.j = 1;
          }
        }
        // a non-finite s_0 (a zero or non-finite diagonal): the residual runs as a product and
        // reports the matrix as diverged
        if (!isfinite(s0)) s0 = 0.f;
      }
      if (threadIdx.x == 0) slot_s[s] = make_float2(s0, s0);  // read after later barriers only
    }
    if (s == 0)
      sl0 = t;
    else
      sl1 = t;
    tc_fence_before();
    tc_wsync();
    tc_fence_after();
  };
  // every thread learns the same outcome of the wait on the last issued MMA chain
  auto wait_mma = [&]() -> bool {
    if (!outstanding) return true;
    // (the lanes leave the polling loop at different times: reconverge before the TMEM loads)
    const bool got = mbar_wait(mma_bar, phase, abort_word, p.err);
    __syncwarp();
    const bool r = tc_wsync_and(got);
    phase ^= 1u;
    outstanding = false;
    tc_fence_after();
    return r;
  };
  // stage slot s's next product, then one thread issues its MMA chain
  auto stage = [&](int s) {
    const uint32_t sb = uint32_t(s) * btc::SLOT_COLS;
    const TcProd pr = tc_product(s == 0 ? sl0 : sl1, sb, p.depth);
    tc_stage<U>(tmem, pr.mode != BM_RESID, pr.cP, pr.cQ, ops + btc::L_STAGE, ops + btc::B_STAGE, q, h, l);
    fence_proxy_async_smem();
    tc_fence_before();
    if (threadIdx.x == 0) {
      cmd->d_tmem = tmem + sb + btc::ACC;
      cmd->l_saddr = pr.mode == BM_RESID ? ops_s + uint32_t(btc::A_CACHE + s * btc::OPND) : ops_s + uint32_t(btc::L_STAGE);
      cmd->b_saddr = ops_s + uint32_t(btc::B_STAGE);
      cmd->exit = 0;
    }
    tc_handoff_arrive();
    outstanding = true;
  };
  // finish slot s's product (its MMAs complete): epilogue, residual test, next state; a
  // finished matrix is written out and the slot refilled
  auto finish = [&](int s) {
    const uint32_t sb = uint32_t(s) * btc::SLOT_COLS;
    TcSlot t = s == 0 ? sl0 : sl1;
    const TcProd pr = tc_product(t, sb, p.depth);
    const float ss = tc_epilogue<U>(tmem, sb + btc::ACC, pr.cD, pr.cOut, pr.mode, q, h, l);
    // the first nest's update X_1 = X_0 (I + T) is a row scaling: right after its last Horner
    // product (each thread reads back what it wrote)
    const bool diag_update = t.diag && t.k == 0 && t.j + 1 == p.depth;
    if (diag_update) tc_diag_update<U>(tmem, pr.cOut, sb + btc::MX, x0s[s], q, h, l);
    tc_fence_before();
    bool done = false, diverged = false;
    if (pr.mode == BM_RESID) {
      const float sv = sqrtf(bt_block_sum(ss, red_warp)) / float(U);
      if (!isfinite(sv) || (t.k >= 1 && sv >= 1.f && sv > slot_s[s].x)) diverged = done = true;
      if (t.k == p.nests) done = true;
      tc_wsync();  // every thread has read s_prev
      tc_fence_after();
      if (threadIdx.x == 0) slot_s[s] = make_float2(sv, sv);
    }
    // (other products need no worker barrier here: each warp reads back only the TMEM columns
    // and lanes it wrote itself, and the next MMA into this slot's accumulator is ordered after
    // every warp's epilogue by the next wait and hand-over)
    if (!done) {
      if (diag_update || ++t.j > p.depth) {
        t.j = 0;
        ++t.k;
      }
      if (s == 0)
        sl0 = t;
      else
        sl1 = t;
      return;
    }
    tc_store_x<U>(p.X + slot_off[s], tmem, sb + btc::MX, ops + btc::A_CACHE + s * btc::OPND, q, h, l);
    if (threadIdx.x == 0) {
      p.residual[t.b] = slot_s[s].y;
      p.status[t.b] = diverged ? NN_ERR_DIVERGED : NN_OK;
    }
    fetch(s);
  };

  for (int s = 0; s < nslots; ++s) fetch(s);
  int pending = -1;  // slot whose product's MMAs are issued and whose epilogue is not done
  while (ok) {
    int m = -1;
    if (pending >= 0)
      m = (nslots == 2 && (pending == 0 ? sl1 : sl0).b >= 0) ? 1 - pending : pending;
    else if (sl0.b >= 0)
      m = 0;
    else if (nslots == 2 && sl1.b >= 0)
      m = 1;
    if (m < 0) break;
    ok = wait_mma();  // staging buffers free, the pending product's accumulator final
    if (!ok) break;
    if (m == pending) {
      // one slot in flight: its product completes before the next is staged
      finish(m);
      pending = -1;
      continue;
    }
    stage(m);
    if (pending >= 0) finish(pending);
    pending = m;
  }
  if (ok) ok = wait_mma();
  // release the MMA warp (after a timeout too; its last chain, if any, was issued) and the
  // claimer
  if (threadIdx.x == 0) {
    cmd->exit = 1;
    *reinterpret_cast<volatile int*>(&mb->exit) = 1;
  }
  tc_handoff_arrive();
  if (!ok) {
    // a bounded wait ran out: the slots' matrices and every item not yet taken report
    // NN_ERR_TIMEOUT (X unspecified; an item left in the mailbox is reported once the claimer
    // has returned); wait (bounded) for the issued MMAs before freeing TMEM
    if (threadIdx.x == 0) {
      if (sl0.b >= 0) {
        p.residual[sl0.b] = slot_s[0].y;
        p.status[sl0.b] = NN_ERR_TIMEOUT;
      }
      if (nslots == 2 && sl1.b >= 0) {
        p.residual[sl1.b] = slot_s[1].y;
        p.status[sl1.b] = NN_ERR_TIMEOUT;
      }
    }
    while (true) {
      if (threadIdx.x == 0) item_sh[0] = first + atomicAdd(p.queue + cls, 1);
      tc_wsync();
      const int it = item_sh[0];
      tc_wsync();
      if (it >= last) break;
      if (threadIdx.x == 0) {
        const int b = p.plan[PLAN_HDR + items[4 * it + 1]];
        p.residual[b] = 0.f;
        p.status[b] = NN_ERR_TIMEOUT;
      }
    }
    if (outstanding) {
      volatile int drain_flag = 0;
      mbar_wait(mma_bar, phase, &drain_flag, p.err);
    }
  }
}

// 18 warps (16 workers, the MMA warp, the claimer warp): at most 96 registers a thread (five
// warps share one scheduler's quarter of the register file)
template <int U>
__global__ void __launch_bounds__(btc::BLOCK, 1) batched_tc_kernel(const BatchedParams p, int cls) {
  extern __shared__ float2 smem[];
  __shared__ float red_warp[btc::WARPS];
  __shared__ int item_sh[2];
  __shared__ long long slot_off[2];  // per slot: the matrix's offset in A and X
  __shared__ float2 slot_s[2];       // per slot: (s_prev, s_last)
  __shared__ TcMailbox mb;
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_word;
  __shared__ TcCmd cmd;
  __shared__ float2 x0s[2][64];  // per slot: the diagonal of X_0
  pdl_launch_dependents();
  const int count = p.plan[1];
  const int first = p.plan[3 + cls], last = p.plan[3 + cls + 1];
  const int32_t* items = p.plan + PLAN_HDR + count;
  if (first < last) {
    uint8_t* ops = reinterpret_cast<uint8_t*>(smem);
    ops += (1024u - (smem_u32(ops) & 1023u)) & 1023u;
    const uint32_t ops_s = smem_u32(ops);
    if (threadIdx.x == 0) {
      mbar_init(&mma_bar, 1);
      abort_word = 0;
      mb.full = 0;
      mb.exit = 0;
      mbar_fence_init();
    }
    if (threadIdx.x < 32) tmem_alloc(&tmem_slot, btc::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    if (threadIdx.x >= btc::THREADS + 32) {
      tc_claimer<U>(p, cls, first, last, items, &mb, &abort_word);
    } else if (threadIdx.x >= btc::THREADS) {
      // the MMA warp: one chain per handed-over product until the workers send exit (test hook:
      // the first chain's completion is never signalled, so the workers' bounded wait runs out)
      bool first_chain = true;
      while (true) {
        tc_handoff_wait();
        const TcCmd c = cmd;
        if (c.exit) break;
        if (threadIdx.x == btc::THREADS) {
          tc_fence_after();
          tc_issue<U>(c.d_tmem, c.l_saddr, c.b_saddr);
          if (!(p.withhold && first_chain)) tc_commit(&mma_bar);
        }
        first_chain = false;
        __syncwarp();
      }
    } else {
      batched_tc_work<U>(p, cls, first, last, items, ops, ops_s, tmem, &mma_bar, &abort_word, item_sh, red_warp,
                         &cmd, x0s, &mb, slot_off, slot_s);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // an item the claimer delivered after a timeout ended the workers
    if (threadIdx.x == 0 && mb.full && mb.b >= 0) {
      p.residual[mb.b] = 0.f;
      p.status[mb.b] = NN_ERR_TIMEOUT;
    }
    if (threadIdx.x < 32) tmem_dealloc(tmem, btc::TMEM_COLS);
  }
  pdl_wait();
}

// ---- warp-per-matrix CUDA-core path (plan configuration 3; U in {8, 16, 24, 32}) ----------
//
// One warp runs one matrix's whole loop; its products need only warp synchronisation, so the
// warps of an SM never wait for each other. Thread (ti, tj) of the 8 x 4 warp grid owns rows
// ti + 8a (a < U/8) and columns tj + 4b (b < U/4) of every product. Matrices live in shared
// memory with rows padded to U + 1 complex (the eight rows a k step reads fall in different
// banks); three buffers per matrix (A, X, R), four at depth >= 3 (T).
namespace bw {
template <int U>
struct Shape {
  static constexpr int TR = U / 8, TC = U / 4, PITCH = U + 1;
  static constexpr int MAT = U * PITCH;  // float2 per buffer
};
// warps per CTA for (U, buffers): shared memory up to about 200 KB, at most 32 warps
__host__ __device__ constexpr int warps_per_cta(int U, int bufs) {
  return (200 * 1024) / (bufs * U * (U + 1) * 8) < 32 ? (200 * 1024) / (bufs * U * (U + 1) * 8) : 32;
}
}  // namespace bw

// acc = P Q for this thread's tile (all U k steps).
template <int U>
__device__ __forceinline__ void warp_acc(const float2* P, const float2* Q, int ti, int tj,
                                         float2 (&acc)[bw::Shape<U>::TR][bw::Shape<U>::TC]) {
  using S = bw::Shape<U>;
#pragma unroll
  for (int a = 0; a < S::TR; ++a)
#pragma unroll
    for (int b = 0; b < S::TC; ++b) acc[a][b] = make_float2(0.f, 0.f);
#pragma unroll 4
  for (int k = 0; k < U; ++k) {
    float2 pa[S::TR], qb[S::TC];
#pragma unroll
    for (int a = 0; a < S::TR; ++a) pa[a] = P[(ti + 8 * a) * S::PITCH + k];
#pragma unroll
    for (int b = 0; b < S::TC; ++b) qb[b] = Q[k * S::PITCH + tj + 4 * b];
#pragma unroll
    for (int a = 0; a < S::TR; ++a)
#pragma unroll
      for (int b = 0; b < S::TC; ++b) {
        acc[a][b].x = fmaf(pa[a].x, qb[b].x, acc[a][b].x);
        acc[a][b].x = fmaf(-pa[a].y, qb[b].y, acc[a][b].x);
        acc[a][b].y = fmaf(pa[a].x, qb[b].y, acc[a][b].y);
        acc[a][b].y = fmaf(pa[a].y, qb[b].x, acc[a][b].y);
      }
  }
}

// out = I - P Q (mode RESID, returns this thread's sum of |out|^2) or D + P Q (mode ADD); out
// may alias P, Q or D (the warp synchronises between the product and the stores).
template <int U>
__device__ __forceinline__ float warp_product(const float2* P, const float2* Q, const float2* D, float2* out,
                                              int mode, int ti, int tj) {
  using S = bw::Shape<U>;
  float2 acc[S::TR][S::TC];
  warp_acc<U>(P, Q, ti, tj, acc);
  __syncwarp();
  float ss = 0.f;
#pragma unroll
  for (int a = 0; a < S::TR; ++a)
#pragma unroll
    for (int b = 0; b < S::TC; ++b) {
      const int i = ti + 8 * a, j = tj + 4 * b;
      float2 v;
      if (mode == BM_RESID) {
        v = make_float2((i == j ? 1.f : 0.f) - acc[a][b].x, -acc[a][b].y);
        ss = fmaf(v.x, v.x, fmaf(v.y, v.y, ss));
      } else {
        const float2 d = D[i * S::PITCH + j];
        v = make_float2(d.x + acc[a][b].x, d.y + acc[a][b].y);
      }
      out[i * S::PITCH + j] = v;
    }
  __syncwarp();
  return ss;
}

// One matrix, the whole NN loop, by one warp (lane = threadIdx.x % 32).
template <int U>
__device__ void warp_item(const BatchedParams& p, int b, float2* buf, int lane) {
  using S = bw::Shape<U>;
  const int ti = lane >> 2, tj = lane & 3;
  float2* Ab = buf;
  float2* Xb = buf + S::MAT;
  float2* Rb = buf + 2 * S::MAT;
  float2* Tb = p.depth >= 3 ? buf + 3 * S::MAT : Rb;
  const int64_t off = p.offsets[b];
  for (int e = lane; e < U * U; e += 32) Ab[(e / U) * S::PITCH + e % U] = p.A[off + e];
  __syncwarp();
  const float c = 1.f / (1.f + p.damping * float(U));
  for (int e = lane; e < U * U; e += 32) {
    const int i = e / U, j = e % U;
    float2 v = make_float2(0.f, 0.f);
    if (i == j) {
      const float2 a = Ab[i * S::PITCH + i];
      const float den = a.x * a.x + a.y * a.y;
      v = make_float2(c * a.x / den, -c * a.y / den);
    }
    Xb[i * S::PITCH + j] = v;
  }
  __syncwarp();
  float s_prev = 0.f, s_last = 0.f;
  int st = NN_OK;
  // the first nest element-wise (X_0 diagonal): R_0 = I - A X_0, X_1 = X_0 (I + T), x0
  // recomputed from A's diagonal exactly as above
  for (int k = 0; k <= p.nests; ++k) {
    const bool diag0 = k == 0;
    float ss = 0.f;
    if (diag0) {
      for (int e = lane; e < U * U; e += 32) {
        const int i = e / U, j = e % U;
        const float2 a = Ab[i * S::PITCH + j];
        const float2 xj = Xb[j * S::PITCH + j];
        const float2 r = make_float2((i == j ? 1.f : 0.f) - (a.x * xj.x - a.y * xj.y), -(a.x * xj.y + a.y * xj.x));
        Rb[i * S::PITCH + j] = r;
        ss = fmaf(r.x, r.x, fmaf(r.y, r.y, ss));
      }
      __syncwarp();
    } else {
      ss = warp_product<U>(Ab, Xb, nullptr, Rb, BM_RESID, ti, tj);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const float s = sqrtf(ss) / float(U);
    s_last = s;
    if (!isfinite(s) || (k >= 1 && s >= 1.f && s > s_prev)) {
      st = NN_ERR_DIVERGED;
      break;
    }
    s_prev = s;
    if (k == p.nests) break;
    // Horner: T_1 = R, T_{j+1} = R + R T_j (depth 2: in place of R); X_{k+1} = X_k + X_k T
    const float2* t_cur = Rb;
    for (int j = 1; j < p.depth; ++j) {
      warp_product<U>(Rb, t_cur, Rb, Tb, BM_ADD, ti, tj);
      t_cur = Tb;
    }
    if (diag0) {
      for (int e = lane; e < U * U; e += 32) {
        const int i = e / U, j = e % U;
        const float2 a = Ab[i * S::PITCH + i];
        const float den = a.x * a.x + a.y * a.y;
        const float2 xi = make_float2(c * a.x / den, -c * a.y / den);
        const float2 tv = t_cur[i * S::PITCH + j];
        const float2 t = make_float2(tv.x + (i == j ? 1.f : 0.f), tv.y);
        Xb[i * S::PITCH + j] = make_float2(xi.x * t.x - xi.y * t.y, xi.x * t.y + xi.y * t.x);
      }
      __syncwarp();
    } else {
      warp_product<U>(Xb, t_cur, Xb, Xb, BM_ADD, ti, tj);
    }
  }
  for (int e = lane; e < U * U; e += 32) p.X[off + e] = Xb[(e / U) * S::PITCH + e % U];
  if (lane == 0) {
    p.residual[b] = s_last;
    p.status[b] = st;
  }
  __syncwarp();
}

// The configuration-3 items of size U (classes 18..21): each warp pulls single matrices.
template <int U>
__global__ void __launch_bounds__(32 * bw::warps_per_cta(U, 3)) batched_warp_kernel(const BatchedParams p, int cls) {
  extern __shared__ float2 smem[];
  pdl_launch_dependents();
  const int count = p.plan[1];
  const int first = p.plan[3 + cls], last = p.plan[3 + cls + 1];
  const int32_t* items = p.plan + PLAN_HDR + count;
  const int lane = int(threadIdx.x & 31), w = int(threadIdx.x >> 5);
  float2* buf = smem + size_t(w) * (p.depth >= 3 ? 4 : 3) * bw::Shape<U>::MAT;
  while (first < last) {
    int it = 0;
    if (lane == 0) it = first + atomicAdd(p.queue + cls, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= last) break;
    warp_item<U>(p, p.plan[PLAN_HDR + items[4 * it + 1]], buf, lane);
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
const SimtKernel kSimtKernels[16] = {
    batched_simt_kernel<16, 4, 64>, batched_simt_kernel<16, 4, 0>, batched_simt_kernel<16, 3, 48>,
    batched_simt_kernel<16, 3, 0>,  batched_simt_kernel<16, 2, 32>, batched_simt_kernel<16, 2, 0>,
    batched_simt_kernel<16, 1, 16>, batched_simt_kernel<16, 1, 0>,  batched_simt_kernel<8, 4, 32>,
    batched_simt_kernel<8, 4, 0>,   batched_simt_kernel<8, 3, 24>,  batched_simt_kernel<8, 3, 0>,
    batched_simt_kernel<8, 2, 16>,  batched_simt_kernel<8, 2, 0>,   batched_simt_kernel<8, 1, 8>,
    batched_simt_kernel<8, 1, 0>};

// Dynamic shared memory of a warp-per-matrix CTA (U, buffers per matrix).
int warp_smem(int U, int bufs) { return bw::warps_per_cta(U, bufs) * bufs * U * (U + 1) * int(sizeof(float2)); }

int g_bt_sms = 0;
bool g_bt_init = false;

int bt_init() {
  if (g_bt_init) return NN_OK;
  int dev = 0;
  NN_CUDA_TRY(cudaGetDevice(&dev));
  NN_CUDA_TRY(cudaDeviceGetAttribute(&g_bt_sms, cudaDevAttrMultiProcessorCount, dev));
  NN_CUDA_TRY(cudaFuncSetAttribute(batched_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, BT_SMEM));
  NN_CUDA_TRY(cudaFuncSetAttribute(batched_tc_kernel<48>, cudaFuncAttributeMaxDynamicSharedMemorySize, BT_SMEM));
  for (auto k : {batched_tc_kernel<64>, batched_tc_kernel<48>}) {
    cudaFuncAttributes fa;
    NN_CUDA_TRY(cudaFuncGetAttributes(&fa, k));
    if (fa.maxThreadsPerBlock < btc::BLOCK) return NN_ERR_UNSUPPORTED;  // registers do not fit
  }
  for (SimtKernel k : kSimtKernels)
    NN_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, BT_SMEM_SIMT_DEEP));
  const SimtKernel warp_kernels[4] = {batched_warp_kernel<32>, batched_warp_kernel<24>, batched_warp_kernel<16>,
                                      batched_warp_kernel<8>};
  for (int c = 0; c < 4; ++c) {
    const int U = 32 - 8 * c;
    NN_CUDA_TRY(cudaFuncSetAttribute(warp_kernels[c], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     std::max(warp_smem(U, 3), warp_smem(U, 4))));
  }
  g_bt_init = true;
  return NN_OK;
}

// Matrices per work item for (U, cfg): thread groups available and shared memory.
int group_count(int U, int cfg) {
  if (cfg >= 2) return 1;
  const int by_threads = cfg == 0 ? BT_THREADS / 64 : 1;
  const int per = bt_buffers(2) * U * bt_simt_pitch(U, cfg == 0 ? 8 : 16) * int(sizeof(float2));
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
    if (cfg < 0 || cfg > 3) return NN_ERR_ARG;
    if (cfg == 2 && U != 48 && U != 64) cfg = U <= 32 ? 0 : 1;
    if (cfg == 3 && (U % 8 != 0 || U > 32)) cfg = U <= 32 ? 0 : 1;
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
  plan_host[2] = class_first[2];
  return NN_OK;
}

size_t nn_batched_workspace_bytes(int64_t count) {
  if (count < 1) return 0;
  return 256;
}

uint32_t nn_batched_plan_classes(const int32_t* plan_host) {
  if (plan_host == nullptr) return 0;
  uint32_t mask = 0;
  for (int c = 0; c < BT_NCLS; ++c)
    if (plan_host[3 + c + 1] > plan_host[3 + c]) mask |= 1u << c;
  return mask;
}

int nn_invert_batched_c64(const void* A, const int64_t* offsets, const int32_t* sizes, int64_t count,
                          const int32_t* plan, uint32_t classes, int depth, int nests, double damping, void* X,
                          float* residual, int32_t* status, void* workspace, size_t ws_bytes, void* stream) {
  if (A == nullptr || offsets == nullptr || sizes == nullptr || plan == nullptr || X == nullptr ||
      residual == nullptr || status == nullptr || count < 1)
    return NN_ERR_ARG;
  classes &= (1u << BT_NCLS) - 1u;
  if (classes == 0) return NN_ERR_ARG;
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
  p.withhold = 0;
  NN_CUDA_TRY(cudaMemsetAsync(p.queue, 0, nn_batched_workspace_bytes(count), st));
  // the classes' kernels in class order; each after the first may start as the previous
  // one's CTAs retire (programmatic dependent launch)
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 0;
  const int bufs = depth >= 3 ? 4 : 3;
  const SimtKernel warp_kernels[4] = {batched_warp_kernel<32>, batched_warp_kernel<24>, batched_warp_kernel<16>,
                                      batched_warp_kernel<8>};
  for (int c = 0; c < BT_NCLS; ++c) {
    if (((classes >> c) & 1u) == 0) continue;
    SimtKernel k;
    if (c < 2) {
      k = c == 0 ? batched_tc_kernel<64> : batched_tc_kernel<48>;
      cfg.gridDim = dim3(unsigned(g_bt_sms));
      cfg.blockDim = dim3(btc::BLOCK);
      cfg.dynamicSmemBytes = size_t(BT_SMEM);
    } else if (c < 18) {
      k = kSimtKernels[c - 2];
      cfg.gridDim = dim3(unsigned(depth <= 2 ? 2 * g_bt_sms : g_bt_sms));
      cfg.blockDim = dim3(BT_THREADS);
      cfg.dynamicSmemBytes = size_t(depth <= 2 ? BT_SMEM_SIMT : BT_SMEM_SIMT_DEEP);
    } else {
      const int U = 8 * (4 - (c - 18));
      k = warp_kernels[c - 18];
      cfg.gridDim = dim3(unsigned(g_bt_sms));
      cfg.blockDim = dim3(unsigned(32 * bw::warps_per_cta(U, bufs)));
      cfg.dynamicSmemBytes = size_t(warp_smem(U, bufs));
    }
    BatchedParams pc = p;
    if (c < 2) pc.withhold = tc_take_withhold();  // the test hook goes to the first tensor-core class
    NN_CUDA_TRY(cudaLaunchKernelEx(&cfg, k, pc, c));
    cfg.numAttrs = 1;
  }
  return NN_OK;
}

int nn_invert_batched(const void* A, const int64_t* offsets, const int32_t* sizes, int64_t count, int depth, int nests,
                      double damping, const int32_t* plan, uint32_t classes, void* X, float* residual,
                      int32_t* status, void* workspace, size_t ws_bytes, void* stream) {
  return nn_invert_batched_c64(A, offsets, sizes, count, plan, classes, depth, nests, damping, X, residual, status,
                               workspace, ws_bytes, stream);
}

}  // extern "C"
