// Sparse NN chain: the explicit product form applied to right-hand sides through a CSR
// matrix (Corollary 1, Eq. (NNexplicit); Corollary 6; Algorithm 2), with the Jacobi start
// phi^(0) = D^-1:
//     X = D^-1 prod_{j=0}^{k-1} ( sum_{n=0}^{L} P^{n (L+1)^j} ) B,     P = I - A D^-1.
// D^-1 is folded into the stored values once (A' = A D^-1, so P v = v - A' v), and the chain
// runs as (L+1)^k - 1 sparse products. Each product streams a contiguous slice of (val, col)
// into shared memory with coalesced streaming loads (one block = 256 consecutive rows), then
// each thread reduces its own row; the vector gathers hit L2 through plain cached loads (the
// read-only path is the texture pipeline, which takes four requests per cycle).
//
// Arithmetic policies: native FP64, native FP32, and double-float ("DF": a value is an
// unevaluated sum hi + lo of two FP32 numbers, 49-bit significand) for FP64 data. GB300's FP64
// pipe is narrow (predicated-off FP64 FMAs alone saturated it in an earlier four-right-hand-side
// form of this kernel, hence the compile-time right-hand-side count R below); the DF policy keeps
// the same 8 bytes per value and does its arithmetic with error-free transformations on the
// FP32 pipes (two-sum after Knuth, two-product with FMA after Dekker, the double-float
// additions and products of the QD library of Hida, Li and Bailey), for FP64 data on parts
// with even less FP64 throughput.
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

// ---- arithmetic policies ----------------------------------------------------------------

struct ArithF64 {
  using V = double;
  using In = double;
  static constexpr bool kBranchTail = true;
  __device__ static V zero() { return 0.0; }
  __device__ static V nmad(V a, V x, V acc) { return fma(-a, x, acc); }
  __device__ static V add(V a, V b) { return a + b; }
  __device__ static double to_d(V a) { return a; }
  __device__ static V from_d(double a) { return a; }
};

struct ArithF32 {
  using V = float;
  using In = float;
  static constexpr bool kBranchTail = false;
  __device__ static V zero() { return 0.f; }
  __device__ static V nmad(V a, V x, V acc) { return fmaf(-a, x, acc); }
  __device__ static V add(V a, V b) { return a + b; }
  __device__ static double to_d(V a) { return double(a); }
  __device__ static V from_d(double a) { return float(a); }
};

// Double-float: (hi, lo) with |lo| <= ulp(hi)/2. The _rn intrinsics keep the compiler from
// contracting the error-free sequences into FMAs.
struct ArithDF {
  using V = float2;
  using In = double;
  static constexpr bool kBranchTail = false;
  __device__ static void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  }
  __device__ static void quick_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
  }
  __device__ static V zero() { return make_float2(0.f, 0.f); }
  // a + b, accurate variant (two two-sums, two renormalisations)
  __device__ static V add(V a, V b) {
    float s1, s2, t1, t2;
    two_sum(a.x, b.x, s1, s2);
    two_sum(a.y, b.y, t1, t2);
    s2 = __fadd_rn(s2, t1);
    quick_two_sum(s1, s2, s1, s2);
    s2 = __fadd_rn(s2, t2);
    quick_two_sum(s1, s2, s1, s2);
    return make_float2(s1, s2);
  }
  // a * x: exact high product from FMA, cross terms into the low part
  __device__ static V mul(V a, V x) {
    const float p = __fmul_rn(a.x, x.x);
    float e = fmaf(a.x, x.x, -p);
    e = fmaf(a.x, x.y, e);
    e = fmaf(a.y, x.x, e);
    float s, t;
    quick_two_sum(p, e, s, t);
    return make_float2(s, t);
  }
  __device__ static V nmad(V a, V x, V acc) { return add(acc, mul(make_float2(-a.x, -a.y), x)); }
  __device__ static double to_d(V a) { return double(a.x) + double(a.y); }
  __device__ static V from_d(double a) {
    const float hi = float(a);
    return make_float2(hi, float(a - double(hi)));
  }
};

// R = right-hand sides handled per launch (compile-time, so nrhs = 1 stays lean in registers).
template <class P, int R>
__global__ void __launch_bounds__(SP_ROWS, R == 1 ? 5 : 1)
spmv_p_kernel(int n, const int* __restrict__ row_ptr, const int* __restrict__ col, const typename P::V* val,
              const typename P::V* v, int64_t ldv, typename P::V* y, int64_t ldy, const typename P::V* acc_in,
              typename P::V* acc_out, int64_t ld_acc, const typename P::In* b, int64_t ldb, int nrhs, int mode,
              double* __restrict__ partial) {
  using V = typename P::V;
  __shared__ V sval[SP_CHUNK];
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
  // sum = v_row - sum_e a_e x_e for the products (one rounding chain started at v_row, so
  // y = v - A'v needs no separate subtraction), sum = -sum_e a_e x_e for the residual
  V sum[R];
#pragma unroll
  for (int r = 0; r < R; ++r)
    sum[r] = (mode != SP_RESID && row < n && r < nrhs) ? __ldca(v + row + r * ldv) : P::zero();

  constexpr int PER = SP_CHUNK / SP_ROWS;
  for (int base = e_begin; base < e_end; base += SP_CHUNK) {
    const int cnt = min(SP_CHUNK, e_end - base);
    // Issue every load of the slice before any shared-memory store, so each thread has PER
    // independent requests in flight; the matrix streams through (evict-first) and leaves
    // L2 to the vector, which the gathers below reuse across rows.
    V vv[PER];
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
      const V a0 = sval[e - base], a1 = sval[e + 1 - base], a2 = sval[e + 2 - base], a3 = sval[e + 3 - base];
      const int c0 = scol[e - base], c1 = scol[e + 1 - base], c2 = scol[e + 2 - base], c3 = scol[e + 3 - base];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (r < nrhs) {
          const V* vr = v + r * ldv;
          const V x0 = __ldca(vr + c0), x1 = __ldca(vr + c1), x2 = __ldca(vr + c2), x3 = __ldca(vr + c3);
          sum[r] = P::nmad(a0, x0, sum[r]);
          sum[r] = P::nmad(a1, x1, sum[r]);
          sum[r] = P::nmad(a2, x2, sum[r]);
          sum[r] = P::nmad(a3, x3, sum[r]);
        }
      }
    }
    for (; e < hi; ++e) {
      const V a = sval[e - base];
      const int c = scol[e - base];
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (r < nrhs) sum[r] = P::nmad(a, __ldca(v + c + r * ldv), sum[r]);
    }
    __syncthreads();
  }

  double ss_r = 0.0, ss_b = 0.0;
  if (row < n) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r >= nrhs) break;
      if (mode == SP_RESID) {
        const double bi = double(b[row + r * ldb]);
        const double ri = bi + P::to_d(sum[r]);
        ss_r = fma(ri, ri, ss_r);
        ss_b = fma(bi, bi, ss_b);
      } else {
        const V yi = sum[r];
        if (mode != SP_ACC) y[row + r * ldy] = yi;
        if (mode != SP_Y) acc_out[row + r * ld_acc] = P::add(acc_in[row + r * ld_acc], yi);
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

// ---- one right-hand side: persistent kernel with a bulk-copy ring ----------------------
//
// Each block runs one producer warp and ST_ROWS consumer threads (one per row of a 256-row
// tile). The producer walks the block's tiles (blockIdx.x, + gridDim.x, ...) and, for each
// chunk of at most ST_CAP nonzeros of a tile, issues cp.async.bulk copies of (val, col) and,
// for a tile's first chunk, of row_ptr[r0 .. r0 + 260) into the next free stage of a
// ST_STAGES ring; completion is counted on the stage's full barrier. Consumers reduce their
// row over the staged chunk (vector gathers from L2) and release the stage on its empty
// barrier. The matrix stream therefore stays in flight while the gathers of earlier tiles
// wait on L2, which a load-then-compute block cannot do. The chunk grid starts at the tile's
// first nonzero rounded down to a multiple of 4 (16-byte source alignment for every element
// type); the last elements of the arrays past the last multiple of 4 are read directly.
// Each row's terms are summed in increasing column-slot order, as in spmv_p_kernel, so both
// kernels give identical results.
// sum - a_0 x_0 - ... - a_{K-1} x_{K-1}, in that order
template <class P, int K>
__device__ __forceinline__ typename P::V nmad_chain(const typename P::V (&a)[7], const typename P::V (&x)[7],
                                                    typename P::V sum) {
#pragma unroll
  for (int k = 0; k < K; ++k) sum = P::nmad(a[k], x[k], sum);
  return sum;
}

constexpr int ST_ROWS = 256;
constexpr int ST_THREADS = ST_ROWS + 32;
constexpr int ST_STAGES = 3;
constexpr int ST_CAP = 1288;             // nonzeros per stage, multiple of 4 (a 5-point tile + alignment)
constexpr int ST_ROWBUF = ST_ROWS + 4;   // row_ptr entries staged per tile, multiple of 4

struct StageHdr {
  int base;      // first staged element (multiple of 4)
  int end;       // one past the last nonzero of this chunk
  int copy_end;  // one past the last staged element (elements in [copy_end, end) are read from global)
  int rows;      // row_ptr entries staged (first chunk of a tile), else 0
  int last;      // last chunk of the tile
  int pad[3];
};

template <class P>
struct StLayout {
  using V = typename P::V;
  static constexpr int kVal = ST_CAP * int(sizeof(V));
  static constexpr int kCol = ST_CAP * 4;
  static constexpr int kRow = ST_ROWBUF * 4;
  static constexpr int kStage = kVal + kCol + kRow;
  // control block: full/empty barriers, 4 reduction barriers, stage headers, abort flag,
  // then 4 x 16 doubles of residual reduction scratch at the end
  static constexpr int kRed = 4 * 16 * 8;
  static constexpr int kCtrl = 1024;
  static constexpr int kBytes = ST_STAGES * kStage + kCtrl;
  static_assert(kVal % 16 == 0 && kCol % 16 == 0 && kRow % 16 == 0, "16-byte stage pieces");
  static_assert((2 * ST_STAGES + 4) * 8 + ST_STAGES * int(sizeof(StageHdr)) + 16 + kRed <= kCtrl, "control block");
};

template <class P>
__global__ void __launch_bounds__(ST_THREADS, 4)
spmv_ring_kernel(int n, int nnz, const int* __restrict__ row_ptr, const int* __restrict__ col,
                 const typename P::V* __restrict__ val, const typename P::V* v, typename P::V* y,
                 const typename P::V* acc_in, typename P::V* acc_out, const typename P::In* b, int mode,
                 double* __restrict__ partial, int* err, int withhold) {
  using V = typename P::V;
  using L = StLayout<P>;
  extern __shared__ __align__(128) uint8_t st_smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(st_smem + ST_STAGES * L::kStage);
  uint64_t* empty = full + ST_STAGES;
  uint64_t* red_bar = empty + ST_STAGES;
  StageHdr* hdr = reinterpret_cast<StageHdr*>(red_bar + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(hdr + ST_STAGES);
  double* red = reinterpret_cast<double*>(st_smem + ST_STAGES * L::kStage + L::kCtrl - L::kRed);

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int tiles = (n + ST_ROWS - 1) / ST_ROWS;
  // Programmatic dependent launch: the next product may be scheduled as soon as every block of
  // this one is resident; its producer then streams the matrix (which no product writes) while
  // this product finishes, and its consumers wait for this grid to complete before reading the
  // vectors.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (tid == 0) {
    for (int s = 0; s < ST_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], ST_ROWS / 32);
    }
    for (int s = 0; s < 4; ++s) mbar_init(&red_bar[s], ST_ROWS / 32);
    *abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();

  if (warp == ST_ROWS / 32) {
    // ---- producer warp ----
    const uint64_t pol = l2_evict_first_policy();
    const int nnz4 = nnz & ~3;
    const int rows4 = (n + 1) & ~3;
    int stage = 0;
    uint32_t phase = 0;
    bool stop = false;
    // failure-detection test hook: block 0 never fills its first stage, so its consumers'
    // bounded wait on it runs out (the later stages' copies land long before)
    bool skip_first = withhold != 0 && blockIdx.x == 0;
    for (int t0 = blockIdx.x; t0 < tiles && !stop; t0 += 32 * int(gridDim.x)) {
      // lane j fetches the nonzero range of the block's j-th next tile
      const int tj = t0 + lane * int(gridDim.x);
      int eb = 0, ee = 0;
      if (tj < tiles) {
        eb = row_ptr[tj * ST_ROWS];
        ee = row_ptr[min((tj + 1) * ST_ROWS, n)];
      }
      for (int j = 0; j < 32; ++j) {
        const int t = t0 + j * int(gridDim.x);
        if (t >= tiles) break;
        const int e0 = __shfl_sync(0xffffffffu, eb, j);
        const int e1 = __shfl_sync(0xffffffffu, ee, j);
        const int r0 = t * ST_ROWS;
        int base = e0 & ~3;
        bool first = true;
        while (true) {
          const int end = min(base + ST_CAP, e1);
          if (lane == 0 && skip_first) {
            skip_first = false;
          } else if (lane == 0) {
            if (mbar_wait(&empty[stage], phase ^ 1u, abort_flag, err)) {
              const int copy_end = max(base, min((end + 3) & ~3, nnz4));
              const int rows = first ? max(0, min(ST_ROWBUF, rows4 - r0)) : 0;
              StageHdr& h = hdr[stage];
              h.base = base;
              h.end = end;
              h.copy_end = copy_end;
              h.rows = rows;
              h.last = end >= e1 ? 1 : 0;
              uint8_t* sp = st_smem + stage * L::kStage;
              const uint32_t cnt = uint32_t(copy_end - base);
              mbar_arrive_expect_tx(&full[stage], cnt * uint32_t(sizeof(V) + 4) + uint32_t(rows) * 4u);
              if (cnt > 0) {
                bulk_load(sp, val + base, cnt * uint32_t(sizeof(V)), &full[stage], pol);
                bulk_load(sp + L::kVal, col + base, cnt * 4u, &full[stage], pol);
              }
              if (rows > 0) bulk_load(sp + L::kVal + L::kCol, row_ptr + r0, uint32_t(rows) * 4u, &full[stage], pol);
            }
          }
          __syncwarp();
          if (*abort_flag) {
            stop = true;
            break;
          }
          if (++stage == ST_STAGES) {
            stage = 0;
            phase ^= 1u;
          }
          first = false;
          base += ST_CAP;
          if (end >= e1) break;
        }
        if (stop) break;
      }
    }
    // Leave only after the consumers have released every stage, so no copy is in flight.
    if (lane == 0 && !stop) {
      for (int i = 0; i < ST_STAGES; ++i) {
        if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, err)) break;
        if (++stage == ST_STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    return;
  }

  // ---- consumers: thread tid owns row r0 + tid of every tile ----
  // every vector read and write comes after the previous grid in the stream has completed
  asm volatile("griddepcontrol.wait;" ::: "memory");
  int stage = 0;
  uint32_t phase = 0;
  int local = 0;
  for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++local) {
    const int row = t * ST_ROWS + tid;
    const bool has_row = row < n;
    // row-wise operands, fetched before the matrix arrives
    V v_row = P::zero(), a_row = P::zero();
    double b_row = 0.0;
    if (has_row) {
      if (mode == SP_RESID) {
        b_row = double(b[row]);
      } else {
        v_row = __ldca(v + row);
        if (mode != SP_Y) a_row = acc_in[row];
      }
    }
    V sum = mode == SP_RESID ? P::zero() : v_row;  // same rounding chain as spmv_p_kernel
    int my_b = 0, my_e = 0;
    bool first = true;
    while (true) {
      if (!mbar_wait(&full[stage], phase, abort_flag, err)) return;
      const StageHdr h = hdr[stage];
      const uint8_t* sp = st_smem + stage * L::kStage;
      const V* sval = reinterpret_cast<const V*>(sp);
      const int* scol = reinterpret_cast<const int*>(sp + L::kVal);
      const int* srow = reinterpret_cast<const int*>(sp + L::kVal + L::kCol);
      if (first && has_row) {
        my_b = tid < h.rows ? srow[tid] : row_ptr[row];
        my_e = tid + 1 < h.rows ? srow[tid + 1] : row_ptr[row + 1];
      }
      const int lo = max(my_b, h.base), hi = min(my_e, h.end);
      const int hs = min(hi, h.copy_end);
      int e = lo;
      // Eight gathers in flight: a row of up to eight terms costs one L2 round trip. For FP64
      // the multiply-adds of the last partial group run in a branch per count, so no
      // predicated-off FMA takes a slot of the narrow FP64 pipe.
      for (; e + 8 <= hs; e += 8) {
        const int q = e - h.base;
        V a[8], x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = sval[q + k];
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = __ldca(v + scol[q + k]);
#pragma unroll
        for (int k = 0; k < 8; ++k) sum = P::nmad(a[k], x[k], sum);
      }
      const int rem = hs - e;
      if (rem > 0) {
        const int q = e - h.base;
        V a[7], x[7];
#pragma unroll
        for (int k = 0; k < 7; ++k) {
          a[k] = P::zero();
          x[k] = P::zero();
          if (k < rem) {
            a[k] = sval[q + k];
            x[k] = __ldca(v + scol[q + k]);
          }
        }
        if (P::kBranchTail) {
          switch (rem) {
            case 1: sum = nmad_chain<P, 1>(a, x, sum); break;
            case 2: sum = nmad_chain<P, 2>(a, x, sum); break;
            case 3: sum = nmad_chain<P, 3>(a, x, sum); break;
            case 4: sum = nmad_chain<P, 4>(a, x, sum); break;
            case 5: sum = nmad_chain<P, 5>(a, x, sum); break;
            case 6: sum = nmad_chain<P, 6>(a, x, sum); break;
            default: sum = nmad_chain<P, 7>(a, x, sum); break;
          }
        } else {
#pragma unroll
          for (int k = 0; k < 7; ++k)
            if (k < rem) sum = P::nmad(a[k], x[k], sum);
        }
        e = hs;
      }
      for (; e < hi; ++e) sum = P::nmad(val[e], __ldca(v + col[e]), sum);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[stage]);
      if (++stage == ST_STAGES) {
        stage = 0;
        phase ^= 1u;
      }
      first = false;
      if (h.last) break;
    }
    if (mode == SP_RESID) {
      double ss_r = 0.0, ss_b = 0.0;
      if (has_row) {
        const double ri = b_row + P::to_d(sum);
        ss_r = ri * ri;
        ss_b = b_row * b_row;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ss_r += __shfl_down_sync(0xffffffffu, ss_r, o);
        ss_b += __shfl_down_sync(0xffffffffu, ss_b, o);
      }
      // Per-tile sums over the 8 warps through scratch slot local % 4 and its mbarrier (no
      // CTA-wide barrier: a warp can be at most ST_STAGES tiles ahead of warp 0, because the
      // stages it needs are only refilled after warp 0 has released them).
      const int slot = local & 3;
      double* rs = red + 16 * slot;
      if (lane == 0) {
        rs[warp] = ss_r;
        rs[8 + warp] = ss_b;
        mbar_arrive(&red_bar[slot]);
      }
      if (tid == 0) {
        if (!mbar_wait(&red_bar[slot], uint32_t(local >> 2) & 1u, abort_flag, err)) return;
        double a = 0, c = 0;
        for (int w = 0; w < ST_ROWS / 32; ++w) {
          a += rs[w];
          c += rs[8 + w];
        }
        partial[2 * t] = a;
        partial[2 * t + 1] = c;
      }
    } else if (has_row) {
      const V yi = sum;
      if (mode != SP_ACC) y[row] = yi;
      if (mode != SP_Y) acc_out[row] = P::add(a_row, yi);
    }
  }
}

// dinv[i] = 1 / A_ii (in the input precision); flags a missing or zero diagonal in *err.
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

// A' = A D^-1 (column scaling), formed in the input precision and stored in the policy's type.
template <class P>
__global__ void scale_cols_kernel(int64_t nnz, const int* __restrict__ col, const typename P::In* __restrict__ val,
                                  const typename P::In* __restrict__ dinv, typename P::V* __restrict__ out) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e < nnz) out[e] = P::from_d(double(val[e] * dinv[col[e]]));
}

// dst (policy type, n x nrhs, leading dim n) = src (input type, lds)
template <class P>
__global__ void load_cols_kernel(int n, int nrhs, const typename P::In* __restrict__ src, int64_t lds,
                                 typename P::V* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (i >= n || r >= nrhs) return;
  dst[i + int64_t(r) * n] = P::from_d(double(src[i + r * lds]));
}

// X (input type, ldx) = D^-1 z
template <class P>
__global__ void store_cols_kernel(int n, int nrhs, const typename P::V* __restrict__ z,
                                  const typename P::In* __restrict__ dinv, typename P::In* __restrict__ X,
                                  int64_t ldx) {
  using In = typename P::In;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (i >= n || r >= nrhs) return;
  X[i + r * ldx] = In(P::to_d(z[i + int64_t(r) * n])) * dinv[i];
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

template <class P>
void carve_csr(Carver& c, int64_t n, int64_t nnz, int64_t nrhs, CsrWs& w) {
  using V = typename P::V;
  using In = typename P::In;
  const size_t vec = size_t(n) * size_t(nrhs);
  w.dinv = c.take<In>(size_t(n));
  w.vals = c.take<V>(size_t(nnz));
  w.z[0] = c.take<V>(vec);
  w.z[1] = c.take<V>(vec);
  w.u[0] = c.take<V>(vec);
  w.u[1] = c.take<V>(vec);
  const int64_t slices = (nrhs + SP_MAXR - 1) / SP_MAXR;
  w.partial = c.take<double>(size_t(2 * slices * ((n + SP_ROWS - 1) / SP_ROWS)));
  w.scal = c.take<double>(8);
  w.err = c.take<int>(8);
}

int g_spmv_variant = 0;  // 0 automatic (bulk-copy ring for one right-hand side), 1 staged loads only

// Grid of the ring kernel: every SM filled with as many blocks as fit (cached per policy).
template <class P>
struct RingOccupancy {
  int sms = 0, per_sm = 0;
  RingOccupancy() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(spmv_ring_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, StLayout<P>::kBytes) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spmv_ring_kernel<P>, ST_THREADS, StLayout<P>::kBytes) !=
            cudaSuccess) {
      (void)cudaGetLastError();
      per_sm = 0;
    }
  }
};

template <class P>
int ring_grid(int tiles) {
  static const RingOccupancy<P> occ;  // thread-safe one-time initialisation
  if (occ.per_sm <= 0) return 0;
  const int g = occ.sms * occ.per_sm;
  return tiles < g ? tiles : g;
}

template <class P>
int spmv(cudaStream_t st, int n, int nnz, const int* rp, const int* col, const typename P::V* vals,
         const typename P::V* v, typename P::V* y, const typename P::V* acc_in, typename P::V* acc_out,
         const typename P::In* b, int64_t ldb, int nrhs, int mode, double* partial, int* err) {
  const int blocks = (n + SP_ROWS - 1) / SP_ROWS;
  // the ring copies (val, col, row_ptr) with 16-byte aligned bulk copies
  const bool aligned = ((reinterpret_cast<uintptr_t>(rp) | reinterpret_cast<uintptr_t>(col) |
                         reinterpret_cast<uintptr_t>(vals)) & 15u) == 0;
  for (int r0 = 0; r0 < nrhs; r0 += SP_MAXR) {
    const int nr = nrhs - r0 < SP_MAXR ? nrhs - r0 : SP_MAXR;
    const int64_t off = int64_t(r0) * n;
    // residual partials of slice r0/SP_MAXR follow those of the previous slices
    double* part = partial ? partial + int64_t(2) * blocks * (r0 / SP_MAXR) : nullptr;
    const int grid = (nr == 1 && aligned && g_spmv_variant != 1) ? ring_grid<P>(blocks) : 0;
    if (grid > 0) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(unsigned(grid));
      cfg.blockDim = dim3(ST_THREADS);
      cfg.dynamicSmemBytes = size_t(StLayout<P>::kBytes);
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      NN_CUDA_TRY(cudaLaunchKernelEx(&cfg, spmv_ring_kernel<P>, n, nnz, rp, col, vals, v + off,
                                     y ? y + off : nullptr, acc_in ? acc_in + off : nullptr,
                                     acc_out ? acc_out + off : nullptr, b ? b + int64_t(r0) * ldb : nullptr, mode,
                                     part, err, tc_take_withhold()));
    } else if (nr == 1) {
      spmv_p_kernel<P, 1><<<blocks, SP_ROWS, 0, st>>>(n, rp, col, vals, v + off, n, y ? y + off : nullptr, n,
                                                      acc_in ? acc_in + off : nullptr, acc_out ? acc_out + off : nullptr,
                                                      n, b ? b + int64_t(r0) * ldb : nullptr, ldb, nr, mode, part);
    } else {
      spmv_p_kernel<P, SP_MAXR><<<blocks, SP_ROWS, 0, st>>>(
          n, rp, col, vals, v + off, n, y ? y + off : nullptr, n, acc_in ? acc_in + off : nullptr,
          acc_out ? acc_out + off : nullptr, n, b ? b + int64_t(r0) * ldb : nullptr, ldb, nr, mode, part);
    }
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

template <class P>
int solve_csr(const int* rp, const int* col, const typename P::In* val, int64_t n64, int64_t nnz,
              const typename P::In* B, int64_t ldb, int64_t nrhs64, const int* depths, int nests, double tol,
              typename P::In* X, int64_t ldx, nn_result* res, void* ws, size_t ws_bytes, cudaStream_t st) {
  using V = typename P::V;
  using In = typename P::In;
  const int n = int(n64), nrhs = int(nrhs64);
  Carver c(ws, ws_bytes);
  CsrWs w;
  carve_csr<P>(c, n64, nnz, nrhs64, w);
  if (!c.ok) return NN_ERR_OOM_BUDGET;
  In* dinv = static_cast<In*>(w.dinv);
  V* vals = static_cast<V*>(w.vals);
  V* z = static_cast<V*>(w.z[0]);
  V* znew = static_cast<V*>(w.z[1]);
  V* u[2] = {static_cast<V*>(w.u[0]), static_cast<V*>(w.u[1])};
  const int blocks = (n + SP_ROWS - 1) / SP_ROWS;

  NN_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  diag_inv_kernel<In><<<(n + 255) / 256, 256, 0, st>>>(n, rp, col, val, dinv, w.err);
  NN_CUDA_TRY(cudaGetLastError());
  scale_cols_kernel<P><<<unsigned((nnz + 255) / 256), 256, 0, st>>>(nnz, col, val, dinv, vals);
  NN_CUDA_TRY(cudaGetLastError());
  load_cols_kernel<P><<<dim3((n + 255) / 256, nrhs), 256, 0, st>>>(n, nrhs, B, ldb, z);
  NN_CUDA_TRY(cudaGetLastError());
  res->launches += 3;
  int dev_err = 0;
  NN_CUDA_TRY(cudaMemcpyAsync(&dev_err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  NN_CUDA_TRY(cudaStreamSynchronize(st));
  if (dev_err != DEV_OK) return NN_ERR_ARG;

  auto residual = [&](const V* zz, double* out) -> int {
    // r = B - A X = B - A' z (since A X = A D^-1 z); relative Frobenius norm.
    NN_TRY(spmv<P>(st, n, int(nnz), rp, col, vals, zz, nullptr, nullptr, nullptr, B, ldb, nrhs, SP_RESID, w.partial,
                   w.err));
    const int slices = (nrhs + SP_MAXR - 1) / SP_MAXR;
    reduce_pair_kernel<<<1, 256, 0, st>>>(w.partial, blocks * slices, w.scal);
    NN_CUDA_TRY(cudaGetLastError());
    res->launches += 1 + slices;
    res->flops += 2.0 * double(nnz) * nrhs;
    int e = DEV_OK;
    NN_CUDA_TRY(cudaMemcpyAsync(out, w.scal, sizeof(double), cudaMemcpyDeviceToHost, st));
    NN_CUDA_TRY(cudaMemcpyAsync(&e, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    NN_CUDA_TRY(cudaStreamSynchronize(st));
    return e == DEV_OK ? NN_OK : NN_ERR_TIMEOUT;  // the ring kernel's bounded waits
  };

  int applied = 0;
  res->status = NN_OK;
  long long t = 1;  // m_j = prod_{q<j} (L_q + 1): the power of P one block of factor j applies
  for (int j = 0; j < nests; ++j) {
    const int depth = depths[j];
    if (j > 0) t *= (depths[j - 1] + 1);
    const V* src = z;
    int ping = 0;
    for (int blk = 1; blk <= depth; ++blk) {
      for (long long s = 1; s <= t; ++s) {
        const bool last_of_block = (s == t);
        const bool last_of_factor = last_of_block && (blk == depth);
        V* dst = u[ping];
        int mode = SP_Y;
        const V* acc_in = nullptr;
        V* acc_out = nullptr;
        if (last_of_block) {
          mode = last_of_factor ? SP_ACC : SP_Y_ACC;
          acc_in = (blk == 1) ? z : znew;
          acc_out = znew;
        }
        NN_TRY(spmv<P>(st, n, int(nnz), rp, col, vals, src, mode == SP_ACC ? nullptr : dst, acc_in, acc_out, nullptr, 0,
                       nrhs, mode, nullptr, w.err));
        res->launches += (nrhs + SP_MAXR - 1) / SP_MAXR;
        res->flops += 2.0 * double(nnz) * nrhs;
        src = dst;
        ping ^= 1;
      }
    }
    // znew = z + sum of the L blocks: swap
    V* tmp = z;
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
  store_cols_kernel<P><<<dim3((n + 255) / 256, nrhs), 256, 0, st>>>(n, nrhs, z, dinv, X, ldx);
  NN_CUDA_TRY(cudaGetLastError());
  res->launches += 1;
  int e = DEV_OK;
  NN_CUDA_TRY(cudaMemcpyAsync(&e, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  NN_CUDA_TRY(cudaStreamSynchronize(st));
  if (e != DEV_OK) res->status = NN_ERR_TIMEOUT;
  return res->status;
}

// Both sums of the residual partials (sum r^2, sum b^2), for an all-reduce across row strips.
__global__ void reduce_pair_sums_kernel(const double* __restrict__ partial, int count, double* out) {
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
  if (threadIdx.x == 0) {
    out[0] = a[0];
    out[1] = c[0];
  }
}

// Workspace of the row-strip entry points: residual partials, two sums, the error word.
struct StripWs {
  double* partial;
  double* sums;
  int* err;
};
void carve_strip(Carver& c, int64_t n_local, StripWs& w) {
  w.partial = c.take<double>(size_t(2 * ((n_local + SP_ROWS - 1) / SP_ROWS)));
  w.sums = c.take<double>(2);
  w.err = c.take<int>(8);
}

bool strip_args_ok(const int32_t* row_ptr, const int32_t* col, const void* val, int64_t n_local, int64_t nnz,
                   int dtype) {
  return row_ptr != nullptr && col != nullptr && val != nullptr && n_local >= 1 && n_local <= (int64_t(1) << 30) &&
         nnz >= 0 && nnz <= (int64_t(1) << 31) - 1 && (dtype == NN_F64 || dtype == NN_F32);
}

size_t csr_ws_bytes(int64_t n, int64_t nnz, int64_t nrhs, int dtype) {
  Carver c(nullptr, 0);
  CsrWs w;
  if (dtype == NN_F64)
    carve_csr<ArithF64>(c, n, nnz, nrhs, w);
  else if (dtype == NN_F32)
    carve_csr<ArithF32>(c, n, nnz, nrhs, w);
  else
    carve_csr<ArithDF>(c, n, nnz, nrhs, w);
  return align_up(c.used, 256);
}

}  // namespace
}  // namespace nn

using namespace nn;

extern "C" {

int nn_set_spmv_variant(int variant) {
  if (variant < 0 || variant > 1) return NN_ERR_ARG;
  g_spmv_variant = variant;
  return NN_OK;
}

size_t nn_csr_workspace_bytes(int64_t n, int64_t nnz, int64_t nrhs, int dtype) {
  if (n < 1 || nnz < n || nrhs < 1 || n > (int64_t(1) << 30) || nnz > (int64_t(1) << 31) - 1) return 0;
  if (dtype != NN_F64 && dtype != NN_F32 && dtype != NN_F64_DF) return 0;
  return csr_ws_bytes(n, nnz, nrhs, dtype);
}

static int solve_csr_any(const int32_t* row_ptr, const int32_t* col, const void* val, int64_t n, int64_t nnz,
                         int dtype, const void* B, int64_t ldb, int64_t nrhs, const int* depths, int nests,
                         double tol, void* X, int64_t ldx, nn_result* res, void* workspace, size_t ws_bytes,
                         void* stream) {
  if (res == nullptr) return NN_ERR_ARG;
  memset(res, 0, sizeof(*res));
  res->status = NN_ERR_ARG;
  if (row_ptr == nullptr || col == nullptr || val == nullptr || B == nullptr || X == nullptr) return NN_ERR_ARG;
  if (nests < 0 || nests > NN_MAX_HISTORY - 1 || ldb < n || ldx < n || isnan(tol)) return NN_ERR_ARG;
  if (nests > 0 && depths == nullptr) return NN_ERR_ARG;
  // prod (L_j + 1) - 1 sparse products must stay countable
  double total = 1.0;
  for (int j = 0; j < nests; ++j) {
    if (depths[j] < 1 || depths[j] > 16) return NN_ERR_ARG;
    total *= double(depths[j] + 1);
  }
  if (total > 2147483647.0) return NN_ERR_ARG;
  const size_t need = nn_csr_workspace_bytes(n, nnz, nrhs, dtype);
  if (need == 0) return NN_ERR_ARG;
  if (workspace == nullptr || ws_bytes < need) {
    res->status = NN_ERR_OOM_BUDGET;
    return NN_ERR_OOM_BUDGET;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int s;
  if (dtype == NN_F64)
    s = solve_csr<ArithF64>(row_ptr, col, static_cast<const double*>(val), n, nnz, static_cast<const double*>(B), ldb,
                            nrhs, depths, nests, tol, static_cast<double*>(X), ldx, res, workspace, ws_bytes, st);
  else if (dtype == NN_F64_DF)
    s = solve_csr<ArithDF>(row_ptr, col, static_cast<const double*>(val), n, nnz, static_cast<const double*>(B), ldb,
                           nrhs, depths, nests, tol, static_cast<double*>(X), ldx, res, workspace, ws_bytes, st);
  else
    s = solve_csr<ArithF32>(row_ptr, col, static_cast<const float*>(val), n, nnz, static_cast<const float*>(B), ldb,
                            nrhs, depths, nests, tol, static_cast<float*>(X), ldx, res, workspace, ws_bytes, st);
  res->status = s;
  return s;
}

int nn_solve_csr(const int32_t* row_ptr, const int32_t* col, const void* val, int64_t n, int64_t nnz, int dtype,
                 const void* B, int64_t ldb, int64_t nrhs, int depth, int nests, double tol, void* X, int64_t ldx,
                 nn_result* res, void* workspace, size_t ws_bytes, void* stream) {
  if (depth < 1 || depth > 16 || nests < 0 || nests > NN_MAX_HISTORY - 1) {
    if (res != nullptr) {
      memset(res, 0, sizeof(*res));
      res->status = NN_ERR_ARG;
    }
    return NN_ERR_ARG;
  }
  int depths[NN_MAX_HISTORY];
  for (int j = 0; j < nests; ++j) depths[j] = depth;
  return solve_csr_any(row_ptr, col, val, n, nnz, dtype, B, ldb, nrhs, depths, nests, tol, X, ldx, res, workspace,
                       ws_bytes, stream);
}

int nn_solve_csr_sched(const int32_t* row_ptr, const int32_t* col, const void* val, int64_t n, int64_t nnz,
                       int dtype, const void* B, int64_t ldb, int64_t nrhs, const int32_t* depths, int nfactors,
                       double tol, void* X, int64_t ldx, nn_result* res, void* workspace, size_t ws_bytes,
                       void* stream) {
  return solve_csr_any(row_ptr, col, val, n, nnz, dtype, B, ldb, nrhs, depths, nfactors, tol, X, ldx, res, workspace,
                       ws_bytes, stream);
}

size_t nn_csr_strip_workspace_bytes(int64_t n_local) {
  if (n_local < 1 || n_local > (int64_t(1) << 30)) return 0;
  Carver c(nullptr, 0);
  StripWs w;
  carve_strip(c, n_local, w);
  return align_up(c.used, 256);
}

int nn_csr_strip_diag_inv(const int32_t* row_ptr, const int32_t* col_local, const void* val, int64_t n_local,
                          int64_t nnz, int dtype, void* dinv_local, void* workspace, size_t ws_bytes, void* stream) {
  if (!strip_args_ok(row_ptr, col_local, val, n_local, nnz, dtype) || dinv_local == nullptr) return NN_ERR_ARG;
  Carver c(workspace, ws_bytes);
  StripWs w;
  carve_strip(c, n_local, w);
  if (workspace == nullptr || !c.ok) return NN_ERR_OOM_BUDGET;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = int(n_local);
  NN_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  if (dtype == NN_F64)
    diag_inv_kernel<double><<<(n + 255) / 256, 256, 0, st>>>(n, row_ptr, col_local, static_cast<const double*>(val),
                                                              static_cast<double*>(dinv_local), w.err);
  else
    diag_inv_kernel<float><<<(n + 255) / 256, 256, 0, st>>>(n, row_ptr, col_local, static_cast<const float*>(val),
                                                             static_cast<float*>(dinv_local), w.err);
  NN_CUDA_TRY(cudaGetLastError());
  int e = DEV_OK;
  NN_CUDA_TRY(cudaMemcpyAsync(&e, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  NN_CUDA_TRY(cudaStreamSynchronize(st));
  return e == DEV_OK ? NN_OK : NN_ERR_ARG;
}

int nn_csr_strip_scale(const int32_t* col_local, const void* val, int64_t nnz, int dtype, const void* dinv_ext,
                       void* val_scaled, void* stream) {
  if (col_local == nullptr || val == nullptr || dinv_ext == nullptr || val_scaled == nullptr || nnz < 0 ||
      nnz > (int64_t(1) << 31) - 1 || (dtype != NN_F64 && dtype != NN_F32))
    return NN_ERR_ARG;
  if (nnz == 0) return NN_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned blocks = unsigned((nnz + 255) / 256);
  if (dtype == NN_F64)
    scale_cols_kernel<ArithF64><<<blocks, 256, 0, st>>>(nnz, col_local, static_cast<const double*>(val),
                                                        static_cast<const double*>(dinv_ext),
                                                        static_cast<double*>(val_scaled));
  else
    scale_cols_kernel<ArithF32><<<blocks, 256, 0, st>>>(nnz, col_local, static_cast<const float*>(val),
                                                        static_cast<const float*>(dinv_ext),
                                                        static_cast<float*>(val_scaled));
  NN_CUDA_TRY(cudaGetLastError());
  return NN_OK;
}

int nn_csr_strip_product(const int32_t* row_ptr, const int32_t* col_local, const void* val_scaled, int64_t n_local,
                         int64_t nnz, int dtype, const void* v_ext, void* y, const void* acc_in, void* acc_out,
                         void* workspace, size_t ws_bytes, void* stream) {
  if (!strip_args_ok(row_ptr, col_local, val_scaled, n_local, nnz, dtype) || v_ext == nullptr) return NN_ERR_ARG;
  if (y == nullptr && acc_out == nullptr) return NN_ERR_ARG;
  if (acc_out != nullptr && acc_in == nullptr) return NN_ERR_ARG;
  Carver c(workspace, ws_bytes);
  StripWs w;
  carve_strip(c, n_local, w);
  if (workspace == nullptr || !c.ok) return NN_ERR_OOM_BUDGET;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int mode = acc_out == nullptr ? SP_Y : (y == nullptr ? SP_ACC : SP_Y_ACC);
  if (dtype == NN_F64)
    return spmv<ArithF64>(st, int(n_local), int(nnz), row_ptr, col_local, static_cast<const double*>(val_scaled),
                          static_cast<const double*>(v_ext), static_cast<double*>(y),
                          static_cast<const double*>(acc_in), static_cast<double*>(acc_out), nullptr, 0, 1, mode,
                          nullptr, w.err);
  return spmv<ArithF32>(st, int(n_local), int(nnz), row_ptr, col_local, static_cast<const float*>(val_scaled),
                        static_cast<const float*>(v_ext), static_cast<float*>(y), static_cast<const float*>(acc_in),
                        static_cast<float*>(acc_out), nullptr, 0, 1, mode, nullptr, w.err);
}

int nn_csr_strip_residual(const int32_t* row_ptr, const int32_t* col_local, const void* val_scaled, int64_t n_local,
                          int64_t nnz, int dtype, const void* z_ext, const void* b_local, double* sums,
                          void* workspace, size_t ws_bytes, void* stream) {
  if (!strip_args_ok(row_ptr, col_local, val_scaled, n_local, nnz, dtype) || z_ext == nullptr ||
      b_local == nullptr || sums == nullptr)
    return NN_ERR_ARG;
  Carver c(workspace, ws_bytes);
  StripWs w;
  carve_strip(c, n_local, w);
  if (workspace == nullptr || !c.ok) return NN_ERR_OOM_BUDGET;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = int(n_local);
  const int blocks = (n + SP_ROWS - 1) / SP_ROWS;
  if (dtype == NN_F64)
    NN_TRY(spmv<ArithF64>(st, n, int(nnz), row_ptr, col_local, static_cast<const double*>(val_scaled),
                          static_cast<const double*>(z_ext), nullptr, nullptr, nullptr,
                          static_cast<const double*>(b_local), n, 1, SP_RESID, w.partial, w.err));
  else
    NN_TRY(spmv<ArithF32>(st, n, int(nnz), row_ptr, col_local, static_cast<const float*>(val_scaled),
                          static_cast<const float*>(z_ext), nullptr, nullptr, nullptr,
                          static_cast<const float*>(b_local), n, 1, SP_RESID, w.partial, w.err));
  reduce_pair_sums_kernel<<<1, 256, 0, st>>>(w.partial, blocks, w.sums);
  NN_CUDA_TRY(cudaGetLastError());
  int e = DEV_OK;
  NN_CUDA_TRY(cudaMemcpyAsync(sums, w.sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  NN_CUDA_TRY(cudaMemcpyAsync(&e, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  NN_CUDA_TRY(cudaStreamSynchronize(st));
  return e == DEV_OK ? NN_OK : NN_ERR_TIMEOUT;
}

int nn_csr_strip_finish(const void* z_local, const void* dinv_local, int64_t n_local, int dtype, void* x_local,
                        void* stream) {
  if (z_local == nullptr || dinv_local == nullptr || x_local == nullptr || n_local < 1 ||
      n_local > (int64_t(1) << 30) || (dtype != NN_F64 && dtype != NN_F32))
    return NN_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = int(n_local);
  if (dtype == NN_F64)
    store_cols_kernel<ArithF64><<<dim3((n + 255) / 256, 1), 256, 0, st>>>(
        n, 1, static_cast<const double*>(z_local), static_cast<const double*>(dinv_local),
        static_cast<double*>(x_local), n);
  else
    store_cols_kernel<ArithF32><<<dim3((n + 255) / 256, 1), 256, 0, st>>>(
        n, 1, static_cast<const float*>(z_local), static_cast<const float*>(dinv_local), static_cast<float*>(x_local),
        n);
  NN_CUDA_TRY(cudaGetLastError());
  return NN_OK;
}

int nn_solve(const int32_t* row_ptr, const int32_t* col, const void* val, int64_t n, int64_t nnz, const void* B,
             int64_t ldb, int64_t nrhs, int depth, double tol, const nn_opts* opts, void* X, int64_t ldx,
             nn_result* res, void* workspace, size_t ws_bytes, void* stream) {
  if (opts == nullptr || opts->schedule_len < 0 || opts->schedule_len > NN_MAX_HISTORY ||
      (opts->schedule_len > 0 && opts->depth_schedule == nullptr)) {
    if (res != nullptr) {
      memset(res, 0, sizeof(*res));
      res->status = NN_ERR_ARG;
    }
    return NN_ERR_ARG;
  }
  if (opts->schedule_len > 0)
    return solve_csr_any(row_ptr, col, val, n, nnz, opts->dtype, B, ldb, nrhs, opts->depth_schedule,
                         opts->schedule_len, tol, X, ldx, res, workspace, ws_bytes, stream);
  return nn_solve_csr(row_ptr, col, val, n, nnz, opts->dtype, B, ldb, nrhs, depth, opts->max_nests, tol, X, ldx, res,
                      workspace, ws_bytes, stream);
}

}  // extern "C"
