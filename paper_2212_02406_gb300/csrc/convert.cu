// O(N^2) kernels around the nest chain: precision splitting into BF16 pieces (row-major
// and transposed), FP32/FP64 conversions, the starting matrix X_0 (preconditioners of
// Section II-A and Appendix 1) and the deterministic reduction of sum(R_ij^2) partials.
#include <utility>

#include "common.cuh"
#include "kernels.h"

namespace nn {

namespace {

constexpr int TILE = 32;
constexpr int ROWS = 8;  // 32 x 8 threads per 32 x 32 tile

// BF16 pieces of a value with FP32 arithmetic after one FP64 split (the FP64 pipe is narrow):
// v = hi + lo with hi = fp32(v), lo = fp32(v - hi); p0 = bf16(hi), p1 = bf16((hi - p0) + lo),
// p2 = bf16(((hi - p0) + lo) - p1). hi - p0 and t - p1 are exact in FP32; the only rounding
// beyond the pieces themselves is (hi - p0) + lo, at most 2^-24 |hi - p0| <= 2^-33 |v|.
// hi and lo, both rounded to nearest even, come from the FP64 bit pattern without FP64
// arithmetic: hi by rounding the significand's top 24 bits (a carry into the exponent field is
// the correct rounding), lo as the 29-bit remainder (an integer, |r| <= 2^28) converted with
// one int -> float rounding and scaled by the exact power of two 2^(e-52). Returns false,
// leaving the work to FP64 arithmetic, for |v| outside [2^-60, 2^101) (zeros, subnormals, inf
// and NaN included); the results are identical to the FP64 conversions.
__device__ __forceinline__ bool split_hi_lo_int(double v, float& hi, float& lo) {
  const unsigned hw = unsigned(__double2hiint(v)), lw = unsigned(__double2loint(v));
  const int e = int((hw >> 20) & 0x7FFu) - 1023;
  if (e < -60 || e > 100) return false;
  const unsigned sign = hw & 0x80000000u;
  const unsigned mtop = ((hw & 0xFFFFFu) << 3) | (lw >> 29);  // the 23 fraction bits FP32 keeps
  const unsigned rest = lw & 0x1FFFFFFFu;                     // the 29 bits below them
  const unsigned up = (rest > 0x10000000u || (rest == 0x10000000u && (mtop & 1u))) ? 1u : 0u;
  hi = __uint_as_float(sign | ((unsigned(e + 127) << 23) + mtop + up));
  const int r = int(rest) - int(up << 29);  // (v - hi) / 2^(e-52), sign of v factored out
  const float mag = __int2float_rn(r) * __uint_as_float(unsigned(e - 52 + 127) << 23);
  lo = sign ? -mag : mag;
  return true;
}

// v = hi + lo (hi = fp32(v), lo = fp32(v - hi)), by split_hi_lo_int where it applies.
__device__ __forceinline__ void split_hi_lo(double v, float& hi, float& lo) {
  const unsigned long long vb = static_cast<unsigned long long>(__double_as_longlong(v));
  if ((vb << 1) == 0) {
    hi = __uint_as_float(unsigned(vb >> 32) & 0x80000000u);  // +-0
    lo = 0.0f;
  } else if (!split_hi_lo_int(v, hi, lo)) {
    hi = static_cast<float>(v);
    lo = static_cast<float>(v - static_cast<double>(hi));
  }
}

// The three pieces (bit patterns, BF16 or FP16) of s (hi + lo) (|lo| at most half an FP32 ulp of
// hi, s a power of two: the scaling is exact); returns hi. Each remainder before a rounding is
// exact in FP32.
__device__ __forceinline__ float pieces3_hl(float hi, float lo, float s, bool half, uint16_t (&p)[3],
                                            bool r8 = false) {
  float v0, v1, v2;
  const float hs = hi * s;
  p[0] = piece_bits(hs, half, &v0, r8);
  const float t = (hs - v0) + lo * s;
  p[1] = piece_bits(t, half, &v1);
  p[2] = piece_bits(t - v1, half, &v2);
  return hi;
}

__device__ __forceinline__ float pieces3(double v, float s, bool half, uint16_t (&p)[3], bool r8 = false) {
  float hi, lo;
  split_hi_lo(v, hi, lo);
  return pieces3_hl(hi, lo, s, half, p, r8);
}

// The piece scale of padded row i under fmt.
__device__ __forceinline__ float row_piece_scale(const PieceFmt& fmt, int i) {
  return fmt.row_scale != nullptr ? fmt.scale * fmt.row_scale[i] : fmt.scale;
}

// scale v + d as an unevaluated FP32 pair (hi, lo), hi the FP32 rounding of the pair's sum, from
// v = vh + vl, scale = sh + sl and d = dh + dl without FP64 arithmetic (the FP64 pipe is
// narrow): the product sh vh exactly as p + pe (FMA), the cross terms sh vl + sl vh rounded in
// FP32 (they are below 2^-23 |scale v|; sl vl, below 2^-46, is dropped), p + dh exactly as a
// two-sum, then one renormalisation. The pair carries scale v + d to about 2^-45
// max(|scale v|, |d|), far below the 2^-24 of the three BF16 pieces made from it.
__device__ __forceinline__ void affine_hi_lo(float vh, float vl, float sh, float sl, float dh, float dl, float& hi,
                                             float& lo) {
  const float p = sh * vh;
  const float pe = fmaf(sh, vh, -p);
  const float cross = fmaf(sh, vl, sl * vh) + pe;
  const float s = p + dh;
  const float bp = s - p;
  const float se = (p - (s - bp)) + (dh - bp);
  const float t = (se + cross) + dl;
  hi = s + t;
  lo = t - (hi - s);
}

// Four consecutive FP32 source values of row i from column jj (zeros past n), widened to FP64
// (exact).
__device__ __forceinline__ void split_load4(const float* src, int64_t lds, int n, int i, int jj, double (&v)[4]) {
  if (i < n && jj + 3 < n && ((lds & 3) | (reinterpret_cast<uintptr_t>(src) & 15)) == 0) {
    const float4 a = *reinterpret_cast<const float4*>(src + int64_t(i) * lds + jj);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = (i < n && jj + e < n) ? double(src[int64_t(i) * lds + jj + e]) : 0.0;
  }
}

struct PiecePtrs {
  __nv_bfloat16* p[3];
};

// Tile of 32 rows x 128 columns per block of 32 x 8 threads; each thread handles four
// consecutive columns (32-byte loads, 8-byte piece stores, 16-byte FP32 stores), and the
// transposed pieces go out through shared memory as 4-byte pairs along the output rows.
constexpr int SPLIT_R = 32, SPLIT_C = 128;

// Four consecutive source values of row i from column jj (zeros past n), as FP64.
__device__ __forceinline__ void split_load4(const double* src, int64_t lds, int n, int i, int jj, double (&v)[4]) {
  if (i < n && jj + 3 < n && ((lds & 1) | (reinterpret_cast<uintptr_t>(src) & 15)) == 0) {
    const double2* p2 = reinterpret_cast<const double2*>(src + int64_t(i) * lds + jj);
    const double2 a = p2[0], b = p2[1];
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = (i < n && jj + e < n) ? src[int64_t(i) * lds + jj + e] : 0.0;
  }
}

// Splits the n x n matrix scale * src + diag * I (FP64 arithmetic; AFFINE = false: src as is)
// into its FP32 rounding and operand pieces (format and piece scales: fmt).
// DUAL (with AFFINE): the same pass also writes the three row-major pieces of src itself to
// dual_row (format dual_fmt), with its per-block sums of squares in dual_sumsq (one read of src
// for both).
template <typename S, bool AFFINE, bool DUAL = false>
__global__ void split_kernel(const S* __restrict__ src, int64_t lds, int n, int np, float* __restrict__ f32,
                             PiecePtrs row, int n_row, PiecePtrs col, int n_col, double* __restrict__ sumsq,
                             double scale, double diag, PieceFmt fmt, PiecePtrs dual_row = PiecePtrs{},
                             double* __restrict__ dual_sumsq = nullptr, int yb0 = 0, PieceFmt dual_fmt = PieceFmt{}) {
  __shared__ uint16_t tile[3][SPLIT_R][SPLIT_C + 2];  // odd word pitch: conflict-free columns
  __shared__ float red[ROWS];
  // yb0: first block row (a launch may cover a panel of rows; partial sums keep global indices)
  const int yb = int(blockIdx.y) + yb0;
  const int i0 = yb * SPLIT_R, j0 = blockIdx.x * SPLIT_C;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int jj = j0 + 4 * tx;
  float ss = 0.f, ss_src = 0.f;
  // all of the thread's source rows are loaded before any is processed: four 32-byte loads
  // in flight per thread instead of one
  constexpr int RPT = SPLIT_R / ROWS;
  double vin[RPT][4];
#pragma unroll
  for (int rr = 0; rr < RPT; ++rr) split_load4(src, lds, n, i0 + ty + rr * ROWS, jj, vin[rr]);
#pragma unroll
  for (int rr = 0; rr < RPT; ++rr) {
    const int r = ty + rr * ROWS;
    const int i = i0 + r;
    double v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = vin[rr][e];
    // AFFINE: the source's FP32 pairs, shared by its own pieces (DUAL) and the affine output
    float vh[4], vl[4];
    if (AFFINE) {
#pragma unroll
      for (int e = 0; e < 4; ++e) split_hi_lo(v[e], vh[e], vl[e]);
    }
    const float ps = row_piece_scale(fmt, i);
    if (DUAL) {
      uint16_t pd[4][3];
      const float ds = row_piece_scale(dual_fmt, i);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float h = pieces3_hl(vh[e], vl[e], ds, dual_fmt.half, pd[e], dual_fmt.r8);
        ss_src = fmaf(h, h, ss_src);
      }
      const int64_t off = int64_t(i) * np + jj;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const uint32_t lo2 = uint32_t(pd[0][q]) | (uint32_t(pd[1][q]) << 16);
        const uint32_t hi2 = uint32_t(pd[2][q]) | (uint32_t(pd[3][q]) << 16);
        *reinterpret_cast<uint2*>(dual_row.p[q] + off) = make_uint2(lo2, hi2);
      }
    }
    uint16_t pc[4][3];
    float hi[4];
    if (AFFINE) {
      // scale v + diag I in FP32 pairs (padding rows and columns stay zero)
      const float sh = static_cast<float>(scale), sl = static_cast<float>(scale - static_cast<double>(sh));
      const float dh = static_cast<float>(diag), dl = static_cast<float>(diag - static_cast<double>(dh));
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float h = 0.f, l = 0.f;
        if (i < n && jj + e < n) {
          const bool on = i == jj + e;
          affine_hi_lo(vh[e], vl[e], sh, sl, on ? dh : 0.f, on ? dl : 0.f, h, l);
        }
        hi[e] = pieces3_hl(h, l, ps, fmt.half, pc[e], fmt.r8);
        ss = fmaf(hi[e], hi[e], ss);
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        hi[e] = pieces3(v[e], ps, fmt.half, pc[e], fmt.r8);
        ss = fmaf(hi[e], hi[e], ss);
      }
    }
    const int64_t off = int64_t(i) * np + jj;
    if (f32) *reinterpret_cast<float4*>(f32 + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
    // static piece indices (q unrolled) keep pc in registers
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (q >= n_row) break;
      const uint32_t lo2 = uint32_t(pc[0][q]) | (uint32_t(pc[1][q]) << 16);
      const uint32_t hi2 = uint32_t(pc[2][q]) | (uint32_t(pc[3][q]) << 16);
      *reinterpret_cast<uint2*>(row.p[q] + off) = make_uint2(lo2, hi2);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (q >= n_col) break;
#pragma unroll
      for (int e = 0; e < 4; ++e) tile[q][r][4 * tx + e] = pc[e][q];
    }
  }
  if (sumsq != nullptr) {
    // per-block sum of squares (FP32 within the block, fixed order), for ||src||_F
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
    if (tx == 0) red[ty] = ss;
    __syncthreads();
    if (tx == 0 && ty == 0) {
      float t = 0.f;
      for (int w = 0; w < ROWS; ++w) t += red[w];
      sumsq[int64_t(yb) * gridDim.x + blockIdx.x] = double(t);
    }
  }
  if (DUAL) {
    // the same for src itself (the affine output's sums above)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss_src += __shfl_down_sync(0xffffffffu, ss_src, o);
    __syncthreads();
    if (tx == 0) red[ty] = ss_src;
    __syncthreads();
    if (tx == 0 && ty == 0) {
      float t = 0.f;
      for (int w = 0; w < ROWS; ++w) t += red[w];
      dual_sumsq[int64_t(yb) * gridDim.x + blockIdx.x] = double(t);
    }
  }
  if (n_col > 0) {
    __syncthreads();
    // transposed: output row j0 + c (c < 128) holds input column j0 + c, entries i0 .. i0 + 31;
    // thread t writes entries 8 (t % 4) .. + 7 of output row c = t / 4 (+ 64) as one 16-byte store
    const int t = ty * 32 + tx;
    const int r0 = 8 * (t % 4);
    for (int c = t / 4; c < SPLIT_C; c += (ROWS * 32) / 4) {
      const int64_t off = int64_t(j0 + c) * np + i0 + r0;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (q >= n_col) break;
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
          w[e] = uint32_t(tile[q][r0 + 2 * e][c]) | (uint32_t(tile[q][r0 + 2 * e + 1][c]) << 16);
        *reinterpret_cast<uint4*>(col.p[q] + off) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
  }
}

template <typename S, typename D>
__global__ void convert_kernel(const S* __restrict__ src, int64_t lds, int n, D* __restrict__ dst, int64_t ldd) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (i < n && j < n) dst[int64_t(i) * ldd + j] = static_cast<D>(src[int64_t(i) * lds + j]);
}

// FP32 -> FP64 with 16-byte loads and stores: four consecutive elements of row blockIdx.y per
// thread (src rows 16-byte aligned, dst rows 16-byte aligned).
__global__ void f32_to_f64_vec_kernel(const float* __restrict__ src, int64_t lds, int n, double* __restrict__ dst,
                                      int64_t ldd) {
  const int j = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int i = blockIdx.y;
  if (j >= n) return;
  const float* s = src + int64_t(i) * lds + j;
  double* d = dst + int64_t(i) * ldd + j;
  if (j + 4 <= n) {
    const float4 f = *reinterpret_cast<const float4*>(s);
    reinterpret_cast<double2*>(d)[0] = make_double2(double(f.x), double(f.y));
    reinterpret_cast<double2*>(d)[1] = make_double2(double(f.z), double(f.w));
  } else {
    for (int e = 0; j + e < n; ++e) d[e] = double(s[e]);
  }
}

__global__ void reduce_rms_kernel(const double* __restrict__ partial, int count, double scale, double* out) {
  __shared__ double buf[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < count; i += 256) s += partial[i];
  buf[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) buf[threadIdx.x] += buf[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sqrt(buf[0]) * scale;
}

// Per-block sum of squares of an n x n matrix, grid-stride over rows (fixed block order).
__global__ void sumsq_rows_kernel(const double* __restrict__ src, int64_t lds, int n, double* partial) {
  __shared__ double buf[256];
  double s = 0.0;
  for (int i = blockIdx.x; i < n; i += gridDim.x)
    for (int j = threadIdx.x; j < n; j += 256) {
      const double v = src[int64_t(i) * lds + j];
      s = fma(v, v, s);
    }
  buf[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) buf[threadIdx.x] += buf[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = buf[0];
}

// Non-negative doubles order like their bit patterns, so max() can use the 64-bit integer atomic.
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), static_cast<unsigned long long>(__double_as_longlong(v)));
}

// ||A||_inf: one warp per row.
__global__ void row_abs_max_kernel(const double* __restrict__ A, int64_t lda, int n, double* out) {
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += fabs(A[int64_t(row) * lda + j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) atomic_max_nonneg(out, s);
}

// ||A||_1: one thread per column (coalesced across the warp).
__global__ void col_abs_max_kernel(const double* __restrict__ A, int64_t lda, int n, double* out) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= n) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += fabs(A[int64_t(i) * lda + col]);
  atomic_max_nonneg(out, s);
}

__global__ void trace_kernel(const double* __restrict__ A, int64_t lda, int n, double* out) {
  __shared__ double buf[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += A[int64_t(i) * lda + i];
  buf[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) buf[threadIdx.x] += buf[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = buf[0];
}

// X0 = A^T / (||A||_1 ||A||_inf), tiled transpose.
__global__ void pan_schreiber_kernel(const double* __restrict__ A, int64_t lda, int n, const double* norms,
                                     double* __restrict__ X, int64_t ldx) {
  __shared__ double tile[TILE][TILE + 1];
  const double c = 1.0 / (norms[0] * norms[1]);
  const int i0 = blockIdx.y * TILE, j0 = blockIdx.x * TILE;
  for (int r = threadIdx.y; r < TILE; r += ROWS) {
    const int i = i0 + r, j = j0 + threadIdx.x;
    tile[r][threadIdx.x] = (i < n && j < n) ? A[int64_t(i) * lda + j] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < TILE; r += ROWS) {
    const int i = j0 + r, j = i0 + threadIdx.x;  // X[i][j] = A[j][i] * c
    if (i < n && j < n) X[int64_t(i) * ldx + j] = tile[threadIdx.x][r] * c;
  }
}

// y = A x, one warp per row (coalesced row reads), FP64.
__global__ void gemv_rows_kernel(const double* __restrict__ A, int64_t lda, int n, const double* __restrict__ x,
                                 double* __restrict__ y) {
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s = fma(A[int64_t(row) * lda + j], x[j], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = s;
}

__global__ void fill_value_kernel(double* __restrict__ x, int n, double v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

// out[0] = (k/(k+1)) <u,u> / <u,w>, fixed summation order (one block).
__global__ void theta2_kernel(const double* __restrict__ u, const double* __restrict__ w, int n, double kfac,
                              double* out) {
  __shared__ double a[256], b[256];
  double x = 0, y = 0;
  for (int i = threadIdx.x; i < n; i += 256) {
    x = fma(u[i], u[i], x);
    y = fma(u[i], w[i], y);
  }
  a[threadIdx.x] = x;
  b[threadIdx.x] = y;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      a[threadIdx.x] += a[threadIdx.x + s];
      b[threadIdx.x] += b[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = kfac * a[0] / b[0];
}

// Diagonal starting matrices: kind SCALAR (value), TRACE (1 / *dev), JACOBI (value / A_ii),
// THETA2 (*dev).
__global__ void fill_diag_kernel(const double* __restrict__ A, int64_t lda, int n, int kind, double value,
                                 const double* dev, double* __restrict__ X, int64_t ldx) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (i >= n || j >= n) return;
  double v = 0.0;
  if (i == j) {
    if (kind == NN_PC_SCALAR)
      v = value;
    else if (kind == NN_PC_TRACE)
      v = 1.0 / dev[0];
    else if (kind == NN_PC_THETA2)
      v = dev[0];
    else
      v = value / A[int64_t(i) * lda + i];
  }
  X[int64_t(i) * ldx + j] = v;
}

// One warp per padded row i in [row0, row1): scale[i] = 2^e with max_j |src_ij| 2^e in
// [2^13, 2^14) (exponent of the maximum from frexp), inv[i] = 2^-e; zero, non-finite and
// padding rows get 1.
__global__ void row_piece_scale_kernel(const double* __restrict__ src, int64_t lds, int n, int row0, int row1,
                                       float* __restrict__ scale, float* __restrict__ inv) {
  const int i = row0 + int(blockIdx.x) * 8 + int(threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= row1) return;
  double m = 0.0;
  if (i < n) {
    // four independent maxima, four loads in flight per lane
    const double* row = src + int64_t(i) * lds;
    double m4[4] = {0.0, 0.0, 0.0, 0.0};
    int j = lane;
    for (; j + 96 < n; j += 128) {
#pragma unroll
      for (int u = 0; u < 4; ++u) m4[u] = fmax(m4[u], fabs(row[j + 32 * u]));
    }
    for (; j < n; j += 32) m4[0] = fmax(m4[0], fabs(row[j]));
    m = fmax(fmax(m4[0], m4[1]), fmax(m4[2], m4[3]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) {
    int e = 0;
    if (m > 0.0 && isfinite(m)) {
      int ex = 0;
      (void)frexp(m, &ex);  // m = f 2^ex, f in [0.5, 1): m 2^(14 - ex) in [2^13, 2^14)
      e = 14 - ex;
      e = e > 100 ? 100 : (e < -100 ? -100 : e);
    }
    scale[i] = ldexpf(1.0f, e);
    inv[i] = ldexpf(1.0f, -e);
  }
}

}  // namespace

// Rows [row0, row1) of the padded matrix (row1 < 0: to np); both multiples of the block height.
static bool split_rows(int np, int& row0, int& row1) {
  if (row1 < 0) row1 = np;
  return row0 >= 0 && row0 < row1 && row1 <= np && row0 % SPLIT_R == 0 && row1 % SPLIT_R == 0;
}

int split_matrix(cudaStream_t st, const double* src, int64_t lds, int n, int np, float* f32,
                 __nv_bfloat16* const* row_pieces, int n_row, __nv_bfloat16* const* col_pieces, int n_col,
                 double* sumsq_partial, int row0, int row1, PieceFmt fmt) {
  if (np % SPLIT_C != 0 || n > np || n_row < 0 || n_row > 3 || n_col < 0 || n_col > 3) return NN_ERR_ARG;
  if (!split_rows(np, row0, row1)) return NN_ERR_ARG;
  PiecePtrs r{}, c{};
  for (int q = 0; q < n_row; ++q) r.p[q] = row_pieces[q];
  for (int q = 0; q < n_col; ++q) c.p[q] = col_pieces[q];
  dim3 grid(np / SPLIT_C, (row1 - row0) / SPLIT_R), block(32, ROWS);
  split_kernel<double, false><<<grid, block, 0, st>>>(src, lds, n, np, f32, r, n_row, c, n_col, sumsq_partial, 1.0,
                                                      0.0, fmt, PiecePtrs{}, nullptr, row0 / SPLIT_R);
  NN_CUDA_TRY(cudaGetLastError());
  return NN_OK;
}

int split_matrix_f32(cudaStream_t st, const float* src, int64_t lds, int n, int np, __nv_bfloat16* const* row_pieces,
                     int n_row, __nv_bfloat16* const* col_pieces, int n_col, PieceFmt fmt) {
  if (np % SPLIT_C != 0 || n > np || n_row < 0 || n_row > 3 || n_col < 0 || n_col > 3) return NN_ERR_ARG;
  PiecePtrs r{}, c{};
  for (int q = 0; q < n_row; ++q) r.p[q] = row_pieces[q];
  for (int q = 0; q < n_col; ++q) c.p[q] = col_pieces[q];
  dim3 grid(np / SPLIT_C, np / SPLIT_R), block(32, ROWS);
  split_kernel<float, false><<<grid, block, 0, st>>>(src, lds, n, np, nullptr, r, n_row, c, n_col, nullptr, 1.0, 0.0,
                                                     fmt);
  NN_CUDA_TRY(cudaGetLastError());
  return NN_OK;
}

static int split_affine(cudaStream_t st, const double* src, int64_t lds, int n, int np, float* f32,
                        __nv_bfloat16* const* row_pieces, int n_row, __nv_bfloat16* const* col_pieces, int n_col,
                        double* sumsq_partial, double scale, double diag, PieceFmt fmt) {
  if (np % SPLIT_C != 0 || n > np || n_row < 0 || n_row > 3 || n_col < 0 || n_col > 3) return NN_ERR_ARG;
  PiecePtrs r{}, c{};
  for (int q = 0; q < n_row; ++q) r.p[q] = row_pieces[q];
  for (int q = 0; q < n_col; ++q) c.p[q] = col_pieces[q];
  dim3 grid(np / SPLIT_C, np / SPLIT_R), block(32, ROWS);
  split_kernel<double, true><<<grid, block, 0, st>>>(src, lds, n, np, f32, r, n_row, c, n_col, sumsq_partial, scale, diag,
                                                     fmt);
  NN_CUDA_TRY(cudaGetLastError());
  return NN_OK;
}

int split_matrix_dual(cudaStream_t st, const double* src, int64_t lds, int n, int np,
                      __nv_bfloat16* const* src_row_pieces, double* src_sumsq_partial, float* f32,
                      __nv_bfloat16* const* row_pieces, int n_row, __nv_bfloat16* const* col_pieces, int n_col,
                      double* sumsq_partial, double scale, double diag, int row0, int row1, PieceFmt fmt,
                      PieceFmt src_fmt) {
  if (np % SPLIT_C != 0 || n > np || n_row < 0 || n_row > 3 || n_col < 0 || n_col > 3 || sumsq_partial == nullptr ||
      src_sumsq_partial == nullptr)
    return NN_ERR_ARG;
  if (!split_rows(np, row0, row1)) return NN_ERR_ARG;
  PiecePtrs r{}, c{}, d{};
  for (int q = 0; q < n_row; ++q) r.p[q] = row_pieces[q];
  for (int q = 0; q < n_col; ++q) c.p[q] = col_pieces[q];
  for (int q = 0; q < 3; ++q) {
    if (src_row_pieces[q] == nullptr) return NN_ERR_ARG;
    d.p[q] = src_row_pieces[q];
  }
  dim3 grid(np / SPLIT_C, (row1 - row0) / SPLIT_R), block(32, ROWS);
  if (fmt.half != src_fmt.half) return NN_ERR_ARG;  // one product reads both in one format
  split_kernel<double, true, true><<<grid, block, 0, st>>>(src, lds, n, np, f32, r, n_row, c, n_col, sumsq_partial,
                                                           scale, diag, fmt, d, src_sumsq_partial, row0 / SPLIT_R,
                                                           src_fmt);
  NN_CUDA_TRY(cudaGetLastError());
  return NN_OK;
}

int split_matrix_affine(cudaStream_t st, const double* src, int64_t lds, int n, int np, float* f32,
                        __nv_bfloat16* const* row_pieces, int n_row, __nv_bfloat16* const* col_pieces, int n_col,
                        double* sumsq_partial, double scale, double diag, PieceFmt fmt) {
  return split_affine(st, src, lds, n, np, f32, row_pieces, n_row, col_pieces, n_col, sumsq_partial, scale, diag,
                      fmt);
}

int row_piece_scales(cudaStream_t st, const double* src, int64_t lds, int n, int np, float* scale, float* inv,
                     int row0, int row1) {
  if (row1 < 0) row1 = np;
  if (n > np || row0 < 0 || row0 > row1 || row1 > np || scale == nullptr || inv == nullptr) return NN_ERR_ARG;
  if (row1 == row0) return NN_OK;
  row_piece_scale_kernel<<<(row1 - row0 + 7) / 8, 256, 0, st>>>(src, lds, n, row0, row1, scale, inv);
  NN_CUDA_TRY(cudaGetLastError());
  return NN_OK;
}

int split_blocks(int np) { return (np / SPLIT_C) * (np / SPLIT_R); }

template <typename S, typename D>
static int convert(cudaStream_t st, const S* src, int64_t lds, int n, D* dst, int64_t ldd) {
  if (n <= 0) return NN_OK;
  dim3 grid((n + 255) / 256, n), block(256);
  convert_kernel<S, D><<<grid, block, 0, st>>>(src, lds, n, dst, ldd);
  NN_CUDA_TRY(cudaGetLastError());
  return NN_OK;
}

int f32_to_f64(cudaStream_t st, const float* src, int64_t lds, int n, double* dst, int64_t ldd) {
  if (n > 0 && lds % 4 == 0 && ldd % 2 == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0 &&
      (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
    dim3 grid((n + 1023) / 1024, n), block(256);
    f32_to_f64_vec_kernel<<<grid, block, 0, st>>>(src, lds, n, dst, ldd);
    NN_CUDA_TRY(cudaGetLastError());
    return NN_OK;
  }
  return convert(st, src, lds, n, dst, ldd);
}
int copy_f64(cudaStream_t st, const double* src, int64_t lds, int n, double* dst, int64_t ldd) {
  return convert(st, src, lds, n, dst, ldd);
}
int f64_to_f32(cudaStream_t st, const double* src, int64_t lds, int n, float* dst, int64_t ldd) {
  return convert(st, src, lds, n, dst, ldd);
}

int frob_f64(cudaStream_t st, const double* src, int64_t lds, int n, double* partial, int count, double* out) {
  int blocks = count < 1024 ? count : 1024;
  if (blocks > n) blocks = n;
  if (blocks < 1) return NN_ERR_ARG;
  sumsq_rows_kernel<<<blocks, 256, 0, st>>>(src, lds, n, partial);
  NN_CUDA_TRY(cudaGetLastError());
  return reduce_rms(st, partial, blocks, 1.0, out);
}

int reduce_rms(cudaStream_t st, const double* partial, int count, double scale, double* out) {
  reduce_rms_kernel<<<1, 256, 0, st>>>(partial, count, scale, out);
  NN_CUDA_TRY(cudaGetLastError());
  return NN_OK;
}

int precond_fill(cudaStream_t st, const double* A, int64_t lda, int n, int kind, double scalar, double* X0,
                 int64_t ldx, double* scratch, double* vec_scratch) {
  if (n <= 0) return NN_ERR_ARG;
  if (kind == NN_PC_PAN_SCHREIBER) {
    NN_CUDA_TRY(cudaMemsetAsync(scratch, 0, 2 * sizeof(double), st));
    col_abs_max_kernel<<<(n + 255) / 256, 256, 0, st>>>(A, lda, n, scratch + 0);
    NN_CUDA_TRY(cudaGetLastError());
    row_abs_max_kernel<<<(n + 7) / 8, 256, 0, st>>>(A, lda, n, scratch + 1);
    NN_CUDA_TRY(cudaGetLastError());
    dim3 grid((n + TILE - 1) / TILE, (n + TILE - 1) / TILE), block(TILE, ROWS);
    pan_schreiber_kernel<<<grid, block, 0, st>>>(A, lda, n, scratch, X0, ldx);
    NN_CUDA_TRY(cudaGetLastError());
    return NN_OK;
  }
  if (kind == NN_PC_TRACE) {
    trace_kernel<<<1, 256, 0, st>>>(A, lda, n, scratch + 2);
    NN_CUDA_TRY(cudaGetLastError());
  } else if (kind == NN_PC_THETA2) {
    // Theta_2(k) = (k/(k+1)) ||A^k v||^2 / <A^k v, A^(k+1) v>, v = ones, k = scalar
    const int k = int(scalar);
    if (k < 1 || vec_scratch == nullptr) return NN_ERR_ARG;
    double* u = vec_scratch;
    double* w = vec_scratch + n;
    fill_value_kernel<<<(n + 255) / 256, 256, 0, st>>>(u, n, 1.0);
    NN_CUDA_TRY(cudaGetLastError());
    for (int it = 0; it <= k; ++it) {
      gemv_rows_kernel<<<(n + 7) / 8, 256, 0, st>>>(A, lda, n, u, w);
      NN_CUDA_TRY(cudaGetLastError());
      if (it < k) std::swap(u, w);
    }
    theta2_kernel<<<1, 256, 0, st>>>(u, w, n, double(k) / double(k + 1), scratch + 2);
    NN_CUDA_TRY(cudaGetLastError());
  } else if (kind != NN_PC_SCALAR && kind != NN_PC_JACOBI) {
    return NN_ERR_ARG;
  }
  dim3 grid((n + 255) / 256, n), block(256);
  fill_diag_kernel<<<grid, block, 0, st>>>(A, lda, n, kind, scalar, scratch + 2, X0, ldx);
  NN_CUDA_TRY(cudaGetLastError());
  return NN_OK;
}

}  // namespace nn
