// FP64 matrix product emulated on the BF16 tensor cores with exact slices (the error-free
// splitting of Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its applications",
// Numerical Algorithms 59 (2012)), arranged for tcgen05:
//
//   * every row i of A gets the exponent e_i with max_j |a_ij| < 2^e_i, every column j of B the
//     exponent f_j (rows of B^T); a_ij 2^-e_i is a fixed-point number in (-1, 1) that is cut into
//     S signed base-2^beta digits q_s (rounded to nearest, |q_0| <= 2^beta, |q_s| <= 2^(beta-1)
//     after), a_ij = 2^e_i sum_s q_s 2^(-beta (s+1)) up to 2^(e_i - 62);
//   * slice s of A is stored in BF16 as q_s 2^(e_i - g_A - beta (s+1)) (g_A = max_i e_i), which
//     is exact: q_s has at most beta + 1 significant bits. Likewise for B^T;
//   * the product of slices s and t summed over k is an integer times 2^(e_i + f_j - g_A - g_B
//     - beta (s+t+2)); with beta chosen so that n 2^(2 beta) <= 2^24 every partial sum of such
//     products is exact in the FP32 accumulator, whatever the order. Products with the same
//     d = s + t share that power of two, so several of them run as segments of one launch as
//     long as their summed bound stays within 2^24;
//   * the epilogue converts each group's exact FP32 result to FP64, scales by 2^(g_A + g_B) and
//     accumulates in FP64; the last group applies the NN epilogue (I - C, D + C) in FP64.
// Products with s + t >= S are dropped; with S beta >= 54 the result matches an FP64 product
// to a few units of 2^-53 relative to (max |a_i.|)(max |b_.j|) n.
#include <limits.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace nn {
namespace {

constexpr int EMU_MAX_SLICES = 14;
constexpr int EMU_EXP_NONE = -100000;  // exponent of an all-zero row / matrix

int ceil_log2(int64_t v) {
  int e = 0;
  while ((int64_t(1) << e) < v) ++e;
  return e;
}

// Digit width: n (2^beta)^2 <= 2^24 keeps every slice product's sum exact in FP32.
int emu_beta(int n) {
  int b = (24 - ceil_log2(n)) / 2;
  return b < 3 ? 3 : (b > 7 ? 7 : b);
}

int emu_slices(int beta) {
  const int s = (54 + beta - 1) / beta;
  return s > EMU_MAX_SLICES ? EMU_MAX_SLICES : s;
}

int64_t emu_np(int64_t n) { return (n + 255) / 256 * 256; }

__global__ void init_exps_kernel(int* g) {
  if (threadIdx.x < 2) g[threadIdx.x] = EMU_EXP_NONE;
}

// exps[i] = e with max_j |src_ij| < 2^e (EMU_EXP_NONE for a zero row); *gmax = max_i exps[i].
__global__ void row_exp_kernel(const double* __restrict__ src, int64_t ld, int n, int* __restrict__ exps,
                               int* __restrict__ gmax) {
  __shared__ double red[8];
  const int i = blockIdx.x;
  double m = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) m = fmax(m, fabs(src[int64_t(i) * ld + j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < int(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    const int e = m > 0.0 ? ilogb(m) + 1 : EMU_EXP_NONE;
    exps[i] = e;
    if (m > 0.0) atomicMax(gmax, e);
  }
}

// dst (ld np) = src^T for the n x n block
__global__ void transpose_kernel(const double* __restrict__ src, int64_t ld, int n, double* __restrict__ dst,
                                 int64_t ldd) {
  __shared__ double tile[32][33];
  const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
  for (int ty = threadIdx.y; ty < 32; ty += blockDim.y) {
    const int i = bi + ty, j = bj + threadIdx.x;
    tile[ty][threadIdx.x] = (i < n && j < n) ? src[int64_t(i) * ld + j] : 0.0;
  }
  __syncthreads();
  for (int ty = threadIdx.y; ty < 32; ty += blockDim.y) {
    const int r = bj + ty, c = bi + threadIdx.x;
    if (r < n && c < n) dst[int64_t(r) * ldd + c] = tile[threadIdx.x][ty];
  }
}

// The S BF16 slice planes (np x np each, zero padding) of an n x n FP64 matrix sliced by rows.
__global__ void slice_rows_kernel(const double* __restrict__ src, int64_t ld, int n, int np,
                                  const int* __restrict__ exps, const int* __restrict__ gmax, int beta, int S,
                                  __nv_bfloat16* __restrict__ out) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t plane = int64_t(np) * np;
  if (e >= plane) return;
  const int i = int(e / np), j = int(e % np);
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
  double x = 0.0;
  if (i < n && j < n) x = src[int64_t(i) * ld + j];
  if (x == 0.0) {
    for (int s = 0; s < S; ++s) out[s * plane + e] = zero;
    return;
  }
  // |x| = mant 2^E exactly
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
  const bool neg = (bits >> 63) != 0;
  const int eb = int((bits >> 52) & 0x7FFull);
  unsigned long long mant = bits & 0xFFFFFFFFFFFFFull;
  int E;
  if (eb != 0) {
    mant |= 1ull << 52;
    E = eb - 1075;
  } else {
    E = -1074;
  }
  // fixed point with 62 fraction bits relative to 2^e_i (|x| < 2^e_i, so u < 2^62)
  const int ei = exps[i];
  const int shift = E + 62 - ei;
  unsigned long long u = 0;
  if (shift >= 0)
    u = mant << shift;
  else if (shift > -64)
    u = mant >> (-shift);
  long long v = neg ? -static_cast<long long>(u) : static_cast<long long>(u);
  const int g = *gmax;
  for (int s = 0; s < S; ++s) {
    const int sh = 62 - beta * (s + 1);
    // nearest digit (ties up): q = floor((v + 2^(sh-1)) / 2^sh)
    const long long q = (v + (1ll << (sh - 1))) >> sh;
    v -= q * (1ll << sh);
    // q 2^(e_i - g - beta (s+1)), exact in BF16 while the exponent stays normal
    const int k = ei - g - beta * (s + 1);
    float val = 0.0f;
    if (q != 0 && k >= -126) val = float(q) * __int_as_float((k + 127) << 23);
    out[s * plane + e] = __float2bfloat16_rn(val);
  }
}

struct EmuWs {
  __nv_bfloat16* a_sl;
  __nv_bfloat16* b_sl;
  double* bt;
  double* acc;
  int* rexp;
  int* cexp;
  int* gexp;
};

void carve_emu(Carver& c, int64_t n, EmuWs& w) {
  const int64_t np = emu_np(n);
  const int S = emu_slices(emu_beta(int(n)));
  const size_t plane = size_t(np) * size_t(np);
  w.a_sl = c.take<__nv_bfloat16>(plane * S);
  w.b_sl = c.take<__nv_bfloat16>(plane * S);
  w.bt = c.take<double>(size_t(n) * size_t(np));
  w.acc = c.take<double>(plane);
  w.rexp = c.take<int>(size_t(np));
  w.cexp = c.take<int>(size_t(np));
  w.gexp = c.take<int>(2);
}

struct EmuGroup {
  int d;
  int cnt;
  int s[kTcMaxSeg];
  int t[kTcMaxSeg];
};

// Products (s, t) with s + t < S, grouped by d = s + t into launches of at most kTcMaxSeg
// segments whose summed worst-case |sum| n M_s M_t stays within 2^24 (M_0 = 2^beta, M_s = 2^(beta-1)).
std::vector<EmuGroup> emu_groups(int n, int beta, int S) {
  std::vector<EmuGroup> out;
  const double cap = 16777216.0;
  auto bound = [&](int s, int t) {
    const double ms = s == 0 ? double(1 << beta) : double(1 << (beta - 1));
    const double mt = t == 0 ? double(1 << beta) : double(1 << (beta - 1));
    return double(n) * ms * mt;
  };
  for (int d = 0; d < S; ++d) {
    EmuGroup g{};
    g.d = d;
    double sum = 0.0;
    for (int s = 0; s <= d; ++s) {
      const int t = d - s;
      if (s >= S || t >= S) continue;
      const double b = bound(s, t);
      if (g.cnt == kTcMaxSeg || sum + b > cap) {
        out.push_back(g);
        g = EmuGroup{};
        g.d = d;
        sum = 0.0;
      }
      g.s[g.cnt] = s;
      g.t[g.cnt] = t;
      ++g.cnt;
      sum += b;
    }
    if (g.cnt > 0) out.push_back(g);
  }
  return out;
}

}  // namespace

size_t emu_workspace_bytes(int64_t n) {
  Carver c(nullptr, 0);
  EmuWs w;
  carve_emu(c, n, w);
  return align_up(c.used, 256);
}

int gemm_f64_emu(cudaStream_t st, int n, const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                 int64_t ldc, int mode, const double* D, int64_t ldd, int n_id, double* partial, int* partials,
                 void* ws, size_t ws_bytes, int* err, double* hw_flops, int min_bits) {
  if (n < 1 || A == nullptr || B == nullptr || C == nullptr || err == nullptr) return NN_ERR_ARG;
  if (mode == EPI_ADD && D == nullptr) return NN_ERR_ARG;
  if (!tc_supported()) return NN_ERR_UNSUPPORTED;
  Carver c(ws, ws_bytes);
  EmuWs w;
  carve_emu(c, n, w);
  if (!c.ok) return NN_ERR_OOM_BUDGET;
  const int np = int(emu_np(n));
  const int beta = emu_beta(n);
  // min_bits > 0: only the slice products with s + t < ceil(min_bits / beta) (relative error
  // about 2^-min_bits instead of FP64's 2^-53)
  int S = emu_slices(beta);
  if (min_bits > 0) S = std::min(S, (min_bits + beta - 1) / beta);

  init_exps_kernel<<<1, 32, 0, st>>>(w.gexp);
  NN_CUDA_TRY(cudaGetLastError());
  row_exp_kernel<<<n, 256, 0, st>>>(A, lda, n, w.rexp, w.gexp + 0);
  NN_CUDA_TRY(cudaGetLastError());
  {
    const dim3 block(32, 8), grid(unsigned((n + 31) / 32), unsigned((n + 31) / 32));
    transpose_kernel<<<grid, block, 0, st>>>(B, ldb, n, w.bt, np);
    NN_CUDA_TRY(cudaGetLastError());
  }
  row_exp_kernel<<<n, 256, 0, st>>>(w.bt, np, n, w.cexp, w.gexp + 1);
  NN_CUDA_TRY(cudaGetLastError());
  const int64_t plane = int64_t(np) * np;
  const unsigned blocks = unsigned((plane + 255) / 256);
  slice_rows_kernel<<<blocks, 256, 0, st>>>(A, lda, n, np, w.rexp, w.gexp + 0, beta, S, w.a_sl);
  NN_CUDA_TRY(cudaGetLastError());
  slice_rows_kernel<<<blocks, 256, 0, st>>>(w.bt, np, n, np, w.cexp, w.gexp + 1, beta, S, w.b_sl);
  NN_CUDA_TRY(cudaGetLastError());

  const std::vector<EmuGroup> groups = emu_groups(n, beta, S);
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const EmuGroup& gr = groups[gi];
    TcGemmArgs g;
    g.np = np;
    g.n_id = n_id;
    g.nseg = gr.cnt;
    for (int q = 0; q < gr.cnt; ++q) {
      g.a_seg[q] = w.a_sl + int64_t(gr.s[q]) * plane;
      g.b_seg[q] = w.b_sl + int64_t(gr.t[q]) * plane;
    }
    g.mode = mode;
    g.err = err;
    g.emu = true;
    g.emu_first = gi == 0;
    g.emu_last = gi + 1 == groups.size();
    g.emu_gexp = w.gexp;
    g.emu_acc = w.acc;
    g.emu_out = C;
    g.emu_ld_out = ldc;
    g.emu_add = D;
    g.emu_ld_add = ldd;
    g.emu_n = n;
    g.partial = g.emu_last ? partial : nullptr;
    int grid = 0;
    NN_TRY(gemm_tc(st, g, &grid));
    if (g.emu_last && partials != nullptr) *partials = grid;
    if (hw_flops != nullptr) *hw_flops += 2.0 * double(np) * double(np) * double(np) * double(gr.cnt);
  }
  return NN_OK;
}

}  // namespace nn
