// C ABI of the dense Nested Neumann path: workspace sizing, X_0, the nest loop on the
// host (one stream, one synchronisation per nest to read s_k), and the residual call.
//
// Nest k (Theorem, Eq. (nestedneumann) multiplied out on the right; Algorithm 1):
//   R   = I - A X_k                       residual GEMM (+ sum R^2 partials)
//   T   = R;  L-1 times  T = R + R T      Horner GEMMs  (T = R + R^2 + ... + R^L)
//   X_{k+1} = X_k + X_k T                 update GEMM   (= X_k (I + R (I + ... (I + R))))
// The stop test rides on the residual GEMM of the next nest (s_k = ||R||_F / N), so k nests
// cost (L+1) k + 1 GEMMs and the returned X is the iterate whose residual was measured.
#include <math.h>
#include <string.h>

#include <mutex>
#include <utility>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace nn {
namespace {

struct Simt64Ws {
  double* X[2];
  double* R;
  double* T[2];
};
struct Simt32Ws {
  float* A;
  float* X[2];
  float* R;
  float* T[2];
};
struct MixedWs {
  int np;
  // FP16 operand pieces (NN_MIXED_F16): A's pieces carry per-row scales a_scale (inverse a_rinv)
  bool half;
  float* a_scale;
  float* a_rinv;
  double* split_partial;  // one per 32 x 32 block of the split kernel
  double* split_partial2;  // the second set of a two-output split
  __nv_bfloat16* a_row[3];
  float* x32[2];
  __nv_bfloat16* x_row[2][3];
  __nv_bfloat16* x_col[2][3];
  float* r32;
  __nv_bfloat16* r_row[3];
  __nv_bfloat16* r_col[3];
  __nv_bfloat16* t_col[2][3];
};
constexpr size_t kErrOffset = 256, kScalBlock = 512;
struct Common {
  double* partial;
  int n_partial;
  double* scal;  // [0] s, [1..3] preconditioner scratch
  int* err;
};

int partial_capacity(int64_t n, int dtype) {
  if (dtype == NN_F64) return gemm_simt_partials<double>(int(n), int(n));
  if (dtype == NN_F32) return gemm_simt_partials<float>(int(n), int(n)) > gemm_simt_partials<double>(int(n), int(n))
                                  ? gemm_simt_partials<float>(int(n), int(n))
                                  : gemm_simt_partials<double>(int(n), int(n));
  return 1024 > gemm_simt_partials<double>(int(n), int(n)) ? 1024 : gemm_simt_partials<double>(int(n), int(n));
}

void carve_common(Carver& c, int64_t n, int dtype, Common& cm) {
  cm.n_partial = partial_capacity(n, dtype);
  cm.partial = c.take<double>(size_t(cm.n_partial));
  // scal[0..8) and the error word 256 bytes further in one block: one read-back per nest
  cm.scal = c.take<double>(kScalBlock / sizeof(double));
  cm.err = cm.scal == nullptr ? nullptr : reinterpret_cast<int*>(cm.scal + kErrOffset / sizeof(double));
}

void carve_f64(Carver& c, int64_t n, Simt64Ws& w) {
  const size_t e = size_t(n) * size_t(n);
  w.X[0] = c.take<double>(e);
  w.X[1] = c.take<double>(e);
  w.R = c.take<double>(e);
  w.T[0] = c.take<double>(e);
  w.T[1] = c.take<double>(e);
}

void carve_f32(Carver& c, int64_t n, Simt32Ws& w) {
  const size_t e = size_t(n) * size_t(n);
  w.A = c.take<float>(e);
  w.X[0] = c.take<float>(e);
  w.X[1] = c.take<float>(e);
  w.R = c.take<float>(e);
  w.T[0] = c.take<float>(e);
  w.T[1] = c.take<float>(e);
}

void carve_mixed(Carver& c, int64_t n, MixedWs& w, int dtype) {
  w.np = int((n + 127) / 128 * 128);
  w.half = dtype == NN_MIXED_F16;
  const size_t e = size_t(w.np) * size_t(w.np);
  w.a_scale = c.take<float>(size_t(w.np));
  w.a_rinv = c.take<float>(size_t(w.np));
  w.split_partial = c.take<double>(size_t(split_blocks(w.np)));
  w.split_partial2 = c.take<double>(size_t(split_blocks(w.np)));
  for (int i = 0; i < 3; ++i) w.a_row[i] = c.take<__nv_bfloat16>(e);
  for (int b = 0; b < 2; ++b) {
    w.x32[b] = c.take<float>(e);
    for (int i = 0; i < 3; ++i) w.x_row[b][i] = c.take<__nv_bfloat16>(e);
    for (int i = 0; i < 3; ++i) w.x_col[b][i] = c.take<__nv_bfloat16>(e);
    for (int i = 0; i < 3; ++i) w.t_col[b][i] = c.take<__nv_bfloat16>(e);
  }
  w.r32 = c.take<float>(e);
  for (int i = 0; i < 3; ++i) {
    w.r_row[i] = c.take<__nv_bfloat16>(e);
    w.r_col[i] = c.take<__nv_bfloat16>(e);
  }
}

size_t ws_bytes(int64_t n, int dtype) {
  Carver c(nullptr, 0);
  Common cm;
  carve_common(c, n, dtype, cm);
  if (dtype == NN_F64 || dtype == NN_F64_EMU) {
    Simt64Ws w;
    carve_f64(c, n, w);
    if (dtype == NN_F64_EMU) (void)c.take<char>(emu_workspace_bytes(n));
  } else if (dtype == NN_F32) {
    Simt32Ws w;
    carve_f32(c, n, w);
    // nn_residual in FP32 converts X into this space as well
  } else {
    MixedWs w;
    carve_mixed(c, n, w, dtype);
    if (dtype == NN_MIXED_EMU) {
      Simt64Ws w64;
      carve_f64(c, n, w64);
      (void)c.take<char>(emu_workspace_bytes(n));
    }
  }
  return align_up(c.used, 256);
}

bool valid_dtype(int d) {
  return d == NN_F64 || d == NN_F32 || d == NN_MIXED_BF16 || d == NN_F64_EMU || d == NN_MIXED_EMU ||
         d == NN_MIXED_F16;
}

// Reads count (<= 8) doubles from cm.scal and the device error word with one copy (they share
// one block) and one stream synchronisation.
int fetch_scalars(cudaStream_t st, const Common& cm, double* vals, int count, int* dev_err) {
  if (count < 1 || count > 8) return NN_ERR_ARG;
  double blk[kErrOffset / sizeof(double) + 1];
  NN_CUDA_TRY(cudaMemcpyAsync(blk, cm.scal, kErrOffset + sizeof(int), cudaMemcpyDeviceToHost, st));
  NN_CUDA_TRY(cudaStreamSynchronize(st));
  for (int i = 0; i < count; ++i) vals[i] = blk[i];
  memcpy(dev_err, reinterpret_cast<const char*>(blk) + kErrOffset, sizeof(int));
  return NN_OK;
}

// Reads s (and the device error word) back to the host; one stream synchronisation.
int fetch_scalar(cudaStream_t st, const Common& cm, double* s, int* dev_err) {
  return fetch_scalars(st, cm, s, 1, dev_err);
}

// Applies the stop and divergence rules to s_k. Returns -1 to continue, else a status.
int judge(const nn_opts& o, int k, const double* hist) {
  const double s = hist[k];
  if (!isfinite(s)) return NN_ERR_DIVERGED;
  if (k >= 1 && s >= 1.0 && s > hist[k - 1]) return NN_ERR_DIVERGED;
  if (o.tol > 0 && s < o.tol) return NN_OK;
  if (k == o.max_nests) return o.tol > 0 ? NN_ERR_NOT_CONVERGED : NN_OK;
  return -1;
}

// Depth of nest k: the schedule's entry (the last one repeats), else opts.depth.
int nest_depth(const nn_opts& o, int k) {
  if (o.schedule_len <= 0 || o.depth_schedule == nullptr) return o.depth;
  return o.depth_schedule[k < o.schedule_len ? k : o.schedule_len - 1];
}

int max_depth(const nn_opts& o) {
  int d = o.depth;
  if (o.schedule_len > 0 && o.depth_schedule != nullptr) {
    d = 1;
    for (int k = 0; k < o.schedule_len; ++k) d = o.depth_schedule[k] > d ? o.depth_schedule[k] : d;
  }
  return d;
}

void init_result(nn_result* r) {
  memset(r, 0, sizeof(*r));
  r->status = NN_ERR_ARG;
}

// CUDA events around each GEMM launch of a chain (NN_FLAG_TIME_KERNELS).
// Timing events are reused across calls (per device): creating two per GEMM in every call
// cost host time between the launches of a nest.
std::mutex g_ev_mu;
std::vector<std::pair<int, cudaEvent_t>> g_ev_pool;  // (device, event)

int event_take(cudaEvent_t* e) {
  int dev = 0;
  NN_CUDA_TRY(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lock(g_ev_mu);
    for (size_t i = g_ev_pool.size(); i-- > 0;) {
      if (g_ev_pool[i].first == dev) {
        *e = g_ev_pool[i].second;
        g_ev_pool.erase(g_ev_pool.begin() + ptrdiff_t(i));
        return NN_OK;
      }
    }
  }
  NN_CUDA_TRY(cudaEventCreate(e));
  return NN_OK;
}

void event_give(cudaEvent_t e) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    cudaEventDestroy(e);
    return;
  }
  std::lock_guard<std::mutex> lock(g_ev_mu);
  if (g_ev_pool.size() < 4096)
    g_ev_pool.emplace_back(dev, e);
  else
    cudaEventDestroy(e);
}

struct LaunchTimer {
  bool on = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  ~LaunchTimer() {
    for (auto& e : ev) {
      event_give(e.first);
      event_give(e.second);
    }
  }
  int pair(cudaEvent_t* a, cudaEvent_t* b) {
    NN_TRY(event_take(a));
    if (event_take(b) != NN_OK) {
      event_give(*a);
      return NN_ERR_CUDA;
    }
    ev.emplace_back(*a, *b);
    return NN_OK;
  }
  // Events around a whole product (several launches: CUDA-core and emulated FP64 products).
  int begin(cudaStream_t st) {
    if (!on) return NN_OK;
    cudaEvent_t a, b;
    NN_TRY(pair(&a, &b));
    NN_CUDA_TRY(cudaEventRecord(a, st));
    return NN_OK;
  }
  int end(cudaStream_t st) {
    if (!on) return NN_OK;
    NN_CUDA_TRY(cudaEventRecord(ev.back().second, st));
    return NN_OK;
  }
  // A pair of events for the next tensor-core GEMM, recorded by gemm_tc around the launch itself.
  int arm(TcGemmArgs& g) {
    if (!on) return NN_OK;
    cudaEvent_t a, b;
    NN_TRY(pair(&a, &b));
    g.ev_before = a;
    g.ev_after = b;
    return NN_OK;
  }
  // After the stream has been synchronised.
  double total_ms() {
    double t = 0;
    for (auto& e : ev) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) t += ms;
    }
    (void)cudaGetLastError();
    return t;
  }
};

// ---------------------------------------------------------------------------------------
// CUDA-core chains (FP64 / FP32).

// Role of a product in the nest, for arithmetics whose precision can follow it.
enum ProductRole { ROLE_RESIDUAL = 0, ROLE_HORNER = 1, ROLE_UPDATE = 2 };

// The GEMM of a CUDA-core-style chain: C = mode(A B) with Σ C^2 partials (count in *nparts).
template <typename T>
struct SimtGemm {
  cudaStream_t st;
  int n;
  int operator()(const T* A, int64_t lda, const T* B, int64_t ldb, T* C, int64_t ldc, int mode, const T* D,
                 int64_t ldd, double* partial, int* nparts, int /*role*/ = ROLE_RESIDUAL, double /*s_k*/ = 0,
                 double /*need*/ = 0) const {
    if (nparts) *nparts = gemm_simt_partials<T>(n, n);
    return gemm_simt<T>(st, n, n, n, A, lda, B, ldb, C, ldc, mode, D, ldd, n, partial);
  }
};

// FP64 products emulated with exact BF16 slices on the tensor cores (NN_F64_EMU).
struct EmuGemm {
  cudaStream_t st;
  int n;
  void* ws;
  size_t ws_bytes;
  int* err;
  double* hw_flops;
  // adaptive: the products' precision follows the nest's needs (the continuation of
  // NN_MIXED_EMU); otherwise every product is FP64-accurate but the Horner products.
  bool adaptive = false;
  // The Horner product R T_j enters the next residual multiplied by the residual again (about
  // 2^-40 s_k^2 from 40-bit products), so it runs on the slice products of a 40-bit result
  // instead of FP64's. With `adaptive`, `need` is the rms error the nest may add to the next
  // residual (s_k the current one); dropping slice products past b bits perturbs
  //   the Horner product by about 2^-b sqrt(N) s_k^2,
  //   the update X T (T ~ R) by about 2^-b K s_k in the next residual, K = ||A|| ||X|| / N <= 1024,
  // and 8 more bits cover the slices' fixed point relative to row / column maxima.
  int operator()(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int mode,
                 const double* D, int64_t ldd, double* partial, int* nparts, int role = ROLE_RESIDUAL,
                 double s_k = 0, double need = 0) const {
    int bits = role == ROLE_HORNER ? 40 : 0;
    if (adaptive && need > 0 && s_k > 0 && isfinite(s_k)) {
      if (role == ROLE_HORNER) {
        const double b = ceil(log2(16.0 * sqrt(double(n)) * s_k * s_k / need)) + 8.0;
        bits = b < 16 ? 16 : (b > 40 ? 40 : int(b));
      } else if (role == ROLE_UPDATE) {
        const double b = ceil(log2(1024.0 * s_k / need)) + 8.0;
        bits = b < 24 ? 24 : (b >= 54 ? 0 : int(b));
      }
    }
    return gemm_f64_emu(st, n, A, lda, B, ldb, C, ldc, mode, D, ldd, n, partial, nparts, ws, ws_bytes, err,
                        hw_flops, bits);
  }
};

template <typename T, typename Gemm>
int run_simt(cudaStream_t st, int n, const T* A, int64_t lda, T* const X[2], T* R, T* const Tb[2],
             const nn_opts& o, const Common& cm, nn_result* res, int* final_idx, const Gemm& gemm) {
  const double gemm_flops = 2.0 * double(n) * double(n) * double(n);
  LaunchTimer timer;
  timer.on = (o.flags & NN_FLAG_TIME_KERNELS) != 0;
  auto timed = [&](auto&& launch) -> int {
    NN_TRY(timer.begin(st));
    NN_TRY(launch());
    NN_TRY(timer.end(st));
    res->tc_launches += 1;
    res->tc_flops += gemm_flops;
    return NN_OK;
  };
  int cur = 0;
  res->nests = 0;
  for (int k = 0;; ++k) {
    int nparts = 0;
    NN_TRY(timed([&] { return gemm(A, lda, X[cur], n, R, n, EPI_RESIDUAL, nullptr, 0, cm.partial, &nparts); }));
    NN_TRY(reduce_rms(st, cm.partial, nparts, 1.0 / double(n), cm.scal));
    res->gemms += 1;
    res->launches += 2;
    double s = 0;
    int dev_err = 0;
    NN_TRY(fetch_scalar(st, cm, &s, &dev_err));
    res->history[k] = s;
    res->pieces[k] = 0;
    res->nests = k;
    res->residual = s;
    res->residual_est = s;
    const int verdict = judge(o, k, res->history);
    if (verdict >= 0) {
      res->status = verdict;
      break;
    }
    // rms error this nest may add to the next residual: under tol / 16 for the final nest, and
    // under s_{k+1} / 16 ~ s_k^(L+1) / 16 before it (the nests after correct what it adds)
    const int lk = nest_depth(o, k);
    const double need = o.tol > 0 ? fmax(o.tol, pow(s, double(lk + 1))) / 16.0 : 0.0;
    const T* t_cur = R;
    for (int j = 1; j < lk; ++j) {
      T* t_nxt = Tb[j & 1];
      NN_TRY(timed([&] {
        return gemm(R, n, t_cur, n, t_nxt, n, EPI_ADD, R, n, nullptr, nullptr, ROLE_HORNER, s, need);
      }));
      t_cur = t_nxt;
      res->gemms += 1;
      res->launches += 1;
    }
    NN_TRY(timed([&] {
      return gemm(X[cur], n, t_cur, n, X[cur ^ 1], n, EPI_ADD, X[cur], n, nullptr, nullptr, ROLE_UPDATE, s, need);
    }));
    res->gemms += 1;
    res->launches += 1;
    cur ^= 1;
  }
  *final_idx = cur;
  // every timed launch precedes the last residual read-back, which synchronised the stream
  if (timer.on) res->tc_ms = timer.total_ms();
  return NN_OK;
}

// ---------------------------------------------------------------------------------------
// Tensor-core mixed chain.

// Operand-piece pairs (i, j) of a split product with pa pieces of the left operand and pb of
// the right: every pair with i < pa, j < pb and i + j < max(pa, pb) (the terms of the product's
// precision), smallest terms first: (3, 3): (2,0) (1,1) (0,2) (1,0) (0,1) (0,0); (2, 2): (1,0)
// (0,1) (0,0); (2, 1): (1,0) (0,0); (1, 1): (0,0).
int seg_pairs(int pa, int pb, int (*pairs)[2]) {
  const int top = pa > pb ? pa : pb;
  int cnt = 0;
  for (int d = top - 1; d >= 0; --d)
    for (int i = d; i >= 0; --i) {
      const int j = d - i;
      if (i < pa && j < pb && cnt < kTcMaxSeg) {
        pairs[cnt][0] = i;
        pairs[cnt][1] = j;
        ++cnt;
      }
    }
  return cnt;
}

int tc_product(cudaStream_t st, TcGemmArgs& g, int pa, int pb, __nv_bfloat16* const* a_pieces,
               __nv_bfloat16* const* b_pieces, const Common& cm, nn_result* res, int* grid, LaunchTimer* tm) {
  int pairs[kTcMaxSeg][2];
  g.nseg = seg_pairs(pa, pb, pairs);
  for (int s = 0; s < g.nseg; ++s) {
    g.a_seg[s] = a_pieces[pairs[s][0]];
    g.b_seg[s] = b_pieces[pairs[s][1]];
  }
  g.err = cm.err;
  NN_TRY(tm->arm(g));
  NN_TRY(gemm_tc(st, g, grid));
  const double np3 = double(g.np) * double(g.np) * double(g.np);
  res->gemms += 1;
  res->launches += 1;
  res->tc_launches += 1;
  res->hw_flops += 2.0 * np3 * g.nseg;
  res->tc_flops += 2.0 * np3 * g.nseg;
  return NN_OK;
}

// Precision levels of the mixed chain (BF16 pieces per operand):
//   level 1: residual 1 piece,  Horner/update 1 piece   (bulk)
//   level 2: residual 2 pieces, Horner product 1 piece, update 2 pieces of X
//   level 3: residual 3 pieces, Horner product 1 piece, update 2 pieces of X
//   level 4: residual 3 pieces, Horner/update 3 pieces
// Error floors (rms error of a residual measured at the level, with c = ||A||_F ||X_k||_F / N^1.5):
// the pieces leave about 2^-8.8 c (1 piece), 2^-17.9 c (2 pieces), 2^-25 c (3 pieces) -- the
// rounding of N terms of size ~|a_i| |x_j| / N with random signs -- and the tensor core's FP32
// accumulation over K = N adds about 5.4e-10 c N, growing with N (both constants measured on
// GB300 by comparing residuals of an FP64 inverse with FP64 ones, N = 1024..8192, kappa = 1e2
// and 1e4). At N = 8192 the accumulation floor of level 3 equals the piece floor of level 2.
// These floors are systematic for a given A: the chain converges to the X whose measured
// residual vanishes, so a measured s_k falls below the truth, which is about
// sqrt(s_k^2 + e(L')^2) with L' the level of the residual that produced X_k. That estimate
// is what a stop must pass (the certified residual). The top level of a run is the lowest one
// whose floor lies under 0.8 tol; levels above it gain nothing for this tol.
// The chain moves up a level (not past the top one) once s_k < 8 e(L), and when it stalls
// (s_k > 0.9 s_{k-1}) within 30 e(L) of the floor.
// Stability: a product with p pieces perturbs the next residual by about
// 2^-(8p+1) ||A||_2 ||X_k||_2 ||T||_2; once that nears 1 the perturbed residual can reach
// spectral radius 1 in a slowly converging direction and the chain diverges later even though
// s_k still falls. K = ||A||_F ||X_k||_F / N estimates ||A||_2 ||X_k||_2 from below, so the
// level must keep 2^-(8p+1) K * 64 <= 1 (64 covers ||T||_2 <= L+1 and the Frobenius-to-spectral
// gap of the spectra this path is built for).
// Levels never go down.
//
// The update X_k T reads X_k with the level's pieces and T with its own count: T ~ R_k, and
// A X_k ~ I, so T's rounding reaches the next residual unamplified (about 2^-9 s_k for one
// piece), while X_k's is amplified by K; one piece of T (one pass less at levels 2 and 3) stays
// under the next residual wherever s_k is small enough for those levels.
// Compile-time tuning of the schedule (defaults as described above).
#ifndef NN_POLICY_RISE
#define NN_POLICY_RISE 8.0
#endif
#ifndef NN_POLICY_T_MID
#define NN_POLICY_T_MID 1
#endif
#ifndef NN_POLICY_STABLE
#define NN_POLICY_STABLE 64.0
#endif
constexpr double kRise = NN_POLICY_RISE;        // level L < 3 rises once s_k < kRise e(L)
constexpr double kStable = NN_POLICY_STABLE;    // 2^-(8p+1) K kStable <= 1 for the X pieces p
static int level_res_pieces(int L) { return L <= 1 ? 1 : (L == 2 ? 2 : 3); }
// pieces of X_k in the update
static int level_x_pieces(int L) { return L <= 1 ? 1 : (L <= 3 ? 2 : 3); }
// pieces of T (and of R as T_1) that the update reads
static int level_t_pieces(int L) { return L <= 1 ? 1 : (L <= 3 ? NN_POLICY_T_MID : 3); }
// pieces of both operands of the Horner products R T_j (second order in the residual)
static int level_h_pieces(int L) { return (L == 2 || L == 3) ? 1 : level_x_pieces(L); }
// FP16 pieces (half) keep 11 significant bits where BF16 keeps 8: every power of 2^-8 below
// becomes one of 2^-11.
static int stable_level(double kest, bool half) {
  const int b = half ? 11 : 8;
  for (int L = 1; L <= 3; ++L) {
    const int p = level_x_pieces(L);
    if (ldexp(kest, -(b * p + 1)) * kStable <= 1.0) return L;
  }
  return 4;
}
// rms error floor of a residual measured at level L (0: exact, the element-wise R_0). FP16
// pieces: the BF16 piece constants times 2^-3 per piece (the ratio of the two formats' unit
// roundoffs), three pieces beyond FP32 (2^-33). The tensor core's accumulation of FP16 products
// (22 significant bits against BF16's 16) loses more to its alignment: 8.0e-10 c N against
// 5.4e-10 c N. Measured on GB300 with X an FP64 inverse (N = 1024..8192, kappa = 1e2 and 1e4):
// one FP16 piece 2.77-2.84e-4 c (2^-11.8 c); two or three pieces 7.1-7.8e-10 c N at kappa = 1e2,
// 5.9e-10 c N at 1e4, where the accumulation term dominates.
static double level_floor(int L, double c, double n, bool half) {
  if (L <= 0) return 0.0;
  const double pieces = half ? c * (L == 1 ? 0x1.27p-12 : (L == 2 ? 0x1.15p-24 : 0x1p-33))
                             : c * (L == 1 ? 0x1.27p-9 : (L == 2 ? 0x1.15p-18 : 0x1p-25));
  const double acc = (half ? 8.0e-10 : 5.4e-10) * c * n;
  return sqrt(pieces * pieces + acc * acc);
}
// lowest level whose floor lies under 0.8 tol (3 if none does, 1 for tol <= 0)
static int top_level(double tol, double c, double n, bool half) {
  if (!(tol > 0)) return 3;
  for (int L = 1; L <= 3; ++L)
    if (level_floor(L, c, n, half) < 0.8 * tol) return L;
  return 3;
}
// FP16 piece scales: R_k and T_j are scaled by kPieceRT (entries below 16 stay under FP16's
// 65504), X_k by the power of two that puts `bound` (an upper bound of its entries) at or under
// 2^14; 1 for BF16 pieces.
constexpr float kPieceRT = 4096.0f;
static float x_piece_scale(double bound, bool half) {
  if (!half || !(bound > 0) || !isfinite(bound)) return 1.0f;
  int ex = 0;
  (void)frexp(16384.0 / bound, &ex);  // 2^14 / bound in [2^(ex-1), 2^ex): exact, scale-covariant
  int e = ex - 1;
  e = e > 60 ? 60 : (e < -60 ? -60 : e);
  return ldexpf(1.0f, e);
}

// Re-splits X_0 into buffer set 0 (pieces, FP32 master) and its norm into cm.scal[1].
struct X0Source {
  const double* x0;
  int64_t ldx0;
  float scale = 1.0f;  // FP16 piece scale of X_0
};
int load_x0(cudaStream_t st, int n, const MixedWs& w, const Common& cm, const X0Source& src) {
  const int sb = split_blocks(w.np);
  PieceFmt fx;
  fx.half = w.half;
  fx.scale = src.scale;
  NN_TRY(split_matrix(st, src.x0, src.ldx0, n, w.np, w.x32[0], w.x_row[0], 3, w.x_col[0], 3, w.split_partial, 0, -1,
                      fx));
  NN_TRY(reduce_rms(st, w.split_partial, sb, 1.0, cm.scal + 1));
  return NN_OK;
}

}  // namespace

// Host-buffer calls: when a nest is predicted to be the last (s_{k+1} < tol), its new iterate is
// converted to FP64 and copied to the host on a side stream while the confirming residual runs
// on the main stream. If the residual confirms the stop, that copy is the result.
struct HostOut {
  double* host = nullptr;     // caller's host X (row-major, ld n)
  double* dev = nullptr;      // device FP64 X (ld n), the conversion target
  int n = 0;
  cudaStream_t side = nullptr;
  cudaEvent_t ready = nullptr, done = nullptr;
  bool pending = false;       // a side-stream copy was issued and may still run
  int spec_buf = -1;          // x32 buffer that copy reads
  int spec_nests = -1;        // nests applied when it was issued
  bool valid = false;         // set at the end: the copy holds the returned iterate
};

// The caller's device X (FP64), written by the epilogue of a residual product whose iterate is
// predicted to be the last one; buf / nests record which iterate the copy holds (-1: none).
struct DevOut {
  double* X = nullptr;
  int64_t ldx = 0;
  int buf = -1;
  int nests = -1;
};

namespace {

int initial_level(const nn_opts& o) { return (o.bulk_pieces >= 1 && o.bulk_pieces <= 4) ? o.bulk_pieces : 1; }

// r0_pre: R_0 = I - alpha A for the initial level is already in the residual layouts, its
// per-block sums of squares in w.split_partial2 (written by the pass that split A).
int run_mixed(cudaStream_t st, int n, const double* A, int64_t lda, const MixedWs& w, const nn_opts& o,
              const Common& cm, double a_frob, const X0Source& x0src, nn_result* res, int* final_idx, HostOut* ho,
              DevOut* dout, bool r0_pre) {
  const int np = w.np;
  // X_0 = alpha I (the caller's assertion): the first nest's residual R_0 = I - alpha A and update
  // X_1 = alpha (I + T) are element-wise, split straight into the chain's layouts from FP64 A
  // and the FP32 T; the chain's other products are unchanged.
  const bool scalar_x0 = o.x0_scalar > 0;
  const double alpha = o.x0_scalar;
  const int sb = split_blocks(np);
  const double sqrt_n = sqrt(double(n));
  const double n15 = double(n) * sqrt(double(n));
  int level = initial_level(o);
  const int r0_pre_hp = level_t_pieces(level);
  // FP16 pieces: the piece scale of each X buffer (set when its pieces are written), R and T at
  // kPieceRT, A per row (w.a_scale). R and T in one piece (levels 1-3) are written at 8
  // significant bits, as BF16 pieces would be: the Horner product R T_j is second order in the
  // residual and T's rounding reaches the next residual unamplified (about 2^-9 s_k), while X
  // and A, whose rounding the residual and the update amplify, keep all 11 bits. Products with
  // 8-bit operands draw less power at the cap.
  const bool half = w.half;
  const float rt_scale = half ? kPieceRT : 1.0f;
  float xs[2] = {half ? x0src.scale : 1.0f, 1.0f};
  PieceFmt rt_fmt;
  rt_fmt.half = half;
  rt_fmt.scale = rt_scale;
  auto x_fmt = [&](int b) {
    PieceFmt f;
    f.half = half;
    f.scale = xs[b];
    return f;
  };
  auto set_half = [&](TcGemmArgs& g, float in_scale, const float* in_row, float out_scale) {
    g.half = half;
    if (half) {
      g.in_scale = in_scale;
      g.in_row = in_row;
      g.out_scale = out_scale;
    }
  };
  int cur = 0;
  int k = 0;
  bool copy_next = false;  // the next residual's iterate is predicted to be returned
  // BF16 pieces of x32[b] present in x_row[b] / x_col[b]: an update writes only what the next
  // nest's predicted level reads; a later level rise or a rollback regenerates them from the
  // FP32 master (the same pieces).
  int xr[2] = {0, 0}, xc[2] = {0, 0};
  if (!scalar_x0) xr[0] = xc[0] = 3;
  // level of the residual that produced each buffer's iterate (0: X_0, exact)
  int xlev[2] = {0, 0};
  auto ensure_pieces = [&](int b, int need_r, int need_c) -> int {
    if (xr[b] >= need_r && xc[b] >= need_c) return NN_OK;
    NN_TRY(split_matrix_f32(st, w.x32[b], np, n, np, w.x_row[b], 3, w.x_col[b], 3, x_fmt(b)));
    xr[b] = xc[b] = 3;
    res->launches += 1;
    return NN_OK;
  };
  double x_frob = 0;  // ||X_k||_F, read back with s_k
  LaunchTimer timer;
  timer.on = (o.flags & NN_FLAG_TIME_KERNELS) != 0;

  auto residual = [&](int L, double* s_out) -> int {
    const int hp = level_t_pieces(L);
    TcGemmArgs g;
    g.np = np;
    g.n_id = n;
    g.mode = EPI_RESIDUAL;
    // R in FP32 and row pieces feed the Horner GEMMs of nests with depth >= 2
    g.out_f32 = (max_depth(o) >= 2) ? w.r32 : nullptr;
    g.n_row = (max_depth(o) >= 2) ? hp : 0;
    g.n_col = hp;
    for (int i = 0; i < 3; ++i) {
      g.row_pieces[i] = w.r_row[i];
      g.col_pieces[i] = w.r_col[i];
    }
    g.partial = cm.partial;
    if (dout != nullptr && copy_next) {
      // the predicted final residual (a multi-pass, tensor-bound product) also widens X_k into
      // the caller's FP64 X from its epilogue
      g.cvt_src = w.x32[cur];
      g.cvt_dst = dout->X;
      g.cvt_ld = dout->ldx;
      g.cvt_n = n;
      dout->buf = cur;
      dout->nests = k;
    }
    NN_TRY(ensure_pieces(cur, 0, level_res_pieces(L)));
    set_half(g, 1.0f / xs[cur], w.a_rinv, rt_scale);
    g.out_r8 = half && hp == 1;
    int grid = 0;
    NN_TRY(tc_product(st, g, level_res_pieces(L), level_res_pieces(L), w.a_row, w.x_col[cur], cm, res, &grid,
                      &timer));
    NN_TRY(reduce_rms(st, cm.partial, grid, 1.0 / double(n), cm.scal));
    res->launches += 1;
    int dev_err = 0;
    double vals[2];
    NN_TRY(fetch_scalars(st, cm, vals, 2, &dev_err));
    if (dev_err != DEV_OK) return NN_ERR_TIMEOUT;
    *s_out = vals[0];
    x_frob = vals[1];
    return NN_OK;
  };
  auto residual0 = [&](int L, double* s_out) -> int {
    const int hp = level_t_pieces(L);
    const bool rows = max_depth(o) >= 2;
    if (r0_pre && hp == r0_pre_hp) {
      NN_TRY(reduce_rms(st, w.split_partial2, sb, 1.0 / double(n), cm.scal));
      res->launches += 1;
    } else {
      PieceFmt f0 = rt_fmt;
      f0.r8 = half && hp == 1;
      NN_TRY(split_matrix_affine(st, A, lda, n, np, rows ? w.r32 : nullptr, w.r_row, rows ? hp : 0, w.r_col, hp,
                                 w.split_partial, -alpha, 1.0, f0));
      NN_TRY(reduce_rms(st, w.split_partial, sb, 1.0 / double(n), cm.scal));
      res->launches += 2;
    }
    r0_pre = false;  // R's buffers are rewritten from here on
    int dev_err = 0;
    double vals[2];
    NN_TRY(fetch_scalars(st, cm, vals, 2, &dev_err));
    if (dev_err != DEV_OK) return NN_ERR_TIMEOUT;
    *s_out = vals[0];
    x_frob = alpha * sqrt(double(n));  // ||X_0||_F
    return NN_OK;
  };

  int rollbacks = 0;
  bool restarted = false;
  double x_frob_prev = 0;  // ||X_{k-1}||_F, kept for a rollback
  // the residual of X_k at level L (element-wise for k = 0 with a scalar X_0)
  auto measure = [&](int L, double* s_out) -> int {
    return (scalar_x0 && k == 0) ? residual0(L, s_out) : residual(L, s_out);
  };
  for (;; ++k) {
    double s = 0;
    NN_TRY(measure(level, &s));
    // Slow first contraction (s_1 > 0.85 s_0) marks a residual spectrum crowded near 1, i.e.
    // large kappa: there the rounding of BF16 bulk nests, amplified by the (L+1)-fold growth of
    // errors along eigenvalues of R close to 1, can push rho(R) past 1 nests later. Discard
    // the bulk nest and start again from X_0 at level 2 (once).
    if (k == 1 && level == 1 && !restarted && isfinite(s) && s > 0.85 * res->history[0]) {
      if (ho != nullptr && ho->pending) {
        NN_CUDA_TRY(cudaStreamWaitEvent(st, ho->done, 0));
        ho->spec_nests = -1;
      }
      restarted = true;
      cur = 0;
      k = 0;
      level = 2;
      xlev[0] = 0;
      if (!scalar_x0) {
        NN_TRY(load_x0(st, n, w, cm, x0src));
        xr[0] = xc[0] = 3;
        xs[0] = half ? x0src.scale : 1.0f;
        res->launches += 2;
      }
      NN_TRY(measure(level, &s));
    }
    const double c = a_frob * x_frob / n15;
    const double dn = double(n);
    // false: tol lies under what BF16 pieces can certify (the level-3 floor is above 0.8 tol)
    const bool certifiable = !(o.tol > 0) || level_floor(3, c, dn, half) < 0.8 * o.tol;
    // NN_MIXED_EMU hands an uncertifiable tol to emulated nests: level 3 would gain nothing
    const int l_top = (o.dtype == NN_MIXED_EMU && !certifiable) ? 2 : top_level(o.tol, c, dn, half);
    {
      int target = level;
      if (isfinite(s)) {
        const int ls = stable_level(a_frob * x_frob / dn, half);
        if (target < ls) target = ls;
        while (target < l_top && s < kRise * level_floor(target, c, dn, half)) ++target;
        if (k >= 1 && s > 0.9 * res->history[k - 1] && s < 30.0 * level_floor(level, c, dn, half) && level < 4)
          target = target > (level <= 2 ? 3 : 4) ? target : (level <= 2 ? 3 : 4);
        if (o.refine_below > 0 && s * sqrt_n < o.refine_below && target < 3) target = 3;
        if (o.tol > 0 && s < o.tol && target < l_top) target = l_top;
      }
      if (target != level) {
        // The residual epilogue writes R's pieces for the Horner/update GEMMs at the level's
        // count of T pieces, so a change in either count needs a new residual.
        const bool remeasure = level_res_pieces(target) != level_res_pieces(level) ||
                               level_t_pieces(target) != level_t_pieces(level);
        level = target;
        if (remeasure) NN_TRY(measure(level, &s));
      }
    }
    // A nest that made the residual grow below the top level was spoiled by rounding
    // (low-precision updates amplify along slowly converging directions when kappa is
    // large): discard X_k, return to X_{k-1} (still in the other buffer) and continue from
    // there at the top level. NN converges from any X with rho(I - A X) < 1 (Appendix 2).
    if (k >= 1 && level < 4 && rollbacks < 2 && !(s <= res->history[k - 1])) {
      if (ho != nullptr) ho->spec_nests = -1;  // a copy of the discarded iterate is stale
      ++rollbacks;
      cur ^= 1;
      --k;
      x_frob = x_frob_prev;
      level = 4;
      NN_TRY(measure(level, &s));
      x_frob = x_frob_prev;
    }
    res->history[k] = s;
    res->pieces[k] = level_res_pieces(level);
    res->nests = k;
    res->residual = s;
    // the residual X_k has, with the floor of the residual that produced it (certified estimate)
    const double e_fix = level_floor(xlev[cur], c, dn, half);
    const double s_cert = sqrt(s * s + e_fix * e_fix);
    res->residual_est = s_cert;
    int verdict = judge(o, k, res->history);
    if (verdict == NN_OK && o.tol > 0 && !(s_cert < o.tol))
      // measured under tol but not certified: a nest from a residual at the top level certifies
      // it where the top level's floor allows, otherwise the floor blocks
      verdict = (certifiable && k < o.max_nests) ? -1 : NN_ERR_NOT_CONVERGED;
    // At the top level, two nests in a row within 30 floors without a 10% gain: the residual
    // has reached the arithmetic floor, so more nests cannot reach tol.
    if (verdict < 0 && level == 4 && k >= 2 && o.tol > 0 && s > 0.9 * res->history[k - 1] &&
        res->history[k - 1] > 0.9 * res->history[k - 2] && s < 30.0 * level_floor(4, c, dn, half))
      verdict = NN_ERR_NOT_CONVERGED;
    // NN_MIXED_EMU: a tolerance below the BF16-piece floors is reached by emulated FP64 nests;
    // hand the iterate over once the pieces can no longer bring s down (within 4 level-2 floors:
    // level 3 only gains the tensor core's FP32 accumulation floor at twice the passes).
    if (verdict < 0 && o.dtype == NN_MIXED_EMU && !certifiable && s < 4.0 * level_floor(2, c, dn, half))
      verdict = NN_ERR_NOT_CONVERGED;
    // NN_MIXED_BF16 with a tol it cannot certify: once s is under the level-3 floor, more nests
    // lower the measured residual but not the true one (about the floor), so the run ends there.
    if (verdict < 0 && (o.dtype == NN_MIXED_BF16 || o.dtype == NN_MIXED_F16) && !certifiable && level >= 3 &&
        s < level_floor(3, c, dn, half))
      verdict = NN_ERR_NOT_CONVERGED;
    if (verdict >= 0) {
      res->status = verdict;
      break;
    }
    const int hp = level_x_pieces(level), ht = level_t_pieces(level), hh = level_h_pieces(level);
    x_frob_prev = x_frob;
    // Predict s_{k+1} from the observed order-(L+1) contraction,
    // log(s_{k+1}/s_k) ~ (L+1) log(s_k/s_{k-1}), and raise the level of the next residual now
    // if it will fall under this level's floor (or under tol), instead of measuring it at the
    // old level first and again at the new one.
    int next_level = level;
    bool likely_final = false;
    double s_pred = -1.0;
    if (k >= 1 && res->history[k - 1] > 0) {
      const double ratio = s / res->history[k - 1];
      if (ratio > 0 && ratio < 1) {
        // s_k / s_{k-1} = rho^(m_{k-1} L_{k-1}) and s_{k+1} / s_k = rho^(m_k L_k), m_k = m_{k-1} (L_{k-1} + 1)
        const double lp = double(nest_depth(o, k - 1)), lk = double(nest_depth(o, k));
        s_pred = s * pow(ratio, (lp + 1.0) * lk / lp);
        if (level < 3) {
          while (next_level < l_top && s_pred < kRise * level_floor(next_level, c, dn, half)) ++next_level;
          if (o.tol > 0 && s_pred < o.tol && next_level < l_top) next_level = l_top;
        }
        likely_final = o.tol > 0 && s_pred < 0.5 * o.tol && next_level >= l_top &&
                       hypot(s_pred, level_floor(level, c, dn, half)) < 0.9 * o.tol;
      }
    }
    // NN_MIXED_EMU with tol below the BF16 pieces' floor: once X_{k+1} is predicted to lie within
    // 4 level-2 floors, the emulated FP64 nests take X_{k+1} over and measure its residual
    // themselves (no piece residual first). The prediction here is the cautious one: near the
    // ends of a continuous spectrum s_k ~ rho^(m_k) m_k^(-1/2) (m_k the Neumann order + 1), so
    // the geometric extrapolation above is multiplied by
    // exp((ln(L_{k-1} + 1) (L_{k-1} + 1) L_k / L_{k-1} - ln(L_k + 1)) / 2) (3 at depth 2).
    auto predict_slow = [](double s_cur, double s_prev, double lp, double lk) {
      const double ratio = s_cur / s_prev;
      return s_cur * pow(ratio, (lp + 1.0) * lk / lp) *
             exp(0.5 * (log(lp + 1.0) * (lp + 1.0) * lk / lp - log(lk + 1.0)));
    };
    double s_slow = -1.0;
    if (s_pred >= 0) {
      const double lp = double(nest_depth(o, k - 1)), lk = double(nest_depth(o, k));
      s_slow = predict_slow(s, res->history[k - 1], lp, lk);
      // Nest k+1 predicted to be the last one (its iterate X_{k+2} under tol): X_{k+2} is only
      // certified if R_{k+1}, which produces it, runs at the top level.
      if (o.tol > 0 && next_level < l_top && s_slow < s) {
        const double s2 = predict_slow(s_slow, s, lk, double(nest_depth(o, k + 1)));
        if (s2 < 0.5 * o.tol) next_level = l_top;
      }
    }
    const bool handover = o.dtype == NN_MIXED_EMU && !certifiable && s_slow >= 0 &&
                          s_slow < 4.0 * level_floor(2, c, dn, half) && k + 1 < o.max_nests;
    if (handover) likely_final = false;
    // Horner: T_1 = R (its column pieces), T_{j+1} = R + R T_j. With a scalar X_0 the first
    // nest's last Horner product also leaves T in FP32 over R's FP32 copy (each element read as
    // the addend, then written), for the element-wise update below. R T_j is second order in
    // the residual (|R T_j| <= s_k |T_j|), so at levels 2 and 3 one piece less (one pass
    // instead of three) perturbs the next residual by about 2^-9 s_k^2, far under the floors
    // those levels serve; its output T keeps the update's pieces.
    const bool update0 = scalar_x0 && k == 0;
    // pieces of X_{k+1} that the next nest reads at its predicted level (none after a handover:
    // the emulated nests read the FP32 master)
    const int wr = handover ? 0 : level_x_pieces(next_level), wc = handover ? 0 : level_res_pieces(next_level);
    // Before a write to x32[cur ^ 1]: a host side copy must finish reading it, and a copy of
    // it is stale from then on.
    auto before_x_write = [&]() -> int {
      if (ho != nullptr && ho->pending) {
        NN_CUDA_TRY(cudaStreamWaitEvent(st, ho->done, 0));
        if (ho->spec_buf == (cur ^ 1)) ho->spec_nests = -1;
      }
      if (dout != nullptr && dout->buf == (cur ^ 1)) dout->nests = -1;
      return NN_OK;
    };
    // FP16 piece scale of X_{k+1} from ||X_{k+1}||_F <= (1 + ||T||_2) ||X_k||_F, ||T||_2 <= L when
    // ||R_k||_2 < 1 (T = R + ... + R^L)
    const float xs_next = x_piece_scale((1.0 + double(nest_depth(o, k))) * x_frob, half);
    __nv_bfloat16* const* t_cur = w.r_col;
    for (int j = 1; j < nest_depth(o, k); ++j) {
      TcGemmArgs g;
      g.np = np;
      g.n_id = n;
      g.mode = EPI_ADD;
      g.add = w.r32;
      g.n_col = ht;
      for (int i = 0; i < 3; ++i) g.col_pieces[i] = w.t_col[j & 1][i];
      set_half(g, 1.0f / (rt_scale * rt_scale), nullptr, rt_scale);
      g.out_r8 = half && ht == 1;
      int grid = 0;
      if (update0 && j == nest_depth(o, k) - 1) {
        // the first nest's last Horner product writes X_1 = alpha (I + T) straight from its
        // epilogue (FP32 master, row and column pieces, ||X_1||_F): no T, no separate pass
        xs[cur ^ 1] = xs_next;
        g.out_scale = half ? xs_next : 1.0f;
        g.out_r8 = false;  // X keeps every FP16 bit
        g.affine = true;
        g.aff_scale = float(alpha);
        g.aff_diag = float(alpha);
        g.out_f32 = w.x32[cur ^ 1];
        g.n_row = wr;
        g.n_col = wc;
        for (int i = 0; i < 3; ++i) {
          g.row_pieces[i] = w.x_row[cur ^ 1][i];
          g.col_pieces[i] = w.x_col[cur ^ 1][i];
        }
        g.partial = cm.partial;
        NN_TRY(before_x_write());
        xlev[cur ^ 1] = level;
        xr[cur ^ 1] = wr;
        xc[cur ^ 1] = wc;
        NN_TRY(tc_product(st, g, hh, hh, w.r_row, t_cur, cm, res, &grid, &timer));
        NN_TRY(reduce_rms(st, cm.partial, grid, 1.0, cm.scal + 1));
        res->launches += 1;
        break;
      }
      NN_TRY(tc_product(st, g, hh, hh, w.r_row, t_cur, cm, res, &grid, &timer));
      t_cur = w.t_col[j & 1];
    }
    // Update: X_{k+1} = X_k + X_k T, with ||X_{k+1}||_F from the epilogue partials.
    if (update0) {
      // depth 1: T = R_0 = I - alpha A, X_1 = 2 alpha I - alpha^2 A element-wise from FP64 A
      if (nest_depth(o, k) == 1) {
        NN_TRY(before_x_write());
        xlev[cur ^ 1] = level;
        xr[cur ^ 1] = xc[cur ^ 1] = 3;
        xs[cur ^ 1] = xs_next;
        NN_TRY(split_matrix_affine(st, A, lda, n, np, w.x32[cur ^ 1], w.x_row[cur ^ 1], 3, w.x_col[cur ^ 1], 3,
                                   w.split_partial, -alpha * alpha, 2.0 * alpha, x_fmt(cur ^ 1)));
        NN_TRY(reduce_rms(st, w.split_partial, sb, 1.0, cm.scal + 1));
        res->launches += 2;
      }
    } else {
      NN_TRY(ensure_pieces(cur, hp, 0));
      NN_TRY(before_x_write());
      xlev[cur ^ 1] = level;
      xr[cur ^ 1] = wr;
      xc[cur ^ 1] = wc;
      TcGemmArgs g;
      g.np = np;
      g.n_id = n;
      g.mode = EPI_ADD;
      g.add = w.x32[cur];
      g.out_f32 = w.x32[cur ^ 1];
      g.n_row = wr;
      g.n_col = wc;
      for (int i = 0; i < 3; ++i) {
        g.row_pieces[i] = w.x_row[cur ^ 1][i];
        g.col_pieces[i] = w.x_col[cur ^ 1][i];
      }
      g.partial = cm.partial;
      xs[cur ^ 1] = xs_next;
      set_half(g, 1.0f / (xs[cur] * rt_scale), nullptr, xs_next);
      int grid = 0;
      NN_TRY(tc_product(st, g, hp, ht, w.x_row[cur], t_cur, cm, res, &grid, &timer));
      NN_TRY(reduce_rms(st, cm.partial, grid, 1.0, cm.scal + 1));
      res->launches += 1;
    }
    if (ho != nullptr && likely_final) {
      NN_CUDA_TRY(cudaEventRecord(ho->ready, st));
      NN_CUDA_TRY(cudaStreamWaitEvent(ho->side, ho->ready, 0));
      NN_TRY(f32_to_f64(ho->side, w.x32[cur ^ 1], np, n, ho->dev, ho->n));
      NN_CUDA_TRY(cudaMemcpyAsync(ho->host, ho->dev, size_t(ho->n) * size_t(ho->n) * sizeof(double),
                                  cudaMemcpyDeviceToHost, ho->side));
      NN_CUDA_TRY(cudaEventRecord(ho->done, ho->side));
      ho->pending = true;
      ho->spec_buf = cur ^ 1;
      ho->spec_nests = k + 1;
      res->launches += 1;
    }
    cur ^= 1;
    level = next_level;
    copy_next = likely_final;
    if (handover) {
      xr[cur] = xc[cur] = 0;
      res->nests = k + 1;
      res->status = NN_ERR_NOT_CONVERGED;
      break;
    }
  }
  *final_idx = cur;
  if (ho != nullptr && ho->pending) ho->valid = ho->spec_buf == cur && ho->spec_nests == res->nests;
  if (timer.on) {
    NN_CUDA_TRY(cudaStreamSynchronize(st));
    res->tc_ms = timer.total_ms();
  }
  return NN_OK;
}

}  // namespace

// A's BF16 pieces with their per-block sums of squares, for the padded rows [row0, row1) (row1 < 0:
// to Np); with X_0 = alpha I the same pass also writes R_0 = I - alpha A at the starting level.
int split_a_panels(cudaStream_t st, const double* A, int64_t lda, int n, const MixedWs& w, const nn_opts& o, int row0,
                   int row1) {
  // FP16 pieces: each row of A at its own power-of-two scale, R_0 at kPieceRT
  PieceFmt fa, fr;
  fa.half = fr.half = w.half;
  if (w.half) {
    NN_TRY(row_piece_scales(st, A, lda, n, w.np, w.a_scale, w.a_rinv, row0, row1));
    fa.row_scale = w.a_scale;
    fr.scale = kPieceRT;
  }
  if (o.x0_scalar > 0) {
    const int hp = level_t_pieces(initial_level(o));
    const bool rows = max_depth(o) >= 2;
    fr.r8 = w.half && hp == 1;  // R_0 in one piece: 8 significant bits (see run_mixed)
    return split_matrix_dual(st, A, lda, n, w.np, w.a_row, w.split_partial, rows ? w.r32 : nullptr, w.r_row,
                             rows ? hp : 0, w.r_col, hp, w.split_partial2, -o.x0_scalar, 1.0, row0, row1, fr, fa);
  }
  return split_matrix(st, A, lda, n, w.np, nullptr, w.a_row, 3, nullptr, 0, w.split_partial, row0, row1, fa);
}

int check_opts(const nn_opts* o, int64_t n) {
  if (o == nullptr) return NN_ERR_ARG;
  if (o->depth < 1 || o->depth > 16) return NN_ERR_ARG;
  if (o->schedule_len < 0 || o->schedule_len > NN_MAX_HISTORY) return NN_ERR_ARG;
  if (o->schedule_len > 0) {
    if (o->depth_schedule == nullptr) return NN_ERR_ARG;
    for (int k = 0; k < o->schedule_len; ++k)
      if (o->depth_schedule[k] < 1 || o->depth_schedule[k] > 16) return NN_ERR_ARG;
  }
  if (o->max_nests < 0 || o->max_nests > NN_MAX_HISTORY - 1) return NN_ERR_ARG;
  if (!valid_dtype(o->dtype)) return NN_ERR_ARG;
  if (n < 1 || n > 32768) return NN_ERR_ARG;
  if (isnan(o->tol)) return NN_ERR_ARG;
  if (!(o->x0_scalar >= 0.0) || !isfinite(o->x0_scalar)) return NN_ERR_ARG;
  if (!(o->fwd_tol >= 0.0) || !isfinite(o->fwd_tol)) return NN_ERR_ARG;
  return NN_OK;
}

// a_presplit (mixed dtypes): the caller already wrote A's pieces (and, with x0_scalar, R_0) into
// the workspace with split_a_panels, panel by panel as A arrived.
int invert_device(const double* A, int64_t n, int64_t lda, const double* X0, int64_t ldx0, const nn_opts* opts,
                  double* X, int64_t ldx, nn_result* res, void* workspace, size_t ws_size, cudaStream_t st,
                  HostOut* ho, bool a_presplit) {
  // the stop threshold with the forward-error target folded in: N s_k bounds the relative error
  nn_opts o = *opts;
  if (o.fwd_tol > 0) {
    const double t = o.fwd_tol / double(n);
    o.tol = (o.tol > 0 && o.tol < t) ? o.tol : t;
  }
  Carver c(workspace, ws_size);
  Common cm;
  carve_common(c, n, o.dtype, cm);
  NN_CUDA_TRY(cudaMemsetAsync(cm.err, 0, sizeof(int), st));
  const int ni = int(n);
  int fin = 0;
  if (o.dtype == NN_F64 || o.dtype == NN_F64_EMU) {
    Simt64Ws w;
    carve_f64(c, n, w);
    const size_t eb = o.dtype == NN_F64_EMU ? emu_workspace_bytes(n) : 0;
    void* ews = eb ? c.take<char>(eb) : nullptr;
    if (!c.ok) return NN_ERR_OOM_BUDGET;
    NN_TRY(copy_f64(st, X0, ldx0, ni, w.X[0], n));
    if (o.dtype == NN_F64)
      NN_TRY(run_simt<double>(st, ni, A, lda, w.X, w.R, w.T, o, cm, res, &fin, SimtGemm<double>{st, ni}));
    else
      NN_TRY(run_simt<double>(st, ni, A, lda, w.X, w.R, w.T, o, cm, res, &fin,
                              EmuGemm{st, ni, ews, eb, cm.err, &res->hw_flops}));
    NN_TRY(copy_f64(st, w.X[fin], n, ni, X, ldx));
    res->launches += 2;
  } else if (o.dtype == NN_F32) {
    Simt32Ws w;
    carve_f32(c, n, w);
    if (!c.ok) return NN_ERR_OOM_BUDGET;
    NN_TRY(f64_to_f32(st, A, lda, ni, w.A, n));
    NN_TRY(f64_to_f32(st, X0, ldx0, ni, w.X[0], n));
    NN_TRY(run_simt<float>(st, ni, w.A, n, w.X, w.R, w.T, o, cm, res, &fin, SimtGemm<float>{st, ni}));
    NN_TRY(f32_to_f64(st, w.X[fin], n, ni, X, ldx));
    res->launches += 3;
  } else {
    if (!tc_supported()) return NN_ERR_UNSUPPORTED;
    MixedWs w;
    carve_mixed(c, n, w, o.dtype);
    Simt64Ws w64{};
    void* ews = nullptr;
    size_t eb = 0;
    if (o.dtype == NN_MIXED_EMU) {
      carve_f64(c, n, w64);
      eb = emu_workspace_bytes(n);
      ews = c.take<char>(eb);
    }
    if (!c.ok) return NN_ERR_OOM_BUDGET;
    // BF16 pieces of A and X_0, with ||A||_F and ||X_0||_F (for the precision-level floors)
    // from the split kernel's per-block sums of squares
    const int sb = split_blocks(w.np);
    // with X_0 = alpha I the same pass over A also writes R_0 = I - alpha A for the first residual
    const bool r0_pre = o.x0_scalar > 0;
    if (!a_presplit) {
      NN_TRY(split_a_panels(st, A, lda, ni, w, o, 0, -1));
      res->launches += w.half ? 2 : 1;  // FP16: the row scales' pass, then the split
    }
    NN_TRY(reduce_rms(st, w.split_partial, sb, 1.0, cm.scal + 2));
    res->launches += 1;
    X0Source x0src{X0, ldx0};
    if (o.x0_scalar <= 0) {  // a scalar X_0 needs no pieces
      if (w.half) {
        // FP16 pieces of X_0 at the scale that puts ||X_0||_F (>= its entries) under 2^14
        NN_TRY(frob_f64(st, X0, ldx0, ni, cm.partial, cm.n_partial, cm.scal + 3));
        double x0_frob = 0;
        NN_CUDA_TRY(cudaMemcpyAsync(&x0_frob, cm.scal + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
        NN_CUDA_TRY(cudaStreamSynchronize(st));
        x0src.scale = x_piece_scale(x0_frob, true);
        res->launches += 2;
      }
      NN_TRY(load_x0(st, ni, w, cm, x0src));
      res->launches += 2;
    }
    double a_frob = 0;
    NN_CUDA_TRY(cudaMemcpyAsync(&a_frob, cm.scal + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
    NN_CUDA_TRY(cudaStreamSynchronize(st));
    // X written before the run ends must not be read by it (X overlapping A or X_0: no early copy)
    auto span = [&](const double* p, int64_t ld) {
      return std::make_pair(reinterpret_cast<uintptr_t>(p),
                            reinterpret_cast<uintptr_t>(p + (n - 1) * ld + n));
    };
    auto overlaps = [&](std::pair<uintptr_t, uintptr_t> a, std::pair<uintptr_t, uintptr_t> b) {
      return a.first < b.second && b.first < a.second;
    };
    const bool early_ok = !overlaps(span(X, ldx), span(A, lda)) &&
                          (X0 == nullptr || !overlaps(span(X, ldx), span(X0, ldx0)));
    DevOut dout;
    dout.X = X;
    dout.ldx = ldx;
    NN_TRY(run_mixed(st, ni, A, lda, w, o, cm, a_frob, x0src, res, &fin, ho,
                     (ho == nullptr && early_ok) ? &dout : nullptr, r0_pre));
    if (ho != nullptr && ho->pending) NN_CUDA_TRY(cudaStreamWaitEvent(st, ho->done, 0));
    if (o.dtype == NN_MIXED_EMU && res->status == NN_ERR_NOT_CONVERGED && res->nests < o.max_nests) {
      // Continue from the mixed chain's last iterate with emulated FP64 nests (NN converges from
      // any X with rho(I - A X) < 1, Appendix 2): their first residual re-measures s_k exactly.
      if (ho != nullptr) ho->valid = false;
      NN_TRY(f32_to_f64(st, w.x32[fin], w.np, ni, w64.X[0], n));
      nn_opts o2 = o;
      o2.dtype = NN_F64_EMU;
      o2.max_nests = o.max_nests - res->nests;
      o2.depth = nest_depth(o, res->nests);
      o2.depth_schedule = nullptr;
      o2.schedule_len = 0;
      nn_result r2;
      init_result(&r2);
      int fin2 = 0;
      EmuGemm eg{st, ni, ews, eb, cm.err, &res->hw_flops};
      eg.adaptive = true;
      NN_TRY(run_simt<double>(st, ni, A, lda, w64.X, w64.R, w64.T, o2, cm, &r2, &fin2, eg));
      const int k0 = res->nests;
      for (int k = 0; k <= r2.nests && k0 + k < NN_MAX_HISTORY; ++k) {
        res->history[k0 + k] = r2.history[k];
        res->pieces[k0 + k] = 0;
      }
      res->nests = k0 + r2.nests;
      res->residual = r2.residual;
      res->residual_est = r2.residual_est;
      res->status = r2.status;
      res->gemms += r2.gemms;
      res->launches += r2.launches + 2;  // with the widening before and the copy after
      res->tc_launches += r2.tc_launches;
      res->tc_ms += r2.tc_ms;
      res->tc_flops += r2.tc_flops;
      NN_TRY(copy_f64(st, w64.X[fin2], n, ni, X, ldx));
    } else if (ho != nullptr ? !ho->valid : !(dout.buf == fin && dout.nests == res->nests)) {
      NN_TRY(f32_to_f64(st, w.x32[fin], w.np, ni, X, ldx));
      res->launches += 1;
    }
  }
  // Algorithmic work of the method: (L+1) GEMMs per nest plus the final residual, less the
  // products that ran element-wise (X_0 = alpha I on the mixed chains: the first nest's residual
  // and update). Precision passes, re-measured residuals and rolled-back nests are not counted.
  double gemms = 1.0;
  for (int k = 0; k < res->nests; ++k) gemms += double(nest_depth(o, k) + 1);
  if ((o.dtype == NN_MIXED_BF16 || o.dtype == NN_MIXED_EMU || o.dtype == NN_MIXED_F16) && o.x0_scalar > 0)
    gemms -= res->nests >= 1 ? 2.0 : 1.0;
  res->flops = 2.0 * double(n) * double(n) * double(n) * gemms;
  NN_CUDA_TRY(cudaStreamSynchronize(st));
  int dev_err = 0;
  NN_CUDA_TRY(cudaMemcpy(&dev_err, cm.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (dev_err != DEV_OK) {
    res->status = NN_ERR_TIMEOUT;
    return NN_ERR_TIMEOUT;
  }
  return res->status;
}

}  // namespace nn

using namespace nn;

extern "C" {

int nn_debug_withhold_signal(int on) {
  gemm_tc_withhold_next(on);
  return NN_OK;
}

int nn_set_gemm_variant(int variant) {
  if (variant != 0 && variant != 1 && variant != 3 && variant != 4) return NN_ERR_ARG;
  gemm_tc_set_variant(variant);
  return NN_OK;
}

size_t nn_workspace_bytes(int64_t n, int dtype) {
  if (n < 1 || n > 32768 || !valid_dtype(dtype)) return 0;
  return ws_bytes(n, dtype);
}

size_t nn_workspace_bytes_host(int64_t n, int dtype) {
  size_t b = nn_workspace_bytes(n, dtype);
  if (b == 0) return 0;
  // A, X_0, X on the device, plus the preconditioner's scratch (8 + 2n doubles)
  return b + 3 * align_up(size_t(n) * size_t(n) * sizeof(double), 256) +
         align_up(8 * sizeof(double), 256) + align_up(2 * size_t(n) * sizeof(double), 256) + 256;
}

int nn_init_precond(const double* A, int64_t n, int64_t lda, int kind, double scalar, double* X0, int64_t ldx,
                    void* workspace, size_t ws_bytes_, void* stream) {
  if (A == nullptr || X0 == nullptr || n < 1 || n > 32768 || lda < n || ldx < n) return NN_ERR_ARG;
  if (kind < NN_PC_PAN_SCHREIBER || kind > NN_PC_THETA2) return NN_ERR_ARG;
  if (kind == NN_PC_SCALAR && !(scalar > 0)) return NN_ERR_ARG;
  if (kind == NN_PC_THETA2 && !(scalar >= 1 && scalar <= 1024)) return NN_ERR_ARG;
  Carver c(workspace, ws_bytes_);
  Common cm;
  carve_common(c, n, NN_F64, cm);
  double* vec = c.take<double>(size_t(2 * n));
  if (!c.ok) return NN_ERR_OOM_BUDGET;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  NN_TRY(precond_fill(st, A, lda, int(n), kind, kind == NN_PC_JACOBI && scalar == 0 ? 1.0 : scalar, X0, ldx,
                      cm.scal + 1, vec));
  return NN_OK;
}

int nn_invert(const double* A, int64_t n, int64_t lda, const double* X0, int64_t ldx0, const nn_opts* opts,
              double* X, int64_t ldx, nn_result* res, void* workspace, size_t ws_size, void* stream) {
  if (res == nullptr) return NN_ERR_ARG;
  init_result(res);
  NN_TRY(check_opts(opts, n));
  if (A == nullptr || X0 == nullptr || X == nullptr || lda < n || ldx0 < n || ldx < n) return NN_ERR_ARG;
  if (workspace == nullptr || ws_size < nn_workspace_bytes(n, opts->dtype)) return NN_ERR_OOM_BUDGET;
  const int s = invert_device(A, n, lda, X0, ldx0, opts, X, ldx, res, workspace, ws_size,
                              static_cast<cudaStream_t>(stream));
  if (s != res->status) res->status = s;
  return s;
}

}  // extern "C"

namespace nn {
namespace {

// Shared body of the host-buffer entry points: copy A (and X_0 when given) in, build X_0 on the
// device otherwise, run the chain, and return X through the speculative side-stream copy when
// it holds the final iterate.
int invert_host_impl(const double* A_host, int64_t n, const double* X0_host, int pc_kind, double pc_scalar,
                     const nn_opts* opts, double* X_host, nn_result* res, void* workspace, size_t ws_size,
                     void* stream) {
  if (res == nullptr) return NN_ERR_ARG;
  init_result(res);
  NN_TRY(check_opts(opts, n));
  if (A_host == nullptr || X_host == nullptr) return NN_ERR_ARG;
  const size_t need = nn_workspace_bytes_host(n, opts->dtype);
  if (workspace == nullptr || ws_size < need) return NN_ERR_OOM_BUDGET;
  const size_t inner = nn_workspace_bytes(n, opts->dtype);
  Carver c(static_cast<char*>(workspace) + inner, ws_size - inner);
  const size_t e = size_t(n) * size_t(n);
  double* dA = c.take<double>(e);
  double* dX0 = c.take<double>(e);
  double* dX = c.take<double>(e);
  double* pc_scratch = c.take<double>(8);
  double* pc_vec = c.take<double>(2 * size_t(n));
  if (!c.ok) return NN_ERR_OOM_BUDGET;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // a scalar preconditioner on the mixed chain: X_0 = pc_scalar I is never materialised
  nn_opts oh = *opts;
  const bool mixed = opts->dtype == NN_MIXED_BF16 || opts->dtype == NN_MIXED_EMU || opts->dtype == NN_MIXED_F16;
  if (X0_host == nullptr && pc_kind == NN_PC_SCALAR && mixed && pc_scalar > 0) oh.x0_scalar = pc_scalar;
  // Mixed chain, large N: A travels in row panels on a copy stream, and each panel is split into
  // its BF16 pieces (and R_0) as soon as it has arrived, so the split overlaps the copy.
  bool presplit = false;
  if (mixed && n >= 2048 && tc_supported()) {
    Carver cw(workspace, inner);
    Common cmw;
    carve_common(cw, n, oh.dtype, cmw);
    MixedWs ww;
    carve_mixed(cw, n, ww, oh.dtype);  // the same carving as invert_device's
    if (!cw.ok) return NN_ERR_OOM_BUDGET;
    constexpr int kPanels = 8;
    cudaStream_t cs = nullptr;
    cudaEvent_t start = nullptr, ev[kPanels] = {};
    bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&start, cudaEventDisableTiming) == cudaSuccess;
    // the copies start after the work already queued on the caller's stream
    ok = ok && cudaEventRecord(start, st) == cudaSuccess && cudaStreamWaitEvent(cs, start, 0) == cudaSuccess;
    const int rb = ((ww.np / kPanels + 31) / 32) * 32;
    int p = 0;
    for (int r0 = 0; ok && r0 < ww.np && p < kPanels; r0 += rb, ++p) {
      const int r1 = (p == kPanels - 1) ? ww.np : std::min(r0 + rb, ww.np);
      const int64_t h0 = std::min<int64_t>(r0, n), h1 = std::min<int64_t>(r1, n);
      ok = cudaEventCreateWithFlags(&ev[p], cudaEventDisableTiming) == cudaSuccess;
      if (ok && h1 > h0)
        ok = cudaMemcpyAsync(dA + h0 * n, A_host + h0 * n, size_t(h1 - h0) * size_t(n) * sizeof(double),
                             cudaMemcpyHostToDevice, cs) == cudaSuccess;
      ok = ok && cudaEventRecord(ev[p], cs) == cudaSuccess && cudaStreamWaitEvent(st, ev[p], 0) == cudaSuccess;
      ok = ok && split_a_panels(st, dA, n, int(n), ww, oh, r0, r1) == NN_OK;
      res->launches += ww.half ? 2 : 1;
      if (r1 == ww.np) break;
    }
    // On failure, queued copies and splits may still read the caller's A and write the
    // workspace: wait for them (statuses ignored) so that nothing references caller memory after
    // the error returns.
    if (!ok) {
      if (cs) (void)cudaStreamSynchronize(cs);
      (void)cudaStreamSynchronize(st);
    }
    // (destroying a stream or event with work pending releases it once that work is done)
    for (auto& x : ev)
      if (x) cudaEventDestroy(x);
    if (start) cudaEventDestroy(start);
    if (cs) cudaStreamDestroy(cs);
    if (!ok) {
      (void)cudaGetLastError();
      return NN_ERR_CUDA;
    }
    presplit = true;
  } else {
    NN_CUDA_TRY(cudaMemcpyAsync(dA, A_host, e * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  if (X0_host != nullptr) {
    NN_CUDA_TRY(cudaMemcpyAsync(dX0, X0_host, e * sizeof(double), cudaMemcpyHostToDevice, st));
  } else if (!(mixed && oh.x0_scalar > 0 && pc_kind == NN_PC_SCALAR)) {
    NN_TRY(precond_fill(st, dA, n, int(n), pc_kind, pc_scalar, dX0, n, pc_scratch, pc_vec));
    res->launches += 2;
  }
  HostOut ho;
  ho.host = X_host;
  ho.dev = dX;
  ho.n = int(n);
  const bool spec =
      (opts->dtype == NN_MIXED_BF16 || opts->dtype == NN_MIXED_F16) && (opts->tol > 0 || opts->fwd_tol > 0);
  if (spec) {
    NN_CUDA_TRY(cudaStreamCreateWithFlags(&ho.side, cudaStreamNonBlocking));
    if (cudaEventCreateWithFlags(&ho.ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ho.done, cudaEventDisableTiming) != cudaSuccess) {
      if (ho.ready) cudaEventDestroy(ho.ready);
      cudaStreamDestroy(ho.side);
      (void)cudaGetLastError();
      return NN_ERR_CUDA;
    }
  }
  int s = invert_device(dA, n, n, dX0, n, &oh, dX, n, res, workspace, inner, st, spec ? &ho : nullptr, presplit);
  int rc = s;
  if (!(s == NN_ERR_CUDA || s == NN_ERR_ARG || s == NN_ERR_UNSUPPORTED || s == NN_ERR_OOM_BUDGET)) {
    if (!ho.valid && cudaMemcpyAsync(X_host, dX, e * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      rc = NN_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = NN_ERR_CUDA;
  }
  if (spec) {
    if (cudaStreamSynchronize(ho.side) != cudaSuccess && rc == s) rc = NN_ERR_CUDA;
    cudaEventDestroy(ho.ready);
    cudaEventDestroy(ho.done);
    cudaStreamDestroy(ho.side);
  }
  (void)cudaGetLastError();
  return rc;
}

}  // namespace
}  // namespace nn

extern "C" {

int nn_invert_host(const double* A_host, int64_t n, const double* X0_host, const nn_opts* opts, double* X_host,
                   nn_result* res, void* workspace, size_t ws_size, void* stream) {
  if (X0_host == nullptr) {
    if (res != nullptr) init_result(res);
    return NN_ERR_ARG;
  }
  return invert_host_impl(A_host, n, X0_host, 0, 0.0, opts, X_host, res, workspace, ws_size, stream);
}

int nn_invert_host_pc(const double* A_host, int64_t n, int pc_kind, double pc_scalar, const nn_opts* opts,
                      double* X_host, nn_result* res, void* workspace, size_t ws_size, void* stream) {
  if (pc_kind < NN_PC_PAN_SCHREIBER || pc_kind > NN_PC_THETA2 || (pc_kind == NN_PC_SCALAR && !(pc_scalar > 0)) ||
      (pc_kind == NN_PC_THETA2 && !(pc_scalar >= 1 && pc_scalar <= 1024))) {
    if (res != nullptr) init_result(res);
    return NN_ERR_ARG;
  }
  if (pc_kind == NN_PC_JACOBI && pc_scalar == 0) pc_scalar = 1.0;
  return invert_host_impl(A_host, n, nullptr, pc_kind, pc_scalar, opts, X_host, res, workspace, ws_size, stream);
}

int nn_residual(const double* A, int64_t lda, const double* X, int64_t ldx, int64_t n, int dtype, double* rms_frob,
                void* workspace, size_t ws_size, void* stream) {
  if (A == nullptr || X == nullptr || rms_frob == nullptr || n < 1 || n > 32768 || lda < n || ldx < n)
    return NN_ERR_ARG;
  if (dtype != NN_F64 && dtype != NN_F32 && dtype != NN_F64_EMU) return NN_ERR_ARG;
  if (workspace == nullptr || ws_size < nn_workspace_bytes(n, dtype)) return NN_ERR_OOM_BUDGET;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carver c(workspace, ws_size);
  Common cm;
  carve_common(c, n, dtype, cm);
  const int ni = int(n);
  if (dtype == NN_F64) {
    Simt64Ws w;
    carve_f64(c, n, w);
    if (!c.ok) return NN_ERR_OOM_BUDGET;
    NN_TRY(gemm_simt<double>(st, ni, ni, ni, A, lda, X, ldx, w.R, n, EPI_RESIDUAL, nullptr, 0, ni, cm.partial));
    NN_TRY(reduce_rms(st, cm.partial, gemm_simt_partials<double>(ni, ni), 1.0 / double(n), cm.scal));
  } else if (dtype == NN_F64_EMU) {
    Simt64Ws w;
    carve_f64(c, n, w);
    const size_t eb = emu_workspace_bytes(n);
    void* ews = c.take<char>(eb);
    if (!c.ok) return NN_ERR_OOM_BUDGET;
    NN_CUDA_TRY(cudaMemsetAsync(cm.err, 0, sizeof(int), st));
    int nparts = 0;
    NN_TRY(gemm_f64_emu(st, ni, A, lda, X, ldx, w.R, n, EPI_RESIDUAL, nullptr, 0, ni, cm.partial, &nparts, ews, eb,
                        cm.err));
    NN_TRY(reduce_rms(st, cm.partial, nparts, 1.0 / double(n), cm.scal));
  } else {
    Simt32Ws w;
    carve_f32(c, n, w);
    if (!c.ok) return NN_ERR_OOM_BUDGET;
    NN_TRY(f64_to_f32(st, A, lda, ni, w.A, n));
    NN_TRY(f64_to_f32(st, X, ldx, ni, w.X[0], n));
    NN_TRY(gemm_simt<float>(st, ni, ni, ni, w.A, n, w.X[0], n, w.R, n, EPI_RESIDUAL, nullptr, 0, ni, cm.partial));
    NN_TRY(reduce_rms(st, cm.partial, gemm_simt_partials<float>(ni, ni), 1.0 / double(n), cm.scal));
  }
  int dev_err = 0;
  NN_TRY(fetch_scalar(st, cm, rms_frob, &dev_err));
  return NN_OK;
}

}  // extern "C"
