// Serving runtime: continuous batching of NN inversions and solves on one GPU.
//
// Requests (a dense matrix A, optional right-hand sides B) arrive at any time through
// nn_server_submit. The server allocates no device memory: the caller hands it one device
// arena (the HBM budget), and a first-fit allocator carves every admitted request's buffers
// (A, X_0, X, B, Y and the nn_invert workspace) out of it. A request is admitted as soon as a
// worker slot and enough arena are free, in arrival order, except that a request that does
// not fit yet lets up to kBypass later ones that do go first. Each worker thread owns one
// CUDA stream and runs its request: X_0 from the chosen preconditioner, the NN nest loop of
// nn_invert (one residual read-back per nest), then the solve Y = X B on the device, and the
// copies back to the host. Requests on different workers overlap on the GPU, and a request
// admitted while others run starts as soon as its slot and memory are free.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace nn {
namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, cap) with 256-byte granularity; free blocks coalesce.
class Arena {
 public:
  explicit Arena(size_t cap) : cap_(cap) {
    if (cap) free_[0] = cap;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align_up(std::max<size_t>(bytes, 1), 256);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(std::max<size_t>(bytes, 1), 256);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  size_t cap_;
  size_t used_ = 0;
  std::map<size_t, size_t> free_;
};

size_t request_bytes(int64_t n, int64_t nrhs, int dtype) {
  const size_t ws = nn_workspace_bytes(n, dtype);
  if (ws == 0 || nrhs < 0) return 0;
  const size_t mat = align_up(size_t(n) * size_t(n) * sizeof(double), 256);
  const size_t vec = align_up(size_t(n) * size_t(std::max<int64_t>(nrhs, 1)) * sizeof(double), 256);
  return 3 * mat + 2 * vec + align_up(ws, 256);
}

struct Job {
  nn_request req;
  size_t off = 0;
  size_t bytes = 0;
  double t_submit = 0;
};

}  // namespace
}  // namespace nn

struct nn_server {
  nn_server_opts opts{};
  nn::Arena* arena = nullptr;
  std::mutex mu;
  std::condition_variable cv_work;
  std::condition_variable cv_done;
  std::deque<nn::Job> pending;
  std::deque<nn::Job> admitted;
  std::vector<nn_completion> done;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  int busy = 0;
  bool stop = false;
  int device = 0;
  size_t peak_used = 0;
};

namespace nn {
namespace {

constexpr int kBypass = 8;

// Moves pending requests to the admitted queue while worker slots and arena allow.
// Caller holds s->mu.
void admit_locked(nn_server* s) {
  int slots = s->opts.max_active - s->busy - int(s->admitted.size());
  int skipped = 0;
  for (auto it = s->pending.begin(); it != s->pending.end() && slots > 0 && skipped <= kBypass;) {
    size_t off = 0;
    if (s->arena->alloc(it->bytes, &off)) {
      it->off = off;
      s->admitted.push_back(*it);
      it = s->pending.erase(it);
      --slots;
    } else {
      ++it;
      ++skipped;
    }
  }
  s->peak_used = std::max(s->peak_used, s->arena->used());
  if (!s->admitted.empty()) s->cv_work.notify_all();
}

int run_job(nn_server* s, const Job& j, cudaStream_t st, nn_completion* c) {
  const nn_request& r = j.req;
  const int64_t n = r.n;
  const int64_t nrhs = r.nrhs;
  Carver cv(static_cast<char*>(s->opts.arena) + j.off, j.bytes);
  const size_t e = size_t(n) * size_t(n);
  double* dA = cv.take<double>(e);
  double* dX0 = cv.take<double>(e);
  double* dX = cv.take<double>(e);
  double* dB = cv.take<double>(size_t(n) * size_t(std::max<int64_t>(nrhs, 1)));
  double* dY = cv.take<double>(size_t(n) * size_t(std::max<int64_t>(nrhs, 1)));
  const size_t wsb = nn_workspace_bytes(n, r.dtype);
  void* ws = cv.take<char>(wsb);
  if (!cv.ok) return NN_ERR_OOM_BUDGET;
  NN_CUDA_TRY(cudaMemcpyAsync(dA, r.A, e * sizeof(double), cudaMemcpyHostToDevice, st));
  if (nrhs > 0)
    NN_CUDA_TRY(cudaMemcpyAsync(dB, r.B, size_t(n) * size_t(nrhs) * sizeof(double), cudaMemcpyHostToDevice, st));
  // A scalar X_0 on the mixed chain (the scalar preconditioner, or Theta_1 = I / Tr(A) from the
  // host copy of A) is passed as the x0_scalar hint and never materialised.
  double alpha = 0.0;
  const bool mixed = r.dtype == NN_MIXED_BF16 || r.dtype == NN_MIXED_EMU || r.dtype == NN_MIXED_F16;
  if (mixed && r.precond == NN_PC_SCALAR) alpha = r.pc_scalar;
  if (mixed && r.precond == NN_PC_TRACE) {
    double tr = 0.0;
    for (int64_t i = 0; i < n; ++i) tr += r.A[i * n + i];
    alpha = tr > 0.0 ? 1.0 / tr : 0.0;
  }
  if (!(alpha > 0.0 && std::isfinite(alpha))) {
    alpha = 0.0;
    NN_TRY(nn_init_precond(dA, n, n, r.precond, r.pc_scalar, dX0, n, ws, wsb, st));
  }
  nn_opts o;
  memset(&o, 0, sizeof(o));
  o.depth = s->opts.depth;
  o.tol = s->opts.tol;
  o.max_nests = s->opts.max_nests;
  o.dtype = r.dtype;
  o.x0_scalar = alpha;
  nn_result res;
  memset(&res, 0, sizeof(res));
  const int st_inv = invert_device(dA, n, n, dX0, n, &o, dX, n, &res, ws, wsb, st);
  c->status = st_inv;
  c->nests = res.nests;
  c->residual = res.residual_est;
  // X_0: one reduction for the scalar (trace / Theta_2 power steps / none) and the fill
  const int pc_launches = alpha > 0.0                         ? 0
                          : r.precond == NN_PC_PAN_SCHREIBER ? 3
                          : r.precond == NN_PC_TRACE         ? 2
                          : r.precond == NN_PC_THETA2        ? 3 + int(r.pc_scalar)
                                                             : 1;
  c->launches = pc_launches + res.launches + (nrhs > 0 ? 1 : 0);
  if (st_inv == NN_ERR_CUDA || st_inv == NN_ERR_ARG || st_inv == NN_ERR_UNSUPPORTED || st_inv == NN_ERR_OOM_BUDGET)
    return st_inv;
  if (nrhs > 0) {
    // Solve: Y = X B (B, Y row-major n x nrhs), FP64 on the CUDA cores.
    NN_TRY(gemm_simt<double>(st, int(n), int(nrhs), int(n), dX, n, dB, nrhs, dY, nrhs, EPI_COPY, nullptr, 0, 0,
                             nullptr));
    if (r.Y != nullptr)
      NN_CUDA_TRY(cudaMemcpyAsync(r.Y, dY, size_t(n) * size_t(nrhs) * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  if (r.X != nullptr) NN_CUDA_TRY(cudaMemcpyAsync(r.X, dX, e * sizeof(double), cudaMemcpyDeviceToHost, st));
  NN_CUDA_TRY(cudaStreamSynchronize(st));
  return st_inv;
}

void worker_main(nn_server* s, int wi) {
  cudaSetDevice(s->device);
  cudaStream_t st = s->streams[size_t(wi)];
  for (;;) {
    Job j;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || !s->admitted.empty(); });
      if (s->admitted.empty()) return;  // stop requested and nothing left
      j = s->admitted.front();
      s->admitted.pop_front();
      ++s->busy;
    }
    nn_completion c;
    memset(&c, 0, sizeof(c));
    c.id = j.req.id;
    c.t_submit = j.t_submit;
    c.t_start = now_s();
    const int rc = run_job(s, j, st, &c);
    if (rc != NN_OK && c.status == NN_OK) c.status = rc;
    if (rc == NN_ERR_CUDA || rc == NN_ERR_ARG || rc == NN_ERR_UNSUPPORTED || rc == NN_ERR_OOM_BUDGET) c.status = rc;
    cudaStreamSynchronize(st);
    (void)cudaGetLastError();
    c.t_done = now_s();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->arena->release(j.off, j.bytes);
      --s->busy;
      s->done.push_back(c);
      admit_locked(s);
    }
    s->cv_done.notify_all();
  }
}

}  // namespace
}  // namespace nn

using namespace nn;

extern "C" {

size_t nn_server_request_bytes(int64_t n, int64_t nrhs, int dtype) {
  if (n < 1 || n > 32768 || nrhs < 0) return 0;
  return request_bytes(n, nrhs, dtype);
}

int nn_server_create(const nn_server_opts* opts, nn_server** out) {
  if (opts == nullptr || out == nullptr) return NN_ERR_ARG;
  *out = nullptr;
  if (opts->arena == nullptr || opts->arena_bytes < 256 || opts->max_active < 1 || opts->max_active > 64)
    return NN_ERR_ARG;
  nn_opts probe;
  memset(&probe, 0, sizeof(probe));
  probe.depth = opts->depth;
  probe.tol = opts->tol;
  probe.max_nests = opts->max_nests;
  probe.dtype = NN_F64;
  NN_TRY(check_opts(&probe, 16));
  nn_server* s = new nn_server();
  s->opts = *opts;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    (void)cudaGetLastError();
    return NN_ERR_CUDA;
  }
  s->arena = new Arena(opts->arena_bytes);
  for (int i = 0; i < opts->max_active; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      (void)cudaGetLastError();
      for (auto x : s->streams) cudaStreamDestroy(x);
      delete s->arena;
      delete s;
      return NN_ERR_CUDA;
    }
    s->streams.push_back(st);
  }
  for (int i = 0; i < opts->max_active; ++i) s->workers.emplace_back(worker_main, s, i);
  *out = s;
  return NN_OK;
}

int nn_server_submit(nn_server* s, const nn_request* r) {
  if (s == nullptr || r == nullptr || r->A == nullptr || r->n < 1 || r->nrhs < 0) return NN_ERR_ARG;
  if (r->nrhs > 0 && r->B == nullptr) return NN_ERR_ARG;
  if (r->dtype != NN_F64 && r->dtype != NN_F32 && r->dtype != NN_MIXED_BF16 && r->dtype != NN_MIXED_EMU &&
      r->dtype != NN_MIXED_F16)
    return NN_ERR_ARG;
  if (r->precond < NN_PC_PAN_SCHREIBER || r->precond > NN_PC_THETA2) return NN_ERR_ARG;
  const size_t bytes = request_bytes(r->n, r->nrhs, r->dtype);
  if (bytes == 0) return NN_ERR_ARG;
  if (bytes > s->opts.arena_bytes) return NN_ERR_OOM_BUDGET;  // can never be admitted
  Job j;
  j.req = *r;
  j.bytes = bytes;
  j.t_submit = now_s();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return NN_ERR_ARG;
  s->pending.push_back(j);
  admit_locked(s);
  return NN_OK;
}

int nn_server_poll(nn_server* s, nn_completion* out, int max_out, int* count) {
  if (s == nullptr || count == nullptr || (max_out > 0 && out == nullptr)) return NN_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  const int k = std::min<int>(max_out, int(s->done.size()));
  for (int i = 0; i < k; ++i) out[i] = s->done[size_t(i)];
  s->done.erase(s->done.begin(), s->done.begin() + k);
  *count = k;
  return NN_OK;
}

int nn_server_wait_idle(nn_server* s, double timeout_s) {
  if (s == nullptr) return NN_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9), [&] {
    return s->pending.empty() && s->admitted.empty() && s->busy == 0;
  });
  return ok ? NN_OK : NN_ERR_TIMEOUT;
}

int nn_server_stats(nn_server* s, size_t* arena_used, size_t* arena_peak, int* pending, int* active) {
  if (s == nullptr) return NN_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (arena_used) *arena_used = s->arena->used();
  if (arena_peak) *arena_peak = s->peak_used;
  if (pending) *pending = int(s->pending.size());
  if (active) *active = s->busy + int(s->admitted.size());
  return NN_OK;
}

int nn_server_destroy(nn_server* s) {
  if (s == nullptr) return NN_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->pending.clear();  // not yet admitted: dropped
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto st : s->streams) cudaStreamDestroy(st);
  (void)cudaGetLastError();
  delete s->arena;
  delete s;
  return NN_OK;
}

}  // extern "C"
