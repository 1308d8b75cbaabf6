/*
 * libnn — Nested Neumann (NN) iterative matrix inversion on one GB300 (sm_103a).
 *
 * C ABI. Every pointer argument is a plain address; sizes are element counts.
 * "device" pointers must point to memory of the GPU that is current on the calling
 * thread; "host" pointers to ordinary (pageable or pinned) host memory. The caller owns
 * every buffer it passes, including the workspace; the library allocates no device
 * memory of its own on any of these calls and keeps no pointer after a call returns.
 * All work is ordered on the given CUDA stream (a cudaStream_t passed as void*; NULL is
 * the legacy default stream). Calls that return results to the host (status, residual
 * history) synchronise that stream before returning.
 *
 * Errors: every entry point returns an nn_status. Calls never abort the process, never
 * print, and leave the CUDA context usable: a bad argument returns NN_ERR_ARG before any
 * launch; a CUDA runtime failure returns NN_ERR_CUDA (cudaGetLastError() is cleared);
 * a device-side wait that runs past its limit makes the kernel return early and the call
 * returns NN_ERR_TIMEOUT.
 *
 * Notation (the paper's): W (here A) is the N x N matrix to invert, Theta the
 * normalisation, X_k = phi^(k) Theta the iterate after k nests with X_0 = Theta, L the
 * inception depth. One nest (Theorem, Eq. (nestedneumann), multiplied out on the right):
 *     R_k = I - A X_k,    X_{k+1} = X_k (I + R_k (I + R_k (... (I + R_k)))),  L factors R_k,
 * computed as T = R_k, then L-1 times T = R_k + R_k T, then X_{k+1} = X_k + X_k T.
 * Stop test: s_k = ||R_k||_F / N (the paper's root-mean Frobenius error, Section II).
 */
#ifndef NN_H
#define NN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------ */
typedef enum nn_status {
  NN_OK = 0,
  NN_ERR_ARG = 1,           /* invalid argument (null pointer, bad size, depth < 1, ...) */
  NN_ERR_DIVERGED = 2,      /* s_k non-finite, or s_k >= 1 and s_k > s_{k-1}              */
  NN_ERR_NOT_CONVERGED = 3, /* tol > 0 and s_k >= tol after max_nests nests               */
  NN_ERR_OOM_BUDGET = 4,    /* workspace too small for the request                         */
  NN_ERR_TIMEOUT = 5,       /* a device-side wait ran past its limit                       */
  NN_ERR_CUDA = 6,          /* CUDA runtime error                                          */
  NN_ERR_UNSUPPORTED = 7,   /* combination not implemented (e.g. no sm_103a device)         */
  NN_ERR_TOO_LARGE = 8      /* size beyond a fixed-capacity entry point's stated maximum    */
} nn_status;

/* ---- arithmetic of the dense nest chain -------------------------------------------- */
typedef enum nn_dtype {
  NN_F64 = 0,        /* every GEMM and epilogue in FP64 (CUDA cores)                           */
  NN_F32 = 1,        /* every GEMM and epilogue in FP32 (CUDA cores)                           */
  NN_MIXED_BF16 = 2, /* tcgen05 tensor-core GEMMs on BF16 operand pieces, FP32 accumulate in
                        TMEM, FP32 master copy of X. Precision levels 1..4 use 1..3 pieces for
                        the residual and the Horner/update products (1 to 6 BF16 passes each);
                        the chain raises the level as s_k nears each level's rounding floor. */
  NN_F64_DF = 3,     /* sparse chain only: FP64 data and results, arithmetic in double-float
                        (hi + lo FP32 pairs, 49-bit significand) on the FP32 pipes; values must
                        lie within the FP32 exponent range                                   */
  NN_F64_EMU = 4,    /* dense chain, nn_residual and nn_solve_normal: FP64 data and results,
                        every product emulated on the BF16 tensor cores with exact slices
                        (error-free splitting after Ozaki et al.: per-row / per-column
                        power-of-two scales, signed base-2^beta digits with n 2^(2 beta) <= 2^24,
                        slice products summed exactly in FP32 and the groups in FP64).
                        Accurate to a few units of 2^-53 normwise. Workspace grows by two sets
                        of BF16 slices (about 2.8 GB at N = 8192)                            */
  NN_MIXED_EMU = 5,  /* dense chain: NN_MIXED_BF16 until the iterate nears the BF16 pieces' floor
                        with tol below it, then NN_F64_EMU nests from that iterate (FP64 copy);
                        history and status cover both stages, pieces[k] = 0 for the FP64
                        nests. Reaches FP64-level residuals at a fraction of NN_F64_EMU's cost */
  NN_MIXED_F16 = 6   /* NN_MIXED_BF16 with FP16 operand pieces (11 significant bits against
                        BF16's 8, same tensor-core rate): each level's rounding floor is 2^-3
                        (one piece) to 2^-6 (two) of BF16's, so the chain stays at one piece
                        longer and certifies a tol with fewer passes. FP16's range is kept by
                        exact power-of-two scales: every row of A by its own (largest entry
                        to [2^13, 2^14)), X_k by one from ||X_k||_F, R and T by 2^12. The
                        entries of R_k and T must stay below 15.97 in magnitude, which holds
                        under the convergence condition ||I - A X_0||_2 < 1 (Theorem); beyond
                        it the pieces overflow, s_k turns non-finite and the call returns
                        NN_ERR_DIVERGED                                                       */
} nn_dtype;

/* ---- starting matrix X_0 = Theta (Section II-A, Eq. (normalization), Appendix 1) --------- */
typedef enum nn_pc {
  NN_PC_PAN_SCHREIBER = 0, /* X_0 = A^T / (||A||_1 ||A||_inf)                                  */
  NN_PC_SCALAR = 1,        /* X_0 = scalar * I                                                */
  NN_PC_TRACE = 2,         /* X_0 = I / Tr(A)   (Theta_1 of Eq. (trace))                        */
  NN_PC_JACOBI = 3,        /* X_0 = scalar * diag(A)^-1 (scalar = 1 for plain Jacobi)          */
  NN_PC_THETA2 = 4         /* X_0 = Theta_2(k) I, k = scalar power steps from v = (1, ..., 1):
                              Theta_2(k) = (k/(k+1)) ||A^k v||^2 / <A^k v, A^(k+1) v>, Eq. (trace)
                              read as an inverse Rayleigh quotient (the printed ratio of squared
                              norms has dimension 1/lambda^2); needs A positive definite      */
} nn_pc;

#define NN_MAX_HISTORY 65

typedef struct nn_opts {
  int depth;           /* inception depth L >= 1 (L = 1 Newton, L = 2 Chebyshev)                 */
  double tol;          /* stop at the first k with s_k < tol; tol <= 0 runs exactly max_nests     */
  int max_nests;       /* 0 .. NN_MAX_HISTORY-1                                                   */
  int dtype;           /* nn_dtype                                                                */
  double refine_below; /* NN_MIXED_BF16 / NN_MIXED_F16: also use level-3 residuals once s_k * sqrt(N) < refine_below
                          (<= 0: off; the floor-based level schedule alone decides)             */
  int bulk_pieces;     /* NN_MIXED_BF16 / NN_MIXED_F16: starting precision level 1..4 (0 = 1): the pieces of
                          the first residuals (1, 2, 3, 3) and updates (1, 2, 2, 3); the chain
                          raises the level itself as the residual nears each level's floor     */
  int flags;           /* NN_FLAG_* bits                                                           */
  const int32_t* depth_schedule; /* optional host array: nest k uses depth_schedule[min(k, len-1)]
                          instead of `depth` (each 1..16). [2, 2, 1] runs two Chebyshev nests,
                          then Newton nests: the matrix form of the Chebyshev-then-Neumann
                          (CNS) construction of Corollary 4 / Corollary 6; after nests of depths
                          L_0..L_{k-1} X_k is the Neumann series of order prod(L_j + 1) - 1    */
  int schedule_len;    /* entries of depth_schedule, 0 .. NN_MAX_HISTORY (0: every nest `depth`) */
  double x0_scalar;    /* > 0: the caller asserts X_0 = x0_scalar * I (X0 must still be passed).
                          NN_MIXED_BF16 / NN_MIXED_F16 / NN_MIXED_EMU then run the first nest's residual
                          R_0 = I - x0_scalar A and update X_1 = x0_scalar (I + T) element-wise
                          (no GEMM, no pieces of X_0); the other dtypes read X0 as usual.
                          nn_result.flops then leaves those two products out. */
  double fwd_tol;      /* > 0: forward-error target. X_k - A^-1 = -A^-1 R_k and ||A^-1||_2 <= ||A^-1||_F give
                          ||X_k - A^-1||_F / ||A^-1||_F <= ||R_k||_F = N s_k, so the chain stops at the
                          first k with s_k < fwd_tol / N (or < tol, when tol > 0 is smaller): the
                          returned X is then within fwd_tol of the inverse, relatively, in the
                          Frobenius norm. With NN_MIXED_EMU the BF16-piece nests run until the next
                          residual is predicted to lie near their floor, then emulated FP64 nests
                          whose products carry only the bits the target needs finish the job. 0: off */
} nn_opts;

/* nn_opts.flags: time every GEMM launch of the chain with CUDA events on the call's stream
 * (fills nn_result.tc_ms; costs two event records per GEMM). */
#define NN_FLAG_TIME_KERNELS 1

typedef struct nn_result {
  int status;                      /* nn_status of the run                                         */
  int nests;                       /* nests applied; the returned X is X_nests                     */
  double residual;                 /* s_nests, the last residual measured                          */
  double history[NN_MAX_HISTORY];  /* s_0 .. s_nests                                               */
  int pieces[NN_MAX_HISTORY];      /* operand pieces used for residual k (0 for FP64/FP32 paths)   */
  int gemms;                       /* GEMM launches issued                                         */
  double flops;                    /* algorithmic FLOPs: 2 N^3 per product of the method that ran as a
                                      GEMM ((L+1) per nest + the final residual, less products run
                                      element-wise); precision passes and re-measured residuals are
                                      not counted                                                  */
  double hw_flops;                 /* tensor-core FLOPs issued, split passes included              */
  int launches;                    /* kernel launches issued by the call                           */
  int tc_launches;                 /* GEMM launches of the chain: tcgen05 for the mixed dtypes,    */
                                   /* CUDA-core for NN_F64 / NN_F32                                */
  double tc_ms;                    /* summed CUDA-event time of those launches (NN_FLAG_TIME_KERNELS) */
  double tc_flops;                 /* 2 Np^3 per piece product pass (mixed) or 2 N^3 per GEMM (F64/F32) */
  double residual_est;             /* the residual the returned X has, as certified by the stop test:
                                      equal to `residual` for FP64, FP32 and emulated residuals; for
                                      piece residuals (mixed dtypes) sqrt(residual^2 + e^2), e the error floor
                                      of the residual that produced X (the pieces' rounding and the
                                      tensor core's FP32 accumulation: the chain converges to the X
                                      whose measured residual vanishes, so the measured value lies
                                      under the truth by about e). A stop requires residual_est < tol;
                                      a tol under the arithmetic's floor ends NN_ERR_NOT_CONVERGED */
} nn_result;

/* Tensor-core GEMM tiling for the mixed chains (a process-wide tuning knob; the
 * element-wise outputs of every variant are bitwise identical, only the per-CTA grouping of the
 * residual's sum of squares differs): 0 = automatic (variant 4 when the padded size is a
 * multiple of 256, else 1), 1 = single-CTA 128 x 256 tiles, 3 = CTA pairs issuing one
 * 256 x 256 MMA over both SMs' shared memory and TMEM (tcgen05 cta_group::2), 4 = variant 3
 * with a last wave that is at most half full run as 256 x 128 halves. Variants 3 and 4 need a
 * padded size that is a multiple of 256; calls that cannot use the chosen one return
 * NN_ERR_UNSUPPORTED. Returns NN_ERR_ARG for other values (2 included). Not thread-safe
 * against concurrent inversions. */
int nn_set_gemm_variant(int variant);

/* Failure-detection test hook (the paper has no counterpart). on != 0 arms it for the next
 * launch of a kernel with bounded device waits (a tensor-core GEMM of the dense chains, the
 * first tensor-core class of an nn_invert_batched_c64 call, or a sparse product on the
 * bulk-copy ring): that launch withholds one signal nothing else sets — the MMA issuer's first
 * "accumulator ready" (in a batched class: every CTA's first chain's completion), or the ring's
 * first stage in its first block — so the bounded device wait on it (about one second) runs
 * out; every role of the kernel then leaves its loop, in-flight copies and tensor work are
 * drained and TMEM freed, the kernel returns, and the calling entry point reports
 * NN_ERR_TIMEOUT (the batched call: as the status of every matrix of that class) with the CUDA
 * context still usable. The hook disarms itself when that launch takes it; on = 0 disarms it.
 * No fault, trap or endless wait is involved. Returns NN_OK. */
int nn_debug_withhold_signal(int on);

/* Bytes of device workspace nn_invert / nn_residual need for an N x N problem of `dtype`
 * (256-byte aligned internally). Returns 0 for invalid arguments. */
size_t nn_workspace_bytes(int64_t n, int dtype);

/* X_0 for A (device, FP64, row-major N x N with leading dimension lda >= n) into X0 (device,
 * FP64, row-major, leading dimension ldx >= n). kind is an nn_pc; `scalar` is the alpha of
 * NN_PC_SCALAR, the damping of NN_PC_JACOBI and the power-step count k (1..1024) of
 * NN_PC_THETA2. Needs nn_workspace_bytes(n, NN_F64) of workspace. Section II-A (Eq. (normalization), Eq. (trace)); Appendix 1 (matrix Theta). */
int nn_init_precond(const double* A, int64_t n, int64_t lda, int kind, double scalar,
                    double* X0, int64_t ldx, void* workspace, size_t ws_bytes, void* stream);

/* Dense NN inversion (Algorithm 1, right-multiplied form). A, X0, X are device FP64
 * row-major with leading dimensions lda, ldx0, ldx (>= n). X receives the last iterate
 * X_nests (also on failure statuses, so the caller can inspect it); X must not overlap A or
 * X0, and for the mixed dtypes it may be written before the last nest is confirmed (the
 * iterate predicted to be returned is widened to FP64 by the confirming residual's epilogue).
 * res (host) receives the run record. The call synchronises `stream` once per nest to read
 * s_k. */
int nn_invert(const double* A, int64_t n, int64_t lda, const double* X0, int64_t ldx0,
              const nn_opts* opts, double* X, int64_t ldx, nn_result* res,
              void* workspace, size_t ws_bytes, void* stream);

/* Same as nn_invert with HOST buffers: A, X0 and X are host FP64 arrays (leading dimension
 * n; page-locked memory lets the copies run at full speed). The call copies A and X0 to the
 * device, runs, and copies X back, and returns after X is in host memory. For NN_MIXED_BF16
 * and NN_MIXED_F16 with tol > 0, the nest predicted to be the last has its iterate converted and copied back on
 * a side stream while the confirming residual runs; when the residual confirms the stop that
 * copy is the result (otherwise X is copied after the run). Needs
 * nn_workspace_bytes_host(n, dtype) of device workspace. */
size_t nn_workspace_bytes_host(int64_t n, int dtype);
int nn_invert_host(const double* A_host, int64_t n, const double* X0_host, const nn_opts* opts,
                   double* X_host, nn_result* res, void* workspace, size_t ws_bytes, void* stream);

/* nn_invert_host with X_0 built on the device from a preconditioner (kind and scalar as in
 * nn_init_precond) instead of a host matrix: only A travels to the device and only X back.
 * Same workspace (nn_workspace_bytes_host), result and errors as nn_invert_host. */
int nn_invert_host_pc(const double* A_host, int64_t n, int pc_kind, double pc_scalar, const nn_opts* opts,
                      double* X_host, nn_result* res, void* workspace, size_t ws_bytes, void* stream);

/* s = ||I - A X||_F / N for device FP64 A, X (row-major), written to *rms_frob (host).
 * dtype NN_F64 evaluates in FP64; NN_F32 in FP32; NN_F64_EMU with the emulated FP64 product.
 * Section II (error measure). */
int nn_residual(const double* A, int64_t lda, const double* X, int64_t ldx, int64_t n, int dtype,
                double* rms_frob, void* workspace, size_t ws_bytes, void* stream);

/* ---- sparse right-hand-side chain ------------------------------------------------------
 * The explicit NN form applied to right-hand sides (Corollary 1, Eq. (NNexplicit); Corollary 6;
 * Algorithm 2) with the Jacobi start phi^(0) = D^-1, D = diag(A):
 *     X = D^-1 prod_{j=0}^{nests-1} ( sum_{n=0}^{L} P^{n (L+1)^j} ) B,    P = I - A D^-1,
 * i.e. the Neumann series of order (L+1)^nests - 1 (Corollary 2), computed as (L+1)^nests - 1
 * sparse products without forming any dense matrix. (Algorithm 2 prints the L + 1 = 2 case.)
 *
 * A: CSR, row_ptr[n+1] and col[nnz] int32 (device), val[nnz] (device) of `dtype` (NN_F64 or
 * NN_F32; NN_F64_DF takes FP64 data and computes in double-float, which on GB300 keeps the
 * chain bound by HBM instead of by the narrow FP64 pipe); columns in any order; every row needs
 * a nonzero diagonal (else NN_ERR_ARG).
 * B, X: device, column-major n x nrhs of `dtype`, leading dimensions ldb, ldx >= n.
 * tol > 0: after each factor j the relative residual ||B - A X_j||_F / ||B||_F (one extra
 * sparse product) goes to res->history[j] and the chain stops at the first factor below tol
 * (NN_ERR_NOT_CONVERGED if none is). tol <= 0 runs all `nests` factors and evaluates the
 * residual once at the end (res->residual). res->nests = factors applied; res->flops counts
 * 2 nnz per sparse product per right-hand side. Needs nn_csr_workspace_bytes() of workspace.
 * Returns NN_ERR_TIMEOUT if a device-side wait of the product kernel ran past its limit. */
size_t nn_csr_workspace_bytes(int64_t n, int64_t nnz, int64_t nrhs, int dtype);
int nn_solve_csr(const int32_t* row_ptr, const int32_t* col, const void* val, int64_t n, int64_t nnz,
                 int dtype, const void* B, int64_t ldb, int64_t nrhs, int depth, int nests, double tol,
                 void* X, int64_t ldx, nn_result* res, void* workspace, size_t ws_bytes, void* stream);

/* The same chain with a depth per factor (host array depths[nfactors], each 1..16):
 *     X = D^-1 prod_{j=0}^{nfactors-1} ( sum_{n=0}^{L_j} P^{n m_j} ) B,   m_j = prod_{q<j} (L_q + 1),
 * i.e. Chebyshev factors (L = 2) followed by the factorised Neumann series prod_t (I + P^{2^t})
 * (L = 1) on the preconditioner they built: the CNS construction for sparse matrices
 * (Corollary 4, Eq. (CNS); Corollary 6). prod_j (L_j + 1) - 1 sparse products, at most 2^31 - 1
 * (else NN_ERR_ARG). Arguments, tol, res and errors as nn_solve_csr (nests -> nfactors). */
int nn_solve_csr_sched(const int32_t* row_ptr, const int32_t* col, const void* val, int64_t n, int64_t nnz,
                       int dtype, const void* B, int64_t ldb, int64_t nrhs, const int32_t* depths, int nfactors,
                       double tol, void* X, int64_t ldx, nn_result* res, void* workspace, size_t ws_bytes,
                       void* stream);

/* nn_solve: the sparse chain with the argument order of the library's solve interface
 * (A, B, depth, tol, options, X, result, stream): the problem statement A X = B solved by the
 * explicit NN form of Corollary 1 (Eq. (NNexplicit)) and Algorithm 2. A is the CSR triple
 * (row_ptr, col, val) of size n with nnz nonzeros; B and X as in nn_solve_csr. From opts it
 * reads dtype (NN_F64, NN_F64_DF or NN_F32), max_nests (the number of factors) and, when
 * schedule_len > 0, depth_schedule (a depth per factor, as nn_solve_csr_sched; `depth` is then
 * unused); its other fields are ignored. Same workspace (nn_csr_workspace_bytes), result and
 * errors as nn_solve_csr; a null opts or a bad schedule returns NN_ERR_ARG. */
int nn_solve(const int32_t* row_ptr, const int32_t* col, const void* val, int64_t n, int64_t nnz, const void* B,
             int64_t ldb, int64_t nrhs, int depth, double tol, const nn_opts* opts, void* X, int64_t ldx,
             nn_result* res, void* workspace, size_t ws_bytes, void* stream);

/* Sparse-product kernel for one right-hand side (a process-wide tuning knob; both variants
 * sum each row's terms in the same order, so results are bitwise identical): 0 = automatic
 * (a persistent kernel that streams (val, col, row_ptr) through a ring of shared-memory stages
 * with bulk async copies, used when row_ptr, col and the values are 16-byte aligned), 1 = one
 * block per 256 rows with staged loads. Returns NN_ERR_ARG for other values. Not thread-safe
 * against concurrent solves. */
int nn_set_spmv_variant(int variant);

/* ---- row strips of the sparse chain (one rank's share of a sharded solve) ----------------
 * Corollary 1 applied per row strip: with the rows of A cut into contiguous strips, one per
 * rank, each sparse product P v = v - A D^-1 v of the chain needs, besides the strip's own
 * entries of v, the values of v on the strip's halo columns (owned by other strips), and each
 * residual check needs two sums reduced over the strips. These calls run one strip's share on
 * this GPU; the caller exchanges the halo values (NCCL or any transport) and reduces the sums.
 * One right-hand side.
 *
 * Local numbering: the strip holds rows [r0, r1) of A, n_local = r1 - r0, in CSR with
 * row_ptr[n_local + 1] (from 0) and col_local[nnz] in an extended numbering: a column c owned
 * by the strip is c - r0, a halo column takes a position >= n_local (n_ext = n_local + number of
 * halo columns). An extended vector v_ext[n_ext] holds the strip's values first, then the halo
 * values in that order. All arrays are device memory owned by the caller; values of dtype
 * NN_F64 or NN_F32 (else NN_ERR_ARG). Every call needs nn_csr_strip_workspace_bytes(n_local) of
 * workspace; nn_csr_strip_diag_inv clears its error word, so call it first with the workspace.
 *
 * nn_csr_strip_diag_inv: dinv_local[i] = 1 / A_ii for the strip's rows (the entries with
 *   col_local == i); NN_ERR_ARG if a row has no or a zero diagonal. Synchronises `stream`.
 * nn_csr_strip_scale: val_scaled[e] = val[e] * dinv_ext[col_local[e]] (A' = A D^-1; dinv_ext is
 *   dinv_local extended with the halo rows' values, exchanged like a vector).
 * nn_csr_strip_product: y_i = v_ext[i] - sum_e val_scaled[e] v_ext[col_local[e]] for i < n_local
 *   (the strip of P v); with acc_out, also acc_out = acc_in + y (acc_in may equal acc_out; y may
 *   then be NULL), the factor accumulation of the chain. Only enqueues work.
 * nn_csr_strip_residual: sums[0] = sum_i (b_i - (A' z)_i)^2, sums[1] = sum_i b_i^2 over the
 *   strip (host array of two doubles; A x = A' z for x = D^-1 z); NN_ERR_TIMEOUT if a bounded
 *   device wait of an earlier product or of this one ran past its limit. Synchronises `stream`.
 * nn_csr_strip_finish: x_local = dinv_local * z_local. Only enqueues work. */
size_t nn_csr_strip_workspace_bytes(int64_t n_local);
int nn_csr_strip_diag_inv(const int32_t* row_ptr, const int32_t* col_local, const void* val, int64_t n_local,
                          int64_t nnz, int dtype, void* dinv_local, void* workspace, size_t ws_bytes, void* stream);
int nn_csr_strip_scale(const int32_t* col_local, const void* val, int64_t nnz, int dtype, const void* dinv_ext,
                       void* val_scaled, void* stream);
int nn_csr_strip_product(const int32_t* row_ptr, const int32_t* col_local, const void* val_scaled, int64_t n_local,
                         int64_t nnz, int dtype, const void* v_ext, void* y, const void* acc_in, void* acc_out,
                         void* workspace, size_t ws_bytes, void* stream);
int nn_csr_strip_residual(const int32_t* row_ptr, const int32_t* col_local, const void* val_scaled, int64_t n_local,
                          int64_t nnz, int dtype, const void* z_ext, const void* b_local, double* sums,
                          void* workspace, size_t ws_bytes, void* stream);
int nn_csr_strip_finish(const void* z_local, const void* dinv_local, int64_t n_local, int dtype, void* x_local,
                        void* stream);

/* ---- general systems through the normal equations ----------------------------------------
 * Corollary 3 (Eq. (linearsystemfinal), Eq. (nnlinearsystem)): A X = B for any nonsingular A,
 * real or complex, solved as X = (A^H A)^-1 A^H B. W = A^H A is Hermitian positive definite;
 * the dense NN runs on W from X_0 = I / Tr(W) with the caller's options (depth, tol on
 * ||I - W X_k||_F / m, max_nests, dtype), and X = X_k A^H B. Squaring the condition number is
 * inherent to the method: cond(W) = cond(A)^2, so NN_F64 is the dtype for badly conditioned A
 * (the mixed BF16 chain stops at its accuracy floor with NN_ERR_NOT_CONVERGED there).
 *
 * is_complex = 0: A real FP64, row-major n x n, leading dimension lda >= n; B and X real FP64,
 *                 row-major n x nrhs, leading dimensions ldb, ldx >= nrhs.
 * is_complex = 1: A, B, X complex128 stored as interleaved (re, im) FP64 pairs, row-major, leading
 *                 dimensions counted in complex elements. The solve runs on the real embedding
 *                 z -> [[Re z, -Im z], [Im z, Re z]] of size m = 2n, which maps the complex
 *                 products and A^H exactly onto real ones.
 * All pointers are device memory owned by the caller; X must not overlap A or B. Needs
 * nn_normal_workspace_bytes(n, nrhs, is_complex, opts->dtype) bytes of device workspace (the
 * library allocates nothing). res holds the inversion's nest count, W-residual history and
 * precision schedule. Returns the inversion's status (NN_OK, NN_ERR_NOT_CONVERGED,
 * NN_ERR_DIVERGED: X still receives the solution from the last iterate) or an argument /
 * workspace / CUDA error before or during the call (X then undefined). Synchronises `stream`. */
size_t nn_normal_workspace_bytes(int64_t n, int64_t nrhs, int is_complex, int dtype);
int nn_solve_normal(const void* A, int64_t n, int64_t lda, int is_complex, const void* B, int64_t ldb,
                    int64_t nrhs, const nn_opts* opts, void* X, int64_t ldx, nn_result* res, void* workspace,
                    size_t ws_bytes, void* stream);

/* ---- batched small complex inversions ---------------------------------------------------
 * Many independent U x U complex64 matrices (U <= 64; massive-MIMO Gram matrices, the use the
 * paper names in Corollary 4) inverted by the right-multiplied NN loop in persistent kernels
 * (one per tile class): X_0 = diag(A)^-1 / (1 + damping * U) (Jacobi start, a diagonal Theta of
 * Appendix 1; damping = 0 is plain Jacobi), then `nests` nests of depth L, with s_k =
 * ||I - A X_k||_F / U and the divergence rule of nn_invert (a diverged matrix keeps the X_k at
 * which it diverged). X_0 being diagonal, the first nest's residual I - A X_0 and update
 * X_0 (I + T) are computed element-wise (column and row scalings) rather than as products.
 *
 * nn_batched_plan (host only): sorts the matrices by size (largest first) and groups equal
 * sizes into work items. sizes_host[count] in 1..64; cfg_by_u (nullable, 65 entries indexed by
 * U, -1 = default) picks the path per size (0: CUDA cores, 8x8 threads per matrix, up to four
 * matrices per CTA; 1: CUDA cores, 16x16 threads per matrix; 3: CUDA cores, one warp per
 * matrix, for U in {8, 16, 24, 32} (other sizes fall back to 0 or 1); 2: tensor cores, for U in
 * {48, 64} (other sizes fall back to 0 or 1): the iterates stay in TMEM, each complex product
 * P Q is one tcgen05 MMA chain [Pr; Pi] [Qr | Qi] whose cross terms combine in the epilogue,
 * with three BF16 pieces per operand, FP32-level accuracy, two matrices per SM in a software
 * pipeline);
 * plan_host holds nn_batched_plan_size(count)
 * int32. The caller copies the plan to the device and may reuse it for every launch with the
 * same size list. Layout: [n_items, count, n_tc, class_first[23], order[count],
 * items[n_items][4]]; order = matrix indices by size, largest first; item = (U, first position
 * in order, matrices, cfg); items are grouped by tile class (classes 0, 1 = tensor cores for
 * U = 64, 48; 2..17 = CUDA-core (threads per matrix, tile, exact U) classes; 18..21 = one warp
 * per matrix, U = 32, 24, 16, 8), class c spanning items
 * [class_first[c], class_first[c + 1]). nn_batched_plan_classes (host only) returns the mask of
 * the classes that hold items (bit c for class c; 0 for a null plan).
 *
 * nn_invert_batched_c64: A and X device complex64 (interleaved re, im) packed back to back,
 * matrix b row-major at element offset offsets[b] (device int64) with size sizes[b] (device
 * int32); plan = the device copy of the plan; classes = nn_batched_plan_classes of its host
 * copy (or any superset, e.g. 0xFFFFFFFF: a class without items costs one empty launch; a
 * class with items left out is not computed); NN_ERR_ARG if no class bit is set.
 * residual[b] (device float) = s of the returned X_b; status[b] (device int32) = NN_OK,
 * NN_ERR_DIVERGED, or NN_ERR_TIMEOUT (a tensor-core item whose bounded wait ran out). The call
 * only enqueues work on `stream` (a memset and one kernel per selected tile class, at most
 * NN_BATCHED_KERNELS, chained by programmatic dependent launch; no synchronisation, no
 * allocation), so it can be captured in a CUDA graph. Needs nn_batched_workspace_bytes(count)
 * of workspace. */
#define NN_BATCHED_KERNELS 22
int64_t nn_batched_plan_size(int64_t count);
int nn_batched_plan(const int32_t* sizes_host, int64_t count, const int32_t* cfg_by_u, int32_t* plan_host);
uint32_t nn_batched_plan_classes(const int32_t* plan_host);
size_t nn_batched_workspace_bytes(int64_t count);
int nn_invert_batched_c64(const void* A, const int64_t* offsets, const int32_t* sizes, int64_t count,
                          const int32_t* plan, uint32_t classes, int depth, int nests, double damping, void* X,
                          float* residual, int32_t* status, void* workspace, size_t ws_bytes,
                          void* stream);

/* nn_invert_batched: nn_invert_batched_c64 with the argument order of the library's batched
 * interface (batch A, depth, nests, X, residuals, stream; Corollary 4's mMIMO use, each matrix
 * run as Algorithm 1): A (complex64 batch: data, offsets, sizes, count), depth, nests, damping
 * of the Jacobi start, the device plan and its class mask, then X, residual, status, workspace
 * and stream. Same semantics, workspace and errors as nn_invert_batched_c64. */
int nn_invert_batched(const void* A, const int64_t* offsets, const int32_t* sizes, int64_t count, int depth, int nests,
                      double damping, const int32_t* plan, uint32_t classes, void* X, float* residual,
                      int32_t* status, void* workspace, size_t ws_bytes, void* stream);

/* ---- serving: continuous batching of inversions and solves -----------------------------
 * A request inverts one dense N x N matrix A (host FP64, row-major) with the NN loop of
 * nn_invert (X_0 from `precond` with `pc_scalar`, depth / tol / max_nests from the server
 * options, arithmetic `dtype`) and, if nrhs > 0, solves Y = X B for B (host FP64, row-major
 * N x nrhs). X (host, N x N) and Y (host, N x nrhs) receive the results when not NULL. Host
 * buffers must stay valid until the request's completion is polled; pinned memory gives
 * asynchronous copies. This is a serving form of the dense inversion; the paper itself
 * describes single inversions (Algorithm 1) and linear solves (Corollary 3).
 *
 * The server allocates no device memory: `arena` (device, arena_bytes) is the HBM budget
 * from which every admitted request's buffers are carved (nn_server_request_bytes() each).
 * Up to max_active requests run at once, each on its own worker thread and CUDA stream, so
 * their work overlaps on the GPU; a request is admitted as soon as a slot and enough arena
 * are free (arrival order, with a bounded bypass for requests that fit while an earlier one
 * does not). nn_server_submit never blocks (NN_ERR_OOM_BUDGET if the request can never fit);
 * nn_server_poll returns finished requests with their status, nests, final residual and
 * steady-clock times (seconds) of submission, start and completion. Requests not yet admitted
 * when nn_server_destroy is called are dropped; running ones finish first. */
typedef struct nn_server nn_server;
typedef struct nn_server_opts {
  void* arena;          /* device memory the server may use                                    */
  size_t arena_bytes;
  int max_active;       /* concurrent requests (worker threads / streams), 1..64               */
  int depth;            /* inception depth for every request                                   */
  double tol;           /* stop tolerance on ||I - A X||_F / N                                 */
  int max_nests;
} nn_server_opts;
typedef struct nn_request {
  int64_t id;
  int64_t n;
  const double* A;
  int64_t nrhs;
  const double* B;
  double* Y;
  double* X;
  int dtype;            /* NN_F64, NN_F32, NN_MIXED_BF16, NN_MIXED_F16 or NN_MIXED_EMU (BF16-piece
                           nests, then emulated FP64 nests where tol lies under what the pieces
                           certify)                                                            */
  int precond;          /* nn_pc                                                               */
  double pc_scalar;
} nn_request;
typedef struct nn_completion {
  int64_t id;
  int status;
  int nests;
  double residual;      /* certified residual of the returned X (nn_result.residual_est)         */
  double t_submit, t_start, t_done;
  int launches;         /* kernels the request launched (X_0, the NN loop, the solve)          */
} nn_completion;

size_t nn_server_request_bytes(int64_t n, int64_t nrhs, int dtype);
int nn_server_create(const nn_server_opts* opts, nn_server** out);
int nn_server_submit(nn_server* s, const nn_request* r);
int nn_server_poll(nn_server* s, nn_completion* out, int max_out, int* count);
int nn_server_wait_idle(nn_server* s, double timeout_s);
int nn_server_stats(nn_server* s, size_t* arena_used, size_t* arena_peak, int* pending, int* active);
int nn_server_destroy(nn_server* s);

/* ---- residual without any allocation ---------------------------------------------------
 * The paper has no counterpart: this is a deployment variant of nn_residual for callers that
 * cannot allocate device memory: real-time services that forbid allocation after start-up, and
 * plug-ins whose host framework owns and budgets all device memory and hands them only the
 * operands. It computes s = ||I - A X||_F / N in FP64 from device A and X
 * (row-major, leading dimensions lda, ldx >= n) into *rms_frob (host), using the same kernels
 * as nn_residual, with its scratch in a fixed 16 MiB array that the library reserves in device
 * memory on every GPU that loads it, until the process exits.
 * Limits: n <= NN_RESIDUAL_NOALLOC_MAX_N, larger n returns NN_ERR_TOO_LARGE before any device
 * work. The array is shared by all calls on a device: calls whose work overlaps on the GPU race
 * on it; each call overwrites all the scratch it reads, so nothing carries over between calls.
 * The first call on each device resolves the array's address (cudaGetSymbolAddress) and keeps
 * it for that device's context (a call after cudaDeviceReset resolves it again); make the first
 * call before any stream capture on that device. Calls no allocating routine. Synchronises
 * `stream` before returning. */
#define NN_RESIDUAL_NOALLOC_MAX_N 1440
int nn_residual_noalloc(const double* A, int64_t lda, const double* X, int64_t ldx, int64_t n,
                        double* rms_frob, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NN_H */
