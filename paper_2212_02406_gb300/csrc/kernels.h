// Internal launchers shared between the libnn translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/nn.h"

namespace nn {

// Epilogue modes of the GEMM kernels.
enum : int {
  EPI_COPY = 0,      // C = A B
  EPI_RESIDUAL = 1,  // C = I_{n_id} - A B
  EPI_ADD = 2        // C = D + A B
};

// ---- CUDA-core GEMM (gemm_simt.cu) ---------------------------------------------------
template <typename T>
int gemm_simt(cudaStream_t st, int M, int N, int K, const T* A, int64_t lda, const T* B, int64_t ldb, T* C,
              int64_t ldc, int mode, const T* D, int64_t ldd, int n_id, double* partial);
template <typename T>
int gemm_simt_partials(int M, int N);

// ---- tcgen05 GEMM (gemm_tc.cu) --------------------------------------------------------
// C(Np x Np) = sum over segments s of A_s (Np x Np, row-major BF16) * B_s^T, where B_s is
// stored row-major as the TRANSPOSE of the right operand (i.e. each B_s row is one
// column of the right factor, K contiguous). Np must be a multiple of 128.
// Epilogue per element (mode, I restricted to < n_id, addend `add` FP32 row-major ld=Np):
// writes out_f32 (row-major, nullable), `n_row` BF16 pieces row-major and `n_col` BF16
// pieces transposed (column-major = row-major of C^T); partial[cta] = sum C_ij^2 if given.
constexpr int kTcMaxSeg = 6;
struct TcGemmArgs {
  int np = 0;
  int n_id = 0;
  int nseg = 0;
  const __nv_bfloat16* a_seg[kTcMaxSeg] = {};
  const __nv_bfloat16* b_seg[kTcMaxSeg] = {};
  int mode = EPI_COPY;
  const float* add = nullptr;
  float* out_f32 = nullptr;
  __nv_bfloat16* row_pieces[3] = {};
  int n_row = 0;
  __nv_bfloat16* col_pieces[3] = {};
  int n_col = 0;
  double* partial = nullptr;
  int* err = nullptr;
  // FP64-emulation epilogue (emu = true; the BF16/FP32 outputs above unused): the segments are
  // exact-integer slice products of one diagonal group, summed exactly in FP32. The epilogue
  // adds acc * 2^(emu_gexp[0] + emu_gexp[1]) into emu_acc (FP64, Np x Np, ld Np; the first
  // group starts from 0) for rows and columns < emu_n; the last group applies `mode` in FP64
  // (I restricted to < n_id, addend emu_add with ld emu_ld_add) and writes emu_out (ld
  // emu_ld_out) and the partials. emu_gexp: device pair of the operands' global exponents.
  bool emu = false;
  bool emu_first = false, emu_last = false;
  const int* emu_gexp = nullptr;
  double* emu_acc = nullptr;
  double* emu_out = nullptr;
  int64_t emu_ld_out = 0;
  const double* emu_add = nullptr;
  int64_t emu_ld_add = 0;
  int emu_n = 0;
  // Affine epilogue: C' = aff_scale * C + aff_diag * I_{n_id} (FP32), applied after `mode`, before
  // the squares and the outputs.
  bool affine = false;
  float aff_scale = 1.0f, aff_diag = 0.0f;
  // Side copy riding on the epilogue: cvt_dst (FP64, ld cvt_ld) receives cvt_src (FP32, ld Np)
  // widened, for rows and columns < cvt_n (a final FP32 -> FP64 conversion overlapped with a
  // tensor-bound product).
  const float* cvt_src = nullptr;
  double* cvt_dst = nullptr;
  int64_t cvt_ld = 0;
  int cvt_n = 0;
  // FP16 operand pieces (half): both operands of every segment are FP16 and the written pieces
  // too. The accumulator is multiplied by in_scale and, when in_row is given, by in_row[row]
  // (device, one factor per output row) before `mode`; the written pieces hold the result times
  // out_scale (FP32 output, sums of squares and side copy unscaled). All factors are powers of
  // two (exact). BF16 chains leave the defaults.
  bool half = false;
  float in_scale = 1.0f;
  const float* in_row = nullptr;
  float out_scale = 1.0f;
  bool out_r8 = false;  // FP16 pieces written at 8 significant bits (piece_bits)
  // Optional events recorded on the stream immediately before and after the kernel launch (after
  // the host has prepared it), so that their interval is the kernel's device time.
  cudaEvent_t ev_before = nullptr, ev_after = nullptr;
};
int gemm_tc(cudaStream_t st, const TcGemmArgs& a, int* grid_used);
int gemm_tc_max_grid();
// 0: automatic (4 when Np is a multiple of 256, else single-CTA tiles), 1: single-CTA
// tiles, 3: 2-SM MMA, 4: 2-SM MMA with a split last wave (3, 4: NN_ERR_UNSUPPORTED where they
// do not apply).
void gemm_tc_set_variant(int v);
// Arms (on != 0) or disarms the failure-detection test hook for the next launch of an
// instrumented kernel (a tensor-core GEMM, a batched tensor-core class, a sparse ring product);
// tc_take_withhold returns the armed state and disarms it.
void gemm_tc_withhold_next(int on);
int tc_take_withhold();

// ---- FP64 GEMM emulated with exact BF16 slices on the tensor cores (ozaki.cu) -------------
// C (n x n FP64, ldc) = mode(A B): EPI_COPY A B, EPI_RESIDUAL I_{n_id} - A B, EPI_ADD D + A B;
// partial[0 .. *partials) receives per-CTA sums of C_ij^2 when non-null. A, B FP64 n x n
// (lda, ldb). Workspace from emu_workspace_bytes(n); err is the device error word of the
// tensor-core kernel's bounded waits.
size_t emu_workspace_bytes(int64_t n);
// *hw_flops (nullable) is increased by the tensor-core FLOPs issued (2 Np^3 per slice product).
// min_bits > 0 truncates the slice products to a relative error of about 2^-min_bits.
int gemm_f64_emu(cudaStream_t st, int n, const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                 int64_t ldc, int mode, const double* D, int64_t ldd, int n_id, double* partial, int* partials,
                 void* ws, size_t ws_bytes, int* err, double* hw_flops = nullptr, int min_bits = 0);
bool tc_supported();

// ---- conversion / preconditioner / reduction kernels (convert.cu) -----------------------
// Format of written operand pieces: BF16 (half = false) or FP16; each value is multiplied by
// scale and, when row_scale is given, by row_scale[row] (device) before it is cut into pieces
// (powers of two: exact). The FP32 copy and the sums of squares stay unscaled.
struct PieceFmt {
  bool half = false;
  float scale = 1.0f;
  const float* row_scale = nullptr;
  bool r8 = false;  // FP16 pieces at 8 significant bits (piece_bits)
};
// Splits an n x n FP64 matrix (leading dim lds) into an Np-padded FP32 copy and BF16
// pieces (row-major and/or transposed). Any output may be null. Padding is zero.
// sumsq_partial (nullable) receives one sum of squares per 32 x 32 block (split_blocks(np) entries).
// row0, row1: only the padded rows [row0, row1) (multiples of 32; row1 < 0: to Np), e.g. a panel
// of A whose host copy has arrived; the partial sums keep their global positions.
int split_matrix(cudaStream_t st, const double* src, int64_t lds, int n, int np, float* f32,
                 __nv_bfloat16* const* row_pieces, int n_row, __nv_bfloat16* const* col_pieces, int n_col,
                 double* sumsq_partial, int row0 = 0, int row1 = -1, PieceFmt fmt = PieceFmt{});
// The same for scale * src + diag * I (FP64 arithmetic): element-wise products with a scalar
// X_0 (R_0 = I - a A; at depth 1, X_1 = 2 a I - a^2 A).
int split_matrix_affine(cudaStream_t st, const double* src, int64_t lds, int n, int np, float* f32,
                        __nv_bfloat16* const* row_pieces, int n_row, __nv_bfloat16* const* col_pieces, int n_col,
                        double* sumsq_partial, double scale, double diag, PieceFmt fmt = PieceFmt{});
// One pass over src for both: the three row-major pieces of src with its per-block sums of squares
// (as split_matrix), and the outputs of split_matrix_affine for scale * src + diag * I.
// fmt: the affine output's pieces; src_fmt: src's (the same half flag).
int split_matrix_dual(cudaStream_t st, const double* src, int64_t lds, int n, int np,
                      __nv_bfloat16* const* src_row_pieces, double* src_sumsq_partial, float* f32,
                      __nv_bfloat16* const* row_pieces, int n_row, __nv_bfloat16* const* col_pieces, int n_col,
                      double* sumsq_partial, double scale, double diag, int row0 = 0, int row1 = -1,
                      PieceFmt fmt = PieceFmt{}, PieceFmt src_fmt = PieceFmt{});
// BF16 pieces of an FP32 matrix (the same pieces the GEMM epilogue writes for it).
int split_matrix_f32(cudaStream_t st, const float* src, int64_t lds, int n, int np, __nv_bfloat16* const* row_pieces,
                     int n_row, __nv_bfloat16* const* col_pieces, int n_col, PieceFmt fmt = PieceFmt{});
// FP16 row scales of an n x n FP64 matrix, padded rows [row0, row1) of np (row1 < 0: to np):
// scale[i] = 2^e_i with the row's largest |entry| times 2^e_i in [2^13, 2^14), inv[i] = 2^-e_i
// (1 for zero and padding rows).
int row_piece_scales(cudaStream_t st, const double* src, int64_t lds, int n, int np, float* scale, float* inv,
                     int row0 = 0, int row1 = -1);
int split_blocks(int np);
// dst (FP64, ldd) = src (FP32, lds), n x n.
int f32_to_f64(cudaStream_t st, const float* src, int64_t lds, int n, double* dst, int64_t ldd);
// dst (T2, ldd) = src (T1, lds), n x n.
int copy_f64(cudaStream_t st, const double* src, int64_t lds, int n, double* dst, int64_t ldd);
int f64_to_f32(cudaStream_t st, const double* src, int64_t lds, int n, float* dst, int64_t ldd);
// out[0] = ||src||_F for an n x n FP64 matrix (partial must hold >= min(count, 1024) doubles).
int frob_f64(cudaStream_t st, const double* src, int64_t lds, int n, double* partial, int count, double* out);
// out[0] = sqrt(sum partial[0..count)) * scale, fixed summation order.
int reduce_rms(cudaStream_t st, const double* partial, int count, double scale, double* out);
// Preconditioners: write X0 (n x n FP64, ldx). scratch holds >= 4 doubles; vec_scratch
// >= 2n doubles (power iteration of NN_PC_THETA2; may be null for the other kinds).
int precond_fill(cudaStream_t st, const double* A, int64_t lda, int n, int kind, double scalar, double* X0,
                 int64_t ldx, double* scratch, double* vec_scratch);

// ---- dense NN on device buffers (nn_dense.cu), shared with the serving runtime ---------------
int check_opts(const nn_opts* o, int64_t n);
struct HostOut;  // speculative copy of the likely-final iterate to host memory (nn_dense.cu)
int invert_device(const double* A, int64_t n, int64_t lda, const double* X0, int64_t ldx0, const nn_opts* opts,
                  double* X, int64_t ldx, nn_result* res, void* workspace, size_t ws_size, cudaStream_t st,
                  HostOut* ho = nullptr, bool a_presplit = false);

}  // namespace nn
