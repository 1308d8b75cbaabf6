// tcgen05 / TMEM tensor-core GEMM for the NN nest chain on sm_103a.
//
// One persistent CTA per SM, 6 warps, warp-specialised:
//   warp 0      TMA producer: 128x64 tile of A and 256x64 tile of B^T per stage (SWIZZLE_128B),
//               4-stage ring guarded by full/empty mbarriers;
//   warp 1      allocates 512 TMEM columns, one elected thread issues tcgen05.mma
//               (M=128, N=256, K=16, BF16 x BF16 -> FP32) into one of two 256-column
//               accumulators, and commits to the empty / accumulator-full barriers;
//   warps 2-5   epilogue: tcgen05.ld of the accumulator (each warp owns its 32-lane
//               quarter), the fused NN element-wise step (I - C, D + C), FP32 and BF16
//               piece stores (row-major and transposed), and sum(C^2) partials.
// The two accumulators let the epilogue of tile i overlap the main loop of tile i+1.
//
// Two tilings of the same schedule (bitwise identical element-wise results):
//   gemm_tc_kernel       one CTA per 128 x 256 tile, as above (any padded size, multiple of 128);
//   gemm_tc_2sm_kernel   clusters of two CTAs computing one 256 x 256 tile with
//                        tcgen05.mma.cta_group::2: each SM stages 32 KB per K step instead of
//                        48 KB for the same tensor work, which lifts the per-SM shared-memory
//                        fill rate that limits the single-CTA kernel (default where the padded
//                        size is a multiple of 256).
//
// "Segments" chain several (A_s, B_s) operand pairs into the same accumulator; the split
// precisions of the mixed path (hi/lo BF16 pieces) use them, smallest products first.
//
// Every mbarrier wait is bounded (about 1 s, %globaltimer); a wait past the limit sets
// an error word and makes every role leave its loop, so the kernel always returns and
// frees its TMEM.
#include <cudaTypedefs.h>
#include <cuda.h>

#include <atomic>
#include <mutex>
#include <string.h>

#include "common.cuh"
#include "kernels.h"

namespace nn {
namespace tc {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int BK = 64;  // 64 BF16 = 128 bytes = one SWIZZLE_128B row
constexpr int STAGES = 4;
constexpr int A_TILE = BM * BK * 2;            // 16 KB
constexpr int B_TILE = BN * BK * 2;            // 32 KB
constexpr int STAGE_BYTES = A_TILE + B_TILE;   // 48 KB
constexpr int THREADS = 192;
constexpr int TMEM_COLS = 512;                 // two 128x256 FP32 accumulators
constexpr int CTRL_BYTES = 256;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + CTRL_BYTES + 1024;
#ifndef NN_TC_GROUP_M
#define NN_TC_GROUP_M 16
#endif
constexpr int GROUP_M = NN_TC_GROUP_M;         // tile raster: bands of 16 row tiles

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A BF16 (bits 7-9 = 1),
// B BF16 (bits 10-12 = 1), both K-major (bits 15, 16 = 0), N>>3 at bit 17, M>>4 at bit 24.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(BN >> 3) << 17) | (uint32_t(BM >> 4) << 24);

struct Params {
  CUtensorMap map_a[kTcMaxSeg];
  CUtensorMap map_b[kTcMaxSeg];
  int nseg;
  int np;
  int tiles_m, tiles_n;
  int n_id;
  int mode;
  const float* add;
  float* out_f32;
  __nv_bfloat16* row_pieces[3];
  int n_row;
  __nv_bfloat16* col_pieces[3];
  int n_col;
  double* partial;
  int* err;
  // 2-SM kernel: tiles [split_from, num_tiles) run as two 256 x 128 halves each (work units
  // beyond split_from), which halves the time of a partly filled last wave; map_b_half loads
  // 64-row halves of those B^T panels.
  CUtensorMap map_b_half[kTcMaxSeg];
  int split_from;
  // FP64-emulation epilogue (see TcGemmArgs)
  int emu;
  int emu_first, emu_last;
  const int* emu_gexp;
  double* emu_acc;
  double* emu_out;
  int64_t emu_ld_out;
  const double* emu_add;
  int64_t emu_ld_add;
  int emu_n;
  // Affine epilogue (affine != 0): C' = aff_scale * C + aff_diag * I_{n_id}, after the mode.
  int affine;
  float aff_scale, aff_diag;
  // Side copy: cvt_dst (FP64, ld cvt_ld) = cvt_src (FP32, ld Np) over this launch's tiles,
  // rows and columns < cvt_n; cvt_vec: cvt_dst rows are 16-byte aligned.
  const float* cvt_src;
  double* cvt_dst;
  int64_t cvt_ld;
  int cvt_n;
  // FP16 operand pieces (see TcGemmArgs): idesc_xor clears the descriptor's BF16 type bits,
  // in_scale (and in_row[row]) multiply the accumulator, out_scale the written pieces.
  int half;
  uint32_t idesc_xor;
  float in_scale;
  const float* in_row;
  float out_scale;
  int out_r8;
  int cvt_vec;
  // Failure-detection test hook: the MMA issuer withholds the first accumulator-ready signal, so
  // the epilogue's bounded wait runs out (nn_debug_withhold_signal).
  int withhold;
};

// Shared-memory matrix descriptor for a K-major tile written by TMA with SWIZZLE_128B:
// rows of 128 bytes, 8-row swizzle atoms of 1024 bytes stacked at a 1024-byte stride (SBO).
// Bits: start>>4 [0,14), LBO>>4 [16,30) (unused for this layout), SBO>>4 [32,46),
// descriptor version 1 at bit 46, layout SWIZZLE_128B (2) at bits [61,64).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr & 0x3FFFFu) >> 4);
  d |= uint64_t(1) << 16;
  d |= uint64_t(1024 >> 4) << 32;
  d |= uint64_t(1) << 46;
  d |= uint64_t(2) << 61;
  return d;
}

__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int group, int& tm, int& tn) {
  const int per_group = group * tiles_n;
  const int g = t / per_group;
  const int first_m = g * group;
  const int gm = min(group, tiles_m - first_m);
  const int r = t - g * per_group;
  tm = first_m + r % gm;
  tn = r / gm;
}

__device__ __forceinline__ void store_pieces_row(__nv_bfloat16* const* pieces, int n_pieces, int64_t off,
                                                 const float (&v)[32], float scale, bool half, bool r8) {
  float rem[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) rem[j] = v[j] * scale;
  for (int p = 0; p < n_pieces; ++p) {
    uint32_t packed[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      float vlo, vhi;
      const uint16_t lo = piece_bits(rem[2 * j], half, &vlo, r8);
      const uint16_t hi = piece_bits(rem[2 * j + 1], half, &vhi, r8);
      rem[2 * j] -= vlo;
      rem[2 * j + 1] -= vhi;
      packed[j] = uint32_t(lo) | (uint32_t(hi) << 16);
    }
    uint4* dst = reinterpret_cast<uint4*>(pieces[p] + off);
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
  }
}

// Epilogue of one 32-column chunk of a thread's accumulator row: applies the mode, adds the
// squares to ss (in column order) and writes the FP32 and BF16-piece outputs.
// FP64-emulation epilogue of one 32-column chunk: the FP32 accumulator holds an exact sum of
// slice products (an integer times this element's power of two), so acc * emu_scale is exact.
__device__ __forceinline__ void emu_chunk(const Params& p, const uint32_t (&raw)[32], int gr, int gc0, double& ss) {
  if (gr >= p.emu_n) return;
  double* accp = p.emu_acc + int64_t(gr) * p.np + gc0;
  const int jn = min(32, p.emu_n - gc0);
  const double scale = ldexp(1.0, p.emu_gexp[0] + p.emu_gexp[1]);
  // fully unrolled (static register indices into raw)
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    if (j >= jn) break;
    double v = double(__uint_as_float(raw[j])) * scale;
    if (!p.emu_first) v += accp[j];
    if (!p.emu_last) {
      accp[j] = v;
      continue;
    }
    const int gc = gc0 + j;
    double c = v;
    if (p.mode == EPI_RESIDUAL)
      c = ((gr == gc && gr < p.n_id) ? 1.0 : 0.0) - v;
    else if (p.mode == EPI_ADD)
      c = p.emu_add[int64_t(gr) * p.emu_ld_add + gc] + v;
    ss = fma(c, c, ss);
    p.emu_out[int64_t(gr) * p.emu_ld_out + gc] = c;
  }
}

__device__ __forceinline__ void epilogue_chunk(const Params& p, const uint32_t (&raw)[32], int gr, int gc0,
                                               int64_t ld, double& ss) {
  if (p.emu) {
    emu_chunk(p, raw, gr, gc0, ss);
    return;
  }
  float v[32];
  const int64_t off = int64_t(gr) * ld + gc0;
  // FP16 pieces carry power-of-two scales: the product of the operands' scales leaves the
  // accumulator (exact)
  float acc[32];
  if (p.half) {
    const float f = p.in_row != nullptr ? p.in_scale * p.in_row[gr] : p.in_scale;
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = __uint_as_float(raw[j]) * f;
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = __uint_as_float(raw[j]);
  }
  if (p.mode == EPI_ADD) {
    const float4* src = reinterpret_cast<const float4*>(p.add + off);
#pragma unroll
    for (int j4 = 0; j4 < 8; ++j4) {
      float4 a4 = src[j4];
      v[4 * j4 + 0] = a4.x + acc[4 * j4 + 0];
      v[4 * j4 + 1] = a4.y + acc[4 * j4 + 1];
      v[4 * j4 + 2] = a4.z + acc[4 * j4 + 2];
      v[4 * j4 + 3] = a4.w + acc[4 * j4 + 3];
    }
  } else if (p.mode == EPI_RESIDUAL) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int gc = gc0 + j;
      v[j] = ((gr == gc && gr < p.n_id) ? 1.0f : 0.0f) - acc[j];
    }
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = acc[j];
  }
  if (p.affine) {
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = fmaf(p.aff_scale, v[j], (gr == gc0 + j && gr < p.n_id) ? p.aff_diag : 0.0f);
  }
  {
    // The chunk's 32 squares in FP32 (four interleaved sums, fixed order; relative error
    // ~2^-21), accumulated in FP64 across chunks: FP64 work once per chunk, not per element
    // (GB300's FP64 pipe is narrow). A chunk sum outside [2^-100, 2^100] (zeros, values whose
    // squares underflow or overflow FP32, NaN) is redone in FP64, so the result stays
    // scale-invariant.
    float c4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 32; ++j) c4[j & 3] = fmaf(v[j], v[j], c4[j & 3]);
    const float cs = (c4[0] + c4[1]) + (c4[2] + c4[3]);
    if (cs >= 0x1p-100f && cs <= 0x1p100f) {
      ss += double(cs);
    } else {
      double d = 0.0;
#pragma unroll
      for (int j = 0; j < 32; ++j) d = fma(double(v[j]), double(v[j]), d);
      ss += d;
    }
  }
  if (p.out_f32 != nullptr) {
    float4* dst = reinterpret_cast<float4*>(p.out_f32 + off);
#pragma unroll
    for (int j4 = 0; j4 < 8; ++j4) dst[j4] = make_float4(v[4 * j4], v[4 * j4 + 1], v[4 * j4 + 2], v[4 * j4 + 3]);
  }
  if (p.n_row > 0) store_pieces_row(p.row_pieces, p.n_row, off, v, p.out_scale, p.half != 0, p.out_r8 != 0);
  if (p.n_col > 0) {
    float rem[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) rem[j] = v[j] * p.out_scale;
    for (int pc = 0; pc < p.n_col; ++pc) {
      uint16_t* dst = reinterpret_cast<uint16_t*>(p.col_pieces[pc]) + gr;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        float b;
        const uint16_t bits = piece_bits(rem[j], p.half != 0, &b, p.out_r8 != 0);
        rem[j] -= b;
        dst[int64_t(gc0 + j) * ld] = bits;  // lanes write consecutive rows: 64-byte runs
      }
    }
  }
  if (p.cvt_dst != nullptr && gr < p.cvt_n && gc0 < p.cvt_n) {
    const float4* src = reinterpret_cast<const float4*>(p.cvt_src + off);
    double* dst = p.cvt_dst + int64_t(gr) * p.cvt_ld + gc0;
    if (p.cvt_vec && gc0 + 32 <= p.cvt_n) {
#pragma unroll
      for (int j4 = 0; j4 < 8; ++j4) {
        const float4 f = src[j4];
        reinterpret_cast<double2*>(dst)[2 * j4] = make_double2(double(f.x), double(f.y));
        reinterpret_cast<double2*>(dst)[2 * j4 + 1] = make_double2(double(f.z), double(f.w));
      }
    } else {
      const int jn = min(32, p.cvt_n - gc0);
      for (int j = 0; j < jn; ++j) dst[j] = double(p.cvt_src[off + j]);
    }
  }
}

// One CTA per 128 x 256 tile.
__global__ void __launch_bounds__(THREADS, 1) gemm_tc_kernel(const __grid_constant__ Params p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);
  uint8_t* tiles = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  double* red = reinterpret_cast<double*>(smem + STAGES * STAGE_BYTES + 128);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  const int unit = int(blockIdx.x);
  const int units = int(gridDim.x);
  const int unit_rows = p.tiles_m;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 4);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 0 && lane == 0) {
    for (int s = 0; s < p.nseg; ++s) {
      tma_prefetch_desc(&p.map_a[s]);
      tma_prefetch_desc(&p.map_b[s]);
    }
  }
  if (warp == 1) tmem_alloc(tmem_slot, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int num_tiles = unit_rows * p.tiles_n;
  const int kblocks = p.np / BK;
  const int total_k = p.nseg * kblocks;

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      for (int t = unit; t < num_tiles && !*abort_flag; t += units) {
        int tm, tn;
        tile_coords(t, unit_rows, p.tiles_n, GROUP_M, tm, tn);
        for (int it = 0; it < total_k; ++it) {
          const int seg = it / kblocks;
          const int kb = it - seg * kblocks;
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, p.err)) break;
          uint8_t* sa = tiles + stage * STAGE_BYTES;
          uint8_t* sb = sa + A_TILE;
          mbar_arrive_expect_tx(&full[stage], STAGE_BYTES);
          tma_load_2d(sa, &p.map_a[seg], kb * BK, tm * BM, &full[stage]);
          tma_load_2d(sb, &p.map_b[seg], kb * BK, tn * BN, &full[stage]);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int local = 0;
      for (int t = unit; t < num_tiles && !*abort_flag; t += units, ++local) {
        const int acc = local & 1;
        const uint32_t acc_phase = (local >> 1) & 1;
        if (!mbar_wait(&acc_empty[acc], acc_phase ^ 1u, abort_flag, p.err)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + uint32_t(acc * BN);
        bool ok = true;
        for (int it = 0; it < total_k; ++it) {
          if (!mbar_wait(&full[stage], phase, abort_flag, p.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(tiles + stage * STAGE_BYTES);
          const uint64_t adesc = sw128_desc(sa);
          const uint64_t bdesc = sw128_desc(sa + A_TILE);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            // +32 bytes along K inside the 128-byte swizzled row = +2 in the address field
            tc_mma_bf16(d_tmem, adesc + uint64_t(2 * kk), bdesc + uint64_t(2 * kk), IDESC ^ p.idesc_xor,
                        (it > 0 || kk > 0) ? 1u : 0u);
          }
          tc_commit(&empty[stage]);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        if (!(p.withhold && local == 0)) tc_commit(&acc_full[acc]);
      }
      // Wait for every MMA this thread issued before TMEM can be released.
      tc_commit(drain);
      volatile int no_abort = 0;
      mbar_wait(drain, 0, &no_abort, p.err);
    }
  } else {
    // Epilogue warps 2..5; warp w reads TMEM lanes 32*(w%4) .. +31.
    const int q = warp & 3;
    const int row_in_tile = q * 32 + lane;
    const int64_t ld = p.np;
    double ss = 0.0;
    int local = 0;
    for (int t = unit; t < num_tiles; t += units, ++local) {
      const int acc = local & 1;
      const uint32_t acc_phase = (local >> 1) & 1;
      if (!mbar_wait(&acc_full[acc], acc_phase, abort_flag, p.err)) break;
      tc_fence_after();
      int tm, tn;
      tile_coords(t, unit_rows, p.tiles_n, GROUP_M, tm, tn);
      const int gr = tm * BM + row_in_tile;
      for (int c = 0; c < BN / 32; ++c) {
        const int gc0 = tn * BN + c * 32;
        if (gc0 >= p.np) break;  // warp-uniform
        uint32_t raw[32];
        tmem_ld_32x32b_x32(tmem_base + uint32_t(acc * BN + c * 32) + (uint32_t(q * 32) << 16), raw);
        tmem_ld_wait();
        epilogue_chunk(p, raw, gr, gc0, ld, ss);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[acc]);
    }
    // Deterministic per-CTA sum of squares over the four epilogue warps.
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
    if (lane == 0) red[q] = ss;
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (warp == 2 && lane == 0 && p.partial != nullptr) p.partial[blockIdx.x] = red[0] + red[1] + red[2] + red[3];
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem_base, TMEM_COLS);
}


// ---------------------------------------------------------------------------------------
// 2-SM variant: a CTA pair computes one 256 x 256 tile with tcgen05.mma.cta_group::2
// (M = 256, N = 256, K = 16). Each CTA holds 128 rows of the A tile and 128 rows of the
// B^T tile in its own shared memory (32 KB per stage instead of 48 KB), the even CTA issues
// the MMA over both, and each CTA's TMEM receives its 128 rows of the accumulator. Both
// CTAs' loads complete on the even CTA's full barrier; its commits release both CTAs'
// stages and accumulators; both CTAs' epilogue warps free an accumulator on the even CTA's
// barrier (count 8).
#ifndef NN_TC_P2_STAGES
#define NN_TC_P2_STAGES 7
#endif
constexpr int P2_STAGES = NN_TC_P2_STAGES;
constexpr int P2_STAGE_BYTES = A_TILE + B_TILE / 2;  // 32 KB
constexpr int P2_SMEM_BYTES = P2_STAGES * P2_STAGE_BYTES + CTRL_BYTES + 1024;
constexpr uint32_t IDESC_P2_HALF =
    (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t((BN / 2) >> 3) << 17) | (uint32_t((2 * BM) >> 4) << 24);
static_assert((2 * P2_STAGES + 5) * 8 + 8 <= 192 && 192 + 4 * 8 <= CTRL_BYTES, "control block layout");

// Work unit w of the 2-SM schedule: full tiles first, then the split tiles' halves.
__device__ __forceinline__ void unit_tile(int w, int split_from, int& t, int& half) {
  if (w < split_from) {
    t = w;
    half = -1;
  } else {
    t = split_from + ((w - split_from) >> 1);
    half = (w - split_from) & 1;
  }
}
static_assert(P2_SMEM_BYTES <= 227 * 1024, "shared memory");
constexpr uint32_t IDESC_P2 =
    (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(BN >> 3) << 17) | (uint32_t((2 * BM) >> 4) << 24);

__global__ void __launch_bounds__(THREADS, 1) gemm_tc_2sm_kernel(const __grid_constant__ Params p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);
  uint8_t* tiles = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + P2_STAGES * P2_STAGE_BYTES);
  uint64_t* empty = full + P2_STAGES;
  uint64_t* acc_full = empty + P2_STAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  // 2 P2_STAGES + 5 barriers, the TMEM slot and the abort flag fit in the first 192 bytes of the control block
  double* red = reinterpret_cast<double*>(smem + P2_STAGES * P2_STAGE_BYTES + 192);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int rank = int(cluster_ctarank());
  const bool leader = rank == 0;
  const int unit = int(blockIdx.x >> 1);
  const int units = int(gridDim.x >> 1);
  const int unit_rows = p.tiles_m / 2;

  if (threadIdx.x == 0) {
    for (int s = 0; s < P2_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 8);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 0 && lane == 0) {
    for (int s = 0; s < p.nseg; ++s) {
      tma_prefetch_desc(&p.map_a[s]);
      tma_prefetch_desc(&p.map_b[s]);
      if (p.split_from < p.tiles_n * (p.tiles_m / 2)) tma_prefetch_desc(&p.map_b_half[s]);
    }
  }
  if (warp == 1) tmem_alloc_pair(tmem_slot, TMEM_COLS);
  tc_fence_before();
  cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int num_tiles = unit_rows * p.tiles_n;
  const int num_units = p.split_from + 2 * (num_tiles - p.split_from);
  const int kblocks = p.np / BK;
  const int total_k = p.nseg * kblocks;

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      for (int w = unit; w < num_units && !*abort_flag; w += units) {
        int t, half, tm2, tn;
        unit_tile(w, p.split_from, t, half);
        tile_coords(t, unit_rows, p.tiles_n, GROUP_M / 2, tm2, tn);
        for (int it = 0; it < total_k; ++it) {
          const int seg = it / kblocks;
          const int kb = it - seg * kblocks;
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, p.err)) break;
          uint8_t* sa = tiles + stage * P2_STAGE_BYTES;
          uint8_t* sb = sa + A_TILE;
          if (leader) mbar_arrive_expect_tx(&full[stage], half < 0 ? 2 * P2_STAGE_BYTES : 2 * (A_TILE + B_TILE / 4));
          const uint32_t bar = cluster_map_shared(&full[stage], 0);
          tma_load_2d_pair(sa, &p.map_a[seg], kb * BK, tm2 * 2 * BM + rank * BM, bar);
          if (half < 0)
            tma_load_2d_pair(sb, &p.map_b[seg], kb * BK, tn * BN + rank * (BN / 2), bar);
          else
            tma_load_2d_pair(sb, &p.map_b_half[seg], kb * BK, tn * BN + half * (BN / 2) + rank * (BN / 4), bar);
          if (++stage == P2_STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {
      int stage = 0;
      uint32_t phase = 0;
      int local = 0;
      for (int w = unit; w < num_units && !*abort_flag; w += units, ++local) {
        const int acc = local & 1;
        const uint32_t acc_phase = (local >> 1) & 1;
        if (!mbar_wait(&acc_empty[acc], acc_phase ^ 1u, abort_flag, p.err)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + uint32_t(acc * BN);
        const uint32_t idesc = (w < p.split_from ? IDESC_P2 : IDESC_P2_HALF) ^ p.idesc_xor;
        bool ok = true;
        for (int it = 0; it < total_k; ++it) {
          if (!mbar_wait(&full[stage], phase, abort_flag, p.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(tiles + stage * P2_STAGE_BYTES);
          const uint64_t adesc = sw128_desc(sa);
          const uint64_t bdesc = sw128_desc(sa + A_TILE);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            tc_mma_bf16_pair(d_tmem, adesc + uint64_t(2 * kk), bdesc + uint64_t(2 * kk), idesc,
                             (it > 0 || kk > 0) ? 1u : 0u);
          tc_commit_pair_multicast(&empty[stage], uint16_t(0x3));
          if (++stage == P2_STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        if (!(p.withhold && local == 0)) tc_commit_pair_multicast(&acc_full[acc], uint16_t(0x3));
      }
      tc_commit_pair(drain);
      volatile int no_abort = 0;
      mbar_wait(drain, 0, &no_abort, p.err);
    }
  } else {
    const int q = warp & 3;
    const int row_in_tile = q * 32 + lane;
    const int64_t ld = p.np;
    const uint32_t leader_acc_empty[2] = {cluster_map_shared(&acc_empty[0], 0),
                                          cluster_map_shared(&acc_empty[1], 0)};
    double ss = 0.0;
    int local = 0;
    for (int w = unit; w < num_units; w += units, ++local) {
      const int acc = local & 1;
      const uint32_t acc_phase = (local >> 1) & 1;
      if (!mbar_wait(&acc_full[acc], acc_phase, abort_flag, p.err)) break;
      tc_fence_after();
      int t, half, tm2, tn;
      unit_tile(w, p.split_from, t, half);
      tile_coords(t, unit_rows, p.tiles_n, GROUP_M / 2, tm2, tn);
      const int gr = tm2 * 2 * BM + rank * BM + row_in_tile;
      const int col0 = tn * BN + (half < 0 ? 0 : half * (BN / 2));
      const int chunks = half < 0 ? BN / 32 : BN / 64;
      for (int c = 0; c < chunks; ++c) {
        const int gc0 = col0 + c * 32;
        if (gc0 >= p.np) break;
        uint32_t raw[32];
        tmem_ld_32x32b_x32(tmem_base + uint32_t(acc * BN + c * 32) + (uint32_t(q * 32) << 16), raw);
        tmem_ld_wait();
        epilogue_chunk(p, raw, gr, gc0, ld, ss);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(leader_acc_empty[acc]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
    if (lane == 0) red[q] = ss;
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (warp == 2 && lane == 0 && p.partial != nullptr) p.partial[blockIdx.x] = red[0] + red[1] + red[2] + red[3];
  }

  tc_fence_before();
  cluster_sync_all();
  tc_fence_after();
  if (warp == 1) tmem_dealloc_pair(tmem_base, TMEM_COLS);
}

}  // namespace tc

// ---------------------------------------------------------------------------------------
// Host side.

namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
int g_sms = 0;
int g_2sm_clusters = 0;   // co-resident clusters of the 2-SM MMA kernel (0: unavailable)
int g_variant = 0;  // 0 auto (4 where possible, else 1), 1 single-CTA, 3 2-SM MMA, 4 3 + split tail
bool g_tc_ok = false;
std::once_flag g_once;
std::atomic<int> g_withhold{0};  // armed by nn_debug_withhold_signal, consumed by the next launch

cudaLaunchConfig_t cluster_config(int grid, int smem, cudaStream_t st, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(tc::THREADS);
  cfg.dynamicSmemBytes = size_t(smem);
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Co-resident clusters of two for a kernel (0: the kernel cannot run as clusters here).
int max_clusters(void (*kernel)(tc::Params), int smem) {
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cluster_config(2 * (g_sms / 2), smem, nullptr, attr);
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, kernel, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return clusters;
}

void init_once() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return;
  g_sms = prop.multiProcessorCount;
  // sm_103 only: this kernel is compiled for sm_103a.
  if (prop.major != 10 || prop.minor != 3) return;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || fn == nullptr) {
    (void)cudaGetLastError();
    return;
  }
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  if (cudaFuncSetAttribute(tc::gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES) !=
      cudaSuccess) {
    (void)cudaGetLastError();
    return;
  }
  g_tc_ok = true;
  g_2sm_clusters = max_clusters(tc::gemm_tc_2sm_kernel, tc::P2_SMEM_BYTES);
  (void)cudaGetLastError();
}

bool encode_bf16_2d(CUtensorMap* map, const void* ptr, int np, int box_rows) {
  cuuint64_t dims[2] = {cuuint64_t(np), cuuint64_t(np)};
  cuuint64_t strides[1] = {cuuint64_t(np) * 2};
  cuuint32_t box[2] = {cuuint32_t(tc::BK), cuuint32_t(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

bool tc_supported() {
  std::call_once(g_once, init_once);
  return g_tc_ok;
}

void gemm_tc_withhold_next(int on) { g_withhold.store(on ? 1 : 0); }
int tc_take_withhold() { return g_withhold.exchange(0); }

void gemm_tc_set_variant(int v) { g_variant = (v == 1 || v == 3 || v == 4) ? v : 0; }

int gemm_tc_max_grid() {
  std::call_once(g_once, init_once);
  return g_sms > 0 ? g_sms : 1;
}

int gemm_tc(cudaStream_t st, const TcGemmArgs& a, int* grid_used) {
  if (!tc_supported()) return NN_ERR_UNSUPPORTED;
  if (a.np <= 0 || a.np % 128 != 0 || a.nseg < 1 || a.nseg > kTcMaxSeg || a.n_row < 0 || a.n_row > 3 ||
      a.n_col < 0 || a.n_col > 3 || a.err == nullptr)
    return NN_ERR_ARG;
  if (!a.emu && a.mode == EPI_ADD && a.add == nullptr) return NN_ERR_ARG;
  if (a.cvt_dst != nullptr && (a.emu || a.cvt_src == nullptr || a.cvt_n < 1 || a.cvt_n > a.np || a.cvt_ld < a.cvt_n))
    return NN_ERR_ARG;
  if (a.emu && (a.affine || a.half)) return NN_ERR_ARG;
  if (a.emu && (a.emu_acc == nullptr || a.emu_gexp == nullptr || (a.emu_last && a.emu_out == nullptr) ||
                (a.emu_last && a.mode == EPI_ADD && a.emu_add == nullptr) || a.n_row != 0 || a.n_col != 0 ||
                a.out_f32 != nullptr || a.emu_n < 1 || a.emu_n > a.np))
    return NN_ERR_ARG;
  tc::Params p;
  memset(&p, 0, sizeof(p));
  for (int s = 0; s < a.nseg; ++s) {
    if (a.a_seg[s] == nullptr || a.b_seg[s] == nullptr) return NN_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(a.a_seg[s]) & 15) || (reinterpret_cast<uintptr_t>(a.b_seg[s]) & 15))
      return NN_ERR_ARG;
    if (!encode_bf16_2d(&p.map_a[s], a.a_seg[s], a.np, tc::BM)) return NN_ERR_CUDA;
    if (!encode_bf16_2d(&p.map_b[s], a.b_seg[s], a.np, tc::BN)) return NN_ERR_CUDA;
  }
  for (int i = 0; i < a.n_row; ++i)
    if (a.row_pieces[i] == nullptr) return NN_ERR_ARG;
  for (int i = 0; i < a.n_col; ++i)
    if (a.col_pieces[i] == nullptr) return NN_ERR_ARG;
  p.nseg = a.nseg;
  p.np = a.np;
  p.tiles_m = a.np / tc::BM;
  p.tiles_n = (a.np + tc::BN - 1) / tc::BN;
  p.n_id = a.n_id;
  p.mode = a.mode;
  p.add = a.add;
  p.out_f32 = a.out_f32;
  for (int i = 0; i < 3; ++i) {
    p.row_pieces[i] = a.row_pieces[i];
    p.col_pieces[i] = a.col_pieces[i];
  }
  p.n_row = a.n_row;
  p.n_col = a.n_col;
  p.partial = a.partial;
  p.err = a.err;
  p.emu = a.emu ? 1 : 0;
  p.emu_first = a.emu_first ? 1 : 0;
  p.emu_last = a.emu_last ? 1 : 0;
  p.emu_gexp = a.emu_gexp;
  p.emu_acc = a.emu_acc;
  p.emu_out = a.emu_out;
  p.emu_ld_out = a.emu_ld_out;
  p.emu_add = a.emu_add;
  p.emu_ld_add = a.emu_ld_add;
  p.emu_n = a.emu_n;
  p.affine = a.affine ? 1 : 0;
  p.aff_scale = a.aff_scale;
  p.aff_diag = a.aff_diag;
  p.cvt_src = a.cvt_src;
  p.cvt_dst = a.cvt_dst;
  p.cvt_ld = a.cvt_ld;
  p.cvt_n = a.cvt_n;
  p.cvt_vec = (a.cvt_ld % 2 == 0 && (reinterpret_cast<uintptr_t>(a.cvt_dst) & 15) == 0) ? 1 : 0;
  p.half = a.half ? 1 : 0;
  // A and B types (bits 7-9, 10-12): BF16 = 1, FP16 = 0; both operands always share one type
  p.idesc_xor = a.half ? ((1u << 7) | (1u << 10)) : 0u;
  p.in_scale = a.in_scale;
  p.in_row = a.in_row;
  p.out_scale = a.out_scale;
  p.out_r8 = a.out_r8 ? 1 : 0;
  p.withhold = tc_take_withhold();
  // Variant choice: the 2-SM MMA with a split last wave by default where the size allows it, else
  // single-CTA tiles.
  const bool even = a.np % (2 * tc::BM) == 0;
  int variant = g_variant;
  if (variant == 0) variant = (even && g_2sm_clusters > 0) ? 4 : 1;
  if (variant >= 3 && !(even && g_2sm_clusters > 0)) return NN_ERR_UNSUPPORTED;
  int grid = 0;
  if (variant >= 3) {
    // B^T maps load 128-row halves (one per CTA of the pair)
    for (int s = 0; s < a.nseg; ++s)
      if (!encode_bf16_2d(&p.map_b[s], a.b_seg[s], a.np, tc::BN / 2)) return NN_ERR_CUDA;
    const int units = (p.tiles_m / 2) * p.tiles_n;
    const int avail = g_2sm_clusters;
    const int clusters = units < avail ? units : avail;
    grid = 2 * clusters;
    // 2-SM kernel: a last wave at most half full runs its tiles as 256 x 128 halves
    p.split_from = units;
    const int tail = units % clusters;
    if (variant == 4 && units > clusters && tail > 0 && 2 * tail <= clusters) {
      p.split_from = units - tail;
      for (int s = 0; s < a.nseg; ++s)
        if (!encode_bf16_2d(&p.map_b_half[s], a.b_seg[s], a.np, tc::BN / 4)) return NN_ERR_CUDA;
    }
    cudaLaunchAttribute attr[1];
    if (a.ev_before) NN_CUDA_TRY(cudaEventRecord(a.ev_before, st));
    cudaLaunchConfig_t cfg = cluster_config(grid, tc::P2_SMEM_BYTES, st, attr);
    NN_CUDA_TRY(cudaLaunchKernelEx(&cfg, tc::gemm_tc_2sm_kernel, p));
  } else {
    const int tiles = p.tiles_m * p.tiles_n;
    grid = tiles < g_sms ? tiles : g_sms;
    if (a.ev_before) NN_CUDA_TRY(cudaEventRecord(a.ev_before, st));
    tc::gemm_tc_kernel<<<grid, tc::THREADS, tc::SMEM_BYTES, st>>>(p);
    NN_CUDA_TRY(cudaGetLastError());
  }
  if (a.ev_after) NN_CUDA_TRY(cudaEventRecord(a.ev_after, st));
  if (grid_used) *grid_used = grid;
  return NN_OK;
}

}  // namespace nn
