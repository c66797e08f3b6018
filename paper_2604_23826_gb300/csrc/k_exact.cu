// k_exact.cu -- the exact fused pass: n, s = X^T 1 and S = X^T X in one
// streaming pass over a columnar table (arxiv 2604.23826, "Data Representation
// and Sufficient Statistics"; exactness because of "Numerical Considerations").
//
// Every row becomes a vector w of 32 small integer "digits": the ones column
// (so that n and s fall out of the same product), then each column's value split
// into base-256 digits (integers directly; real columns first as a fixed-point
// integer q = round(x * 2^shift) of their declared range).  The digit Gram matrix
// G = sum_rows w w^T is accumulated on the tensor cores with f16 operands
// (every digit |d| <= 255 is exact in f16) and FP32 accumulators.  Each product
// is below 2^16 and a warp flushes its accumulators every 256 of its rows, so
// every partial sum is an integer below 2^24 and FP32 never rounds.  Flushes go
// to int32 partial sums (in registers, or for the shapes with more warps in a
// per-warp shared-memory array), every 64 flushes by integer atomics to an int64
// block accumulator in shared memory, then by global integer atomics to a
// per-call int64 accumulator, which the last block to finish adds to the context
// accumulator (integer addition: the result does not depend on block order or on
// the shape of the launch).  S_jk = sum_{a,b} 256^(a+b) G[(j,a),(k,b)] is
// recombined exactly by the finalize kernel.
//
// Pipeline: one producer warp moves each stage of every column from HBM to
// shared memory with bulk copies (cp.async.bulk, completion on an mbarrier;
// columns whose address is not 16-byte aligned are instead read by the consumers
// with plain loads); W consumer warps take RPW rows of a stage each, turn them
// into digits 32 rows at a time, stage those as a swizzled [32 rows x 32 digits]
// f16 tile, load operand fragments with ldmatrix.trans and issue mma.sync
// m16n8k16 for the 6 upper-triangle 16x8 tiles of the 32x32 digit Gram.  The
// shape (W, RPW) is a launch choice (exact_shape_warps / exact_shape_rpw): more warps hide more latency
// but need fewer registers each and smaller stages.  All waits are bounded; an
// expired wait marks the call failed (the accumulator is then left unchanged).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace ss {

namespace {

constexpr int kDigitTileBytes = 32 * 64;  // 32 rows x 32 f16 digits
constexpr int kFlushRows = 256;           // per warp: FP32 partial sums stay below 2^24
constexpr int kI32Flushes = 64;           // int32 partial sums stay below 2^30
// int32 partial sums of a warp held in shared memory (shapes with more than 15 consumer
// warps, whose threads have too few registers for them): 24 per lane, lane-major
constexpr int kI32Bytes = 24 * 32 * 4;
__host__ __device__ constexpr bool i32_in_smem(int warps) { return warps > 15; }

// ---- sources of raw column values: a shared-memory stage or global memory ----
struct SmemSrc {
  const uint8_t* base;  // stage base
  const ExactParams* P;
  int r;                // row inside the stage
  __device__ __forceinline__ int32_t i32(int j) const {
    return *reinterpret_cast<const int32_t*>(base + P->col_off[j] + r * 4);
  }
  __device__ __forceinline__ int32_t i16(int j) const {
    return *reinterpret_cast<const int16_t*>(base + P->col_off[j] + r * 2);
  }
  __device__ __forceinline__ int64_t i64(int j) const {
    return *reinterpret_cast<const int64_t*>(base + P->col_off[j] + r * 8);
  }
  __device__ __forceinline__ double f64(int j) const {
    return *reinterpret_cast<const double*>(base + P->col_off[j] + r * 8);
  }
  __device__ __forceinline__ float f32(int j) const {
    return *reinterpret_cast<const float*>(base + P->col_off[j] + r * 4);
  }
};
struct GlobalSrc {
  const ExactParams* P;
  int64_t r;  // row of the call
  __device__ __forceinline__ int32_t i32(int j) const { return static_cast<const int32_t*>(P->cols[j])[r]; }
  __device__ __forceinline__ int32_t i16(int j) const { return static_cast<const int16_t*>(P->cols[j])[r]; }
  __device__ __forceinline__ int64_t i64(int j) const { return static_cast<const int64_t*>(P->cols[j])[r]; }
  __device__ __forceinline__ double f64(int j) const { return static_cast<const double*>(P->cols[j])[r]; }
  __device__ __forceinline__ float f32(int j) const { return static_cast<const float*>(P->cols[j])[r]; }
};

// Stage layout of the Table 1 layouts for a stage of TILE rows, known at compile time
// (the host lays a stage out with the same rule: columns in order, stage_col_bytes() each).
template <bool L16, int TILE>
struct T1Layout {
  __host__ __device__ static constexpr int bytes(int j) { return (j == 0 || j == 8 || j == 10) ? 8 : (L16 && j != 5) ? 2 : 4; }
  __host__ __device__ static constexpr int off(int j) {
    int o = 0;
    for (int i = 0; i < j; ++i) o += stage_col_bytes(bytes(i), TILE);
    return o;
  }
};
template <bool L16, int TILE>
struct SmemT1Src {
  const uint8_t* base;  // stage base
  int r;                // row inside the stage
  __device__ __forceinline__ int32_t i32(int j) const { return *reinterpret_cast<const int32_t*>(base + T1Layout<L16, TILE>::off(j) + r * 4); }
  __device__ __forceinline__ int32_t i16(int j) const { return *reinterpret_cast<const int16_t*>(base + T1Layout<L16, TILE>::off(j) + r * 2); }
  __device__ __forceinline__ int64_t i64(int j) const { return *reinterpret_cast<const int64_t*>(base + T1Layout<L16, TILE>::off(j) + r * 8); }
  __device__ __forceinline__ double f64(int j) const { return *reinterpret_cast<const double*>(base + T1Layout<L16, TILE>::off(j) + r * 8); }
};

// The Table 1 real columns convert on the FP64 unit: q = round-to-nearest-even(x * 2^sh),
// the scaling an exponent-field add (exact), zero and subnormal inputs giving 0.  (The
// integer-only fixed_rn keeps the ALU pipe busier; on sm_103a the FP64 conversion
// unit sustains about two per clock per SM, well above what this pass needs.)
__device__ __forceinline__ uint64_t fixed_f2i(double x, int sh) {
  const uint32_t hi = static_cast<uint32_t>(__double2hiint(x)), lo = static_cast<uint32_t>(__double2loint(x));
  const bool normal = ((hi >> 20) & 0x7FF) != 0;
  const long long q =
      __double2ll_rn(__hiloint2double(static_cast<int>(hi + (static_cast<uint32_t>(sh) << 20)), static_cast<int>(lo)));
  return normal ? static_cast<uint64_t>(q) : 0ull;
}

// ---- the Table 1 converter: fixed digit plan, column order A B C D E F G H cotC I J K ----
// slots: 0 ones | 1 B | 2 C | 3 D | 4 E | 5 G | 6 H | 7 K | 8-9 F | 10-11 I | 12-16 A |
//        17-23 cotC (signed, top byte 23) | 24-30 J | 31 zero
// The field checks below are exactly the ranges those digit fields can carry.
template <bool L16>
struct ConvT1 {
  template <int TILE>
  __device__ __forceinline__ static SmemT1Src<L16, TILE> smem_src(const uint8_t* st, const ExactParams&, int r) {
    return SmemT1Src<L16, TILE>{st, r};
  }
  template <class Src>
  __device__ __forceinline__ static void row(const ExactParams& P, const Src& src, uint32_t (&w)[16],
                                             uint32_t& bad) {
    int32_t B, C, D, E, F, G, H, I, K;
    if (L16) {
      B = src.i16(1); C = src.i16(2); D = src.i16(3); E = src.i16(4); G = src.i16(6);
      H = src.i16(7); I = src.i16(9); K = src.i16(11); F = src.i32(5);
    } else {
      B = src.i32(1); C = src.i32(2); D = src.i32(3); E = src.i32(4); F = src.i32(5);
      G = src.i32(6); H = src.i32(7); I = src.i32(9); K = src.i32(11);
    }
    const int64_t A = src.i64(0);
    const double cot = src.f64(8), J = src.f64(10);
    const uint32_t Alo = static_cast<uint32_t>(A), Ahi = static_cast<uint32_t>(static_cast<uint64_t>(A) >> 32);
    // field checks: one unsigned byte each; two unsigned bytes; five unsigned bytes
    bad |= static_cast<uint32_t>(B | C | D | E | G | H | K) & 0xFFFFFF00u;
    bad |= static_cast<uint32_t>(F | I) & 0xFFFF0000u;
    bad |= Ahi & 0xFFFFFF00u;
    const int ec = dbl_exp_field(cot), ej = dbl_exp_field(J);
    const uint64_t uj = static_cast<uint64_t>(__double_as_longlong(J));
    bad |= (ec > P.real_emax[8]) | (ej > P.real_emax[10]) | ((uj >> 63) & ((uj << 1) != 0));  // J >= 0
    const uint64_t qc = fixed_f2i(cot, P.real_shift[8]);
    const uint64_t qj = fixed_f2i(J, P.real_shift[10]);
    const uint32_t qclo = static_cast<uint32_t>(qc), qchi = static_cast<uint32_t>(qc >> 32) ^ 0x00800000u;
    const uint32_t qjlo = static_cast<uint32_t>(qj), qjhi = static_cast<uint32_t>(qj >> 32);
    constexpr uint32_t M = 0x64646464u;  // bytes of the f16 exponent 0x64
    w[0] = small_pair_f16x2(1u, static_cast<uint32_t>(B));
    w[1] = small_pair_f16x2(static_cast<uint32_t>(C), static_cast<uint32_t>(D));
    w[2] = small_pair_f16x2(static_cast<uint32_t>(E), static_cast<uint32_t>(G));
    w[3] = small_pair_f16x2(static_cast<uint32_t>(H), static_cast<uint32_t>(K));
    w[4] = half2_sub(__byte_perm(static_cast<uint32_t>(F), M, 0x4140), kH1024);
    w[5] = half2_sub(__byte_perm(static_cast<uint32_t>(I), M, 0x4140), kH1024);
    w[6] = half2_sub(__byte_perm(Alo, M, 0x4140), kH1024);
    w[7] = half2_sub(__byte_perm(Alo, M, 0x4342), kH1024);
    w[8] = digits2(__byte_perm(Ahi, qclo, 0x1410));          // A byte 4 | cotC byte 0
    w[9] = half2_sub(__byte_perm(qclo, M, 0x4241), kH1024);  // cotC bytes 1, 2
    w[10] = digits2(__byte_perm(qclo, qchi, 0x0403) & 0x00FF00FFu);  // cotC bytes 3, 4
    w[11] = half2_sub(__byte_perm(qchi, M, 0x4241), kH1152hi);       // cotC bytes 5, 6 (6 signed)
    w[12] = half2_sub(__byte_perm(qjlo, M, 0x4140), kH1024);
    w[13] = half2_sub(__byte_perm(qjlo, M, 0x4342), kH1024);
    w[14] = half2_sub(__byte_perm(qjhi, M, 0x4140), kH1024);
    w[15] = half2_sub(__byte_perm(qjhi, M, 0x4342), kH1024);  // J byte 6 | zero (byte 7 of q)
  }
};

// ---- the generic converter: any plan of at most 32 digits over at most 16 columns ----
template <class Src>
__device__ __forceinline__ int64_t load_as_int(const ExactParams& P, const Src& src, int j) {
  switch (P.dtype[j]) {
    case I16: return src.i16(j);
    case I32: return src.i32(j);
    case I64: return src.i64(j);
    case F32: return static_cast<int64_t>(fixed_rn<true>(static_cast<double>(src.f32(j)), P.real_shift[j]));
    default: return static_cast<int64_t>(fixed_rn<true>(src.f64(j), P.real_shift[j]));
  }
}

struct ConvGeneric {
  template <int TILE>
  __device__ __forceinline__ static SmemSrc smem_src(const uint8_t* st, const ExactParams& P, int r) {
    return SmemSrc{st, &P, r};
  }
  template <class Src>
  __device__ __forceinline__ static uint32_t byte_of(const ExactParams& P, const Src& src, int c, int b, int sg) {
    if (c == -1) return 1u;
    if (c < 0) return 0u;
    const uint64_t v = static_cast<uint64_t>(load_as_int(P, src, c));
    return static_cast<uint32_t>((v >> (8 * b)) & 0xFF) ^ (sg ? 0x80u : 0u);
  }
  template <class Src>
  __device__ __forceinline__ static void row(const ExactParams& P, const Src& src, uint32_t (&w)[16],
                                             uint32_t& bad) {
#pragma unroll
    for (int j = 0; j < kMaxCols; ++j) {
      if (j >= P.p) break;
      const int dt = P.dtype[j];
      if (dt == F32 || dt == F64) {
        const double x = dt == F32 ? static_cast<double>(src.f32(j)) : src.f64(j);
        const uint64_t ux = static_cast<uint64_t>(__double_as_longlong(x));
        bad |= dbl_exp_field(x) > P.real_emax[j];
        if (!P.is_signed[j]) bad |= (ux >> 63) & ((ux << 1) != 0);  // negative, not -0
      } else {
        const int64_t v = load_as_int(P, src, j);
        const int k = P.kbytes[j];
        if (k < 8) {
          const uint64_t u = static_cast<uint64_t>(P.is_signed[j] ? v + (int64_t(1) << (8 * k - 1)) : v);
          bad |= (u >> (8 * k)) != 0;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kDigitPairs; ++q) {
      const uint32_t lo = byte_of(P, src, P.pc0[q], P.pb0[q], P.ps0[q]);
      const uint32_t hi = byte_of(P, src, P.pc1[q], P.pb1[q], P.ps1[q]);
      const uint32_t bias = (P.ps0[q] ? 0x80u : 0u) | (P.ps1[q] ? 0x800000u : 0u);
      w[q] = half2_sub(lo | (hi << 16) | kH1024, kH1024 | bias);
    }
  }
};

// Digit tile of one warp: row R (0..31) holds 64 bytes; its 16-byte chunk c
// (digits 8c..8c+7) sits at chunk position c ^ ((R >> 1) & 3), which makes
// both the row-wise 128-bit stores and the 8-row ldmatrix phases conflict-free.
__device__ __forceinline__ uint32_t tile_addr(uint32_t tile, int R, int c) {
  return tile + R * 64 + ((c ^ ((R >> 1) & 3)) << 4);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// The 6 upper-triangle tiles of the 32 x 32 digit Gram as (16-row block i, 8-col block j):
// (0,0) (0,1) (0,2) (0,3) (1,2) (1,3).
__host__ __device__ constexpr int tile_i(int e) { return e < 4 ? 0 : 1; }
__host__ __device__ constexpr int tile_j(int e) { return e < 4 ? e : e - 2; }

struct WarpAcc {
  float f[6][4];
};
struct WarpI32 {  // int32 partial sums in registers
  int32_t i[6][4];
};

// One 32-row sub-step of a warp: stage the digits, two K=16 blocks of MMAs.
__device__ __forceinline__ void warp_mma_32rows(uint32_t tile, int lane, const uint32_t (&w)[16], WarpAcc& acc) {
  const int sw = (lane >> 1) & 3;
  st_shared_v4(tile + lane * 64 + ((0 ^ sw) << 4), w[0], w[1], w[2], w[3]);
  st_shared_v4(tile + lane * 64 + ((1 ^ sw) << 4), w[4], w[5], w[6], w[7]);
  st_shared_v4(tile + lane * 64 + ((2 ^ sw) << 4), w[8], w[9], w[10], w[11]);
  st_shared_v4(tile + lane * 64 + ((3 ^ sw) << 4), w[12], w[13], w[14], w[15]);
  __syncwarp();
#pragma unroll
  for (int kb = 0; kb < 2; ++kb) {
    uint32_t R0, R1, R2, R3, Q0, Q1, Q2, Q3;
    const int rr = 16 * kb + (lane & 7), m = lane >> 3;
    ldsm_x4_trans(tile_addr(tile, rr, m), R0, R1, R2, R3);      // rows 0..7 of the K block
    ldsm_x4_trans(tile_addr(tile, rr + 8, m), Q0, Q1, Q2, Q3);  // rows 8..15
    // A_i = {R[2i], R[2i+1], Q[2i], Q[2i+1]},  B_j = {R[j], Q[j]}
    mma_f16_16816(acc.f[0], R0, R1, Q0, Q1, R0, Q0);
    mma_f16_16816(acc.f[1], R0, R1, Q0, Q1, R1, Q1);
    mma_f16_16816(acc.f[2], R0, R1, Q0, Q1, R2, Q2);
    mma_f16_16816(acc.f[3], R0, R1, Q0, Q1, R3, Q3);
    mma_f16_16816(acc.f[4], R2, R3, Q2, Q3, R2, Q2);
    mma_f16_16816(acc.f[5], R2, R3, Q2, Q3, R3, Q3);
  }
  __syncwarp();
}

// FP32 accumulators (exact integers below 2^24) into int32 partial sums: registers, or the
// warp's shared array (each lane its own 24 words, so plain loads and stores suffice).
__device__ __forceinline__ void flush_f32(WarpAcc& acc, WarpI32& ri) {
#pragma unroll
  for (int e = 0; e < 6; ++e)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      ri.i[e][r] += __float2int_rn(acc.f[e][r]);
      acc.f[e][r] = 0.f;
    }
}
__device__ __forceinline__ void flush_f32(WarpAcc& acc, int32_t* si, int lane) {
#pragma unroll
  for (int e = 0; e < 6; ++e)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      si[(4 * e + r) * 32 + lane] += __float2int_rn(acc.f[e][r]);
      acc.f[e][r] = 0.f;
    }
}

// int32 partial sums into the block's int64 accumulator in shared memory: upper-triangle
// entries only, by integer atomics (order-independent); the partial sums restart at zero.
template <class Get>
__device__ __forceinline__ void flush_i32(Get&& get, unsigned long long* cta_acc, int lane) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int e = 0; e < 6; ++e)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int row = 16 * tile_i(e) + g + ((r >> 1) << 3);
      const int col = 8 * tile_j(e) + 2 * t + (r & 1);
      int32_t& v = get(e, r);
      if (row <= col && v != 0)
        atomicAdd(&cta_acc[row * kDigits + col], static_cast<unsigned long long>(static_cast<long long>(v)));
      v = 0;
    }
}

template <class Conv, int W, int RPW>
__global__ void __launch_bounds__((W + 1) * 32, 1) exact_pass_kernel(const __grid_constant__ ExactParams P) {
  constexpr int kTile = W * RPW;  // rows of a stage
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t* stage_base = smem;
  uint8_t* dtiles = smem + P.stages * P.stage_bytes;
  int32_t* i32s = reinterpret_cast<int32_t*>(dtiles + W * kDigitTileBytes);  // i32_in_smem(W) only
  unsigned long long* cta_acc =
      reinterpret_cast<unsigned long long*>(dtiles + W * kDigitTileBytes + (i32_in_smem(W) ? W * kI32Bytes : 0));
  uint64_t* full = reinterpret_cast<uint64_t*>(cta_acc + kDigits * kDigits);
  uint64_t* empty = full + kExactMaxStages;
  __shared__ uint32_t s_bad;
  __shared__ uint32_t s_last;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int stages = P.stages;
  const int64_t ntiles = (P.nmain + kTile - 1) / kTile;
  const int64_t my_count = (ntiles > blockIdx.x) ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  for (int i = threadIdx.x; i < kDigits * kDigits; i += blockDim.x) cta_acc[i] = 0ull;
  if (threadIdx.x == 0) {
    s_bad = 0;
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], W);
    }
    fence_mbar_init();
  }
  __syncthreads();

  uint32_t bad = 0;       // range violations seen by this thread
  uint32_t failed = 0;    // a bounded wait expired
  if (warp == W) {
    // ---------------- producer: bulk copies of every column of each stage ----------------
    if (lane == 0 && !P.direct) {
      int64_t issued = 0;
      int s = 0;
      uint32_t ph = 0;  // phase parity of stage s's current use
      int64_t row0 = static_cast<int64_t>(blockIdx.x) * kTile;
      const int64_t row_step = static_cast<int64_t>(gridDim.x) * kTile;
      for (int64_t k = 0; k < my_count; ++k, row0 += row_step) {
        // stage s was last used by tile k - stages, whose consumption completed phase ph ^ 1
        if (k >= stages && !mbar_wait_bounded(&empty[s], ph ^ 1u)) {
          failed = 1;
          break;
        }
        const uint32_t rows = static_cast<uint32_t>(min(static_cast<int64_t>(kTile), P.nmain - row0));
        uint32_t total = 0;
        for (int j = 0; j < P.p; ++j) total += rows * P.col_bytes[j];
        mbar_arrive_expect_tx(&full[s], total);
        uint8_t* dst = stage_base + s * P.stage_bytes;
        for (int j = 0; j < P.p; ++j)
          bulk_g2s(dst + P.col_off[j], static_cast<const uint8_t*>(P.cols[j]) + row0 * P.col_bytes[j],
                   rows * P.col_bytes[j], &full[s]);
        issued = k + 1;
        if (++s == stages) {
          s = 0;
          ph ^= 1u;
        }
      }
      // No copy may still be landing in shared memory when the block exits.
      for (int64_t k = max(static_cast<int64_t>(0), issued - stages); k < issued; ++k)
        if (!mbar_wait_bounded(&full[k % stages], static_cast<uint32_t>((k / stages) & 1))) failed = 1;
    }
  } else {
    // ---------------- consumers ----------------
    WarpAcc acc;
    WarpI32 ri;
    int32_t* si = i32s + warp * (kI32Bytes / 4);
#pragma unroll
    for (int e = 0; e < 6; ++e)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        acc.f[e][r] = 0.f;
        if (i32_in_smem(W))
          si[(4 * e + r) * 32 + lane] = 0;
        else
          ri.i[e][r] = 0;
      }
    auto get_i32 = [&](int e, int r) -> int32_t& {
      return i32_in_smem(W) ? si[(4 * e + r) * 32 + lane] : ri.i[e][r];
    };
    const uint32_t tile = smem_u32(dtiles + warp * kDigitTileBytes);
    int sub = 0, flushes = 0;
    int s = 0;
    uint32_t ph = 0;  // phase parity of stage s's current use
    int64_t row0 = static_cast<int64_t>(blockIdx.x) * kTile;
    const int64_t row_step = static_cast<int64_t>(gridDim.x) * kTile;
    for (int64_t k = 0; k < my_count; ++k, row0 += row_step) {
      if (!P.direct && !mbar_wait_bounded(&full[s], ph)) {
        failed = 1;
        break;
      }
      const int valid = static_cast<int>(min(static_cast<int64_t>(kTile), P.nmain - row0));
      const uint8_t* st = stage_base + s * P.stage_bytes;
#pragma unroll 1
      for (int h = 0; h < RPW / 32; ++h) {
        const int r = warp * RPW + h * 32 + lane;
        uint32_t w[16];
        if (r < valid && P.direct) {
          GlobalSrc src{&P, row0 + r};
          Conv::row(P, src, w, bad);
        } else if (r < valid) {
          Conv::row(P, Conv::template smem_src<kTile>(st, P, r), w, bad);
        } else {
#pragma unroll
          for (int q = 0; q < 16; ++q) w[q] = 0u;
        }
        warp_mma_32rows(tile, lane, w, acc);
        if (++sub == kFlushRows / 32) {
          sub = 0;
          if (i32_in_smem(W))
            flush_f32(acc, si, lane);
          else
            flush_f32(acc, ri);
          if (++flushes == kI32Flushes) {
            flushes = 0;
            flush_i32(get_i32, cta_acc, lane);
          }
        }
      }
      __syncwarp();
      if (lane == 0 && !P.direct) mbar_arrive(&empty[s]);
      if (++s == stages) {
        s = 0;
        ph ^= 1u;
      }
    }
    // ragged tail (fewer than 8 rows), read from global memory by warp 0 of block 0
    if (blockIdx.x == 0 && warp == 0 && P.nrows > P.nmain) {
      const int64_t r = P.nmain + lane;
      uint32_t w[16];
      if (r < P.nrows) {
        GlobalSrc src{&P, r};
        Conv::row(P, src, w, bad);
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) w[q] = 0u;
      }
      warp_mma_32rows(tile, lane, w, acc);
    }
    if (i32_in_smem(W))
      flush_f32(acc, si, lane);
    else
      flush_f32(acc, ri);
    flush_i32(get_i32, cta_acc, lane);
  }
  if (bad) atomicOr(&s_bad, DEV_ERANGE);
  if (failed) atomicOr(&s_bad, DEV_ETIMEOUT);
  __syncthreads();

  // block partial -> per-call accumulator (integer atomics: order-independent)
  for (int i = threadIdx.x; i < kDigits * kDigits; i += blockDim.x) {
    const unsigned long long v = cta_acc[i];
    if (v) atomicAdd(&P.call_acc[i], v);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_bad) atomicOr(P.err, s_bad);
    __threadfence();
    s_last = (atomicAdd(P.ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  // last block: commit this call's sum to the ctx accumulator unless an error was seen
  __threadfence();
  const unsigned int err = atomicAdd(P.err, 0u);
  for (int i = threadIdx.x; i < kDigits * kDigits; i += blockDim.x) {
    const long long v = static_cast<long long>(atomicExch(&P.call_acc[i], 0ull));
    if (!err) P.acc[i] += v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (err) atomicOr(P.status, err);
    *P.err = 0u;
    *P.ticket = 0u;
    __threadfence();
  }
}

template <class Conv, int W, int RPW>
cudaError_t launch_conv(const ExactParams& P, int grid, cudaStream_t stream) {
  const size_t smem = exact_smem_bytes(P.shape, P.stages, P.stage_bytes);
  auto* fn = exact_pass_kernel<Conv, W, RPW>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  fn<<<grid, (W + 1) * 32, smem, stream>>>(P);
  return cudaGetLastError();
}

template <class Conv, int W, int RPW>
int max_active(size_t smem) {
  auto* fn = exact_pass_kernel<Conv, W, RPW>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
    return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, (W + 1) * 32, smem) != cudaSuccess) return 0;
  return n;
}

// The kernel of a (converter, shape) pair: F<Conv, W, RPW>::run(args...).
template <template <class, int, int> class F, class... A>
auto dispatch(int conv, int shape, A... a) {
  switch (conv * kExactShapes + shape) {
    case CONV_T1_L32 * kExactShapes + 0: return F<ConvT1<false>, exact_shape_warps(0), exact_shape_rpw(0)>::run(a...);
    case CONV_T1_L32 * kExactShapes + 1: return F<ConvT1<false>, exact_shape_warps(1), exact_shape_rpw(1)>::run(a...);
    case CONV_T1_L32 * kExactShapes + 2: return F<ConvT1<false>, exact_shape_warps(2), exact_shape_rpw(2)>::run(a...);
    case CONV_T1_L16 * kExactShapes + 0: return F<ConvT1<true>, exact_shape_warps(0), exact_shape_rpw(0)>::run(a...);
    case CONV_T1_L16 * kExactShapes + 1: return F<ConvT1<true>, exact_shape_warps(1), exact_shape_rpw(1)>::run(a...);
    case CONV_T1_L16 * kExactShapes + 2: return F<ConvT1<true>, exact_shape_warps(2), exact_shape_rpw(2)>::run(a...);
    case CONV_GENERIC * kExactShapes + 1: return F<ConvGeneric, exact_shape_warps(1), exact_shape_rpw(1)>::run(a...);
    case CONV_GENERIC * kExactShapes + 2: return F<ConvGeneric, exact_shape_warps(2), exact_shape_rpw(2)>::run(a...);
    default: return F<ConvGeneric, exact_shape_warps(0), exact_shape_rpw(0)>::run(a...);
  }
}

template <class Conv, int W, int RPW>
struct Launch {
  static cudaError_t run(const ExactParams* P, int grid, cudaStream_t stream) {
    return launch_conv<Conv, W, RPW>(*P, grid, stream);
  }
};
template <class Conv, int W, int RPW>
struct MaxActive {
  static int run(size_t smem) { return max_active<Conv, W, RPW>(smem); }
};

}  // namespace

size_t exact_smem_bytes(int shape, int stages, int stage_bytes) {
  const int W = exact_shape_warps(shape);
  return static_cast<size_t>(stages) * stage_bytes + W * kDigitTileBytes + (i32_in_smem(W) ? W * kI32Bytes : 0) +
         kDigits * kDigits * sizeof(unsigned long long) + 2 * kExactMaxStages * sizeof(uint64_t);
}

int exact_pick_stages(int shape, int stage_bytes) {
  for (int st = kExactMaxStages; st >= 2; --st)
    if (exact_smem_bytes(shape, st, stage_bytes) <= 226 * 1024) return st;
  return 0;
}

bool exact_layout(ExactParams& P, int shape) {
  if (shape < 0 || shape >= kExactShapes) return false;
  const int tile = exact_tile_rows(shape);
  int off = 0;
  for (int j = 0; j < P.p; ++j) {
    P.col_off[j] = off;
    off += stage_col_bytes(P.col_bytes[j], tile);
  }
  const int stages = exact_pick_stages(shape, off);
  if (stages == 0) return false;
  P.shape = shape;
  P.stage_bytes = off;
  P.stages = stages;
  return true;
}

cudaError_t launch_exact(const ExactParams& P, int conv, int max_grid, cudaStream_t stream) {
  const int64_t tile = exact_tile_rows(P.shape);
  const int64_t tiles = (P.nmain + tile - 1) / tile;
  const int grid = static_cast<int>(std::min<int64_t>(std::max(max_grid, 1), std::max<int64_t>(tiles, 1)));
  return dispatch<Launch>(conv, P.shape, &P, grid, stream);
}

int exact_max_active_blocks(int conv, int shape, int stages, int stage_bytes) {
  return dispatch<MaxActive>(conv, shape, exact_smem_bytes(shape, stages, stage_bytes));
}

}  // namespace ss
