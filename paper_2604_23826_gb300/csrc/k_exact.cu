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
// but need fewer registers each and smaller stages.  Launch shape 3 replaces the
// mma.sync step by tcgen05 MMAs on shared-memory operand slots (below); it gives the same
// integers, moves about 1.3x the shared-memory bytes per row (the slots are written, then
// read twice as the MMA's A and B) and measured about 17 % slower on GB300, so shape 0 is
// the default.  All waits are bounded; an expired wait marks the call failed (the
// accumulator is then left unchanged).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tc05.cuh"

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

// The block's partial (int64, upper triangle) into the per-call accumulator by integer
// atomics; the last block to finish (ticket) adds the call's sum to the ctx accumulator unless
// a block recorded an error.  Every thread of the block calls this after the block's last
// shared-memory accumulation.
__device__ __forceinline__ void commit_block(const ExactParams& P, unsigned long long* cta_acc, uint32_t& s_bad,
                                             uint32_t& s_last) {
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

  commit_block(P, cta_acc, s_bad, s_last);
}

// ---- the tcgen05 form (launch shape 3) ----
// Each of kTcW converting warps turns its 64 rows of a stage into digits (in registers, which
// frees the stage for the next bulk copy), then, once the previous stage's MMA on its slot
// has completed, stores them in its own 4 KB operand slot: four sets of 16 rows side by side,
// slot row k (0..15) holding the 128 digits [set 0 | set 1 | set 2 | set 3] of stage rows
// 64 w + 16 b + k.  When every slot of the stage is stored, one thread issues per slot
// D += S^T S (M = N = 128, K = 16, f16 operands read MN-major, FP32 in tensor memory), each
// MMA followed by a commit that frees its slot: the diagonal 32 x 32 block b of D is the
// digit Gram of set b; the off-diagonal blocks (products of different rows) are never read.  A stage is one accumulation chain (kTcW slots:
// 16 kTcW = 224 rows per set, every partial sum an integer below 2^24, exact in FP32) into one
// of two 128-column accumulators.  Four reader warps take the diagonal blocks of each finished
// chain into int32 partial sums, every 64 chains into the block's int64 accumulator.
constexpr int kTcW = exact_shape_warps(3);
constexpr int kTcRpw = exact_shape_rpw(3);
static_assert(kTcRpw == 64, "a slot is one K = 16 step of four 16-row sets");
constexpr int kTcSlotBytes = kTcRpw * kDigits * 2;  // 4 KB
constexpr int kTcThreads = (kTcW + 6) * 32;         // + producer, MMA warp, 4 readers
constexpr int kTcProducer = kTcW, kTcMma = kTcW + 1;  // then the readers: warps kTcW + 2 ..
static_assert(16 * kTcW * 255 * 255 < (1 << 24), "a chain's partial sums stay exact in FP32");
constexpr int kTcI32Chains = 64;  // int32 partial sums stay below 64 x 16 kTcW x 255^2 < 2^31
static_assert(static_cast<long long>(kTcI32Chains) * 16 * kTcW * 255 * 255 < (1ll << 31), "int32 partial sums");
constexpr uint32_t kTcTmemCols = 256;
// MN-major with the 128-byte swizzle: a 1 KB atom holds 64 digits (128 B) of 8 slot rows, the
// 16-byte chunk x of row kk at chunk position x ^ kk (without the swizzle the chunks of one
// slot row would share four banks); LBO = next 64 digits (2 KB), SBO = next 8 slot rows (1 KB).
constexpr uint32_t kTcLbo = 2048, kTcSbo = 1024;
// kind::f16 instruction descriptor: D f32, A and B f16, both MN-major, M = N = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 15) | (1u << 16) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
constexpr int kTcTailTileBytes = kDigitTileBytes;  // the ragged tail's mma.sync tile
__host__ __device__ constexpr int tc_barriers() { return 2 * kExactMaxStages + kTcW + 6; }

// Byte offset in a slot of digits 8c..8c+7 of row r (0..63) of the warp's stage slice: set
// b = r / 16 holds slot digits 32 b .. 32 b + 31 of slot row k = r % 16.
__device__ __forceinline__ uint32_t tc_slot_off(int r, int c) {
  const int b = r >> 4, k = r & 15, x = 4 * (b & 1) + c, kk = k & 7;
  return static_cast<uint32_t>((b >> 1) * kTcLbo + (k >> 3) * kTcSbo + kk * 128 + ((x ^ kk) << 4));
}

// Shared-memory descriptor of a slot: MN-major, 128-byte swizzle (atoms 1024-byte aligned).
__device__ __forceinline__ uint64_t tc_slot_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((kTcLbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((kTcSbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;  // descriptor version
  d |= static_cast<uint64_t>(2) << 61;  // layout: 128-byte swizzle
  return d;
}

// bounded wait that also gives up once another role has given up
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, volatile unsigned int* dead) {
  return tc05::wait_live(bar, parity, dead);
}

// digits of row r of the stage (zeros past the valid rows)
template <class Conv, int TILE>
__device__ __forceinline__ void tc_row(const ExactParams& P, const uint8_t* st, int64_t row0, int r, int valid,
                                       uint32_t (&w)[16], uint32_t& bad) {
  if (r < valid && P.direct) {
    GlobalSrc src{&P, row0 + r};
    Conv::row(P, src, w, bad);
  } else if (r < valid) {
    Conv::row(P, Conv::template smem_src<TILE>(st, P, r), w, bad);
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) w[q] = 0u;
  }
}

template <class Conv>
__global__ void __launch_bounds__(kTcThreads, 1) exact_tc_kernel(const __grid_constant__ ExactParams P) {
  constexpr int kTile = kTcW * kTcRpw;  // rows of a stage
  extern __shared__ __align__(128) uint8_t smem[];
  // first: the operand slots, 1024-byte aligned for the swizzle (the size allows for the pad)
  uint8_t* slots = smem + ((1024u - (smem_u32(smem) & 1023u)) & 1023u);
  uint8_t* stage_base = slots + kTcW * kTcSlotBytes;
  uint8_t* tail_tile = stage_base + P.stages * P.stage_bytes;
  unsigned long long* cta_acc = reinterpret_cast<unsigned long long*>(tail_tile + kTcTailTileBytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(cta_acc + kDigits * kDigits);  // the copy has landed
  uint64_t* empty = full + kExactMaxStages;      // every converting warp has read the stage
  uint64_t* slots_full = empty + kExactMaxStages;  // every converting warp has stored its slot
  uint64_t* slot_free = slots_full + 1;            // the MMA reading slot w has completed (kTcW)
  uint64_t* acc_full = slot_free + kTcW;           // a chain's accumulator is complete (2)
  uint64_t* acc_empty = acc_full + 2;              // the readers have taken it (2)
  uint64_t* fin = acc_empty + 2;                   // every issued MMA has completed
  __shared__ uint32_t s_bad, s_last, s_tmem;
  __shared__ volatile unsigned int s_dead;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int stages = P.stages;
  const int64_t ntiles = (P.nmain + kTile - 1) / kTile;
  const int64_t my_count = (ntiles > blockIdx.x) ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  for (int i = threadIdx.x; i < kDigits * kDigits; i += blockDim.x) cta_acc[i] = 0ull;
  if (threadIdx.x == 0) {
    s_bad = 0;
    s_dead = 0;
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kTcW);
    }
    mbar_init(slots_full, kTcW);
    for (int w = 0; w < kTcW; ++w) mbar_init(&slot_free[w], 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(fin, 1);
    fence_mbar_init();
  }
  if (warp == kTcMma) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  uint32_t bad = 0;     // range violations seen by this thread
  uint32_t failed = 0;  // a bounded wait expired
  if (warp == kTcProducer) {
    // ---------------- producer: bulk copies of every column of each stage ----------------
    if (lane == 0 && !P.direct) {
      int64_t issued = 0;
      int s = 0;
      uint32_t ph = 0;
      int64_t row0 = static_cast<int64_t>(blockIdx.x) * kTile;
      const int64_t row_step = static_cast<int64_t>(gridDim.x) * kTile;
      for (int64_t k = 0; k < my_count; ++k, row0 += row_step) {
        // stage s was last used by tile k - stages, whose reading completed phase ph ^ 1
        if (k >= stages && !tc_wait(&empty[s], ph ^ 1u, &s_dead)) {
          failed = 1;
          s_dead = 1;
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
  } else if (warp < kTcW) {
    // ---------------- converting warps: 64 rows of each stage into the warp's slot ----------------
    const uint32_t slot = smem_u32(slots + warp * kTcSlotBytes);
    int s = 0;
    uint32_t ph = 0;
    int64_t row0 = static_cast<int64_t>(blockIdx.x) * kTile;
    const int64_t row_step = static_cast<int64_t>(gridDim.x) * kTile;
    for (int64_t k = 0; k < my_count; ++k, row0 += row_step) {
      if (!__all_sync(0xffffffffu, P.direct || tc_wait(&full[s], ph, &s_dead))) {
        failed = 1;
        s_dead = 1;
        break;
      }
      const int valid = static_cast<int>(min(static_cast<int64_t>(kTile), P.nmain - row0));
      const uint8_t* st = stage_base + s * P.stage_bytes;
      uint32_t wa[16], wb[16];
      tc_row<Conv, kTile>(P, st, row0, warp * kTcRpw + lane, valid, wa, bad);
      tc_row<Conv, kTile>(P, st, row0, warp * kTcRpw + 32 + lane, valid, wb, bad);
      __syncwarp();
      if (lane == 0 && !P.direct) mbar_arrive(&empty[s]);
      // the slot is read by the previous stage's MMA until it completes
      if (!__all_sync(0xffffffffu, k == 0 || tc_wait(&slot_free[warp], static_cast<uint32_t>((k - 1) & 1), &s_dead))) {
        failed = 1;
        s_dead = 1;
        break;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        st_shared_v4(slot + tc_slot_off(lane, c), wa[4 * c], wa[4 * c + 1], wa[4 * c + 2], wa[4 * c + 3]);
        st_shared_v4(slot + tc_slot_off(32 + lane, c), wb[4 * c], wb[4 * c + 1], wb[4 * c + 2], wb[4 * c + 3]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the slot, to the tensor cores
      __syncwarp();
      if (lane == 0) mbar_arrive(slots_full);
      if (++s == stages) {
        s = 0;
        ph ^= 1u;
      }
    }
    // ragged tail (fewer than 8 rows), read from global memory by warp 0 of block 0 and
    // multiplied with mma.sync in a tile of its own
    if (blockIdx.x == 0 && warp == 0 && P.nrows > P.nmain && !failed) {
      const int64_t r = P.nmain + lane;
      uint32_t w[16];
      if (r < P.nrows) {
        GlobalSrc src{&P, r};
        Conv::row(P, src, w, bad);
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) w[q] = 0u;
      }
      WarpAcc acc;
      WarpI32 ri;
#pragma unroll
      for (int e = 0; e < 6; ++e)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc.f[e][q] = 0.f;
          ri.i[e][q] = 0;
        }
      warp_mma_32rows(smem_u32(tail_tile), lane, w, acc);
      flush_f32(acc, ri);
      flush_i32([&](int e, int q) -> int32_t& { return ri.i[e][q]; }, cta_acc, lane);
    }
  } else if (warp == kTcMma) {
    // ---------------- MMA issuer: one chain of kTcW K = 16 steps per stage ----------------
    int b = 0;
    uint32_t pb = 0;  // phase parity of accumulator b's current use
    for (int64_t k = 0; k < my_count; ++k) {
      const bool ok = __shfl_sync(
          0xffffffffu,
          lane == 0 ? (tc_wait(slots_full, static_cast<uint32_t>(k & 1), &s_dead) &&
                       (k < 2 || tc_wait(&acc_empty[b], pb ^ 1u, &s_dead)))
                    : false,
          0);
      if (!ok) {
        if (lane == 0) {
          failed = 1;
          s_dead = 1;
        }
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // the slots' descriptors differ only in the address field ((address >> 4), no carry
      // inside the 227 KB of shared memory)
      const uint64_t d0 = tc_slot_desc(smem_u32(slots));
      const uint32_t dt = tmem + static_cast<uint32_t>(b * 128);
      if (tc05::elect_one()) {
#pragma unroll
        for (int w = 0; w < kTcW; ++w) {
          const uint64_t d = d0 + static_cast<uint64_t>(w * (kTcSlotBytes >> 4));
          tc05::mma_bf16(dt, d, d, kTcIdesc, w != 0 ? 1u : 0u);
          tc05::umma_commit(&slot_free[w]);  // slot w is free once this MMA has read it
        }
        tc05::umma_commit(&acc_full[b]);  // the chain is complete
      }
      __syncwarp();
      if (++b == 2) {
        b = 0;
        pb ^= 1u;
      }
    }
    if (tc05::elect_one()) tc05::umma_commit(fin);  // every issued MMA completes before the exit
    __syncwarp();
    if (lane == 0 && !mbar_wait_bounded(fin, 0)) failed = 1;
    __syncwarp();
  } else {
    // ---------------- readers: diagonal block q of each finished chain ----------------
    // Warp q (= warp % 4) reads tensor-memory lanes 32 q .. 32 q + 31, i.e. digit rows of set q;
    // lane l holds G_q[l][0..31], added to the int32 partial sums of row l.
    const int q = warp & 3;
    int32_t part[kDigits];
#pragma unroll
    for (int i = 0; i < kDigits; ++i) part[i] = 0;
    auto flush = [&]() {
#pragma unroll
      for (int i = 0; i < kDigits; ++i) {
        if (i >= lane && part[i] != 0)
          atomicAdd(&cta_acc[lane * kDigits + i], static_cast<unsigned long long>(static_cast<long long>(part[i])));
        part[i] = 0;
      }
    };
    int since = 0;
    for (int64_t c = 0; c < my_count; ++c) {
      const int b = static_cast<int>(c & 1);
      const bool ok = __shfl_sync(
          0xffffffffu, lane == 0 ? tc_wait(&acc_full[b], static_cast<uint32_t>((c >> 1) & 1), &s_dead) : false, 0);
      if (!ok) {
        if (lane == 0) {
          failed = 1;
          s_dead = 1;
        }
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t taddr = tmem + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(b * 128 + 32 * q);
      uint32_t v0[16], v1[16];
      tc05::tmem_ld16_issue(taddr, v0);
      tc05::tmem_ld16_issue(taddr + 16, v1);
      tc05::tmem_wait_ld();
      tc05::tmem_hold16(v0);
      tc05::tmem_hold16(v1);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        part[i] += __float2int_rn(__uint_as_float(v0[i]));
        part[16 + i] += __float2int_rn(__uint_as_float(v1[i]));
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
      if (++since == kTcI32Chains) {
        since = 0;
        flush();
      }
    }
    flush();
  }
  if (bad) atomicOr(&s_bad, DEV_ERANGE);
  if (failed) atomicOr(&s_bad, DEV_ETIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kTcMma) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
  }
  commit_block(P, cta_acc, s_bad, s_last);
}

// The kernel and block size of a (converter, shape) pair.
template <class Conv, int Shape>
struct ExactKernel {
  static constexpr int kThreads = exact_shape_tc(Shape) ? kTcThreads : (exact_shape_warps(Shape) + 1) * 32;
  static auto fn() {
    if constexpr (exact_shape_tc(Shape))
      return exact_tc_kernel<Conv>;
    else
      return exact_pass_kernel<Conv, exact_shape_warps(Shape), exact_shape_rpw(Shape)>;
  }
};

template <class Conv, int Shape>
cudaError_t launch_conv(const ExactParams& P, int grid, cudaStream_t stream) {
  const size_t smem = exact_smem_bytes(P.shape, P.stages, P.stage_bytes);
  auto* fn = ExactKernel<Conv, Shape>::fn();
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  fn<<<grid, ExactKernel<Conv, Shape>::kThreads, smem, stream>>>(P);
  return cudaGetLastError();
}

template <class Conv, int Shape>
int max_active(size_t smem) {
  auto* fn = ExactKernel<Conv, Shape>::fn();
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
    return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, ExactKernel<Conv, Shape>::kThreads, smem) != cudaSuccess)
    return 0;
  return n;
}

// The kernel of a (converter, shape) pair: F<Conv, Shape>::run(args...).
template <template <class, int> class F, class... A>
auto dispatch(int conv, int shape, A... a) {
  switch (conv * kExactShapes + shape) {
    case CONV_T1_L32 * kExactShapes + 0: return F<ConvT1<false>, 0>::run(a...);
    case CONV_T1_L32 * kExactShapes + 1: return F<ConvT1<false>, 1>::run(a...);
    case CONV_T1_L32 * kExactShapes + 2: return F<ConvT1<false>, 2>::run(a...);
    case CONV_T1_L32 * kExactShapes + 3: return F<ConvT1<false>, 3>::run(a...);
    case CONV_T1_L16 * kExactShapes + 0: return F<ConvT1<true>, 0>::run(a...);
    case CONV_T1_L16 * kExactShapes + 1: return F<ConvT1<true>, 1>::run(a...);
    case CONV_T1_L16 * kExactShapes + 2: return F<ConvT1<true>, 2>::run(a...);
    case CONV_T1_L16 * kExactShapes + 3: return F<ConvT1<true>, 3>::run(a...);
    case CONV_GENERIC * kExactShapes + 1: return F<ConvGeneric, 1>::run(a...);
    case CONV_GENERIC * kExactShapes + 2: return F<ConvGeneric, 2>::run(a...);
    case CONV_GENERIC * kExactShapes + 3: return F<ConvGeneric, 3>::run(a...);
    default: return F<ConvGeneric, 0>::run(a...);
  }
}

template <class Conv, int Shape>
struct Launch {
  static cudaError_t run(const ExactParams* P, int grid, cudaStream_t stream) {
    return launch_conv<Conv, Shape>(*P, grid, stream);
  }
};
template <class Conv, int Shape>
struct MaxActive {
  static int run(size_t smem) { return max_active<Conv, Shape>(smem); }
};

}  // namespace

size_t exact_smem_bytes(int shape, int stages, int stage_bytes) {
  if (exact_shape_tc(shape))
    return 1024 + static_cast<size_t>(kTcW) * kTcSlotBytes + static_cast<size_t>(stages) * stage_bytes + kTcTailTileBytes +
           kDigits * kDigits * sizeof(unsigned long long) + tc_barriers() * sizeof(uint64_t);
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
