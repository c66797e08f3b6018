// k_split.cu -- sufficient statistics of FP32 tables on the tensor cores with a
// two-term bf16 split ("BF16x3" / "BF16x4"), the floating-point variant of the
// fused pass (arxiv 2604.23826, "Data Representation and Sufficient
// Statistics"; the shift against cancellation follows "Numerical
// Considerations": X^T X and N mu mu^T must not be formed separately).
//
// Every value is shifted by a pivot c_j (the mean of the table's first rows), r = x - c,
// and split r = h + l with h = bf16(r), l = bf16(r - h).  Then
//   S' = sum_rows r r^T  ~  H^T H + H^T L + L^T H      (BF16x3)
//                         + L^T L                      (BF16x4)
// with FP32 accumulation on the tensor cores (mma.sync m16n8k16 bf16): every
// 16-row K block is a fresh chain, smallest products first, added into FP32
// accumulators rounding to nearest (the tensor core's own accumulation
// truncates); every `flush_rows` rows of a warp those are added into FP32
// (hi, lo) pairs with TwoSum, so long sums keep ~48 bits.  BF16x3 keeps L^T L
// on the diagonal sub-tiles (the positive bias of the dropped term's diagonal).  Column sums
// s' = sum r come from the same products with an extra operand column of ones.
//
// Work split: the p x p output is cut into T x T tiles (T = 32 or 64) and only
// tiles on or above the diagonal are computed; block b takes tile b % ntiles
// over the b / ntiles-th contiguous range of rows.  In a block, each of 4 warps
// owns one 32 x 32 sub-tile (T = 64) or a quarter of the rows (T = 32).  Every
// warp writes its FP32-pair partials to its own slot; the last block to finish
// (ticket) adds all slots, in slot order, into the context's double-double
// accumulators -- a fixed order, so a given grid reproduces its bits exactly.
#include "common.cuh"
#include "kernels.h"

namespace ss {

namespace {

constexpr int kKC = 64;            // rows per chunk
constexpr int kThreads = 128;      // 4 warps
constexpr int kSlotFloats = 2 * (32 * 32 + 32);  // (hi, lo) of a 32x32 sub-tile + 32 column sums

__device__ __forceinline__ uint32_t bf16x2_pack(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (v - bp);
  hi = s;
  lo += err;
}

// Row R of a [64 rows x T] bf16 tile: 2T bytes, 16-byte chunk c stored at c ^ swz(R).
template <int T>
__device__ __forceinline__ uint32_t chunk_addr(uint32_t base, int R, int c) {
  if (T == 64) return base + R * 128 + ((c ^ (R & 7)) << 4);
  return base + R * 64 + ((c ^ ((R >> 1) & 3)) << 4);
}

struct Frags {
  uint32_t r[4], q[4];  // chunks 0..3 of the 32-column group: rows 0..7 (r) and 8..15 (q) of a K block
};

template <int T>
__device__ __forceinline__ void load_frags(uint32_t tile, int kb, int c0, int lane, Frags& f) {
  const int m = lane >> 3, rr = 16 * kb + (lane & 7);
  ldsm_x4_trans(chunk_addr<T>(tile, rr, c0 + m), f.r[0], f.r[1], f.r[2], f.r[3]);
  ldsm_x4_trans(chunk_addr<T>(tile, rr + 8, c0 + m), f.q[0], f.q[1], f.q[2], f.q[3]);
}

// One block's share of one table: tile local_block % ntiles over the
// (local_block / ntiles)-th row range.  `units` = ntiles * ksplit blocks of the table.
template <int T, bool X4, class Cols>
__device__ __forceinline__ void split_block(const Cols& cols, const SplitParams& P, int local_block, int units,
                                            uint8_t* sbuf, unsigned int* s_last_ptr) {
  constexpr int NS = T / 32;        // sub-tiles per side
  constexpr int NSUB = NS * NS;     // 4 (T=64) or 1 (T=32)
  constexpr int RG = 4 / NSUB;      // row groups: 1 (T=64) or 4 (T=32)
  unsigned int& s_last = *s_last_ptr;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = local_block % P.ntiles, ks = local_block / P.ntiles;
  int I = 0, rem = tile;
  while (rem >= P.nblk - I) {
    rem -= P.nblk - I;
    ++I;
  }
  const int J = I + rem;
  const bool diag_tile = I == J;
  const int64_t r_begin = P.nrows * ks / P.ksplit, r_end = P.nrows * (ks + 1) / P.ksplit;

  const int sub = warp % NSUB, rg = warp / NSUB;
  const int sa = sub / NS, sb = sub % NS;
  const bool active = !(diag_tile && sa > sb);
  const bool diag_sub = diag_tile && sa == sb;

  const uint32_t base = smem_u32(sbuf);
  const uint32_t tHI = base, tLI = base + kKC * T * 2, tHJ = base + 2 * kKC * T * 2, tLJ = base + 3 * kKC * T * 2;
  const uint32_t tHB = diag_tile ? tHI : tHJ, tLB = diag_tile ? tLI : tLJ;

  float acc[2][4][4], hi[2][4][4], lo[2][4][4];
  float sacc[2][4], shi[2][4], slo[2][4];  // column sums (diagonal sub-tiles): the ones operand column
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      sacc[a][b] = shi[a][b] = slo[a][b] = 0.f;
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = hi[a][b][c] = lo[a][b][c] = 0.f;
    }
  // B fragment of a [16 x 8] block whose column 0 is ones: lanes with g == 0 hold (1, 1)
  const uint32_t ones_b = (lane >> 2) == 0 ? 0x3F803F80u : 0u;

  const int nblocks = diag_tile ? 1 : 2;
  const int flush_kblocks = max(1, P.flush_rows / 16);  // K blocks of 16 rows between flushes
  int since = 0;

  for (int64_t c0 = r_begin; c0 < r_end; c0 += kKC) {
    const int rows = static_cast<int>(min(static_cast<int64_t>(kKC), r_end - c0));
    // ---- load, shift, split: task = (block, 8-column chunk, row) ----
    const int ntask = nblocks * (T / 8) * kKC;
    for (int task = threadIdx.x; task < ntask; task += kThreads) {
      const int k = task % kKC, c8 = (task / kKC) % (T / 8), blk = task / (kKC * (T / 8));
      const int colbase = (blk == 0 ? I : J) * T + c8 * 8;
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float r2[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int col = colbase + 2 * e + u;
          float x = 0.f;
          if (col < P.p && k < rows) x = __ldg(cols[col] + (c0 + k)) - __ldg(P.shift + col);
          r2[u] = x;
        }
        hw[e] = bf16x2_pack(r2[0], r2[1]);
        lw[e] = bf16x2_pack(r2[0] - bf16_lo(hw[e]), r2[1] - bf16_hi(hw[e]));
      }
      const uint32_t th = blk == 0 ? tHI : tHJ, tl = blk == 0 ? tLI : tLJ;
      asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(chunk_addr<T>(th, k, c8)), "r"(hw[0]), "r"(hw[1]),
                   "r"(hw[2]), "r"(hw[3])
                   : "memory");
      asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(chunk_addr<T>(tl, k, c8)), "r"(lw[0]), "r"(lw[1]),
                   "r"(lw[2]), "r"(lw[3])
                   : "memory");
    }
    __syncthreads();
    // ---- tensor-core products on this warp's sub-tile ----
    if (active) {
#pragma unroll 1
      for (int kb = rg; kb < kKC / 16; kb += RG) {
        Frags AH, AL, BH, BL;
        load_frags<T>(tHI, kb, 4 * sa, lane, AH);
        load_frags<T>(tLI, kb, 4 * sa, lane, AL);
        if (diag_sub) {
          BH = AH;
          BL = AL;
        } else {
          load_frags<T>(tHB, kb, 4 * sb, lane, BH);
          load_frags<T>(tLB, kb, 4 * sb, lane, BL);
        }
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
          const uint32_t ah0 = AH.r[2 * mi], ah1 = AH.r[2 * mi + 1], ah2 = AH.q[2 * mi], ah3 = AH.q[2 * mi + 1];
          const uint32_t al0 = AL.r[2 * mi], al1 = AL.r[2 * mi + 1], al2 = AL.q[2 * mi], al3 = AL.q[2 * mi + 1];
#pragma unroll
          for (int nj = 0; nj < 4; ++nj) {
            if (diag_sub && 8 * nj + 7 < 16 * mi) continue;  // below the diagonal
            // a fresh chain per K block, smallest products first, added to the FP32
            // accumulators rounding to nearest; BF16x3 keeps L^T L on diagonal sub-tiles
            // (the positive bias of its diagonal)
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            if (X4 || diag_sub) mma_bf16_16816(d, al0, al1, al2, al3, BL.r[nj], BL.q[nj]);
            mma_bf16_16816(d, al0, al1, al2, al3, BH.r[nj], BH.q[nj]);
            mma_bf16_16816(d, ah0, ah1, ah2, ah3, BL.r[nj], BL.q[nj]);
            mma_bf16_16816(d, ah0, ah1, ah2, ah3, BH.r[nj], BH.q[nj]);
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[mi][nj][c] += d[c];
          }
          if (diag_sub) {
            // column sums: A rows (columns of X) against a ones column; H^T 1 + L^T 1 = sum (h + l)
            float t4[4] = {0.f, 0.f, 0.f, 0.f};
            mma_bf16_16816(t4, al0, al1, al2, al3, ones_b, ones_b);
            mma_bf16_16816(t4, ah0, ah1, ah2, ah3, ones_b, ones_b);
#pragma unroll
            for (int c = 0; c < 4; ++c) sacc[mi][c] += t4[c];
          }
        }
        if (++since >= flush_kblocks) {
          since = 0;
#pragma unroll
          for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              two_sum_acc(shi[a][b], slo[a][b], sacc[a][b]);
              sacc[a][b] = 0.f;
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                two_sum_acc(hi[a][b][c], lo[a][b][c], acc[a][b][c]);
                acc[a][b][c] = 0.f;
              }
            }
        }
      }
    }
    __syncthreads();
  }
  // final flush and slot write: slot (block, warp) holds (hi, lo) of its 32x32 sub-tile and 32 sums
  float* slot = P.slots + (static_cast<size_t>(local_block) * 4 + warp) * kSlotFloats;
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      two_sum_acc(shi[a][b], slo[a][b], sacc[a][b]);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        two_sum_acc(hi[a][b][c], lo[a][b][c], acc[a][b][c]);
        const int row = 16 * a + g + ((c >> 1) << 3), col = 8 * b + 2 * t + (c & 1);
        slot[2 * (row * 32 + col)] = active ? hi[a][b][c] : 0.f;
        slot[2 * (row * 32 + col) + 1] = active ? lo[a][b][c] : 0.f;
      }
    }
  // sums: the ones column is column 0 of the extra N block, held by lanes t == 0 in c = 0 and c = 2
  if (t == 0) {
#pragma unroll
    for (int a = 0; a < 2; ++a) {
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const int row = 16 * a + g + 8 * h2;  // column of X within the sub-tile
        // sums were accumulated in sacc[a][c] with c = 0 (rows g) and c = 2 (rows g + 8); the other
        // entries of the ones block are zero
        const int c = 2 * h2;
        slot[2 * 1024 + 2 * row] = diag_sub ? shi[a][c] : 0.f;
        slot[2 * 1024 + 2 * row + 1] = diag_sub ? slo[a][c] : 0.f;
      }
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(P.ticket, 1u) == static_cast<unsigned int>(units - 1)) ? 1u : 0u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last block: every packed-upper entry of p x p, slots added in slot order
  const int p = P.p;
  const int Tn = p * (p + 1) / 2;
  for (int e = threadIdx.x; e < Tn + p; e += kThreads) {
    int j, k;
    if (e < Tn) {
      j = 0;
      int rm = e;
      while (rm >= p - j) {
        rm -= p - j;
        ++j;
      }
      k = j + rm;
    } else {
      j = k = e - Tn;  // column sum of j
    }
    const int Ib = j / T, Jb = k / T;  // tile (Ib, Jb) with Ib <= Jb
    const int tidx = Ib * P.nblk - Ib * (Ib - 1) / 2 + (Jb - Ib);
    const int sa2 = (j % T) / 32, sb2 = (k % T) / 32;
    const int subw = sa2 * NS + sb2;
    const int rr = j % 32, cc = k % 32;
    float h = 0.f, l = 0.f;
    for (int kk = 0; kk < P.ksplit; ++kk) {
      const size_t blk = static_cast<size_t>(kk) * P.ntiles + tidx;
      for (int w = 0; w < 4; ++w) {
        if (w % NSUB != (e < Tn ? subw : (sa2 * NS + sa2))) continue;
        const float* sl = P.slots + (blk * 4 + w) * kSlotFloats;
        const int off = e < Tn ? 2 * (rr * 32 + cc) : 2 * 1024 + 2 * rr;
        two_sum_acc(h, l, __ldcg(sl + off));
        two_sum_acc(h, l, __ldcg(sl + off + 1));
      }
    }
    double* dh = e < Tn ? &P.acc_S[e] : &P.acc_s[e - Tn];
    double* dl = e < Tn ? &P.acc_S_lo[e] : &P.acc_s_lo[e - Tn];
    const double v = static_cast<double>(h) + static_cast<double>(l);
    const double s = *dh + v;
    const double bp = s - *dh;
    *dl += (*dh - (s - bp)) + (v - bp);
    *dh = s;
  }
  if (threadIdx.x == 0) {
    *P.acc_n += P.nrows;
    *P.ticket = 0u;
  }
}

template <int T, bool X4>
__global__ void __launch_bounds__(kThreads) split_kernel(const __grid_constant__ SplitParams P) {
  __shared__ __align__(128) uint8_t sbuf[4 * kKC * T * 2];  // H_I, L_I, H_J, L_J
  __shared__ unsigned int s_last;
  split_block<T, X4>(P.cols, P, blockIdx.x, gridDim.x, sbuf, &s_last);
}

// Many tables in one launch: block b runs unit units[b] = (table, local block) of table
// descriptors tabs[] (their column pointer arrays live in device memory).
template <int T, bool X4>
__global__ void __launch_bounds__(kThreads) split_batched_kernel(const SplitParams* __restrict__ tabs,
                                                                 const int2* __restrict__ units) {
  __shared__ __align__(128) uint8_t sbuf[4 * kKC * T * 2];
  __shared__ unsigned int s_last;
  const int2 u = units[blockIdx.x];
  const SplitParams& P = tabs[u.x];
  split_block<T, X4>(P.col_ptrs, P, u.y, P.ntiles * P.ksplit, sbuf, &s_last);
}

// pivot c_j = the mean of the first min(rows, kPivotRows) rows of FP32 columns, rounded to FP32
// (called once, rows >= 1)
__device__ void split_pivot(const SplitParams& P, int64_t rows, double* shift_d) {
  const int k = static_cast<int>(min(static_cast<int64_t>(kPivotRows), rows));
  for (int j = threadIdx.x; j < P.p; j += blockDim.x) {
    const float* col = P.col_ptrs ? P.col_ptrs[j] : P.cols[j];
    double sum = 0.0;
    for (int i = 0; i < k; ++i) sum += static_cast<double>(col[i]);
    const float v = static_cast<float>(sum / k);
    const_cast<float*>(P.shift)[j] = v;
    shift_d[j] = static_cast<double>(v);
  }
}

__global__ void split_shift_kernel(const __grid_constant__ SplitParams P, int64_t rows, double* shift_d) {
  split_pivot(P, rows, shift_d);
}

__global__ void split_shift_batched_kernel(const SplitParams* __restrict__ tabs, const int* __restrict__ which) {
  const SplitParams& P = tabs[which[blockIdx.x]];
  split_pivot(P, P.nrows, P.shift_d);
}

}  // namespace

size_t split_slot_floats(int grid) { return static_cast<size_t>(grid) * 4 * kSlotFloats; }

int split_tile(int p) { return p <= 32 ? 32 : 64; }

cudaError_t launch_split(const SplitParams& P, int T, bool x4, int grid, cudaStream_t stream) {
  if (T == 32) {
    if (x4)
      split_kernel<32, true><<<grid, kThreads, 0, stream>>>(P);
    else
      split_kernel<32, false><<<grid, kThreads, 0, stream>>>(P);
  } else {
    if (x4)
      split_kernel<64, true><<<grid, kThreads, 0, stream>>>(P);
    else
      split_kernel<64, false><<<grid, kThreads, 0, stream>>>(P);
  }
  return cudaGetLastError();
}

cudaError_t launch_split_batched(const SplitParams* tabs, const int2* units, int nunits, int T, bool x4,
                                 cudaStream_t stream) {
  if (nunits <= 0) return cudaSuccess;
  if (T == 32) {
    if (x4)
      split_batched_kernel<32, true><<<nunits, kThreads, 0, stream>>>(tabs, units);
    else
      split_batched_kernel<32, false><<<nunits, kThreads, 0, stream>>>(tabs, units);
  } else {
    if (x4)
      split_batched_kernel<64, true><<<nunits, kThreads, 0, stream>>>(tabs, units);
    else
      split_batched_kernel<64, false><<<nunits, kThreads, 0, stream>>>(tabs, units);
  }
  return cudaGetLastError();
}

cudaError_t launch_split_shift_batched(const SplitParams* tabs, const int* which, int count, cudaStream_t stream) {
  if (count <= 0) return cudaSuccess;
  split_shift_batched_kernel<<<count, 64, 0, stream>>>(tabs, which);
  return cudaGetLastError();
}

cudaError_t launch_split_shift(const SplitParams& P, int64_t rows, double* shift_d, cudaStream_t stream) {
  split_shift_kernel<<<1, 256, 0, stream>>>(P, rows, shift_d);
  return cudaGetLastError();
}

}  // namespace ss
