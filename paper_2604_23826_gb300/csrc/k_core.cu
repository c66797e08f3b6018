// k_core.cu -- CUDA-core comparators of the fused pass for tables of any width:
// the plain FP64 pass (raw or shifted moments) for p > 12 and the FP32-core
// pass (shifted, FP32 FMA flushed into FP32 (hi, lo) pairs), arxiv 2604.23826
// "Data Representation and Sufficient Statistics" (column sums and X^T X in
// one pass) with the shift of "Numerical Considerations".
//
// The p x p output is cut into 64 x 64 tiles on or above the diagonal; block b
// takes tile b % ntiles over the (b / ntiles)-th range of rows, stages 64 rows
// of its two column blocks in shared memory (column-major, shifted), and each
// of its 4 warps accumulates one 32 x 32 sub-tile with a 4 x 8 register
// micro-tile per lane.  Warps write their partials to their own slots; the
// last block adds the slots in slot order into the context's double-double
// accumulators (fixed order: a given grid reproduces its bits).
#include "common.cuh"
#include "kernels.h"

namespace ss {

namespace {

constexpr int kT = 64;         // tile width
constexpr int kKC = 64;        // rows per chunk
constexpr int kLd = kKC + 1;   // padded column stride in shared memory
constexpr int kThreads = 128;

__device__ __forceinline__ double load_as_double(const void* col, int dt, int64_t r) {
  switch (dt) {
    case I16: return static_cast<double>(static_cast<const int16_t*>(col)[r]);
    case I32: return static_cast<double>(static_cast<const int32_t*>(col)[r]);
    case I64: return static_cast<double>(static_cast<const int64_t*>(col)[r]);
    case F32: return static_cast<double>(static_cast<const float*>(col)[r]);
    default: return static_cast<const double*>(col)[r];
  }
}

template <typename Acc>
__device__ __forceinline__ void pair_add(Acc& hi, Acc& lo, Acc v) {
  const Acc s = hi + v;
  const Acc bp = s - hi;
  lo += (hi - (s - bp)) + (v - bp);
  hi = s;
}

template <typename Acc>
__global__ void __launch_bounds__(kThreads) core_kernel(const __grid_constant__ CoreParams P) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  Acc* Xi = reinterpret_cast<Acc*>(smem_raw);  // [kT columns][kLd rows]
  Acc* Xj = Xi + kT * kLd;
  __shared__ unsigned int s_last;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x % P.ntiles, ks = blockIdx.x / P.ntiles;
  int I = 0, rem = tile;
  while (rem >= P.nblk - I) {
    rem -= P.nblk - I;
    ++I;
  }
  const int J = I + rem;
  const bool diag_tile = I == J;
  const int64_t r_begin = P.nrows * ks / P.ksplit, r_end = P.nrows * (ks + 1) / P.ksplit;
  const int sa = warp >> 1, sb = warp & 1;
  const bool active = !(diag_tile && sa > sb);
  const bool diag_sub = diag_tile && sa == sb;
  const Acc* XB = diag_tile ? Xi : Xj;
  const int ty = lane >> 2, tx = lane & 3;  // rows 4ty..4ty+3, cols 8tx..8tx+7 of the sub-tile

  Acc acc[4][8], hi[4][8], lo[4][8], sacc[4], shi[4], slo[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    sacc[i] = shi[i] = slo[i] = Acc(0);
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = hi[i][j] = lo[i][j] = Acc(0);
  }
  const bool flush_pairs = sizeof(Acc) == 4;
  int since = 0;

  for (int64_t c0 = r_begin; c0 < r_end; c0 += kKC) {
    const int rows = static_cast<int>(min(static_cast<int64_t>(kKC), r_end - c0));
    const int nblocks = diag_tile ? 1 : 2;
    for (int task = threadIdx.x; task < nblocks * kT * kKC; task += kThreads) {
      const int k = task % kKC, c = (task / kKC) % kT, blk = task / (kT * kKC);
      const int col = (blk == 0 ? I : J) * kT + c;
      Acc v = Acc(0);
      if (col < P.p && k < rows) {
        const double x = load_as_double(P.cols[col], P.dtype[col], c0 + k);
        v = static_cast<Acc>(P.shift ? x - P.shift[col] : x);
      }
      (blk == 0 ? Xi : Xj)[c * kLd + k] = v;
    }
    __syncthreads();
    if (active) {
      const Acc* a_base = Xi + (32 * sa + 4 * ty) * kLd;
      const Acc* b_base = XB + (32 * sb + 8 * tx) * kLd;
      for (int k = 0; k < rows; ++k) {
        Acc a[4], b[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = a_base[i * kLd + k];
#pragma unroll
        for (int j = 0; j < 8; ++j) b[j] = b_base[j * kLd + k];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
          if (diag_sub && tx == 0) sacc[i] += a[i];
        }
      }
      if (flush_pairs && (since += rows) >= P.flush_rows) {
        since = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          pair_add(shi[i], slo[i], sacc[i]);
          sacc[i] = Acc(0);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            pair_add(hi[i][j], lo[i][j], acc[i][j]);
            acc[i][j] = Acc(0);
          }
        }
      }
    }
    __syncthreads();
  }
  // slot (block, warp): (hi, lo) doubles of the 32 x 32 sub-tile, then 32 column sums
  double* slot = P.slots + (static_cast<size_t>(blockIdx.x) * 4 + warp) * kCoreSlotDoubles;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    pair_add(shi[i], slo[i], sacc[i]);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      pair_add(hi[i][j], lo[i][j], acc[i][j]);
      const int row = 4 * ty + i, col = 8 * tx + j;
      slot[2 * (row * 32 + col)] = active ? static_cast<double>(hi[i][j]) : 0.0;
      slot[2 * (row * 32 + col) + 1] = active ? static_cast<double>(lo[i][j]) : 0.0;
    }
    if (tx == 0) {
      slot[2 * 1024 + 2 * (4 * ty + i)] = diag_sub ? static_cast<double>(shi[i]) : 0.0;
      slot[2 * 1024 + 2 * (4 * ty + i) + 1] = diag_sub ? static_cast<double>(slo[i]) : 0.0;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(P.ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int p = P.p, Tn = p * (p + 1) / 2;
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
      j = k = e - Tn;
    }
    const int Ib = j / kT, Jb = k / kT;
    const int tidx = Ib * P.nblk - Ib * (Ib - 1) / 2 + (Jb - Ib);
    const int w = ((j % kT) / 32) * 2 + (k % kT) / 32;
    const int off = e < Tn ? 2 * ((j % 32) * 32 + (k % 32)) : 2 * 1024 + 2 * (j % 32);
    double h = 0.0, l = 0.0;
    for (int kk = 0; kk < P.ksplit; ++kk) {
      const double* sl = P.slots + ((static_cast<size_t>(kk) * P.ntiles + tidx) * 4 + w) * kCoreSlotDoubles;
      pair_add(h, l, __ldcg(sl + off));
      pair_add(h, l, __ldcg(sl + off + 1));
    }
    double* dh = e < Tn ? &P.acc_S[e] : &P.acc_s[e - Tn];
    double* dl = e < Tn ? &P.acc_S_lo[e] : &P.acc_s_lo[e - Tn];
    pair_add(*dh, *dl, h);
    *dl += l;
  }
  if (threadIdx.x == 0) {
    *P.acc_n += P.nrows;
    *P.ticket = 0u;
  }
}

}  // namespace

size_t core_slot_doubles(int grid) { return static_cast<size_t>(grid) * 4 * kCoreSlotDoubles; }

cudaError_t launch_core(const CoreParams& P, bool fp32, int grid, cudaStream_t stream) {
  const size_t smem = 2 * kT * kLd * (fp32 ? sizeof(float) : sizeof(double));
  if (fp32) {
    cudaError_t e = cudaFuncSetAttribute(core_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    core_kernel<float><<<grid, kThreads, smem, stream>>>(P);
  } else {
    cudaError_t e = cudaFuncSetAttribute(core_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    core_kernel<double><<<grid, kThreads, smem, stream>>>(P);
  }
  return cudaGetLastError();
}

}  // namespace ss
