// k_fp64.cu -- the plain FP64 CUDA-core pass, the comparator of the exact pass.
//
// arxiv 2604.23826 ("Data Representation and Sufficient Statistics", and the
// "intentionally simple" reduction kernels of "Discussion and Lessons
// Learned"): rows are double-precision values; each thread accumulates its rows
// into the column sums and the upper triangle of X^T X (90 FP64 registers for
// p = 12) with FMA, warps reduce with shuffles, each block writes one slot, and
// the last block to finish adds the slots in block order (a fixed order, so a
// given grid gives bit-identical results run to run) into the context's
// double-double accumulator.  With a shift vector c the same pass runs on
// x - c (the "shifted" comparator of equal accuracy).
#include "common.cuh"
#include "kernels.h"

namespace ss {

namespace {

constexpr int kP = 12;                         // columns handled by the row-parallel kernel
constexpr int kT = kP * (kP + 1) / 2;          // 78
constexpr int kE = kT + kP;                    // values per row-set: S upper + s
constexpr int kThreads = 256;

__device__ __forceinline__ double load_d(const void* col, int dt, int64_t r) {
  switch (dt) {
    case I16: return static_cast<double>(static_cast<const int16_t*>(col)[r]);
    case I32: return static_cast<double>(static_cast<const int32_t*>(col)[r]);
    case I64: return static_cast<double>(static_cast<const int64_t*>(col)[r]);
    case F32: return static_cast<double>(static_cast<const float*>(col)[r]);
    default: return static_cast<const double*>(col)[r];
  }
}

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__global__ void __launch_bounds__(kThreads, 1) fp64_rows_kernel(const __grid_constant__ Fp64Params P,
                                                                unsigned int* ticket) {
  __shared__ double red[kThreads / 32][kE];
  __shared__ unsigned int s_last;
  double s[kP], S[kT];
#pragma unroll
  for (int j = 0; j < kP; ++j) s[j] = 0.0;
#pragma unroll
  for (int t = 0; t < kT; ++t) S[t] = 0.0;
  double c[kP];
#pragma unroll
  for (int j = 0; j < kP; ++j) c[j] = (P.shift && j < P.p) ? P.shift[j] : 0.0;

  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < P.nrows; r += stride) {
    double x[kP];
#pragma unroll
    for (int j = 0; j < kP; ++j) x[j] = (j < P.p) ? load_d(P.cols[j], P.dtype[j], r) - c[j] : 0.0;
    int t = 0;
#pragma unroll
    for (int j = 0; j < kP; ++j) {
      s[j] += x[j];
#pragma unroll
      for (int k = j; k < kP; ++k, ++t) S[t] = fma(x[j], x[k], S[t]);
    }
  }
  // warp reduction (butterfly, fixed pattern)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int j = 0; j < kP; ++j) s[j] += __shfl_xor_sync(0xffffffffu, s[j], off);
#pragma unroll
    for (int t = 0; t < kT; ++t) S[t] += __shfl_xor_sync(0xffffffffu, S[t], off);
  }
  if (lane == 0) {
#pragma unroll
    for (int t = 0; t < kT; ++t) red[warp][t] = S[t];
#pragma unroll
    for (int j = 0; j < kP; ++j) red[warp][kT + j] = s[j];
  }
  __syncthreads();
  // block slot: warps summed in warp order
  for (int e = threadIdx.x; e < kE; e += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) v += red[w][e];
    P.slots[static_cast<size_t>(blockIdx.x) * kE + e] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last block: slots in block order, then into the double-double accumulator
  const int T = P.p * (P.p + 1) / 2;
  for (int e = threadIdx.x; e < kE; e += blockDim.x) {
    double v = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) v += __ldcg(&P.slots[static_cast<size_t>(b) * kE + e]);
    // map the padded (kP) layout to the packed layout of p columns
    double *hi, *lo;
    if (e < kT) {
      int j = 0, t = e;
      while (t >= kP - j) { t -= kP - j; ++j; }
      const int k = j + t;
      if (j >= P.p || k >= P.p) continue;
      const int idx = j * P.p - j * (j - 1) / 2 + (k - j);
      hi = &P.acc_S[idx];
      lo = &P.acc_S_lo[idx];
      (void)T;
    } else {
      const int j = e - kT;
      if (j >= P.p) continue;
      hi = &P.acc_s[j];
      lo = &P.acc_s_lo[j];
    }
    double sum, err;
    two_sum(*hi, v, sum, err);
    *hi = sum;
    *lo += err;
  }
  if (threadIdx.x == 0) {
    *P.acc_n += P.nrows;
    *ticket = 0u;
  }
}

// shift = the mean of the first min(nrows, kPivotRows) rows of the columns (nrows >= 1); for
// FP32 columns rounded to FP32, so that x - c is exact wherever x and c are within a factor
// of two of each other (and the FP32-core pass's rounding of x - c to FP32 is exact there)
__global__ void set_shift_kernel(Fp64Params P) {
  const int j = threadIdx.x;
  const int k = static_cast<int>(min(static_cast<int64_t>(kPivotRows), P.nrows));
  if (j < P.p) {
    double sum = 0.0;
    for (int i = 0; i < k; ++i) sum += load_d(P.cols[j], P.dtype[j], i);
    const double c = sum / k;
    const_cast<double*>(P.shift)[j] = P.dtype[j] == F32 ? static_cast<double>(static_cast<float>(c)) : c;
  }
}

}  // namespace

cudaError_t launch_fp64(const Fp64Params& P, int grid, cudaStream_t stream) {
  // the slot buffer starts with the ticket word (one double), the slots follow
  unsigned int* ticket = reinterpret_cast<unsigned int*>(P.slots);
  Fp64Params Q = P;
  Q.slots = P.slots + 1;
  fp64_rows_kernel<<<grid, kThreads, 0, stream>>>(Q, ticket);
  return cudaGetLastError();
}

size_t fp64_slot_doubles(int grid) { return static_cast<size_t>(grid) * kE + 1; }

namespace {
__global__ void merge_i64_kernel(long long* dst, const long long* src, int count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) dst[i] += src[i];
}
__global__ void merge_dd_kernel(double* hi, double* lo, const double* shi, const double* slo, int count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    double s, e;
    two_sum(hi[i], shi[i], s, e);
    hi[i] = s;
    lo[i] += e + slo[i];
  }
}
}  // namespace

// dd helpers for the pivot change
__device__ __forceinline__ void dd_add(double& hi, double& lo, double bhi, double blo) {
  double s, e;
  two_sum(hi, bhi, s, e);
  e += lo + blo;
  hi = s + e;
  lo = e - (hi - s);
}
__device__ __forceinline__ void dd_mul(double ahi, double alo, double bhi, double blo, double& hi, double& lo) {
  const double p = ahi * bhi;
  const double e = fma(ahi, bhi, -p) + (ahi * blo + alo * bhi);
  hi = p + e;
  lo = e - (hi - p);
}

// Shifted moments about pivot c_s (n_s rows: s' = sum (x - c_s), S' = sum (x - c_s)(x - c_s)^T)
// re-expressed about c_d and added to the destination's: with d = c_s - c_d,
//   sum (x - c_d)              = s' + n_s d
//   sum (x - c_d)(x - c_d)^T   = S' + d s'^T + s' d^T + n_s d d^T      (packed upper)
// in double-double (Chan, Golub and LeVeque's pairwise update with the two means replaced by pivots).
__global__ void merge_shifted_kernel(double* s, double* s_lo, double* S, double* S_lo, const double* c_d,
                                     const double* ss, const double* ss_lo, const double* Ss, const double* Ss_lo,
                                     const double* c_s, const long long* n_s, int p) {
  const int T = p * (p + 1) / 2;
  const double ns = static_cast<double>(*n_s);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < T + p; e += gridDim.x * blockDim.x) {
    if (e < T) {
      int j = 0, rm = e;
      while (rm >= p - j) {
        rm -= p - j;
        ++j;
      }
      const int k = j + rm;
      double dj, dj_lo, dk, dk_lo;
      two_sum(c_s[j], -c_d[j], dj, dj_lo);
      two_sum(c_s[k], -c_d[k], dk, dk_lo);
      double hi = Ss[e], lo = Ss_lo[e], th, tl;
      dd_mul(dj, dj_lo, ss[k], ss_lo[k], th, tl);
      dd_add(hi, lo, th, tl);
      dd_mul(dk, dk_lo, ss[j], ss_lo[j], th, tl);
      dd_add(hi, lo, th, tl);
      double dd_hi, dd_lo;
      dd_mul(dj, dj_lo, dk, dk_lo, dd_hi, dd_lo);
      dd_mul(dd_hi, dd_lo, ns, 0.0, th, tl);
      dd_add(hi, lo, th, tl);
      dd_add(S[e], S_lo[e], hi, lo);
    } else {
      const int j = e - T;
      double dj, dj_lo, th, tl;
      two_sum(c_s[j], -c_d[j], dj, dj_lo);
      double hi = ss[j], lo = ss_lo[j];
      dd_mul(dj, dj_lo, ns, 0.0, th, tl);
      dd_add(hi, lo, th, tl);
      dd_add(s[j], s_lo[j], hi, lo);
    }
  }
}

__global__ void pivot_to_float_kernel(const double* src, float* dst, int p) {
  for (int j = threadIdx.x; j < p; j += blockDim.x) dst[j] = static_cast<float>(src[j]);
}

cudaError_t launch_pivot_to_float(const double* src, float* dst, int p, cudaStream_t stream) {
  pivot_to_float_kernel<<<1, 256, 0, stream>>>(src, dst, p);
  return cudaGetLastError();
}

cudaError_t launch_merge_shifted(double* s, double* s_lo, double* S, double* S_lo, const double* c_d,
                                 const double* ss, const double* ss_lo, const double* Ss, const double* Ss_lo,
                                 const double* c_s, const long long* n_s, int p, cudaStream_t stream) {
  const int count = p * (p + 1) / 2 + p;
  merge_shifted_kernel<<<(count + 255) / 256, 256, 0, stream>>>(s, s_lo, S, S_lo, c_d, ss, ss_lo, Ss, Ss_lo, c_s,
                                                                 n_s, p);
  return cudaGetLastError();
}

cudaError_t launch_merge_i64(long long* dst, const long long* src, int count, cudaStream_t stream) {
  merge_i64_kernel<<<(count + 255) / 256, 256, 0, stream>>>(dst, src, count);
  return cudaGetLastError();
}

cudaError_t launch_merge_dd(double* dst_hi, double* dst_lo, const double* src_hi, const double* src_lo, int count,
                            cudaStream_t stream) {
  merge_dd_kernel<<<(count + 255) / 256, 256, 0, stream>>>(dst_hi, dst_lo, src_hi, src_lo, count);
  return cudaGetLastError();
}

cudaError_t launch_set_shift(const void* const* cols, const int32_t* dtypes, int p, int64_t rows, double* shift,
                             cudaStream_t stream) {
  Fp64Params P{};
  P.nrows = rows;
  for (int j = 0; j < p && j < 256; ++j) {
    P.cols[j] = cols[j];
    P.dtype[j] = dtypes[j];
  }
  P.p = p;
  P.shift = shift;
  set_shift_kernel<<<1, 256, 0, stream>>>(P);
  return cudaGetLastError();
}

}  // namespace ss
