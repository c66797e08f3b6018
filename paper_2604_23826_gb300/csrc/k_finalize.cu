// k_finalize.cu -- from the sufficient statistics (n, s, S) to mean,
// covariance, correlation and the PCA eigenpairs, in one thread block on the
// device (arxiv 2604.23826: "Data Representation and Sufficient Statistics" --
// mean, covariance and correlation from the aggregated matrices only;
// "Numerical Considerations" -- cancellation between X^T X and N mu mu^T, and the
// identifier dropped from the analysis; "Principal Component Analysis Results"
// -- eigenpairs of the p x p matrix).
//
// STATS_EXACT: the digit Gram G is recombined into exact integers
//   r_j = sum_a 256^a G[0][(j,a)],  R_jk = sum_{a,b} 256^(a+b) G[(j,a)][(k,b)]
// (values scaled by 2^-shift for real columns), in 256-bit two's complement
// arithmetic, and centred exactly: C_jk = n R_jk - r_j r_k, so no cancellation
// can occur; cov_jk = C_jk 2^-(shift_j + shift_k) / (n (n - 1)) is then rounded.
// STATS_FP64: the paper's raw-moment formula (S_jk - s_j s_k / n) / (n - 1) in FP64.
// Eigenpairs: cyclic Jacobi with the parallel round-robin ordering (Brent & Luk):
// each round applies n/2 rotations on disjoint index pairs at once.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace ss {

namespace {

constexpr int kThreads = 256;

// ------------------------------- 256-bit integers -------------------------------
struct i256 {
  uint64_t w[4];  // two's complement, w[0] least significant
};

__device__ __forceinline__ i256 i256_from(int64_t v) {
  const uint64_t ext = v < 0 ? ~0ull : 0ull;
  return i256{{static_cast<uint64_t>(v), ext, ext, ext}};
}
__device__ __forceinline__ bool i256_neg(const i256& a) { return static_cast<int64_t>(a.w[3]) < 0; }
__device__ __forceinline__ bool i256_zero(const i256& a) { return !(a.w[0] | a.w[1] | a.w[2] | a.w[3]); }

__device__ __forceinline__ i256 i256_add(const i256& a, const i256& b) {
  i256 r;
  uint64_t c = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint64_t s = a.w[i] + b.w[i];
    const uint64_t c1 = s < a.w[i];
    r.w[i] = s + c;
    const uint64_t c2 = r.w[i] < s;
    c = c1 | c2;
  }
  return r;
}
__device__ __forceinline__ i256 i256_negate(const i256& a) {
  i256 r;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.w[i] = ~a.w[i];
  return i256_add(r, i256_from(1));
}
__device__ __forceinline__ i256 i256_sub(const i256& a, const i256& b) { return i256_add(a, i256_negate(b)); }
__device__ __forceinline__ i256 i256_abs(const i256& a) { return i256_neg(a) ? i256_negate(a) : a; }

// a << bits, 0 <= bits < 256
__device__ __forceinline__ i256 i256_shl(const i256& a, int bits) {
  i256 r{{0, 0, 0, 0}};
  const int lw = bits >> 6, b = bits & 63;
  for (int i = 3; i >= 0; --i) {
    const int src = i - lw;
    if (src < 0) continue;
    uint64_t v = a.w[src] << b;
    if (b && src > 0) v |= a.w[src - 1] >> (64 - b);
    r.w[i] = v;
  }
  return r;
}

// |a| * |b| modulo 2^256, unsigned limbs
__device__ __forceinline__ i256 u256_mul(const i256& a, const i256& b) {
  i256 r{{0, 0, 0, 0}};
  for (int i = 0; i < 4; ++i) {
    uint64_t carry = 0;
    for (int j = 0; i + j < 4; ++j) {
      const uint64_t lo = a.w[i] * b.w[j];
      const uint64_t hi = __umul64hi(a.w[i], b.w[j]);
      uint64_t s = r.w[i + j] + lo;
      uint64_t c = s < lo;
      s += carry;
      c += s < carry;
      r.w[i + j] = s;
      carry = hi + c;
    }
  }
  return r;
}
__device__ __forceinline__ i256 i256_mul(const i256& a, const i256& b) {
  const bool neg = i256_neg(a) != i256_neg(b);
  const i256 m = u256_mul(i256_abs(a), i256_abs(b));
  return neg ? i256_negate(m) : m;
}

// Correctly rounded conversion to double (round to nearest even): the top 64
// significant bits with a sticky bit for everything below them.
__device__ double i256_to_double(const i256& a) {
  if (i256_zero(a)) return 0.0;
  const bool neg = i256_neg(a);
  const i256 m = i256_abs(a);
  int top = 3;
  while (top > 0 && m.w[top] == 0) --top;
  const int lz = __clzll(static_cast<long long>(m.w[top]));
  const int msb = top * 64 + 63 - lz;  // index of the highest set bit
  double d;
  if (msb < 64) {
    d = __ull2double_rn(m.w[0]);
  } else {
    const int sh = msb - 63;  // drop sh low bits
    const i256 t = i256{{0, 0, 0, 0}};
    (void)t;
    const int lw = sh >> 6, b = sh & 63;
    uint64_t hi64 = m.w[lw] >> b;
    if (b && lw + 1 < 4) hi64 |= m.w[lw + 1] << (64 - b);
    uint64_t sticky = 0;
    for (int i = 0; i < lw; ++i) sticky |= m.w[i];
    if (b) sticky |= m.w[lw] & ((1ull << b) - 1);
    d = ldexp(__ull2double_rn(hi64 | (sticky ? 1ull : 0ull)), sh);
  }
  return neg ? -d : d;
}

__device__ bool i256_fits_i128(const i256& a, int64_t& lo, int64_t& hi) {
  lo = static_cast<int64_t>(a.w[0]);
  hi = static_cast<int64_t>(a.w[1]);
  const uint64_t ext = hi < 0 ? ~0ull : 0ull;
  return a.w[2] == ext && a.w[3] == ext;
}

// ------------------------------- Jacobi (one block) -------------------------------
// A (m x m padded, row-major, lda = pa) symmetric in global scratch; V likewise.
__device__ void jacobi_block(double* A, double* V, int pa, double* evals, double* evecs, double* flags) {
  __shared__ double s_c[kThreads], s_s[kThreads];
  __shared__ int s_p[kThreads], s_q[kThreads];
  __shared__ double s_red[kThreads];
  __shared__ int s_done;
  const int tid = threadIdx.x;
  const int m = pa + (pa & 1);  // even number of indices; index pa is a dummy when pa is odd
  for (int i = tid; i < pa * pa; i += blockDim.x) V[i] = (i / pa == i % pa) ? 1.0 : 0.0;
  __syncthreads();
  // Frobenius norm for the stopping test
  double loc = 0.0;
  for (int i = tid; i < pa * pa; i += blockDim.x) loc += A[i] * A[i];
  s_red[tid] = loc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) s_red[tid] += s_red[tid + w];
    __syncthreads();
  }
  const double fro2 = s_red[0];
  __syncthreads();
  int sweep = 0;
  for (; sweep < 60; ++sweep) {
    loc = 0.0;
    for (int i = tid; i < pa * pa; i += blockDim.x)
      if (i / pa != i % pa) loc += A[i] * A[i];
    s_red[tid] = loc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (tid < w) s_red[tid] += s_red[tid + w];
      __syncthreads();
    }
    if (tid == 0) s_done = (s_red[0] == 0.0 || s_red[0] <= 1e-34 * fro2) ? 1 : 0;
    __syncthreads();
    if (s_done) break;
    for (int round = 0; round < m - 1; ++round) {
      // pairs of this round: (m-1, round) and ((round+i) mod (m-1), (round-i) mod (m-1))
      for (int i = tid; i < m / 2; i += blockDim.x) {
        int p, q;
        if (i == 0) {
          p = round;
          q = m - 1;
        } else {
          p = (round + i) % (m - 1);
          q = (round - i + (m - 1)) % (m - 1);
        }
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double c = 1.0, s = 0.0;
        if (q < pa) {
          const double apq = A[p * pa + q];
          if (apq != 0.0) {
            const double theta = (A[q * pa + q] - A[p * pa + p]) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        s_c[i] = c;
        s_s[i] = s;
        s_p[i] = p;
        s_q[i] = q;
      }
      __syncthreads();
      // rows: (row p, row q) <- (c row p - s row q, s row p + c row q)
      for (int idx = tid; idx < (m / 2) * pa; idx += blockDim.x) {
        const int i = idx / pa, k = idx % pa;
        const int p = s_p[i], q = s_q[i];
        if (q >= pa || s_s[i] == 0.0) continue;
        const double c = s_c[i], s = s_s[i];
        const double apk = A[p * pa + k], aqk = A[q * pa + k];
        A[p * pa + k] = c * apk - s * aqk;
        A[q * pa + k] = s * apk + c * aqk;
      }
      __syncthreads();
      // columns of A and V
      for (int idx = tid; idx < (m / 2) * pa; idx += blockDim.x) {
        const int i = idx / pa, k = idx % pa;
        const int p = s_p[i], q = s_q[i];
        if (q >= pa || s_s[i] == 0.0) continue;
        const double c = s_c[i], s = s_s[i];
        const double akp = A[k * pa + p], akq = A[k * pa + q];
        A[k * pa + p] = c * akp - s * akq;
        A[k * pa + q] = s * akp + c * akq;
        const double vkp = V[k * pa + p], vkq = V[k * pa + q];
        V[k * pa + p] = c * vkp - s * vkq;
        V[k * pa + q] = s * vkp + c * vkq;
      }
      __syncthreads();
      for (int i = tid; i < m / 2; i += blockDim.x) {
        const int p = s_p[i], q = s_q[i];
        if (q < pa && s_s[i] != 0.0) {
          A[p * pa + q] = 0.0;
          A[q * pa + p] = 0.0;
        }
      }
      __syncthreads();
    }
  }
  // order descending; sign: largest-magnitude component positive
  __shared__ int s_order[256];
  if (tid == 0) {
    for (int i = 0; i < pa; ++i) s_order[i] = i;
    for (int i = 0; i < pa; ++i) {
      int best = i;
      for (int j = i + 1; j < pa; ++j)
        if (A[s_order[j] * pa + s_order[j]] > A[s_order[best] * pa + s_order[best]]) best = j;
      const int t = s_order[i];
      s_order[i] = s_order[best];
      s_order[best] = t;
    }
    flags[2] = sweep;
  }
  __syncthreads();
  for (int k = tid; k < pa; k += blockDim.x) {
    const int col = s_order[k];
    evals[k] = A[col * pa + col];
    int imax = 0;
    for (int i = 1; i < pa; ++i)
      if (fabs(V[i * pa + col]) > fabs(V[imax * pa + col])) imax = i;
    const double sg = V[imax * pa + col] < 0.0 ? -1.0 : 1.0;
    for (int i = 0; i < pa; ++i) evecs[k * pa + i] = sg * V[i * pa + col];
  }
  __syncthreads();
}

__device__ void finalize_body(const FinalParams& P) {
  __shared__ long long G[kDigits * kDigits];
  __shared__ int s_amap[256];  // analysis column index -> table column
  __shared__ int s_pa;
  __shared__ int s_zero;
  __shared__ int s_over;
  const int tid = threadIdx.x;
  const int p = P.p;
  if (tid == 0) {
    int pa = 0;
    for (int j = 0; j < p; ++j)
      if (!P.col[j].is_ident) s_amap[pa++] = j;
    s_pa = pa;
    s_zero = 0;
    s_over = 0;
  }
  const FinalLayout L = final_layout(p, 0);  // offsets of n, s, S and exact blocks do not depend on pa
  __syncthreads();
  const int pa = s_pa;
  const FinalLayout LA = final_layout(p, pa);
  double* out = P.out;
  double* flags = out + LA.flags;
  double* cov = out + LA.cov;
  double* corr = out + LA.corr;
  const int T = p * (p + 1) / 2;
  double n_d = 0.0;

  if (P.mode == 0) {
    // ------------------------------- STATS_EXACT -------------------------------
    for (int i = tid; i < kDigits * kDigits; i += blockDim.x) {
      const int r = i / kDigits, c = i % kDigits;
      G[i] = (r <= c) ? P.g[r * kDigits + c] : P.g[c * kDigits + r];
    }
    __syncthreads();
    const long long n = G[0];
    n_d = static_cast<double>(n);
    if (tid == 0) reinterpret_cast<long long*>(out)[L.n] = n;
    // exact column sums r_j (scaled by 2^-shift_j)
    for (int j = tid; j < p; j += blockDim.x) {
      const FinalPlanCol cj = P.col[j];
      i256 r = i256_from(0);
      for (int a = 0; a < cj.k; ++a) r = i256_add(r, i256_shl(i256_from(G[cj.off + a]), 8 * a));
      out[L.s + j] = ldexp(i256_to_double(r), -cj.shift);
      int64_t lo = 0, hi = 0;
      if (!cj.is_real) {
        if (!i256_fits_i128(r, lo, hi)) atomicOr(&s_over, 1);
      } else {
        lo = hi = 0;
      }
      reinterpret_cast<int64_t*>(out)[L.s_ex + 2 * j] = lo;
      reinterpret_cast<int64_t*>(out)[L.s_ex + 2 * j + 1] = hi;
    }
    // exact cross products R_jk and, for analysis pairs, the exact centred numerator
    const i256 nn = i256_from(n);
    for (int t = tid; t < T; t += blockDim.x) {
      int j = 0, rem = t;
      while (rem >= p - j) {
        rem -= p - j;
        ++j;
      }
      const int k = j + rem;
      const FinalPlanCol cj = P.col[j], ck = P.col[k];
      i256 R = i256_from(0);
      for (int a = 0; a < cj.k; ++a)
        for (int b = 0; b < ck.k; ++b)
          R = i256_add(R, i256_shl(i256_from(G[(cj.off + a) * kDigits + ck.off + b]), 8 * (a + b)));
      out[L.S + t] = ldexp(i256_to_double(R), -(cj.shift + ck.shift));
      int64_t lo = 0, hi = 0;
      if (!cj.is_real && !ck.is_real) {
        if (!i256_fits_i128(R, lo, hi)) atomicOr(&s_over, 1);
      }
      reinterpret_cast<int64_t*>(out)[L.S_ex + 2 * t] = lo;
      reinterpret_cast<int64_t*>(out)[L.S_ex + 2 * t + 1] = hi;
      if (pa > 0 && !cj.is_ident && !ck.is_ident && n >= 2) {
        i256 rj = i256_from(0), rk = i256_from(0);
        for (int a = 0; a < cj.k; ++a) rj = i256_add(rj, i256_shl(i256_from(G[cj.off + a]), 8 * a));
        for (int b = 0; b < ck.k; ++b) rk = i256_add(rk, i256_shl(i256_from(G[ck.off + b]), 8 * b));
        const i256 C = i256_sub(i256_mul(nn, R), i256_mul(rj, rk));
        const i256 den = i256_mul(nn, i256_from(n - 1));
        const double v = ldexp(i256_to_double(C) / i256_to_double(den), -(cj.shift + ck.shift));
        int aj = 0, ak = 0;
        for (int q = 0; q < pa; ++q) {
          if (s_amap[q] == j) aj = q;
          if (s_amap[q] == k) ak = q;
        }
        cov[aj * pa + ak] = v;
        cov[ak * pa + aj] = v;
      }
    }
    __syncthreads();
    for (int a = tid; a < pa; a += blockDim.x) {
      const int j = s_amap[a];
      out[LA.mean + a] = out[L.s + j] / n_d;
      if (out[LA.cov + a * pa + a] == 0.0) atomicAdd(&s_zero, 1);
    }
  } else {
    // ------------------------------- FP64 modes -------------------------------
    const long long n = *P.fn;
    n_d = static_cast<double>(n);
    if (tid == 0) reinterpret_cast<long long*>(out)[L.n] = n;
    // raw sums (shifted sums mapped back: s = s' + n c, S = S' + c s'^T + s' c^T + n c c^T)
    for (int j = tid; j < p; j += blockDim.x) {
      double v = P.fs[j] + P.fs_lo[j];
      if (P.shift) v = fma(n_d, P.shift[j], v);
      out[L.s + j] = v;
      reinterpret_cast<int64_t*>(out)[L.s_ex + 2 * j] = 0;
      reinterpret_cast<int64_t*>(out)[L.s_ex + 2 * j + 1] = 0;
    }
    for (int t = tid; t < T; t += blockDim.x) {
      int j = 0, rem = t;
      while (rem >= p - j) {
        rem -= p - j;
        ++j;
      }
      const int k = j + rem;
      double v = P.fS[t] + P.fS_lo[t];
      const double sj = P.fs[j] + P.fs_lo[j], sk = P.fs[k] + P.fs_lo[k];
      if (P.shift) {
        const double cj = P.shift[j], ck = P.shift[k];
        v += cj * sk + sj * ck + n_d * cj * ck;
      }
      out[L.S + t] = v;
      reinterpret_cast<int64_t*>(out)[L.S_ex + 2 * t] = 0;
      reinterpret_cast<int64_t*>(out)[L.S_ex + 2 * t + 1] = 0;
      if (!P.col[j].is_ident && !P.col[k].is_ident && n >= 2) {
        // the paper's raw-moment formula on the (shifted) sums, in FP64
        const double Sjk = P.fS[t] + P.fS_lo[t];
        const double c = (Sjk - sj * sk / n_d) / (n_d - 1.0);
        int aj = 0, ak = 0;
        for (int q = 0; q < pa; ++q) {
          if (s_amap[q] == j) aj = q;
          if (s_amap[q] == k) ak = q;
        }
        cov[aj * pa + ak] = c;
        cov[ak * pa + aj] = c;
      }
    }
    __syncthreads();
    for (int a = tid; a < pa; a += blockDim.x) {
      const int j = s_amap[a];
      out[LA.mean + a] = out[L.s + j] / n_d;
      if (!(out[LA.cov + a * pa + a] > 0.0)) atomicAdd(&s_zero, 1);
    }
  }
  __syncthreads();
  // correlation: cov_jk / (sqrt(cov_jj) sqrt(cov_kk)); NaN where a variance is not positive
  for (int i = tid; i < pa * pa; i += blockDim.x) {
    const int a = i / pa, b = i % pa;
    const double va = cov[a * pa + a], vb = cov[b * pa + b];
    double r;
    if (!(va > 0.0) || !(vb > 0.0))
      r = __longlong_as_double(0x7ff8000000000000ll);
    else if (a == b)
      r = 1.0;
    else
      r = cov[i] / (sqrt(va) * sqrt(vb));
    corr[i] = r;
  }
  __syncthreads();
  if (tid == 0) {
    flags[0] = s_over ? 1.0 : 0.0;
    flags[1] = s_zero;
    flags[2] = 0.0;
    flags[3] = 0.0;
    flags[5] = 0.0;
    flags[6] = 0.0;
  }
  __syncthreads();
  const bool pca_ok = P.want_pca && pa > 0 && n_d >= 2.0 && !(P.pca_on == 1 && s_zero > 0);
  if (P.defer_ctl && tid == 0) *P.defer_ctl = pca_ok ? 1 : 0;
  if (pca_ok && P.defer_A) {
    // the grid-wide solver takes over: the matrix, zero-padded to even order m
    const int m = P.defer_m;
    const double* src = P.pca_on ? corr : cov;
    for (int i = tid; i < m * m; i += blockDim.x) {
      const int r = i / m, c = i % m;
      P.defer_A[i] = (r < pa && c < pa) ? src[r * pa + c] : 0.0;
    }
  } else if (pca_ok) {
    double* A = P.work;
    double* V = P.work + static_cast<size_t>(pa) * pa;
    const double* src = P.pca_on ? corr : cov;
    for (int i = tid; i < pa * pa; i += blockDim.x) A[i] = src[i];
    __syncthreads();
    jacobi_block(A, V, pa, out + LA.evals, out + LA.evecs, flags);
    if (tid == 0) flags[3] = 1.0;
  } else {
    for (int i = tid; i < pa; i += blockDim.x) out[LA.evals + i] = __longlong_as_double(0x7ff8000000000000ll);
    for (int i = tid; i < pa * pa; i += blockDim.x) out[LA.evecs + i] = __longlong_as_double(0x7ff8000000000000ll);
  }
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 1) finalize_kernel(const __grid_constant__ FinalParams P) {
  finalize_body(P);
}

// many contexts at once: block b finalizes Ps[b] (each with its own scratch and output)
__global__ void __launch_bounds__(kThreads, 1) finalize_batched_kernel(const FinalParams* __restrict__ Ps) {
  finalize_body(Ps[blockIdx.x]);
}

cudaError_t launch_finalize_batched(const FinalParams* d_params, int count, cudaStream_t stream) {
  if (count <= 0) return cudaSuccess;
  finalize_batched_kernel<<<count, kThreads, 0, stream>>>(d_params);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalParams& P, cudaStream_t stream) {
  finalize_kernel<<<1, kThreads, 0, stream>>>(P);
  return cudaGetLastError();
}

// ------------------------------- Jacobi over the whole GPU -------------------------------
// One rotation of the round-robin ordering, on the even order m: in round r, pair 0 is
// (r, m - 1) and pair i > 0 is ((r + i) mod (m - 1), (r - i) mod (m - 1)), sorted.  Every index
// occurs in exactly one pair, so a round's rotations commute and A' = J^T A J splits into
// independent 2 x 2 blocks (pair i's rows, pair j's columns).
namespace {

constexpr int kJacThreads = 256;
constexpr int kJW = 8;         // indices per Jacobi block
constexpr int kJP = 2 * kJW;   // order of a block pair's diagonal problem; kJP x kJP = kJacThreads
static_assert(kJP * kJP == kJacThreads, "one thread per entry of a block-pair tile");
constexpr unsigned long long kGridWaitNs = 2000000000ull;  // a grid-wide wait gives up after 2 s

__device__ __forceinline__ void pair_of(int r, int i, int m, int& p, int& q) {
  if (i == 0) {
    p = r;
    q = m - 1;
  } else {
    p = (r + i) % (m - 1);
    q = (r - i + (m - 1)) % (m - 1);
  }
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* a) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch.  Thread 0 of each block publishes the block's
// writes (fence), arrives, and the last arrival resets the count and advances the
// generation; the others poll the generation.  A poll that outlasts wait_ns sets the
// shared error word; a block that sees it set leaves.  Returns false in every block once
// the error is set.
__device__ bool grid_sync(unsigned int* bar, unsigned int& gen, int* s_ok, unsigned long long wait_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int g = gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&bar[0], 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicExch(&bar[1], g + 1);
    } else {
      const unsigned long long t0 = global_ns();
      while (ld_acquire_u32(&bar[1]) == g) {
        if (ld_acquire_u32(&bar[2]) != 0u) break;
        if (global_ns() - t0 > wait_ns) {
          atomicExch(&bar[2], 1u);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (ld_acquire_u32(&bar[2]) != 0u) ok = 0;
    gen = g + 1;
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// deterministic block sum (fixed shuffle tree, warps added in order); result valid in thread 0
__device__ double block_sum(double v, double* s_red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kJacThreads / 32; ++w) t += s_red[w];
  __syncthreads();
  return t;
}

// Z = op(X) Y for m x m row-major matrices (op(X) = X, or X^T when xt), 16 x 16 tiles shared
// out over the grid.
__device__ void grid_matmul(const double* X, const double* Y, double* Z, int m, bool xt, double (*sx)[17],
                            double (*sy)[17]) {
  const int nt = (m + 15) / 16;
  const int r = threadIdx.x / 16, c = threadIdx.x % 16;
  for (int t = blockIdx.x; t < nt * nt; t += gridDim.x) {
    const int gi = (t / nt) * 16 + r, gj = (t % nt) * 16 + c;
    double acc = 0.0;
    for (int k0 = 0; k0 < m; k0 += 16) {
      const int gk = k0 + c;
      const int ri = (t / nt) * 16 + r;
      sx[r][c] = (ri < m && gk < m) ? (xt ? __ldcg(X + static_cast<size_t>(gk) * m + ri)
                                          : __ldcg(X + static_cast<size_t>(ri) * m + gk))
                                    : 0.0;
      const int rk = k0 + r;
      sy[r][c] = (rk < m && gj < m) ? __ldcg(Y + static_cast<size_t>(rk) * m + gj) : 0.0;
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) acc = fma(sx[r][kk], sy[kk][c], acc);
      __syncthreads();
    }
    if (gi < m && gj < m) __stcg(Z + static_cast<size_t>(gi) * m + gj, acc);
  }
}

}  // namespace

size_t jacobi_scratch_doubles(int pa) {
  const size_t m = (pa + kJP - 1) / kJP * kJP;
  return 4 * m * m + static_cast<size_t>(pa) * pa + (m / kJP) * kJP * kJP + 1024 + 8;
}

int jacobi_grid_blocks(int pa, int sms) {
  const int m = (pa + kJP - 1) / kJP * kJP, np = m / kJP;
  int g = 2 * np * np;  // the work items of a block round's second step
  if (g > sms) g = sms;
  if (g > 512) g = 512;  // two partial sums per block fit the 1024-double slot area
  return g < 1 ? 1 : g;
}

__global__ void __launch_bounds__(kJacThreads, 1) jacobi_grid_kernel(const __grid_constant__ JacobiParams J) {
  __shared__ double s_c[128], s_s[128];
  __shared__ double s_red[kJacThreads / 32];
  __shared__ double s_x[16][17], s_y[16][17];
  __shared__ double s_S[kJP][kJP + 1], s_Q[kJP][kJP + 1], s_X[kJP][kJP + 1], s_T[kJP][kJP + 1],
      s_QA[kJP][kJP + 1], s_QB[kJP][kJP + 1];
  __shared__ double s_d[256];
  __shared__ int s_order[256];
  __shared__ double s_bv[kJacThreads / 32];
  __shared__ int s_bi[kJacThreads / 32];
  __shared__ double s_val;
  __shared__ int s_ok;
  if (__ldcg(J.ctl) == 0) return;  // the finalize kernel found the eigenpairs undefined
  const int tid = threadIdx.x;
  const unsigned long long wait_ns = J.wait_ns > 0 ? static_cast<unsigned long long>(J.wait_ns) : kGridWaitNs;
  const int pa = J.pa, m = J.m;
  const int nthreads = gridDim.x * kJacThreads;
  const int gtid = blockIdx.x * kJacThreads + tid;
  unsigned int gen = 0;
  bool seeded = false;
  double* A = J.a;
  double* B = J.b;
  double* V = J.v;
  double* flags = J.out + J.flags_off;
  // a block told to be absent leaves before its first arrival: the other blocks' waits at
  // that barrier run out after wait_ns and the call reports the timeout (the failure path
  // of a stalled block, taken without a fault)
  if (static_cast<int>(blockIdx.x) == J.absent_block) goto timed_out;

  // V = I, or the previous eigenvectors as columns
  for (int i = gtid; i < m * m; i += nthreads) {
    const int r = i / m, c = i % m;
    double v = (r == c) ? 1.0 : 0.0;
    if (J.basis && r < pa && c < pa) v = J.basis[static_cast<size_t>(c) * pa + r];
    __stcg(V + i, v);
  }
  if (!grid_sync(J.bar, gen, &s_ok, wait_ns)) goto timed_out;
  if (J.basis) {
    // the seed is used only if its columns are orthonormal: max |V^T V - I| <= 1e-9
    grid_matmul(V, V, J.w, m, true, s_x, s_y);
    if (!grid_sync(J.bar, gen, &s_ok, wait_ns)) goto timed_out;
    double dev = 0.0;
    for (int i = gtid; i < m * m; i += nthreads) {
      const double x = __ldcg(J.w + i) - ((i / m == i % m) ? 1.0 : 0.0);
      dev = fmax(dev, x != x ? 1.0 : fabs(x));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    if ((tid & 31) == 0) s_red[tid >> 5] = dev;
    __syncthreads();
    if (tid == 0) {
      double d = 0.0;
      for (int w = 0; w < kJacThreads / 32; ++w) d = fmax(d, s_red[w]);
      __stcg(J.slots + blockIdx.x, d);
    }
    if (!grid_sync(J.bar, gen, &s_ok, wait_ns)) goto timed_out;
    if (tid == 0) {
      double d = 0.0;
      for (int b = 0; b < static_cast<int>(gridDim.x); ++b) d = fmax(d, __ldcg(J.slots + b));
      s_val = d;
    }
    __syncthreads();
    seeded = s_val <= 1e-9;
    __syncthreads();
    if (!seeded) {  // cold start after all
      for (int i = gtid; i < m * m; i += nthreads) __stcg(V + i, (i / m == i % m) ? 1.0 : 0.0);
      if (!grid_sync(J.bar, gen, &s_ok, wait_ns)) goto timed_out;
    }
  }
  if (seeded) {
    // A <- V^T A V, symmetrised: W = A V, B = V^T W, A = (B + B^T) / 2
    grid_matmul(A, V, J.w, m, false, s_x, s_y);
    if (!grid_sync(J.bar, gen, &s_ok, wait_ns)) goto timed_out;
    grid_matmul(V, J.w, B, m, true, s_x, s_y);
    if (!grid_sync(J.bar, gen, &s_ok, wait_ns)) goto timed_out;
    for (int i = gtid; i < m * m; i += nthreads) {
      const int r = i / m, c = i % m;
      __stcg(A + i, 0.5 * (__ldcg(B + static_cast<size_t>(r) * m + c) + __ldcg(B + static_cast<size_t>(c) * m + r)));
    }
    if (!grid_sync(J.bar, gen, &s_ok, wait_ns)) goto timed_out;
  }
  {
    // ||A||_F^2 once; the off-diagonal part before every sweep
    double lf = 0.0, lo = 0.0;
    for (int i = gtid; i < m * m; i += nthreads) {
      const double x = __ldcg(A + i);
      lf += x * x;
      if (i / m != i % m) lo += x * x;
    }
    const double bf = block_sum(lf, s_red);
    const double bo = block_sum(lo, s_red);
    if (tid == 0) {
      __stcg(J.slots + blockIdx.x, bf);
      __stcg(J.slots + gridDim.x + blockIdx.x, bo);
    }
    if (!grid_sync(J.bar, gen, &s_ok, wait_ns)) goto timed_out;
    if (tid == 0) {
      double t = 0.0;
      for (int b = 0; b < static_cast<int>(gridDim.x); ++b) t += __ldcg(J.slots + b);
      s_val = t;
    }
    __syncthreads();
    const double fro2 = s_val;
    __syncthreads();
    const int nb = m / kJW, np = nb / 2;  // index blocks of kJW, and the pairs of a block round
    const int lr_ = tid / kJP, lc_ = tid % kJP;  // this thread's entry of a kJP x kJP tile
    int sweep = 0;
    double prev_off = 0.0;
    for (; sweep < 60; ++sweep) {
      if (tid == 0) {
        double t = 0.0;
        for (int b = 0; b < static_cast<int>(gridDim.x); ++b) t += __ldcg(J.slots + gridDim.x + b);
        s_val = t;
      }
      __syncthreads();
      const double off = s_val;
      __syncthreads();
      // converged: off-diagonal mass negligible, or (block updates leave rounding noise in every
      // off-diagonal entry) no longer falling quadratically once below 1e-26 of ||A||^2
      if (off == 0.0 || off <= 1e-34 * fro2 || (sweep > 0 && off <= 1e-26 * fro2 && off > 0.0625 * prev_off)) break;
      prev_off = off;
      for (int br = 0; br < nb - 1; ++br) {
        // (1) every block pair's kJP x kJP diagonal problem: one cyclic Jacobi sweep in shared
        //     memory, its rotations accumulated in Q (to J.q), its result written to B
        for (int P = blockIdx.x; P < np; P += gridDim.x) {
          int bi, bj;
          pair_of(br, P, nb, bi, bj);
          const int gr = lr_ < kJW ? bi * kJW + lr_ : bj * kJW + lr_ - kJW;
          const int gc = lc_ < kJW ? bi * kJW + lc_ : bj * kJW + lc_ - kJW;
          s_S[lr_][lc_] = __ldcg(A + static_cast<size_t>(gr) * m + gc);
          s_Q[lr_][lc_] = lr_ == lc_ ? 1.0 : 0.0;
          __syncthreads();
          for (int lr = 0; lr < kJP - 1; ++lr) {
            if (tid < kJP / 2) {
              int p, q;
              pair_of(lr, tid, kJP, p, q);
              double c = 1.0, sn = 0.0;
              const double apq = s_S[p][q];
              if (apq != 0.0) {
                // the one-block solver's t = sgn(theta) / (|theta| + sqrt(theta^2 + 1)), theta =
                // d / (2 apq), d = aqq - app, multiplied through by 2 |apq|: one square root and
                // one division in the dependent chain instead of two of each
                const double d = s_S[q][q] - s_S[p][p];
                const double t = (d >= 0.0 ? 2.0 * apq : -2.0 * apq) / (fabs(d) + sqrt(d * d + 4.0 * apq * apq));
                c = rsqrt(t * t + 1.0);
                sn = t * c;
              }
              s_c[tid] = c;
              s_s[tid] = sn;
            }
            __syncthreads();
            if (tid < (kJP / 2) * kJP) {  // rows p, q
              const int i = tid / kJP, k = tid % kJP;
              int p, q;
              pair_of(lr, i, kJP, p, q);
              const double c = s_c[i], sn = s_s[i];
              if (sn != 0.0) {
                const double apk = s_S[p][k], aqk = s_S[q][k];
                s_S[p][k] = c * apk - sn * aqk;
                s_S[q][k] = sn * apk + c * aqk;
              }
            }
            __syncthreads();
            {  // columns p, q of S (first half of the threads) and of Q (second half)
              const int u = tid % ((kJP / 2) * kJP);
              const int i = u / kJP, k = u % kJP;
              int p, q;
              pair_of(lr, i, kJP, p, q);
              const double c = s_c[i], sn = s_s[i];
              const bool onS = tid < (kJP / 2) * kJP;
              double(*X)[kJP + 1] = onS ? s_S : s_Q;
              if (sn != 0.0) {
                const double xkp = X[k][p], xkq = X[k][q];
                // the rotated pair's off-diagonal entries are zero by construction
                X[k][p] = (onS && k == q) ? 0.0 : c * xkp - sn * xkq;
                X[k][q] = (onS && k == p) ? 0.0 : sn * xkp + c * xkq;
              }
            }
            __syncthreads();
          }
          __stcg(J.q + static_cast<size_t>(P) * kJP * kJP + tid, s_Q[lr_][lc_]);
          __stcg(B + static_cast<size_t>(gr) * m + gc, s_S[lr_][lc_]);
          __syncthreads();
        }
        if (!grid_sync(J.bar, gen, &s_ok, wait_ns)) goto timed_out;
        // (2) the other blocks of A, Q_P^T A[P rows][P' cols] Q_P' (into B), and V's columns,
        //     V[rows][P' cols] Q_P' (in place: every entry belongs to one item)
        const int nA = np * np, nItems = nA + (m / kJP) * np;
        for (int it = blockIdx.x; it < nItems; it += gridDim.x) {
          if (it < nA && it / np == it % np) continue;  // diagonal blocks came from step (1)
          const bool isA = it < nA;
          const int P2 = isA ? it % np : (it - nA) % np;
          int ci, cj;
          pair_of(br, P2, nb, ci, cj);
          const int gc = lc_ < kJW ? ci * kJW + lc_ : cj * kJW + lc_ - kJW;
          int gr;
          if (isA) {
            int bi, bj;
            pair_of(br, it / np, nb, bi, bj);
            gr = lr_ < kJW ? bi * kJW + lr_ : bj * kJW + lr_ - kJW;
            s_X[lr_][lc_] = __ldcg(A + static_cast<size_t>(gr) * m + gc);
            s_QA[lr_][lc_] = __ldcg(J.q + static_cast<size_t>(it / np) * kJP * kJP + tid);
          } else {
            gr = ((it - nA) / np) * kJP + lr_;
            s_X[lr_][lc_] = __ldcg(V + static_cast<size_t>(gr) * m + gc);
          }
          s_QB[lr_][lc_] = __ldcg(J.q + static_cast<size_t>(P2) * kJP * kJP + tid);
          __syncthreads();
          if (isA) {
            double t = 0.0;
#pragma unroll
            for (int k = 0; k < kJP; ++k) t = fma(s_QA[k][lr_], s_X[k][lc_], t);
            s_T[lr_][lc_] = t;
            __syncthreads();
          }
          double (*L)[kJP + 1] = isA ? s_T : s_X;
          double y = 0.0;
#pragma unroll
          for (int k = 0; k < kJP; ++k) y = fma(L[lr_][k], s_QB[k][lc_], y);
          __stcg((isA ? B : V) + static_cast<size_t>(gr) * m + gc, y);
          __syncthreads();
        }
        double* t = A;
        A = B;
        B = t;
        if (!grid_sync(J.bar, gen, &s_ok, wait_ns)) goto timed_out;
      }
      double lo2 = 0.0;
      for (int i = gtid; i < m * m; i += nthreads) {
        const double x = __ldcg(A + i);
        if (i / m != i % m) lo2 += x * x;
      }
      const double bo2 = block_sum(lo2, s_red);
      if (tid == 0) __stcg(J.slots + gridDim.x + blockIdx.x, bo2);
      if (!grid_sync(J.bar, gen, &s_ok, wait_ns)) goto timed_out;
    }
    // descending order (ties by index), eigenvector signs: largest-magnitude component positive
    for (int c = tid; c < pa; c += kJacThreads) {
      s_d[c] = __ldcg(A + static_cast<size_t>(c) * m + c);
      s_order[c] = c;  // stays a valid index even if NaNs leave ranks unassigned
    }
    __syncthreads();
    for (int c = tid; c < pa; c += kJacThreads) {
      int rank = 0;
      for (int d = 0; d < pa; ++d) rank += (s_d[d] > s_d[c] || (s_d[d] == s_d[c] && d < c)) ? 1 : 0;
      s_order[rank] = c;
    }
    __syncthreads();
    double* evals = J.out + J.evals_off;
    double* evecs = J.out + J.evecs_off;
    for (int k = blockIdx.x; k < pa; k += gridDim.x) {
      const int col = s_order[k];
      double best = -1.0;
      int bi = 0;
      double vi = 0.0;
      if (tid < pa) {
        vi = __ldcg(V + static_cast<size_t>(tid) * m + col);
        best = fabs(vi);
        bi = tid;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if ((tid & 31) == 0) {
        s_bv[tid >> 5] = best;
        s_bi[tid >> 5] = bi;
      }
      __syncthreads();
      if (tid == 0) {
        double bb = s_bv[0];
        int ii = s_bi[0];
        for (int w = 1; w < kJacThreads / 32; ++w)
          if (s_bv[w] > bb || (s_bv[w] == bb && s_bi[w] < ii)) {
            bb = s_bv[w];
            ii = s_bi[w];
          }
        s_val = __ldcg(V + static_cast<size_t>(ii) * m + col) < 0.0 ? -1.0 : 1.0;
        evals[k] = s_d[col];
      }
      __syncthreads();
      if (tid < pa) evecs[static_cast<size_t>(k) * pa + tid] = s_val * vi;
      __syncthreads();
    }
    if (blockIdx.x == 0 && tid == 0) {
      flags[2] = sweep;
      flags[3] = 1.0;
      flags[6] = seeded ? 1.0 : 0.0;
    }
  }
  return;
timed_out:
  if (tid == 0) flags[5] = 1.0;
}

cudaError_t launch_jacobi_grid(const JacobiParams& J, int grid, cudaStream_t stream) {
  if (grid < 1 || J.m > 256 || J.m < 2) return cudaErrorInvalidValue;
  void* args[] = {const_cast<JacobiParams*>(&J)};
  return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(jacobi_grid_kernel), dim3(grid), dim3(kJacThreads),
                                     args, 0, stream);
}

}  // namespace ss
