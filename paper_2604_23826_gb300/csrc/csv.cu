// csv.cu -- CSV text tables: a host writer, and a parser on the GPU for the first k
// fields of every line (arxiv 2604.23826, "Validation and Infrastructure Verification":
// the validation program streamed the CSV file in chunks and parsed its first column on
// the GPUs; "Data Representation and Sufficient Statistics": text parsing dominated, so
// the table was converted to binary).
//
// Device parse of a text buffer, three launches and one small one:
//   csv_count_kernel   newlines per 4 KB tile (16 bytes per thread, byte compares);
//   csv_scan_kernel    one block: exclusive prefix of the tile counts, the line count
//                      (plus one for a last line without '\n');
//   csv_index_kernel   each tile again: the offsets of its newlines, in order;
//   csv_parse_kernel   one thread per line: the first k fields, converted and stored in
//                      column j at the line's row (adjacent lines -> adjacent rows, so
//                      the stores of a warp are contiguous).
// Number conversion is exact.  A real field is M * 10^E with M < 10^19 (the significant
// digits as an integer, trailing zeros moved into E) and -38 <= E <= 19.  For E >= 0 the product M * 10^E is formed in
// 128-bit integers; for E < 0 the quotient M * 2^s / 10^-E (a 64-bit quotient and a sticky
// remainder bit) comes, for -E <= 27, from one division by the normalised 5^-E with its
// precomputed reciprocal (exact quotient and remainder), and below that from binary long
// division.  Either way the exact value is
// a 64-bit integer q plus a sticky fraction times a power of two, rounded once to
// nearest, ties to even, to the 53 (FP64) or 24 (FP32) bits of the column type, and
// assembled bit by bit.
#include <fcntl.h>
#include <stdio.h>
#include <string.h>
#include <unistd.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

#include "../../include/stats_csv.h"
#include "common.cuh"
#include "kernels.h"

namespace ss {

namespace {

constexpr int kCsvThreads = 256;  // x 16 bytes = one tile
static_assert(kCsvThreads * 16 == kCsvTile, "a tile is 16 bytes per thread");

__device__ __forceinline__ int nl_count16(const char* t, int64_t pos, int64_t n, bool aligned) {
  if (aligned && pos + 16 <= n) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(t + pos));
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    int c = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int b = 0; b < 4; ++b) c += ((w[i] >> (8 * b)) & 0xFFu) == '\n';
    return c;
  }
  int c = 0;
  for (int64_t i = pos; i < pos + 16 && i < n; ++i) c += t[i] == '\n';
  return c;
}

__device__ __forceinline__ int block_exclusive_scan(int v, int* s_warp, int& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = lane < static_cast<int>(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < static_cast<int>(blockDim.x >> 5)) s_warp[lane] = w;
  }
  __syncthreads();
  total = s_warp[(blockDim.x >> 5) - 1];
  const int before = (wid > 0 ? s_warp[wid - 1] : 0) + x - v;
  __syncthreads();
  return before;
}

__global__ void __launch_bounds__(kCsvThreads) csv_count_kernel(const char* __restrict__ t, int64_t n,
                                                               uint32_t* __restrict__ counts) {
  __shared__ int s_warp[32];
  const bool aligned = (reinterpret_cast<uintptr_t>(t) & 15u) == 0;
  const int64_t pos = static_cast<int64_t>(blockIdx.x) * kCsvTile + threadIdx.x * 16;
  int total = 0;
  block_exclusive_scan(nl_count16(t, pos, n, aligned), s_warp, total);
  if (threadIdx.x == 0) counts[blockIdx.x] = static_cast<uint32_t>(total);
}

// one block of 1024 threads; offs[i] = newlines before tile i; *total = lines
__global__ void __launch_bounds__(1024) csv_scan_kernel(const char* __restrict__ t, int64_t n,
                                                       const uint32_t* __restrict__ counts, int64_t ntiles,
                                                       int64_t* __restrict__ offs, int64_t* __restrict__ ends,
                                                       int64_t ends_cap, int64_t* __restrict__ total) {
  __shared__ long long s_part[1024];
  const int tid = threadIdx.x;
  const int64_t per = (ntiles + 1023) / 1024;
  const int64_t t0 = tid * per, t1 = min(ntiles, t0 + per);
  long long sum = 0;
  for (int64_t i = t0; i < t1; ++i) sum += counts[i];
  s_part[tid] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan (Hillis-Steele)
    const long long y = tid >= o ? s_part[tid - o] : 0;
    __syncthreads();
    s_part[tid] += y;
    __syncthreads();
  }
  long long run = s_part[tid] - sum;
  for (int64_t i = t0; i < t1; ++i) {
    offs[i] = run;
    run += counts[i];
  }
  if (tid == 0) {
    const long long nl = s_part[1023];
    long long lines = nl;
    if (n > 0 && t[n - 1] != '\n') {  // a last line without its newline ends at the text's end
      if (nl < ends_cap) ends[nl] = n;
      ++lines;
    }
    *total = lines;
  }
}

__global__ void __launch_bounds__(kCsvThreads) csv_index_kernel(const char* __restrict__ t, int64_t n,
                                                               const int64_t* __restrict__ offs,
                                                               int64_t* __restrict__ ends, int64_t ends_cap) {
  __shared__ int s_warp[32];
  const bool aligned = (reinterpret_cast<uintptr_t>(t) & 15u) == 0;
  const int64_t pos = static_cast<int64_t>(blockIdx.x) * kCsvTile + threadIdx.x * 16;
  int total = 0;
  const int before = block_exclusive_scan(nl_count16(t, pos, n, aligned), s_warp, total);
  int64_t line = offs[blockIdx.x] + before;
  for (int64_t i = pos; i < pos + 16 && i < n; ++i)
    if (t[i] == '\n') {
      if (line < ends_cap) ends[line] = i;
      ++line;
    }
}

// ------------------------------- exact decimal -> binary -------------------------------
constexpr int kCsvFastK = 27;  // 5^27 < 2^63: one-word divisors for 10^-k, k <= 27
struct CsvTables {
  uint64_t p10[20];
  uint64_t dn[kCsvFastK + 1];
  uint64_t v[kCsvFastK + 1];
  int32_t z[kCsvFastK + 1];
  int32_t pad;
};
static_assert(sizeof(CsvTables) % 8 == 0, "copied as 64-bit words");

// Built on the host in exact integer arithmetic.
CsvTables make_csv_tables() {
  CsvTables T{};
  uint64_t p = 1;
  for (int i = 0; i < 20; ++i, p *= 10u) T.p10[i] = p;
  uint64_t f = 1;
  for (int k = 1; k <= kCsvFastK; ++k) {
    f *= 5u;
    const int z = __builtin_clzll(f);
    const uint64_t dn = f << z;
    const unsigned __int128 all = ~static_cast<unsigned __int128>(0);
    T.dn[k] = dn;
    T.z[k] = z;
    T.v[k] = static_cast<uint64_t>(all / dn - (static_cast<unsigned __int128>(1) << 64));
  }
  return T;
}

struct U128 {
  uint64_t lo, hi;
};
__device__ __forceinline__ int bitlen64(uint64_t x) { return x ? 64 - __clzll(static_cast<long long>(x)) : 0; }
__device__ __forceinline__ int bitlen128(const U128& x) { return x.hi ? 64 + bitlen64(x.hi) : bitlen64(x.lo); }
__device__ __forceinline__ bool ge128(const U128& a, const U128& b) { return a.hi != b.hi ? a.hi > b.hi : a.lo >= b.lo; }
__device__ __forceinline__ U128 sub128(const U128& a, const U128& b) {
  U128 r;
  r.lo = a.lo - b.lo;
  r.hi = a.hi - b.hi - (a.lo < b.lo ? 1u : 0u);
  return r;
}
__device__ __forceinline__ U128 shl128(const U128& a, int s) {  // 0 <= s < 128
  if (s == 0) return a;
  if (s >= 64) return U128{0, a.lo << (s - 64)};
  return U128{a.lo << s, (a.hi << s) | (a.lo >> (64 - s))};
}
__device__ __forceinline__ U128 mul64x64(uint64_t a, uint64_t b) { return U128{a * b, __umul64hi(a, b)}; }
__device__ __forceinline__ U128 mul128x10(const U128& a) {  // a < 2^124
  const U128 lo = mul64x64(a.lo, 10u);
  return U128{lo.lo, lo.hi + a.hi * 10u};
}

// Round (q + f) * 2^e2 (0 <= f < 1, f > 0 iff sticky) to t bits, nearest, ties to even, and
// return the IEEE bits of the column type (53: FP64, 24: FP32).  status: kCsvRange when
// the result overflows or would be subnormal.
__device__ uint64_t round_assemble(uint64_t q, bool sticky, int e2, int t, bool neg, uint32_t& status) {
  const int bq = bitlen64(q);  // q > 0
  uint64_t mant;
  if (bq > t) {
    const int sh = bq - t;
    mant = q >> sh;
    const uint64_t rem = q & ((uint64_t(1) << sh) - 1), half = uint64_t(1) << (sh - 1);
    const bool up = rem > half || (rem == half && (sticky || (mant & 1u)));
    mant += up ? 1u : 0u;
    e2 += sh;
    if (mant >> t) {  // carried into a new bit
      mant >>= 1;
      ++e2;
    }
  } else {
    mant = q << (t - bq);  // exact (sticky is 0 here: see the callers)
    e2 -= t - bq;
  }
  const int etop = e2 + t - 1;  // exponent of the leading bit
  const int emax = t == 53 ? 1023 : 127, emin = t == 53 ? -1022 : -126;
  if (etop > emax || etop < emin) {
    status |= kCsvRange;
    return 0;
  }
  if (t == 53) {
    const uint64_t bits = (static_cast<uint64_t>(etop + 1023) << 52) | (mant & ((uint64_t(1) << 52) - 1));
    return bits | (neg ? (uint64_t(1) << 63) : 0);
  }
  const uint32_t bits = (static_cast<uint32_t>(etop + 127) << 23) | static_cast<uint32_t>(mant & ((1u << 23) - 1));
  return bits | (neg ? (1u << 31) : 0u);
}

// M * 10^E correctly rounded to t bits (M > 0, -38 <= E <= 19), as IEEE bits.  T holds
// 10^0 .. 10^19 and, for 1 <= k <= kCsvFastK, 5^k normalised (shifted left until its top
// bit is set) with its reciprocal v = floor((2^128 - 1) / (5^k << z)) - 2^64.
__device__ uint64_t decimal_to_bits(uint64_t M, int E, int t, bool neg, uint32_t& status, const CsvTables& T) {
  if (E >= 0) {
    const U128 P = mul64x64(M, T.p10[E]);  // 10^19 < 2^64, the product < 2^128
    const int bl = bitlen128(P);
    uint64_t q;
    bool sticky = false;
    int e2 = 0;
    if (bl > 64) {
      const int sh = bl - 64;  // 1 .. 63
      q = (P.lo >> sh) | (P.hi << (64 - sh));
      sticky = (P.lo & ((uint64_t(1) << sh) - 1)) != 0;
      e2 = sh;
    } else {
      q = P.lo;
    }
    return round_assemble(q, sticky, e2, t, neg, status);
  }
  const int k = -E, bM = bitlen64(M);
  if (k <= kCsvFastK) {
    // M / 10^k = (M 2^a / 5^k) 2^-(a + k) with a = 63 + bitlen(5^k) - bitlen(M), so that
    // q = floor(M 2^a / 5^k) lies in [2^62, 2^64).  With 5^k normalised to dn = 5^k 2^z,
    // q = floor(u / dn) for u = M 2^(a + z) = M 2^(127 - bitlen(M)) (a 128-bit numerator
    // whose high word is below dn): one division by an invariant word with its
    // precomputed reciprocal (Moller and Granlund 2011) and the exact remainder.
    const uint64_t dn = T.dn[k], v = T.v[k];
    const int bD = 64 - T.z[k];
    const int sh = 127 - bM;  // 63 .. 126
    const uint64_t u1 = sh >= 64 ? M << (sh - 64) : M >> 1;
    const uint64_t u0 = sh >= 64 ? 0 : M << 63;
    const U128 qq = mul64x64(v, u1);
    const uint64_t q0 = qq.lo + u0;
    uint64_t q1 = qq.hi + u1 + (q0 < qq.lo ? 1u : 0u) + 1u;
    uint64_t r = u0 - q1 * dn;
    if (r > q0) {
      q1 -= 1u;
      r += dn;
    }
    if (r >= dn) {
      q1 += 1u;
      r -= dn;
    }
    return round_assemble(q1, r != 0, -(63 + bD - bM + k), t, neg, status);
  }
  // 10^k above 2^64: binary long division, one quotient bit per step
  U128 D{1, 0};
  for (int i = 0; i < k; ++i) D = mul128x10(D);  // 10^38 < 2^127
  const int bD = bitlen128(D);
  const int s = 63 + bD - bM;  // M 2^s / D lies in [2^62, 2^64)
  U128 R = shl128(U128{M, 0}, bD - 1 - bM);  // M < 2^64 < D here: the leading quotient bits are zero
  const int steps = s - (bD - 1 - bM);
  uint64_t q = 0;
  for (int i = 0; i < steps; ++i) {
    R = shl128(R, 1);
    q <<= 1;
    if (ge128(R, D)) {
      R = sub128(R, D);
      q |= 1u;
    }
  }
  return round_assemble(q, (R.lo | R.hi) != 0, -s, t, neg, status);
}

__device__ __forceinline__ bool is_digit(char c) { return c >= '0' && c <= '9'; }

// Parse the field that starts at p (ended by ',' or the line end e) as column type dt and
// store it at dst.  Returns the terminator's position, or -1 (status set) on an error.
__device__ int64_t parse_field(const char* t, int64_t p, int64_t e, int32_t dt, void* dst, uint32_t& status,
                               const CsvTables& T) {
  char c = p < e ? t[p] : ',';
  bool neg = false;
  if (c == '+' || c == '-') {
    neg = c == '-';
    ++p;
    c = p < e ? t[p] : ',';
  }
  if (dt == STATS_I16 || dt == STATS_I32 || dt == STATS_I64) {
    uint64_t v = 0;
    int nd = 0;
    while (c != ',') {
      if (!is_digit(c) || ++nd > STATS_CSV_MAX_DIGITS) {
        status |= kCsvFormat;
        return -1;
      }
      v = v * 10u + static_cast<uint64_t>(c - '0');
      ++p;
      c = p < e ? t[p] : ',';
    }
    if (nd == 0) {
      status |= kCsvFormat;
      return -1;
    }
    const uint64_t lim = dt == STATS_I16 ? 32767u : dt == STATS_I32 ? 2147483647u : 9223372036854775807ull;
    if (v > lim + (neg ? 1u : 0u)) {
      status |= kCsvRange;
      return -1;
    }
    const int64_t x = neg ? static_cast<int64_t>(0 - v) : static_cast<int64_t>(v);
    if (dt == STATS_I16)
      *static_cast<int16_t*>(dst) = static_cast<int16_t>(x);
    else if (dt == STATS_I32)
      *static_cast<int32_t*>(dst) = static_cast<int32_t>(x);
    else
      *static_cast<int64_t*>(dst) = x;
    return p;
  }
  // real: digits [. digits] [e|E [+-] digits]
  uint64_t M = 0;
  int nsig = 0, E = 0, ndig = 0, tz = 0;  // tz: trailing zero digits of M
  bool point = false;
  for (;; ++p, c = p < e ? t[p] : ',') {
    if (c == '.') {
      if (point) break;
      point = true;
      continue;
    }
    if (!is_digit(c)) break;
    ++ndig;
    const int d = c - '0';
    if (nsig == 0 && d == 0) {  // leading zeros
      if (point) --E;
      continue;
    }
    if (nsig < STATS_CSV_MAX_DIGITS) {
      M = M * 10u + static_cast<uint64_t>(d);
      ++nsig;
      tz = d == 0 ? tz + 1 : 0;
      if (point) --E;
    } else if (d != 0) {
      status |= kCsvFormat;  // more significant digits than supported
      return -1;
    } else if (!point) {
      ++E;  // a zero past the kept digits, before the point
    }
  }
  if (ndig == 0) {
    status |= kCsvFormat;
    return -1;
  }
  if (c == 'e' || c == 'E') {
    ++p;
    c = p < e ? t[p] : ',';
    bool eneg = false;
    if (c == '+' || c == '-') {
      eneg = c == '-';
      ++p;
      c = p < e ? t[p] : ',';
    }
    int x = 0, nx = 0;
    for (; is_digit(c); ++p, c = p < e ? t[p] : ',', ++nx) x = x * 10 + (c - '0');
    if (nx == 0 || nx > 4) {
      status |= kCsvFormat;
      return -1;
    }
    E += eneg ? -x : x;
  }
  if (c != ',') {
    status |= kCsvFormat;
    return -1;
  }
  const bool f64 = dt == STATS_F64;
  uint64_t bits = 0;
  if (M == 0) {
    bits = neg ? (f64 ? (uint64_t(1) << 63) : (uint64_t(1) << 31)) : 0;
  } else {
    // the same value with the exponent moved toward the supported range
    if (E < 0 && tz > 0) {  // trailing zeros of M (counted while parsing: no 64-bit remainders)
      const int n = min(tz, -E);
      M /= T.p10[n];
      E += n;
    }
    while (E > 19 && M < 1000000000000000000ull) {
      M *= 10u;
      --E;
    }
    if (E < -38 || E > 19) {
      status |= kCsvFormat;  // outside the supported exponent range
      return -1;
    }
    uint32_t st = 0;
    bits = decimal_to_bits(M, E, f64 ? 53 : 24, neg, st, T);
    if (st) {
      status |= st;
      return -1;
    }
  }
  if (f64)
    *static_cast<uint64_t*>(dst) = bits;
  else
    *static_cast<uint32_t*>(dst) = static_cast<uint32_t>(bits);
  return p;
}

__device__ __forceinline__ int dtype_size(int32_t dt) {
  return dt == STATS_I16 ? 2 : (dt == STATS_I32 || dt == STATS_F32) ? 4 : 8;
}

__global__ void __launch_bounds__(256) csv_parse_kernel(const char* __restrict__ t, CsvScratch S, int k,
                                                       int64_t row_cap, const __grid_constant__ CsvTables TP) {
  __shared__ CsvTables T;
  for (int i = threadIdx.x; i < static_cast<int>(sizeof(CsvTables) / 8); i += blockDim.x)
    reinterpret_cast<uint64_t*>(&T)[i] = reinterpret_cast<const uint64_t*>(&TP)[i];
  __syncthreads();
  const int64_t nl = min(*S.total, S.ends_cap);
  for (int64_t row = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; row < nl;
       row += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int64_t p = row == 0 ? 0 : S.ends[row - 1] + 1;
    int64_t e = S.ends[row];
    if (e > p && t[e - 1] == '\r') --e;
    uint32_t status = 0;
    const bool store = row < row_cap;
    for (int j = 0; j < k; ++j) {
      const int32_t dt = S.dts[j];
      uint64_t scratch;
      void* dst = store ? static_cast<void*>(static_cast<char*>(S.cols[j]) + row * dtype_size(dt))
                        : static_cast<void*>(&scratch);
      const int64_t f = parse_field(t, p, e, dt, dst, status, T);
      if (f < 0) break;
      if (j + 1 < k) {
        if (f >= e) {  // fewer than k fields
          status |= kCsvFormat;
          break;
        }
        p = f + 1;
      }
    }
    if (status) {  // one error bit per line (its parse stops there); the smallest line wins
      atomicOr(S.status, status);
      atomicMin(S.bad, (static_cast<unsigned long long>(row) << 2) | status);
    }
  }
}

size_t pad256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

size_t csv_scratch_bytes(int64_t nbytes, int64_t ends_cap, int k) {
  const int64_t ntiles = (nbytes + kCsvTile - 1) / kCsvTile + 1;
  return pad256(4 * ntiles) + pad256(8 * ntiles) + pad256(8 * (ends_cap + 1)) + 256 + 256 + 256 + pad256(8 * k) +
         pad256(4 * k);
}

void csv_scratch_carve(void* base, int64_t nbytes, int64_t ends_cap, int k, CsvScratch& s) {
  const int64_t ntiles = (nbytes + kCsvTile - 1) / kCsvTile + 1;
  char* b = static_cast<char*>(base);
  s.counts = reinterpret_cast<uint32_t*>(b);
  b += pad256(4 * ntiles);
  s.offs = reinterpret_cast<int64_t*>(b);
  b += pad256(8 * ntiles);
  s.ends = reinterpret_cast<int64_t*>(b);
  s.ends_cap = ends_cap;
  b += pad256(8 * (ends_cap + 1));
  s.total = reinterpret_cast<int64_t*>(b);
  b += 256;
  s.status = reinterpret_cast<uint32_t*>(b);
  b += 256;
  s.bad = reinterpret_cast<unsigned long long*>(b);
  b += 256;
  s.cols = reinterpret_cast<void**>(b);
  b += pad256(8 * k);
  s.dts = reinterpret_cast<int32_t*>(b);
}

cudaError_t launch_csv_lines(const char* d_text, int64_t nbytes, const CsvScratch& s, cudaStream_t st) {
  const int64_t ntiles = (nbytes + kCsvTile - 1) / kCsvTile;
  if (ntiles == 0) return cudaMemsetAsync(s.total, 0, sizeof(int64_t), st);
  if (ntiles > 0x7fffffff) return cudaErrorInvalidValue;
  csv_count_kernel<<<static_cast<unsigned>(ntiles), kCsvThreads, 0, st>>>(d_text, nbytes, s.counts);
  csv_scan_kernel<<<1, 1024, 0, st>>>(d_text, nbytes, s.counts, ntiles, s.offs, s.ends, s.ends_cap, s.total);
  csv_index_kernel<<<static_cast<unsigned>(ntiles), kCsvThreads, 0, st>>>(d_text, nbytes, s.offs, s.ends,
                                                                        s.ends_cap);
  return cudaGetLastError();
}

cudaError_t launch_csv_parse(const char* d_text, const CsvScratch& s, int k, int64_t row_cap, int sms,
                             cudaStream_t st) {
  const int64_t want = (s.ends_cap + 255) / 256;
  const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(sms) * 8)));
  static const CsvTables tables = make_csv_tables();
  csv_parse_kernel<<<grid, 256, 0, st>>>(d_text, s, k, row_cap, tables);
  return cudaGetLastError();
}

}  // namespace ss

// ------------------------------------------------------------------------ host side
using namespace ss;

namespace {

bool valid_dtype(int32_t d) { return d >= STATS_I16 && d <= STATS_F64; }
int host_dtype_bytes(int32_t d) { return d == STATS_I16 ? 2 : (d == STATS_I32 || d == STATS_F32) ? 4 : 8; }

// decimal text of an integer
char* put_int(char* o, int64_t v) {
  char buf[24];
  int n = 0;
  uint64_t u = v < 0 ? 0 - static_cast<uint64_t>(v) : static_cast<uint64_t>(v);
  do {
    buf[n++] = static_cast<char>('0' + u % 10u);
    u /= 10u;
  } while (u);
  if (v < 0) *o++ = '-';
  while (n) *o++ = buf[--n];
  return o;
}

// Format rows [r0, r1) of the columns into out; false if a real value is not finite.
bool format_rows(int p, const int32_t* dt, const void* const* cols, int64_t r0, int64_t r1, std::string& out) {
  out.clear();
  out.reserve(static_cast<size_t>(r1 - r0) * (p * 12 + 8));
  char line[STATS_MAX_P * 28 + 4];
  for (int64_t r = r0; r < r1; ++r) {
    char* o = line;
    for (int j = 0; j < p; ++j) {
      if (j) *o++ = ',';
      switch (dt[j]) {
        case STATS_I16: o = put_int(o, static_cast<const int16_t*>(cols[j])[r]); break;
        case STATS_I32: o = put_int(o, static_cast<const int32_t*>(cols[j])[r]); break;
        case STATS_I64: o = put_int(o, static_cast<const int64_t*>(cols[j])[r]); break;
        case STATS_F32: {
          const float v = static_cast<const float*>(cols[j])[r];
          if (!std::isfinite(v)) return false;
          o += snprintf(o, 24, "%.9g", static_cast<double>(v));
          break;
        }
        default: {
          const double v = static_cast<const double*>(cols[j])[r];
          if (!std::isfinite(v)) return false;
          o += snprintf(o, 28, "%.17g", v);
          break;
        }
      }
    }
    *o++ = '\n';
    out.append(line, static_cast<size_t>(o - line));
  }
  return true;
}

bool write_all(int fd, const char* b, size_t len, off_t off) {
  while (len > 0) {
    const ssize_t w = pwrite(fd, b, len, off);
    if (w <= 0) return false;
    b += w;
    len -= static_cast<size_t>(w);
    off += w;
  }
  return true;
}

// Append rows [0, nrows) of the host columns at *off, formatted by parallel threads.
stats_status append_rows(int fd, off_t* off, int p, const int32_t* dt, const void* const* cols, int64_t nrows) {
  const int nt = static_cast<int>(std::max(1u, std::min(16u, std::thread::hardware_concurrency())));
  const int64_t block = int64_t(1) << 20;
  std::vector<std::string> bufs(nt);
  for (int64_t b0 = 0; b0 < nrows; b0 += block) {
    const int64_t b1 = std::min(nrows, b0 + block);
    std::vector<char> ok(nt, 1);
    std::vector<std::thread> th;
    const int64_t per = (b1 - b0 + nt - 1) / nt;
    for (int i = 0; i < nt; ++i) {
      const int64_t r0 = std::min(b1, b0 + i * per), r1 = std::min(b1, r0 + per);
      th.emplace_back([&, i, r0, r1] { ok[i] = format_rows(p, dt, cols, r0, r1, bufs[i]); });
    }
    for (auto& x : th) x.join();
    for (int i = 0; i < nt; ++i)
      if (!ok[i]) return STATS_EINVAL;
    std::vector<off_t> at(nt);
    for (int i = 0; i < nt; ++i) {
      at[i] = *off;
      *off += static_cast<off_t>(bufs[i].size());
    }
    std::vector<char> wok(nt, 1);
    th.clear();
    for (int i = 0; i < nt; ++i)
      th.emplace_back([&, i] { wok[i] = write_all(fd, bufs[i].data(), bufs[i].size(), at[i]); });
    for (auto& x : th) x.join();
    for (int i = 0; i < nt; ++i)
      if (!wok[i]) return STATS_EIO;
  }
  return STATS_OK;
}

stats_status open_out(const char* path, const char* header, int* fd, off_t* off) {
  *fd = open(path, O_CREAT | O_TRUNC | O_WRONLY, 0644);
  if (*fd < 0) return STATS_EIO;
  *off = 0;
  if (header) {
    std::string h(header);
    h.push_back('\n');
    if (!write_all(*fd, h.data(), h.size(), 0)) return STATS_EIO;
    *off = static_cast<off_t>(h.size());
  }
  return STATS_OK;
}

}  // namespace

extern "C" {

stats_status stats_csv_write(const char* path, int32_t p, const int32_t* dtypes, int64_t nrows,
                             const void* const* hcols, const char* header) {
  if (!path || p < 1 || p > STATS_MAX_P || !dtypes || nrows < 0) return STATS_EINVAL;
  for (int j = 0; j < p; ++j) {
    if (!valid_dtype(dtypes[j])) return STATS_EINVAL;
    if (nrows > 0 && (!hcols || !hcols[j])) return STATS_EINVAL;
  }
  int fd = -1;
  off_t off = 0;
  stats_status st = open_out(path, header, &fd, &off);
  if (st == STATS_OK) st = append_rows(fd, &off, p, dtypes, hcols, nrows);
  if (fd >= 0 && close(fd) != 0 && st == STATS_OK) st = STATS_EIO;
  return st;
}

stats_status stats_csv_write_table1(const char* path, uint64_t seed, uint64_t row0, int64_t nrows, int32_t layout,
                                    int64_t chunk_rows) {
  int32_t dt[STATS_T1_P];
  double lo[STATS_T1_P], hi[STATS_T1_P];
  uint8_t ident[STATS_T1_P];
  if (!path || nrows < 0 || chunk_rows < 0 || stats_table1_config(layout, 1, dt, ident, lo, hi) != STATS_OK)
    return STATS_EINVAL;
  if (chunk_rows == 0) chunk_rows = int64_t(1) << 22;
  chunk_rows = std::max<int64_t>(1, std::min<int64_t>(chunk_rows, std::max<int64_t>(nrows, 1)));
  std::vector<size_t> coff(STATS_T1_P);
  size_t bytes = 0;
  for (int j = 0; j < STATS_T1_P; ++j) {
    coff[j] = bytes;
    bytes += pad256(static_cast<size_t>(chunk_rows) * host_dtype_bytes(dt[j]));
  }
  void* d = nullptr;
  void* h = nullptr;
  if (cudaMalloc(&d, bytes) != cudaSuccess) {
    cudaGetLastError();
    return STATS_ENOMEM;
  }
  if (cudaHostAlloc(&h, bytes, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d);
    return STATS_ENOMEM;
  }
  std::vector<void*> dcols(STATS_T1_P);
  std::vector<const void*> hcols(STATS_T1_P);
  for (int j = 0; j < STATS_T1_P; ++j) {
    dcols[j] = static_cast<char*>(d) + coff[j];
    hcols[j] = static_cast<char*>(h) + coff[j];
  }
  int fd = -1;
  off_t off = 0;
  stats_status st = open_out(path, "A,B,C,D,E,F,G,H,cotC,I,J,K", &fd, &off);
  for (int64_t r = 0; st == STATS_OK && r < nrows; r += chunk_rows) {
    const int64_t m = std::min(chunk_rows, nrows - r);
    st = stats_gen_table1(seed, row0 + static_cast<uint64_t>(r), m, layout, dcols.data(), nullptr);
    if (st == STATS_OK && cudaMemcpy(h, d, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) st = STATS_ECUDA;
    if (st == STATS_OK) st = append_rows(fd, &off, STATS_T1_P, dt, hcols.data(), m);
  }
  if (fd >= 0 && close(fd) != 0 && st == STATS_OK) st = STATS_EIO;
  cudaFreeHost(h);
  cudaFree(d);
  return st;
}

stats_status stats_csv_parse(const char* d_text, int64_t nbytes, int32_t k, const int32_t* dtypes,
                             void* const* d_cols, int64_t max_rows, int64_t* nrows, int64_t* bad_line,
                             void* stream) {
  if (bad_line) *bad_line = -1;
  if (nrows) *nrows = 0;
  if (nbytes < 0 || k < 1 || k > STATS_MAX_P || !dtypes || !d_cols || max_rows < 0 || (nbytes > 0 && !d_text))
    return STATS_EINVAL;
  for (int j = 0; j < k; ++j)
    if (!valid_dtype(dtypes[j]) || !d_cols[j]) return STATS_EINVAL;
  if (nbytes == 0) return STATS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ends_cap = std::min<int64_t>(max_rows, nbytes / 2 + 1);
  void* scratch = nullptr;
  if (cudaMallocAsync(&scratch, csv_scratch_bytes(nbytes, ends_cap, k), st) != cudaSuccess) {
    cudaGetLastError();
    return STATS_ENOMEM;
  }
  CsvScratch S;
  csv_scratch_carve(scratch, nbytes, ends_cap, k, S);
  struct Out {
    int64_t total;
    uint32_t status;
    uint32_t pad;
    unsigned long long bad;
  } out{};
  stats_status res = STATS_OK;
  cudaError_t e = cudaMemcpyAsync(S.cols, d_cols, sizeof(void*) * k, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S.dts, dtypes, sizeof(int32_t) * k, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(S.status, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(S.bad, 0xFF, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = launch_csv_lines(d_text, nbytes, S, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&out.total, S.total, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && out.total > max_rows) res = STATS_EINVAL;
  if (e == cudaSuccess && res == STATS_OK) {
    e = launch_csv_parse(d_text, S, k, max_rows, sms, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&out.status, S.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&out.bad, S.bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFreeAsync(scratch, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return STATS_ECUDA;
  }
  if (res != STATS_OK) return res;
  if (out.status) {
    if (bad_line) *bad_line = static_cast<int64_t>(out.bad >> 2);
    return (out.bad & kCsvFormat) ? STATS_EFORMAT : STATS_ERANGE;
  }
  if (nrows) *nrows = out.total;
  return STATS_OK;
}

}  // extern "C"
