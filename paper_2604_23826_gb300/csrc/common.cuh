// common.cuh -- device helpers shared by the kernels of libsuffstats (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace ss {


// Iteration bound of every device-side spin.  A try_wait that suspends for the
// hardware time limit each round makes this a multi-second bound.
constexpr uint32_t kSpinLimit = 1u << 22;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// multiplies on words 0 and 2, the high halves XORed into words 1 and 3 with
// the key; the key advances by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// ---------------------------------------------------------------------------
// mbarrier + bulk-copy (TMA, non-tensor) helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// try_wait that lets the hardware suspend the thread for up to `ns` nanoseconds
// while the phase is incomplete (fewer polling instructions).
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity to complete.  Returns false
// (and leaves the barrier alone) when the bound expires (kSpinLimit suspended polls
// of at most 1 us each: a few seconds).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  for (uint32_t i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait_sleep(bar, parity, 1000u)) return true;
  return false;
}

// Global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte
// aligned), completing transaction bytes on `bar`.
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gmem_src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(smem_dst)),
      "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// ---------------------------------------------------------------------------
// Legacy warp-level tensor-core MMA, m16n8k16, f16 inputs, f32 accumulators,
// and ldmatrix (transposed) -- fragment layouts as documented for mma.sync.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ldsm_x4_trans(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                              uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr)
               : "memory");
}

__device__ __forceinline__ void mma_f16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                              uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------
// Exact digits as f16.  A byte b (0..255) placed in the low 8 mantissa bits of
// the half 0x6400 (= 1024.0) reads 1024 + b exactly (the half has 10 mantissa
// bits); subtracting 1024 leaves b.  A signed top byte is first XORed with 0x80
// (so 1024 + (b ^ 0x80) holds b_signed + 1152) and 1152 is subtracted.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t half2_sub(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
constexpr uint32_t kMagicLo = 0x6400u;      // 1024.0 in f16
constexpr uint32_t kMagicHi = 0x6400u << 16;
constexpr uint32_t kH1024 = 0x64006400u;    // {1024, 1024}
constexpr uint32_t kH1152lo = 0x64006480u;  // {1152 (low), 1024 (high)}
constexpr uint32_t kH1152hi = 0x64806400u;  // {1024 (low), 1152 (high)}

// Two unsigned bytes (x low, y high), each already in the low byte of its
// register's half (x in bits 0..7, y in bits 16..23), to an f16x2 of (x, y).
__device__ __forceinline__ uint32_t digits2(uint32_t packed_bytes, uint32_t bias = kH1024) {
  return half2_sub(packed_bytes | kH1024, bias);
}

__device__ __forceinline__ uint32_t half2_mul(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("mul.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
// Two small non-negative integers x, y < 256 to an f16x2 of (x, y) on the FMA
// pipe only: x + 65536 y (one IMAD) holds each value as the bit pattern of the
// subnormal half v * 2^-24; two exact multiplications by 2^12 rescale it to v.
__device__ __forceinline__ uint32_t small_pair_f16x2(uint32_t x, uint32_t y) {
  const uint32_t bits = y * 65536u + x;
  constexpr uint32_t k2p12 = 0x6C006C00u;  // {4096, 4096}
  return half2_mul(half2_mul(bits, k2p12), k2p12);
}

// ---------------------------------------------------------------------------
// Fixed point of a double: q = round(x * 2^sh) as a two's complement int64,
// ties rounded up in magnitude, with 32-bit integer operations only (no FP64
// pipe, no branches).  x = m * 2^(E - 1075) with the 53-bit significand m, so
// 2 * |q| + 1 >= T = floor(m * 2^(E - 1075 + sh + 1)) and |q| = (T + 1) >> 1.
// Valid when |x| * 2^sh < 2^62 and the left shift E - 1075 + sh + 1 < 32
// (both hold for every value that passes the field check, |x| < 2^e with
// sh = P - e, P <= 55); values outside are flagged by that check.
// ---------------------------------------------------------------------------
template <bool Signed>
__device__ __forceinline__ uint64_t fixed_rn(double x, int sh) {
  const uint32_t lo = static_cast<uint32_t>(__double2loint(x));
  const uint32_t hi = static_cast<uint32_t>(__double2hiint(x));
  const int e = static_cast<int>((hi >> 20) & 0x7FF);
  const uint32_t mh = (hi & 0x000FFFFFu) | (e ? 0x00100000u : 0u);
  const int k = max(e, 1) - 1075 + sh + 1;  // left shift of m that gives T
  const uint32_t ls = static_cast<uint32_t>(min(max(k, 0), 31));
  const uint32_t rs = static_cast<uint32_t>(min(max(-k, 0), 63));
  // T = m << ls >> rs
  const uint32_t h1 = __funnelshift_l(lo, mh, ls);
  const uint32_t l1 = lo << ls;
  const uint32_t l2 = rs < 32 ? __funnelshift_r(l1, h1, rs) : (h1 >> (rs - 32));
  const uint32_t h2 = rs < 32 ? (h1 >> rs) : 0u;
  // |q| = (T + 1) >> 1
  const uint64_t t = ((static_cast<uint64_t>(h2) << 32) | l2) + 1ull;
  uint64_t q = t >> 1;
  if (Signed) {
    const uint64_t neg = static_cast<uint64_t>(-static_cast<int64_t>(hi >> 31));  // 0 or all ones
    q = (q ^ neg) - neg;
  }
  return q;
}

// Biased binary exponent field of a double (0 for zero / subnormal).
__device__ __forceinline__ int dbl_exp_field(double x) {
  return static_cast<int>((static_cast<uint64_t>(__double_as_longlong(x)) >> 52) & 0x7FF);
}

}  // namespace ss
