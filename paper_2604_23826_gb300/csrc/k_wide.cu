// k_wide.cu -- sufficient statistics of wide FP32 tables (p > 64) on the 5th-generation
// tensor cores (tcgen05, accumulators in tensor memory): arxiv 2604.23826, "Data
// Representation and Sufficient Statistics" (column sums and X^T X in one streaming
// pass; partials over row ranges combined), with the shift of "Numerical
// Considerations" (r = x - c, c = the table's first row).
//
// Work split.  The columns are cut into 128-column blocks; the output's upper block
// triangle is a list of units (I, J), I <= J, each a 128 x 128 block of S'.  CTA b
// works on unit b % U over the 32-row stages q, q + G/U, ... (q = b / U); the CTAs
// with the same q (one per unit) stay within a few stages of each other, so the
// column blocks that two units share are read from HBM once and from L2 by the other.
//
// In a CTA (320 threads, one per SM):
//   warp 0      producer: one 2D tensor copy per column block and stage (32 rows x 128
//               columns, zero past the table's columns, 128-byte swizzle) into a 3-deep
//               FP32 ring;
//   warp 1      MMA issuer: per stage, a fresh accumulation chain in one of two TMEM
//               buffers: L^T L (BF16x4 only), L^T H, H^T L, H^T H, each as two K = 16
//               tcgen05.mma.kind::f16 (M = N = 128, bf16 operands from shared memory);
//   warps 2-5   converters: r = x - c (rows past the table: r = 0), h = bf16(r),
//               l = bf16(r - h), written in the K-major core-matrix layout the MMA reads;
//               column sums of r and (BF16x3) sums of l^2 for diagonal units;
//   warps 6-9   epilogue: each thread owns one row of the 128 x 128 block (its TMEM
//               lane), adds every chain into FP32 registers (round to nearest) and, every
//               flush, into (hi, lo) pairs in the CTA's slot.
// A second kernel adds each unit's CTA slots, in CTA order, into the context's
// double-double accumulators (packed upper triangle); the order of every floating-point
// addition is fixed by the grid.  Every wait is bounded: on expiry the CTA records
// STATS_ETIMEOUT, stops waiting, lets its copies and MMAs complete and frees its tensor
// memory before returning.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace ss {

namespace {

constexpr int kWBlk = 128;           // columns per block
constexpr int kWRows = 32;           // rows per stage (two K = 16 steps)
constexpr int kWFStages = 3;         // FP32 ring depth
constexpr int kWOStages = 2;         // operand ring depth
constexpr int kWThreads = 320;
constexpr int kWFBytes = kWBlk * kWRows * 4;        // 16 KB: one block's FP32 stage
constexpr int kWOBytes = kWBlk * kWRows * 2;        // 8 KB: one block's bf16 operand (h or l)
constexpr uint32_t kWLbo = 128, kWSbo = 512;        // core-matrix strides (K = 32 per stage)
constexpr int kWTmemCols = 256;                     // two 128-column accumulators

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((kWLbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((kWSbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;  // descriptor version; base offset 0, no swizzle
  return d;
}

// instruction descriptor: D f32, A and B bf16, both K-major, M = N = 128
constexpr uint32_t kWIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(kWIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* smem_dst, const void* tmap, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(smem_dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool wait_live(uint64_t* bar, uint32_t parity, volatile unsigned int* dead) {
  if (mbar_try_wait(bar, parity)) return true;
  for (uint32_t i = 0; i < kSpinLimit; ++i) {
    if (mbar_try_wait_sleep(bar, parity, 1000u)) return true;
    if (*dead) return false;
  }
  return false;
}

constexpr int kWLead = 32;  // stages a CTA may run ahead of its peers of the other units

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// bounded wait until the CTAs (q, u') of every other unit u' have issued at least `need`
// stages; `known` caches the slowest peer's count seen last, so the peers' counters are read
// once every few stages
__device__ __forceinline__ bool wait_peers(const int* progress, int q, int U, int unit, int64_t need, int& known,
                                           volatile unsigned int* dead) {
  if (need <= known) return true;
  uint32_t i = 0;
  for (;;) {
    int mn = 0x7fffffff;
    for (int u = 0; u < U; ++u)
      if (u != unit) mn = min(mn, ld_acquire(progress + q * U + u));
    known = mn;
    if (need <= mn) return true;
    if (*dead || ++i > kSpinLimit) return false;
    __nanosleep(500);
  }
}

__device__ __forceinline__ void record_timeout(volatile unsigned int* dead, unsigned int* status) {
  *dead = 1;
  atomicOr(status, DEV_ETIMEOUT);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
__device__ __forceinline__ float bf_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf_hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }

__device__ __forceinline__ void two_sum(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (v - bp);
  hi = s;
}

// 16 consecutive TMEM columns of this warp's 32 lanes into registers
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <bool X4>
__global__ void __launch_bounds__(kWThreads, 1) wide_kernel(const __grid_constant__ WideParams P) {
  extern __shared__ __align__(1024) uint8_t smem[];
  // [FP32 ring: kWFStages x 2 blocks x 16 KB][operands: kWOStages x {Ah, Al, Bh, Bl} x 8 KB]
  uint8_t* fring = smem;
  uint8_t* oring = smem + kWFStages * 2 * kWFBytes;
  __shared__ __align__(8) uint64_t f_full[kWFStages], f_empty[kWFStages], o_full[kWOStages], o_empty[kWOStages],
      d_full[2], d_empty[2], fin;
  __shared__ uint32_t s_tmem;
  __shared__ volatile unsigned int s_dead;
  __shared__ int s_rows[kWFStages];
  __shared__ float s_piv[2 * kWBlk];  // pivots of the A block, then the B block

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int U = P.nunits, Gu = gridDim.x / U;
  const int unit = blockIdx.x % U, q0 = blockIdx.x / U;
  const int I = P.unit_i[unit], J = P.unit_j[unit];
  const bool diag = I == J;
  const int nblk = diag ? 1 : 2;
  const int64_t nst = (P.nrows + kWRows - 1) / kWRows;
  const int64_t my = q0 < nst ? (nst - 1 - q0) / Gu + 1 : 0;  // stages of this CTA

  if (threadIdx.x == 0) {
    for (int s = 0; s < kWFStages; ++s) {
      mbar_init(&f_full[s], 1);
      mbar_init(&f_empty[s], 4);
    }
    for (int s = 0; s < kWOStages; ++s) {
      mbar_init(&o_full[s], 4);
      mbar_init(&o_empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&d_full[s], 1);
      mbar_init(&d_empty[s], 4);
    }
    mbar_init(&fin, 1);
    s_dead = 0;
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < 2 * kWBlk; i += kWThreads) {
    const int col = (i < kWBlk ? I : J) * kWBlk + (i % kWBlk);
    s_piv[i] = col < P.p ? P.shift[col] : 0.f;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(kWTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      int peer_known = 0;
      int64_t k = 0;
      for (; k < my; ++k) {
        const int64_t st = q0 + k * Gu;
        if (k >= kWFStages && !wait_live(&f_empty[s], ph ^ 1u, &s_dead)) {
          record_timeout(&s_dead, P.status);
          break;
        }
        // stay within kWLead stages of the CTAs of the other units that take the same rows
        // (same q): their shared column blocks then come from L2 (all CTAs are resident:
        // cooperative launch; the slowest never waits)
        if (U > 1 && k >= kWLead && !wait_peers(P.progress, q0, U, unit, k - kWLead, peer_known, &s_dead)) {
          record_timeout(&s_dead, P.status);
          break;
        }
        s_rows[s] = static_cast<int>(min(static_cast<int64_t>(kWRows), P.nrows - st * kWRows));
        mbar_arrive_expect_tx(&f_full[s], static_cast<uint32_t>(nblk * kWFBytes));
        uint8_t* dst = fring + s * 2 * kWFBytes;
        tma_load_2d(dst, P.tmap, static_cast<int>(st * kWRows), I * kWBlk, &f_full[s]);
        if (!diag) tma_load_2d(dst + kWFBytes, P.tmap, static_cast<int>(st * kWRows), J * kWBlk, &f_full[s]);
        if (U > 1) st_release(P.progress + blockIdx.x, static_cast<int>(k + 1));
        if (++s == kWFStages) {
          s = 0;
          ph ^= 1u;
        }
      }
      // no copy in flight at exit: the last issued stages land
      for (int d = 0; d < kWFStages && d < k; ++d) {
        int sk = s - 1 - d;
        uint32_t pk = ph;
        while (sk < 0) {
          sk += kWFStages;
          pk ^= 1u;
        }
        mbar_wait_bounded(&f_full[sk], pk);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int so = 0, bd = 0;
      uint32_t pho = 0, phd = 0;
      int64_t k = 0;
      for (; k < my && !s_dead; ++k) {
        if (!wait_live(&o_full[so], pho, &s_dead) || (k >= 2 && !wait_live(&d_empty[bd], phd ^ 1u, &s_dead))) {
          record_timeout(&s_dead, P.status);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ob = smem_u32(oring + so * 4 * kWOBytes);
        const uint32_t ah = ob, al = ob + kWOBytes;
        const uint32_t bh = diag ? ah : ob + 2 * kWOBytes, bl = diag ? al : ob + 3 * kWOBytes;
        const uint32_t dt = tmem + static_cast<uint32_t>(bd * kWBlk);
        uint32_t acc = 0;
        // smallest products first; each as two K = 16 steps (256 bytes apart along K)
        if (X4) {
          for (int ks = 0; ks < 2; ++ks, acc = 1) umma_bf16(dt, umma_desc(al + ks * 256), umma_desc(bl + ks * 256), acc);
        }
        for (int ks = 0; ks < 2; ++ks, acc = 1) umma_bf16(dt, umma_desc(al + ks * 256), umma_desc(bh + ks * 256), acc);
        for (int ks = 0; ks < 2; ++ks, acc = 1) umma_bf16(dt, umma_desc(ah + ks * 256), umma_desc(bl + ks * 256), acc);
        for (int ks = 0; ks < 2; ++ks, acc = 1) umma_bf16(dt, umma_desc(ah + ks * 256), umma_desc(bh + ks * 256), acc);
        umma_commit(&o_empty[so]);
        umma_commit(&d_full[bd]);
        if (++so == kWOStages) {
          so = 0;
          pho ^= 1u;
        }
        if (++bd == 2) {
          bd = 0;
          phd ^= 1u;
        }
      }
      // every issued MMA completes before the tensor memory is released
      umma_commit(&fin);
      mbar_wait_bounded(&fin, 0);
    }
  } else if (warp < 6) {
    // ---------------------------------------------------------------- converters
    // The FP32 stage holds a block's 128 columns as 128-byte lines (32 rows) with the
    // tensor copy's 128-byte swizzle: 16-byte piece j of column c sits at piece j ^ (c & 7).
    // Per step a warp takes 8 consecutive columns x 4 pieces (lane: column c0 + lane % 8,
    // piece 4 half + lane / 8): each quarter warp reads one piece of 8 columns and writes 8
    // consecutive chunks of one core-matrix row, so reads and operand writes are conflict-free.
    const int cw = warp - 2;
    const bool odd = (lane >> 3) & 1;
    float sh[4], sl[4], qh[4], ql[4];  // column sums of r and of l^2 (diagonal units), (hi, lo)
#pragma unroll
    for (int i = 0; i < 4; ++i) sh[i] = sl[i] = qh[i] = ql[i] = 0.f;
    int sf = 0, so = 0;
    uint32_t phf = 0, pho = 0;
    for (int64_t k = 0; k < my; ++k) {
      bool ok = wait_live(&f_full[sf], phf, &s_dead) && (k < kWOStages || wait_live(&o_empty[so], pho ^ 1u, &s_dead));
      ok = __all_sync(0xffffffffu, ok);  // the warp decides together (shuffles follow)
      if (!ok) {
        if (lane == 0) record_timeout(&s_dead, P.status);
        break;
      }
      const int rows = s_rows[sf];
      const uint8_t* fb = fring + sf * 2 * kWFBytes;
      uint8_t* ob = oring + so * 4 * kWOBytes;
      for (int blk = 0; blk < nblk; ++blk) {
        const float* src = reinterpret_cast<const float*>(fb + blk * kWFBytes);
        uint8_t* oh = ob + (2 * blk) * kWOBytes;
        uint8_t* ol = ob + (2 * blk + 1) * kWOBytes;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int c = 32 * cw + 8 * (i & 3) + (lane & 7);  // column within the block
          const int piece = 4 * (i >> 2) + (lane >> 3);      // rows 4 piece .. 4 piece + 3
          const float4 x = *reinterpret_cast<const float4*>(src + c * kWRows + 4 * (piece ^ (c & 7)));
          const float cp = s_piv[blk * kWBlk + c];
          float r[4] = {x.x - cp, x.y - cp, x.z - cp, x.w - cp};
          if (rows < kWRows) {
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if (4 * piece + e >= rows) r[e] = 0.f;
          }
          const uint32_t h01 = pack_bf16x2(r[0], r[1]), h23 = pack_bf16x2(r[2], r[3]);
          const float e0 = r[0] - bf_lo(h01), e1 = r[1] - bf_hi(h01), e2 = r[2] - bf_lo(h23), e3 = r[3] - bf_hi(h23);
          const uint32_t l01 = pack_bf16x2(e0, e1), l23 = pack_bf16x2(e2, e3);
          if (diag && blk == 0) {
            two_sum(sh[i & 3], sl[i & 3], (r[0] + r[1]) + (r[2] + r[3]));
            if (!X4) two_sum(qh[i & 3], ql[i & 3], (e0 * e0 + e1 * e1) + (e2 * e2 + e3 * e3));
          }
          // lanes (even piece, odd piece) = (lane, lane ^ 8) hold rows 8g..8g+3 and 8g+4..8g+7 of
          // column c: the even one writes the h chunk, the odd one the l chunk (K-major core
          // matrices: 8 rows of a column = 16 bytes)
          const uint32_t s0 = odd ? h01 : l01, s1 = odd ? h23 : l23;
          const uint32_t t0 = __shfl_xor_sync(0xffffffffu, s0, 8), t1 = __shfl_xor_sync(0xffffffffu, s1, 8);
          const int g = piece >> 1;
          const uint32_t off = (c >> 3) * kWSbo + g * kWLbo + (c & 7) * 16;
          if (!odd) {
            *reinterpret_cast<uint4*>(oh + off) = make_uint4(h01, h23, t0, t1);
          } else {
            *reinterpret_cast<uint4*>(ol + off) = make_uint4(t0, t1, l01, l23);
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&f_empty[sf]);
        mbar_arrive(&o_full[so]);
      }
      if (++sf == kWFStages) {
        sf = 0;
        phf ^= 1u;
      }
      if (++so == kWOStages) {
        so = 0;
        pho ^= 1u;
      }
    }
    if (diag) {
      // the 4 lanes of a column (lane % 8 equal) add their pairs (fixed order), lanes 0-7 write
#pragma unroll
      for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int d = 8; d < 32; d <<= 1) {
          const float oh_ = __shfl_xor_sync(0xffffffffu, sh[i], d), ol_ = __shfl_xor_sync(0xffffffffu, sl[i], d);
          const float oq_ = __shfl_xor_sync(0xffffffffu, qh[i], d), oql = __shfl_xor_sync(0xffffffffu, ql[i], d);
          two_sum(sh[i], sl[i], oh_);
          sl[i] += ol_;
          two_sum(qh[i], ql[i], oq_);
          ql[i] += oql;
        }
        if (lane < 8) {
          const int c = 32 * cw + 8 * i + lane;
          float2* cs = reinterpret_cast<float2*>(P.slots) + static_cast<size_t>(blockIdx.x) * kWideSlotPairs +
                       kWBlk * kWBlk;
          cs[c] = make_float2(sh[i], sl[i]);
          cs[kWBlk + c] = make_float2(qh[i], ql[i]);
        }
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int quarter = warp & 3;         // TMEM lanes 32 quarter .. 32 quarter + 31
    const int m = 32 * quarter + lane;    // this thread's row of the 128 x 128 block
    float acc[kWBlk];
#pragma unroll
    for (int i = 0; i < kWBlk; ++i) acc[i] = 0.f;
    float2* slot = reinterpret_cast<float2*>(P.slots) + static_cast<size_t>(blockIdx.x) * kWideSlotPairs +
                   static_cast<size_t>(m) * kWBlk;
    bool fresh = true;
    int since = 0;
    auto flush = [&]() {
#pragma unroll
      for (int i0 = 0; i0 < kWBlk; i0 += 8) {
        float2 hl[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) hl[k] = fresh ? make_float2(0.f, 0.f) : __ldcg(slot + i0 + k);
#pragma unroll
        for (int k = 0; k < 8; ++k) {  // slot row m: 128 pairs
          two_sum(hl[k].x, hl[k].y, acc[i0 + k]);
          acc[i0 + k] = 0.f;
          __stcg(slot + i0 + k, hl[k]);
        }
        asm volatile("" ::: "memory");
      }
      fresh = false;
    };
    int bd = 0;
    uint32_t phd = 0;
    for (int64_t k = 0; k < my; ++k) {
      const bool ok = __all_sync(0xffffffffu, wait_live(&d_full[bd], phd, &s_dead));  // .sync.aligned loads follow
      if (!ok) {
        if (lane == 0) record_timeout(&s_dead, P.status);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t taddr = tmem + (static_cast<uint32_t>(32 * quarter) << 16) + static_cast<uint32_t>(bd * kWBlk);
#pragma unroll
      for (int c0 = 0; c0 < kWBlk; c0 += 16) {
        float v[16];
        tmem_ld16(taddr + c0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[c0 + i] += v[i];
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&d_empty[bd]);
      if (++bd == 2) {
        bd = 0;
        phd ^= 1u;
      }
      if (++since >= P.flush_stages) {
        since = 0;
        flush();
      }
    }
    flush();  // also writes the slot of a CTA without stages
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWTmemCols) : "memory");
  }
}

// The units' CTA slots, in CTA order, into the context's double-double accumulators.
// Block (unit, part) takes rows part, part + parts, ... of the unit's 128 x 128 block.
template <bool X4>
__global__ void __launch_bounds__(128) wide_merge_kernel(const __grid_constant__ WideParams P, int grid, int parts) {
  const int U = P.nunits, Gu = grid / U;
  const int unit = blockIdx.x / parts, part = blockIdx.x % parts;
  const int I = P.unit_i[unit], J = P.unit_j[unit];
  const int p = P.p;
  const float2* slots = reinterpret_cast<const float2*>(P.slots);
  for (int m = part; m < kWBlk; m += parts) {
    const int row = I * kWBlk + m;
    if (row >= p) break;
    const int n = threadIdx.x;
    const int col = J * kWBlk + n;
    if (col < row || col >= p) continue;
    float h = 0.f, l = 0.f;
    for (int q = 0; q < Gu; ++q) {
      const float2 x = __ldcg(slots + static_cast<size_t>(q * U + unit) * kWideSlotPairs + m * kWBlk + n);
      two_sum(h, l, x.x);
      two_sum(h, l, x.y);
    }
    if (!X4 && col == row) {  // BF16x3: + the diagonal of L^T L
      for (int q = 0; q < Gu; ++q) {
        const float2 x =
            __ldcg(slots + static_cast<size_t>(q * U + unit) * kWideSlotPairs + kWBlk * kWBlk + kWBlk + m);
        two_sum(h, l, x.x);
        two_sum(h, l, x.y);
      }
    }
    const int64_t e = static_cast<int64_t>(row) * p - static_cast<int64_t>(row) * (row - 1) / 2 + (col - row);
    const double v = static_cast<double>(h) + static_cast<double>(l);
    const double s = P.acc_S[e] + v;
    const double bp = s - P.acc_S[e];
    P.acc_S_lo[e] += (P.acc_S[e] - (s - bp)) + (v - bp);
    P.acc_S[e] = s;
  }
  if (I == J && part == 0) {  // column sums of the block
    const int c = threadIdx.x, col = I * kWBlk + c;
    if (col < p) {
      float h = 0.f, l = 0.f;
      for (int q = 0; q < Gu; ++q) {
        const float2 x = __ldcg(slots + static_cast<size_t>(q * U + unit) * kWideSlotPairs + kWBlk * kWBlk + c);
        two_sum(h, l, x.x);
        two_sum(h, l, x.y);
      }
      const double v = static_cast<double>(h) + static_cast<double>(l);
      const double s = P.acc_s[col] + v;
      const double bp = s - P.acc_s[col];
      P.acc_s_lo[col] += (P.acc_s[col] - (s - bp)) + (v - bp);
      P.acc_s[col] = s;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *P.acc_n += P.nrows;
}

template <bool X4>
cudaError_t launch_w(const WideParams& P, int grid, cudaStream_t st) {
  const int smem = kWFStages * 2 * kWFBytes + kWOStages * 4 * kWOBytes;
  cudaError_t e = cudaFuncSetAttribute(wide_kernel<X4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  // cooperative: the CTAs of different units wait on one another's progress, so all must be
  // resident at once
  WideParams Pc = P;
  void* args[] = {&Pc};
  e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(wide_kernel<X4>), dim3(grid), dim3(kWThreads), args,
                                  static_cast<size_t>(smem), st);
  if (e != cudaSuccess) return e;
  const int parts = 16;
  wide_merge_kernel<X4><<<P.nunits * parts, 128, 0, st>>>(P, grid, parts);
  return cudaGetLastError();
}

}  // namespace

int wide_grid(int p, int sms) {
  const int nb = (p + kWBlk - 1) / kWBlk;
  const int U = nb * (nb + 1) / 2;
  return U * std::max(1, sms / U);
}

int wide_units(int p, int* ui, int* uj, int max_units) {
  const int nb = (p + kWBlk - 1) / kWBlk;
  int u = 0;
  for (int I = 0; I < nb; ++I)
    for (int J = I; J < nb; ++J) {
      if (u >= max_units) return -1;
      ui[u] = I;
      uj[u] = J;
      ++u;
    }
  return u;
}

int wide_rows_per_stage() { return kWRows; }
int wide_block_cols() { return kWBlk; }

cudaError_t launch_wide(const WideParams& P, bool x4, int grid, cudaStream_t st) {
  return x4 ? launch_w<true>(P, grid, st) : launch_w<false>(P, grid, st);
}

}  // namespace ss
