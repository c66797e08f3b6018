// k_wide.cu -- sufficient statistics of wide FP32 tables (p > 64) on the 5th-generation
// tensor cores (tcgen05, accumulators in tensor memory): arxiv 2604.23826, "Data
// Representation and Sufficient Statistics" (column sums and X^T X in one streaming
// pass; partials over row ranges combined), with the shift of "Numerical
// Considerations" (r = x - c, c = the mean of the table's first rows).
//
// Work split.  The columns are cut into 128-column blocks; the output's upper block
// triangle is a list of units (I, J), I <= J, each a 128 x 128 block of S'.  A diagonal
// unit converts one column block per stage (plus its column sums), the others two, so
// the units get CTAs in the proportion of their measured stage times and sweep the rows
// at about the same speed.  CTA q of a unit with G_u CTAs takes the 64-row stages
// q, q + G_u, q + 2 G_u, ...  (Making the units wait for one another, so that the column
// blocks they share come from L2, cost more in stalls than it saved in HBM reads.)
//
// In a CTA (512 threads in four warpgroups, one CTA per SM; after the start the epilogue's
// warpgroup holds 200 registers per thread and the others 104):
//   warp 0      producer: per stage and column block, one 3D tensor copy (32 rows x 2
//               chunks x 128 columns: 256 contiguous bytes per column, 128-byte swizzle)
//               into a ring of 3 (two blocks) or 6 (one block) 32 KB stages; the rows past
//               the last whole 32-row chunk are read by the converters with plain loads;
//   warps 4-11  converters: r = x - c (rows past the table: 0), h = bf16(r), l = bf16(r - h),
//               written IN PLACE over the FP32 stage in the K-major core-matrix layout the
//               MMA reads (each 8-column group's 2 KB of FP32 becomes its h and l core
//               matrices); column sums of r and (BF16x3) sums of l^2 for diagonal units;
//   warp 1      MMA issuer: per 32-row chunk a fresh accumulation chain in one of two TMEM
//               buffers: L^T L (BF16x4 only), L^T H, H^T L, H^T H, each two K = 16
//               tcgen05.mma.kind::f16 (M = N = 128); a BF16x3 diagonal unit, whose l operand
//               holds 2l, takes only H^T (2L) and H^T H (the merge symmetrizes); the stage is
//               released when its MMAs complete;
//   warps 12-15 epilogue: each thread owns one row of the 128 x 128 block (its TMEM
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
#include "tc05.cuh"

namespace ss {

namespace {

constexpr int kWBlk = 128;                    // columns per block
constexpr int kWChunk = 32;                   // rows per 128-byte line of the tensor copy, and per MMA chain
constexpr int kWRows = 64;                    // rows per stage
constexpr int kWChains = kWRows / kWChunk;    // MMA chains per stage
constexpr int kWBlkBytes = kWBlk * kWRows * 4;  // 32 KB: one block's stage (FP32, then h and l in place)
constexpr int kWRingBytes = 6 * kWBlkBytes;     // 192 KB
constexpr int kWMaxStages = 6;
constexpr int kWThreads = 512;                  // four warpgroups
constexpr int kWConv = 8;                       // converter warps (4 .. 11), two 8-column groups each
constexpr int kWRegsLow = 104, kWRegsEpi = 200; // per-thread registers after the split: 3 x 104 + 200 = 4 x 128
constexpr uint32_t kWLbo = 256, kWSbo = 2048;   // core-matrix strides: next 8 rows (K), next 8 columns (M)
constexpr int kWTmemCols = 256;                 // two 128-column accumulators
constexpr int kWFold = 16;                      // stages of FP32 partial sums of l^2 per (hi, lo) fold

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) { return tc05::desc<kWLbo, kWSbo>(saddr); }

// instruction descriptor: D f32, A and B bf16, both K-major, M = N = 128
constexpr uint32_t kWIdesc = tc05::idesc_bf16(128, 128);

__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  tc05::mma_bf16(dtmem, a, b, kWIdesc, accumulate);
}

using tc05::umma_commit;
using tc05::tma_load_3d;
using tc05::wait_live;
using tc05::record_timeout;
using tc05::pack_bf16x2;
using tc05::bf_lo;
using tc05::bf_hi;
using tc05::two_sum;
using tc05::fp32_piece;

template <bool X4>
__global__ void __launch_bounds__(kWThreads, 1) wide_kernel(const __grid_constant__ WideParams P) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t f_full[kWMaxStages], c_full[kWMaxStages], f_empty[kWMaxStages], d_full[2],
      d_empty[2], fin;
  __shared__ uint32_t s_tmem;
  __shared__ volatile unsigned int s_dead;
  __shared__ int s_rows[kWMaxStages];
  __shared__ float s_piv[2 * kWBlk];  // pivots of the A block, then the B block

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int U = P.nunits;
  int unit = 0;
  while (unit + 1 < U && static_cast<int>(blockIdx.x) >= P.unit_first[unit + 1]) ++unit;
  const int Gu = P.unit_ctas[unit], first = P.unit_first[unit], q0 = blockIdx.x - first;
  const int I = P.unit_i[unit], J = P.unit_j[unit];
  const bool diag = I == J;
  const int nblk = diag ? 1 : 2;
  const int S = kWRingBytes / (nblk * kWBlkBytes);  // ring depth: 6 or 3
  const int64_t nst = (P.nrows + kWRows - 1) / kWRows;
  const int64_t my = q0 < nst ? (nst - 1 - q0) / Gu + 1 : 0;  // stages of this CTA

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&f_full[s], 1);
      mbar_init(&c_full[s], kWConv);
      mbar_init(&f_empty[s], 1);
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

  // Registers: launched at 128 per thread; warpgroup 3 (the epilogue's 128 FP32 accumulators)
  // takes 200, warpgroups 0-2 give up to 104 (per SMSP: 3 x 24 released, 72 taken).  Each
  // warpgroup executes its setmaxnreg as a whole, in one branch.
  if (warp < 12) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kWRegsLow));
  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      int64_t k = 0;
      for (; k < my; ++k) {
        const int64_t st = q0 + k * Gu;
        if (k >= S && !wait_live(&f_empty[s], ph ^ 1u, &s_dead)) {
          record_timeout(&s_dead, P.status);
          break;
        }
        s_rows[s] = static_cast<int>(min(static_cast<int64_t>(kWRows), P.nrows - st * kWRows));
        mbar_arrive_expect_tx(&f_full[s], static_cast<uint32_t>(nblk * kWBlkBytes));
        uint8_t* dst = smem + static_cast<size_t>(s) * nblk * kWBlkBytes;
        const int y = static_cast<int>(st * kWChains);
        tma_load_3d(dst, P.tmap, 0, y, I * kWBlk, &f_full[s]);
        if (!diag) tma_load_3d(dst + kWBlkBytes, P.tmap, 0, y, J * kWBlk, &f_full[s]);
        if (++s == S) {
          s = 0;
          ph ^= 1u;
        }
      }
      // no copy in flight at exit: the last issued stages land
      for (int d = 0; d < S && d < k; ++d) {
        int sk = s - 1 - d;
        uint32_t pk = ph;
        while (sk < 0) {
          sk += S;
          pk ^= 1u;
        }
        mbar_wait_bounded(&f_full[sk], pk);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int s = 0, bd = 0;
      uint32_t ph = 0, phd = 0;
      int64_t chain = 0;
      for (int64_t k = 0; k < my && !s_dead; ++k) {
        if (!wait_live(&c_full[s], ph, &s_dead)) {
          record_timeout(&s_dead, P.status);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ab = smem_u32(smem + static_cast<size_t>(s) * nblk * kWBlkBytes);
        const uint32_t bb = diag ? ab : ab + kWBlkBytes;
        bool ok = true;
        for (int ch = 0; ch < kWChains; ++ch, ++chain) {
          if (chain >= 2 && !wait_live(&d_empty[bd], phd ^ 1u, &s_dead)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t dt = tmem + static_cast<uint32_t>(bd * kWBlk);
          // chain ch: rows 32 ch .. 32 ch + 31 = K groups 4 ch .. 4 ch + 3; K step ks covers K
          // groups 4 ch + 2 ks and + 1 (h at +0, l at +128 of each 256-byte K group)
          const uint32_t ah = ab + ch * 4 * 256, al = ah + 128, bh = bb + ch * 4 * 256, bl = bh + 128;
          uint32_t acc = 0;
          // smallest products first
          if (X4) {
            for (int ks = 0; ks < 2; ++ks, acc = 1)
              umma_bf16(dt, umma_desc(al + ks * 512), umma_desc(bl + ks * 512), acc);
          }
          if (X4 || !diag) {
            for (int ks = 0; ks < 2; ++ks, acc = 1)
              umma_bf16(dt, umma_desc(al + ks * 512), umma_desc(bh + ks * 512), acc);
          }
          // (BF16x3 diagonal units: the l operand holds 2l, so this adds 2 H^T L = H^T L + L^T H
          // up to a transpose, taken in the merge)
          for (int ks = 0; ks < 2; ++ks, acc = 1) umma_bf16(dt, umma_desc(ah + ks * 512), umma_desc(bl + ks * 512), acc);
          for (int ks = 0; ks < 2; ++ks, acc = 1) umma_bf16(dt, umma_desc(ah + ks * 512), umma_desc(bh + ks * 512), acc);
          umma_commit(&d_full[bd]);
          if (++bd == 2) {
            bd = 0;
            phd ^= 1u;
          }
        }
        umma_commit(&f_empty[s]);  // the stage is free once its MMAs have read it
        if (!ok) {
          record_timeout(&s_dead, P.status);
          break;
        }
        if (++s == S) {
          s = 0;
          ph ^= 1u;
        }
      }
      // every issued MMA completes before the tensor memory is released
      umma_commit(&fin);
      mbar_wait_bounded(&fin, 0);
    }
  } else if (warp >= 4 && warp < 4 + kWConv) {
    // ---------------------------------------------------------------- converters (in place)
    // Converter warp cw owns the 8-column groups g = 2 cw, 2 cw + 1 of each block.  Group g's FP32
    // lines (columns 8g .. 8g + 7, two 32-row chunks each) are the 2 KB at g * 2048; they
    // become the group's core matrices: K group kk (rows 8 kk .. 8 kk + 7) of h at
    // g * 2048 + kk * 256 and of l at + 128, row c % 8 of each at 16 (c % 8).  Lane: column
    // sub = lane % 8 of the group and, in step it (0, 1), the whole K group
    // kk = 4 j + lane / 8 of chunk j = (sub / 4) ^ it (two 16-byte pieces).  A quarter warp's
    // 8 lanes read 8 distinct swizzled pieces and write 8 distinct core-matrix rows, so both
    // are free of bank conflicts and no lane needs another's values.  A block's 8 pieces per
    // lane are all loaded before any h or l is stored over them.
    const int cw = warp - 4;
    const int sub = lane & 7, qd = lane >> 3;
    // column sums of r (diagonal units): 4 values at a time in FP32, then (hi, lo);
    // sums of l^2 (BF16x3), ~2^-16 of the diagonal they correct: FP32 pairs over kWFold stages
    constexpr int NG = 16 / kWConv;  // groups per converter warp
    float sh[NG], sl[NG], qh[NG], ql[NG];
    float2 pq[NG];
#pragma unroll
    for (int i = 0; i < NG; ++i) {
      sh[i] = sl[i] = qh[i] = ql[i] = 0.f;
      pq[i] = make_float2(0.f, 0.f);
    }
    auto fold_squares = [&]() {
#pragma unroll
      for (int i = 0; i < NG; ++i) {
        two_sum(qh[i], ql[i], pq[i].x + pq[i].y);
        pq[i] = make_float2(0.f, 0.f);
      }
    };
    int since = 0;
    const int64_t tail = P.nrows - P.nfull * kWChunk;  // rows after the last whole chunk (< 32)
    int s = 0;
    uint32_t ph = 0;
    for (int64_t k = 0; k < my; ++k) {
      const bool ok = __all_sync(0xffffffffu, wait_live(&f_full[s], ph, &s_dead));
      if (!ok) {
        if (lane == 0) record_timeout(&s_dead, P.status);
        break;
      }
      const int64_t st = q0 + k * Gu;
      const int rows = s_rows[s];
      uint8_t* stage = smem + static_cast<size_t>(s) * nblk * kWBlkBytes;
      const int64_t jt = P.nfull - st * kWChains;  // chunk of the stage that holds the tail, if 0 or 1
      for (int blk = 0; blk < nblk; ++blk) {
        uint8_t* base = stage + blk * kWBlkBytes;
        const int col0 = (blk ? J : I) * kWBlk;
        if (tail > 0 && (jt == 0 || jt == 1)) {
          // the tail chunk is past the tensor map (zero-filled): this warp's 8 NG columns by plain loads
          const int c = 8 * NG * cw + lane;
          const int L = 2 * c + static_cast<int>(jt);
          if (lane < 8 * NG && col0 + c < P.p) {
            const float* src = P.base + static_cast<int64_t>(col0 + c) * P.ld + P.nfull * kWChunk;
            for (int t = 0; t < static_cast<int>(tail); ++t)
              *reinterpret_cast<float*>(base + fp32_piece(L, t >> 2) + (t & 3) * 4) = src[t];
          }
          __syncwarp();
        }
        float4 x[NG][2][2];
#pragma unroll
        for (int gi = 0; gi < NG; ++gi)
#pragma unroll
          for (int it = 0; it < 2; ++it) {
            const int L = 2 * (8 * (NG * cw + gi) + sub) + ((sub >> 2) ^ it);
            x[gi][it][0] = *reinterpret_cast<const float4*>(base + fp32_piece(L, 2 * qd));
            x[gi][it][1] = *reinterpret_cast<const float4*>(base + fp32_piece(L, 2 * qd + 1));
          }
        __syncwarp();  // the warp's FP32 is all in registers before its h and l overwrite it
#pragma unroll
        for (int gi = 0; gi < NG; ++gi) {
          const int g = NG * cw + gi;
          const float ncp = -s_piv[blk * kWBlk + 8 * g + sub];
          const float2 np = make_float2(ncp, ncp), m1 = make_float2(-1.f, -1.f);
#pragma unroll
          for (int it = 0; it < 2; ++it) {
            const int j = (sub >> 2) ^ it;
            const int row = kWChunk * j + 8 * qd;  // first of the lane's 8 rows within the stage
            float2 r[4] = {__fadd2_rn(make_float2(x[gi][it][0].x, x[gi][it][0].y), np),
                           __fadd2_rn(make_float2(x[gi][it][0].z, x[gi][it][0].w), np),
                           __fadd2_rn(make_float2(x[gi][it][1].x, x[gi][it][1].y), np),
                           __fadd2_rn(make_float2(x[gi][it][1].z, x[gi][it][1].w), np)};
            if (rows < kWRows) {
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                if (row + 2 * q >= rows) r[q].x = 0.f;
                if (row + 2 * q + 1 >= rows) r[q].y = 0.f;
              }
            }
            uint32_t h[4], l[4];
            float2 e[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              h[q] = pack_bf16x2(r[q].x, r[q].y);
              e[q] = __ffma2_rn(make_float2(bf_lo(h[q]), bf_hi(h[q])), m1, r[q]);  // r - h, exact
              // BF16x3 diagonal units store 2l (exact): one product 2 H^T L replaces H^T L + L^T H
              l[q] = (diag && !X4) ? pack_bf16x2(2.f * e[q].x, 2.f * e[q].y) : pack_bf16x2(e[q].x, e[q].y);
            }
            if (diag) {
              const float2 a = __fadd2_rn(r[0], r[1]), b = __fadd2_rn(r[2], r[3]);
              two_sum(sh[gi], sl[gi], a.x + a.y);
              two_sum(sh[gi], sl[gi], b.x + b.y);
              if (!X4) {
#pragma unroll
                for (int q = 0; q < 4; ++q) pq[gi] = __ffma2_rn(e[q], e[q], pq[gi]);
              }
            }
            uint8_t* cm = base + g * 2048 + (4 * j + qd) * 256 + sub * 16;
            *reinterpret_cast<uint4*>(cm) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4*>(cm + 128) = make_uint4(l[0], l[1], l[2], l[3]);
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&c_full[s]);
      if (diag && !X4 && ++since == kWFold) {
        since = 0;
        fold_squares();
      }
      if (++s == S) {
        s = 0;
        ph ^= 1u;
      }
    }
    if (diag) {
      fold_squares();
      // the 4 lanes of a column (sub equal) add their pairs (fixed order), lanes 0-7 write
#pragma unroll
      for (int i = 0; i < NG; ++i) {
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
          const int c = 8 * (NG * cw + i) + lane;
          float2* cs = reinterpret_cast<float2*>(P.slots) + static_cast<size_t>(blockIdx.x) * kWideSlotPairs +
                       kWBlk * kWBlk;
          cs[c] = make_float2(sh[i], sl[i]);
          cs[kWBlk + c] = make_float2(qh[i], ql[i]);
        }
      }
    }
  } else if (warp >= 12) {
    // ---------------------------------------------------------------- epilogue (warpgroup 3)
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kWRegsEpi));
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
    const int64_t chains = my * kWChains;
    for (int64_t k = 0; k < chains; ++k) {
      const bool ok = __all_sync(0xffffffffu, wait_live(&d_full[bd], phd, &s_dead));  // .sync.aligned loads follow
      if (!ok) {
        if (lane == 0) record_timeout(&s_dead, P.status);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t taddr = tmem + (static_cast<uint32_t>(32 * quarter) << 16) + static_cast<uint32_t>(bd * kWBlk);
      // 32 columns per round trip: two loads in flight, one wait
#pragma unroll
      for (int c0 = 0; c0 < kWBlk; c0 += 32) {
        uint32_t v[2][16];
        tc05::tmem_ld16_issue(taddr + c0, v[0]);
        tc05::tmem_ld16_issue(taddr + c0 + 16, v[1]);
        tc05::tmem_wait_ld();
        tc05::tmem_hold16(v[0]);
        tc05::tmem_hold16(v[1]);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          acc[c0 + i] += __uint_as_float(v[0][i]);
          acc[c0 + 16 + i] += __uint_as_float(v[1][i]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&d_empty[bd]);
      if (++bd == 2) {
        bd = 0;
        phd ^= 1u;
      }
      if (++since >= P.flush_chains) {
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

// Sum of slot entry idx over CTAs [q0, q1) into (h, l), eight loads in flight (the entries of
// consecutive CTAs are 133 KB apart: each load is its own L2 round trip).
__device__ __forceinline__ void sum_slots(const float2* slots, int idx, int q0, int q1, float& h, float& l) {
  for (int q = q0; q < q1; q += 8) {
    float2 x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      x[u] = q + u < q1 ? __ldcg(slots + static_cast<size_t>(q + u) * kWideSlotPairs + idx) : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      two_sum(h, l, x[u].x);
      two_sum(h, l, x[u].y);
    }
  }
}

__device__ __forceinline__ void dd_add(double* hi, double* lo, int64_t e, float h, float l) {
  const double v = static_cast<double>(h) + static_cast<double>(l);
  const double s = hi[e] + v;
  const double bp = s - hi[e];
  lo[e] += (hi[e] - (s - bp)) + (v - bp);
  hi[e] = s;
}

// The units' CTA slots into the context's double-double accumulators.  Block (m, unit) takes
// row m of the unit's 128 x 128 block (m = 128: a diagonal unit's column sums); thread
// (n, quarter) adds a quarter of the unit's CTAs, and the quarters are combined in order, so
// the result depends on the grid only.
template <bool X4>
__global__ void __launch_bounds__(512) wide_merge_kernel(const __grid_constant__ WideParams P) {
  __shared__ float4 part[4][kWBlk];
  const int unit = blockIdx.y, m = blockIdx.x;
  const int I = P.unit_i[unit], J = P.unit_j[unit];
  const int first = P.unit_first[unit], G = P.unit_ctas[unit];
  const int n = threadIdx.x & (kWBlk - 1), qq = threadIdx.x / kWBlk;
  const int q0 = first + qq * G / 4, q1 = first + (qq + 1) * G / 4;
  const int p = P.p;
  const float2* slots = reinterpret_cast<const float2*>(P.slots);
  const int row = I * kWBlk + m, col = J * kWBlk + n;
  const bool two_l = !X4 && I == J;  // BF16x3 diagonal unit: the block holds H^T H + 2 H^T L
  bool active;
  float h = 0.f, l = 0.f, qh = 0.f, ql = 0.f;
  if (m < kWBlk) {
    active = row < p && col >= row && col < p;
    if (active) {
      sum_slots(slots, m * kWBlk + n, q0, q1, h, l);
      if (two_l) sum_slots(slots, n * kWBlk + m, q0, q1, h, l);  // S = (D + D^T) / 2
      if (!X4 && col == row) sum_slots(slots, kWBlk * kWBlk + kWBlk + m, q0, q1, qh, ql);  // + diag(L^T L)
    }
  } else {
    active = I == J && col < p;
    if (active) sum_slots(slots, kWBlk * kWBlk + n, q0, q1, h, l);  // column sums
  }
  part[qq][n] = make_float4(h, l, qh, ql);
  __syncthreads();
  if (qq == 0 && active) {
    for (int k = 1; k < 4; ++k) {
      const float4 o = part[k][n];
      two_sum(h, l, o.x);
      l += o.y;
      two_sum(qh, ql, o.z);
      ql += o.w;
    }
    if (m < kWBlk) {
      if (two_l) {
        h *= 0.5f;
        l *= 0.5f;
      }
      two_sum(h, l, qh);
      l += ql;
      dd_add(P.acc_S, P.acc_S_lo, static_cast<int64_t>(row) * p - static_cast<int64_t>(row) * (row - 1) / 2 + (col - row),
             h, l);
    } else {
      dd_add(P.acc_s, P.acc_s_lo, col, h, l);
    }
  }
  if (unit == 0 && m == 0 && threadIdx.x == 0) *P.acc_n += P.nrows;
}

template <bool X4>
cudaError_t launch_w(const WideParams& P, int grid, cudaStream_t st) {
  const int smem = kWRingBytes;
  cudaError_t e = cudaFuncSetAttribute(wide_kernel<X4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  wide_kernel<X4><<<grid, kWThreads, smem, st>>>(P);
  wide_merge_kernel<X4><<<dim3(kWBlk + 1, P.nunits), 512, 0, st>>>(P);
  return cudaGetLastError();
}

}  // namespace

int wide_plan(int p, int sms, bool x4, WideParams& W) {
  // measured CTA time per stage, diagonal : off-diagonal units (BF16x3 diagonal units run two
  // products and convert one block, the others three products and two blocks; BF16x4 four)
  const int wd = x4 ? 7 : 2, wo = x4 ? 8 : 3;
  const int nb = (p + kWBlk - 1) / kWBlk;
  int u = 0, weight = 0;
  for (int I = 0; I < nb; ++I)
    for (int J = I; J < nb; ++J) {
      if (u >= kWideMaxUnits) return 0;
      W.unit_i[u] = I;
      W.unit_j[u] = J;
      weight += I == J ? wd : wo;
      ++u;
    }
  W.nunits = u;
  if (u > sms) return 0;
  // CTAs in proportion to the weights, at least one each, at most sms in all
  int grid = 0;
  for (int i = 0; i < u; ++i) {
    const int w = W.unit_i[i] == W.unit_j[i] ? wd : wo;
    W.unit_ctas[i] = std::max(1, (sms * w) / weight);
    grid += W.unit_ctas[i];
  }
  for (int i = 0; grid > sms; i = (i + 1) % u)
    if (W.unit_ctas[i] > 1) {
      --W.unit_ctas[i];
      --grid;
    }
  for (int i = 0, f = 0; i < u; ++i) {
    W.unit_first[i] = f;
    f += W.unit_ctas[i];
  }
  return grid;
}

int wide_rows_per_stage() { return kWRows; }
int wide_chunk_rows() { return kWChunk; }
int wide_block_cols() { return kWBlk; }

cudaError_t launch_wide(const WideParams& P, bool x4, int grid, cudaStream_t st) {
  return x4 ? launch_w<true>(P, grid, st) : launch_w<false>(P, grid, st);
}

}  // namespace ss
