// k_narrow.cu -- sufficient statistics of FP32 tables of 33 to 64 columns on the tcgen05
// tensor cores: arxiv 2604.23826, "Data Representation and Sufficient Statistics" (column
// sums and X^T X in one streaming pass, partials over row ranges combined), with the shift
// of "Numerical Considerations" (r = x - c, c = the mean of the table's first rows).
//
// The h and l halves of the split r = h + l (bf16 each) are stacked into one operand of
// M = 128 rows, 8-column group by 8-column group: operand row 16 g + i is h of column
// 8 g + i, row 16 g + 8 + i its l (i < 8).  One tcgen05.mma.kind::f16 per 16-row K step then
// gives every product at once (h(c), l(c): the operand rows of column c):
//   BF16x4: A = B = the stacked operand (N = 128), and
//           S[c][d] = D[h(c)][h(d)] + D[h(c)][l(d)] + D[l(c)][h(d)] + D[l(c)][l(d)];
//   BF16x3: A = the stacked operand, B = its h rows only (N = 64, read at twice the row-group
//           stride), and S[c][d] = D[h(c)][d] + D[l(c)][d] + D[l(d)][c] (+ sum l^2 on the
//           diagonal).
// TMEM lane m accumulates its own row, so each epilogue thread keeps 64 FP32 sums (BF16x4
// adds the h and l column of each d first); the merge kernel forms S from the slots.
//
// Work comes in units: a unit is a range of 128-row stages of one table (its own tensor map,
// pivots and tail), and CTA b takes units b, b + grid, ....  A single-table call has one
// unit of consecutive stages per CTA; a batched call deals the units of all its 33..64-column
// tables, largest first.  Every unit is reduced into its own slot and the merge adds a
// table's slots in row order, so the result depends on the units only.
//
// In a CTA (512 threads, four warpgroups; one CTA per SM):
//   warp 0      producer: one 3D tensor copy per 128-row stage (32 rows x 4 chunks x 64
//               columns: 512 contiguous bytes per column, 128-byte swizzle, zero past p) into a
//               ring of six 32 KB stages;
//               rows past the last whole 32-row chunk are read by the converters;
//   warps 4-11  converters, one 8-column group each: the group's 4 KB of FP32 becomes, in
//               place, its h core matrices (first 2 KB) and l core matrices (second 2 KB), K group
//               kk at + kk * 128, so a warp writes only what it read; column sums of r and
//               (BF16x3) sum l^2;
//   warp 1      MMA issuer: per 128-row stage eight K = 16 MMAs and a commit that frees the
//               stage; every two stages of a unit (256 rows) are one fresh chain in one of four
//               TMEM buffers, committed to the epilogue at its end;
//   warps 12-15 epilogue: each thread owns TMEM lane m, adds every chain into 64 FP32
//               registers (round to nearest) and, every flush, into (hi, lo) pairs in the
//               CTA's slot, draining a TMEM buffer per chain.
// Every wait is bounded: on expiry the CTA records STATS_ETIMEOUT and winds down.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tc05.cuh"

namespace ss {

namespace {

using namespace tc05;

constexpr int kNCols = 64;                        // columns of the block
constexpr int kNChunk = 32;                       // rows per tensor-copy line
constexpr int kNRows = 128;                       // rows per stage (8 K steps): 512 contiguous bytes per column
constexpr int kNChunks = kNRows / kNChunk;
constexpr int kNStageBytes = kNCols * kNRows * 4;  // 32 KB: FP32, then h (16 KB) and l (16 KB) in place
constexpr int kNStages = 6;                       // 192 KB ring
constexpr int kNThreads = 512;
constexpr int kNConv = 8;                         // converter warps 4 .. 11
constexpr int kNRegsLow = 104, kNRegsEpi = 200;   // 3 x 104 + 200 = 4 x 128 per SMSP
constexpr uint32_t kNLbo = 128, kNSbo = kNRows * 16;  // next K group, next 8 operand rows (h, l alternate)
constexpr int kNBufs = 4;                         // accumulator buffers in tensor memory (128 columns each)
constexpr int kNChain = 2;                        // stages per accumulation chain (256 rows) within a unit
constexpr int kNTmemCols = 128 * kNBufs;
constexpr int kNFold = 16;                        // stages of FP32 partial sums of l^2 per fold
constexpr int kNSlotStride = 128;                 // pairs per slot row (the wide pass's slot layout)

__device__ __forceinline__ NarrowUnit narrow_unit(const NarrowParams& P, int u) {
  if (P.units) return P.units[u];
  const int64_t nst = (P.tab0.nrows + kNRows - 1) / kNRows;
  const int64_t a = u * nst / P.nunits, b = (u + 1) * nst / P.nunits;
  NarrowUnit U;
  U.st0 = a;
  U.nst = static_cast<int32_t>(b - a);
  U.tab = 0;
  U.slot = u;
  U.pad = 0;
  return U;
}
__device__ __forceinline__ const NarrowTab& narrow_tab(const NarrowParams& P, int t) {
  return P.tabs ? P.tabs[t] : P.tab0;
}

template <bool X4>
__global__ void __launch_bounds__(kNThreads, 1) narrow_kernel(const __grid_constant__ NarrowParams P) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t f_full[kNStages], c_full[kNStages], f_empty[kNStages], d_full[kNBufs], d_empty[kNBufs],
      fin;
  __shared__ uint32_t s_tmem;
  __shared__ volatile unsigned int s_dead;
  __shared__ int s_rows[kNStages];

  constexpr int NB = X4 ? 128 : 64;  // accumulator columns of a chain
  constexpr uint32_t kIdesc = idesc_bf16(128, NB);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kNStages; ++s) {
      mbar_init(&f_full[s], 1);
      mbar_init(&c_full[s], kNConv);
      mbar_init(&f_empty[s], 1);
    }
    for (int s = 0; s < kNBufs; ++s) {
      mbar_init(&d_full[s], 1);
      mbar_init(&d_empty[s], 4);
    }
    mbar_init(&fin, 1);
    s_dead = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(kNTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  // registers: warpgroup 3 (the epilogue) takes 200 per thread, warpgroups 0-2 give up to 104
  if (warp < 12) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kNRegsLow));

  // Every role walks the same units (u = blockIdx.x, + gridDim.x, ...) and, in each, the same
  // stages; the stage ring and the TMEM buffers run on across units.
  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    // (the whole warp runs the loop; one lane waits, one elected lane issues)
    int s = 0;
    uint32_t ph = 0;
    int64_t issued = 0;
    bool live = true;
    for (int u = blockIdx.x; live && u < P.nunits; u += gridDim.x) {
      const NarrowUnit U = narrow_unit(P, u);
      const NarrowTab& T = narrow_tab(P, U.tab);
      for (int k = 0; k < U.nst; ++k, ++issued) {
        const int64_t st = U.st0 + k;
        const bool ok = __shfl_sync(
            0xffffffffu, lane == 0 ? (issued < kNStages || wait_live(&f_empty[s], ph ^ 1u, &s_dead)) : false, 0);
        if (!ok) {
          if (lane == 0) record_timeout(&s_dead, P.status);
          live = false;
          break;
        }
        if (elect_one()) {
          s_rows[s] = static_cast<int>(min(static_cast<int64_t>(kNRows), T.nrows - st * kNRows));
          mbar_arrive_expect_tx(&f_full[s], static_cast<uint32_t>(kNStageBytes));
          tma_load_3d(smem + static_cast<size_t>(s) * kNStageBytes, T.tmap, 0, static_cast<int>(st * kNChunks), 0,
                      &f_full[s]);
        }
        __syncwarp();
        if (++s == kNStages) {
          s = 0;
          ph ^= 1u;
        }
      }
    }
    if (lane == 0) {
      for (int d = 0; d < kNStages && d < issued; ++d) {  // no copy in flight at exit
        int sk = s - 1 - d;
        uint32_t pk = ph;
        while (sk < 0) {
          sk += kNStages;
          pk ^= 1u;
        }
        mbar_wait_bounded(&f_full[sk], pk);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    // The whole warp runs the loop (warp-uniform addresses and descriptors); one elected lane
    // issues the tcgen05 instructions.
    int s = 0, bd = 0;
    uint32_t ph = 0, phd = 0;
    int64_t chains = 0;
    bool live = true;
    for (int u = blockIdx.x; live && u < P.nunits; u += gridDim.x) {
      const int nst = narrow_unit(P, u).nst;
      for (int k = 0; k < nst; ++k) {
        // stage converted, and (at a chain's start) its TMEM buffer drained by the epilogue
        const int in_chain = k % kNChain;
        const bool last = in_chain == kNChain - 1 || k == nst - 1;
        const bool ok = __shfl_sync(
            0xffffffffu,
            lane == 0 ? (wait_live(&c_full[s], ph, &s_dead) &&
                         (in_chain != 0 || chains < kNBufs || wait_live(&d_empty[bd], phd ^ 1u, &s_dead)))
                      : false,
            0);
        if (!ok) {
          if (lane == 0) record_timeout(&s_dead, P.status);
          live = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base = smem_u32(smem + static_cast<size_t>(s) * kNStageBytes);
        const uint32_t dt = tmem + static_cast<uint32_t>(bd * 128);
        // a fresh chain every kNChain stages of a unit: K step ks = K groups 2 ks and 2 ks + 1;
        // A = the stacked operand, B = the same (BF16x4) or its h rows.  The stage is free once
        // its MMAs have read it; the chain's buffer goes to the epilogue at its end.
        if (elect_one()) {
#pragma unroll
          for (int ks = 0; ks < kNRows / 16; ++ks) {
            const uint64_t a = desc<kNLbo, kNSbo>(base + ks * 2 * kNLbo);
            const uint64_t b = X4 ? a : desc<kNLbo, 2 * kNSbo>(base + ks * 2 * kNLbo);
            mma_bf16(dt, a, b, kIdesc, (in_chain != 0 || ks != 0) ? 1u : 0u);
          }
          umma_commit(&f_empty[s]);
          if (last) umma_commit(&d_full[bd]);
        }
        __syncwarp();
        if (last) {
          ++chains;
          if (++bd == kNBufs) {
            bd = 0;
            phd ^= 1u;
          }
        }
        if (++s == kNStages) {
          s = 0;
          ph ^= 1u;
        }
      }
    }
    if (elect_one()) umma_commit(&fin);  // every issued MMA completes before the tensor memory is released
    __syncwarp();
    if (lane == 0) mbar_wait_bounded(&fin, 0);
    __syncwarp();
  } else if (warp >= 4 && warp < 4 + kNConv) {
    // ---------------------------------------------------------------- converters
    // Warp cw owns columns 8 cw .. 8 cw + 7: their FP32 lines L = 4 c + chunk are the 4 KB at
    // cw * 4096, where its h and l core matrices go.  Lane: column sub = lane % 8 of the group
    // and, in step it (0 .. 3), K group kk = 4 j + lane / 8 of chunk j = (sub / 2) ^ it: a quarter
    // warp reads 8 distinct swizzled 16-byte pieces (L mod 8 = 4 (sub mod 2) + j takes 8
    // values) and writes 8 distinct core-matrix rows (no bank conflicts).
    const int cw = warp - 4;
    const int sub = lane & 7, qd = lane >> 3;
    const int c = 8 * cw + sub;
    const float2 m1 = make_float2(-1.f, -1.f);
    int s = 0;
    uint32_t ph = 0;
    bool live = true;
    for (int u = blockIdx.x; live && u < P.nunits; u += gridDim.x) {
      const NarrowUnit U = narrow_unit(P, u);
      const NarrowTab& T = narrow_tab(P, U.tab);
      float sh = 0.f, sl = 0.f, qh = 0.f, ql = 0.f;  // column sums of r and l^2, (hi, lo)
      float2 pq = make_float2(0.f, 0.f);
      int since = 0;
      const int64_t tail = T.nrows - T.nfull * kNChunk;
      const float ncp = c < T.p ? -T.shift[c] : 0.f;
      const float2 np = make_float2(ncp, ncp);
      for (int k = 0; k < U.nst; ++k) {
        const bool ok = __all_sync(0xffffffffu, wait_live(&f_full[s], ph, &s_dead));
        if (!ok) {
          if (lane == 0) record_timeout(&s_dead, P.status);
          live = false;
          break;
        }
        const int64_t st = U.st0 + k;
        const int rows = s_rows[s];
        uint8_t* base = smem + static_cast<size_t>(s) * kNStageBytes;
        const int64_t jt = T.nfull - st * kNChunks;  // chunk of the stage holding the tail, if in range
        if (tail > 0 && jt >= 0 && jt < kNChunks) {
          if (lane < 8 && 8 * cw + lane < T.p) {
            const int cc = 8 * cw + lane;
            const int L = kNChunks * cc + static_cast<int>(jt);
            const float* src = T.base + static_cast<int64_t>(cc) * T.ld + T.nfull * kNChunk;
            for (int t = 0; t < static_cast<int>(tail); ++t)
              *reinterpret_cast<float*>(base + fp32_piece(L, t >> 2) + (t & 3) * 4) = src[t];
          }
          __syncwarp();
        }
        static_assert(kNChunks == 4, "the lane mapping below covers four 32-row chunks per stage");
        float4 x[kNChunks][2];
#pragma unroll
        for (int it = 0; it < kNChunks; ++it) {
          const int L = kNChunks * c + ((sub >> 1) ^ it);
          x[it][0] = *reinterpret_cast<const float4*>(base + fp32_piece(L, 2 * qd));
          x[it][1] = *reinterpret_cast<const float4*>(base + fp32_piece(L, 2 * qd + 1));
        }
        __syncwarp();  // the group's FP32 is in registers before its h and l overwrite it
        float2 t = make_float2(0.f, 0.f);  // two chunks' 16 values of this lane, a depth-4 tree
#pragma unroll
        for (int it = 0; it < kNChunks; ++it) {
          const int j = (sub >> 1) ^ it;
          const int row = kNChunk * j + 8 * qd;
          float2 r[4] = {__fadd2_rn(make_float2(x[it][0].x, x[it][0].y), np),
                         __fadd2_rn(make_float2(x[it][0].z, x[it][0].w), np),
                         __fadd2_rn(make_float2(x[it][1].x, x[it][1].y), np),
                         __fadd2_rn(make_float2(x[it][1].z, x[it][1].w), np)};
          if (rows < kNRows) {
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
            l[q] = pack_bf16x2(e[q].x, e[q].y);
          }
          t = __fadd2_rn(t, __fadd2_rn(__fadd2_rn(r[0], r[1]), __fadd2_rn(r[2], r[3])));
          if (it & 1) {
            two_sum(sh, sl, t.x + t.y);
            t = make_float2(0.f, 0.f);
          }
          if (!X4) {
#pragma unroll
            for (int q = 0; q < 4; ++q) pq = __ffma2_rn(e[q], e[q], pq);
          }
          const int kk = 4 * j + qd;
          uint8_t* hp = base + 2 * cw * kNSbo + kk * kNLbo + sub * 16;
          *reinterpret_cast<uint4*>(hp) = make_uint4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<uint4*>(hp + kNSbo) = make_uint4(l[0], l[1], l[2], l[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&c_full[s]);
        if (!X4 && ++since == kNFold) {
          since = 0;
          two_sum(qh, ql, pq.x + pq.y);
          pq = make_float2(0.f, 0.f);
        }
        if (++s == kNStages) {
          s = 0;
          ph ^= 1u;
        }
      }
      two_sum(qh, ql, pq.x + pq.y);
      // the 4 lanes of a column (sub equal) add their pairs (fixed order), lanes 0-7 write
#pragma unroll
      for (int d = 8; d < 32; d <<= 1) {
        const float oh_ = __shfl_xor_sync(0xffffffffu, sh, d), ol_ = __shfl_xor_sync(0xffffffffu, sl, d);
        const float oq_ = __shfl_xor_sync(0xffffffffu, qh, d), oql = __shfl_xor_sync(0xffffffffu, ql, d);
        two_sum(sh, sl, oh_);
        sl += ol_;
        two_sum(qh, ql, oq_);
        ql += oql;
      }
      if (lane < 8) {
        float2* cs = reinterpret_cast<float2*>(P.slots) + static_cast<size_t>(U.slot) * kWideSlotPairs +
                     128 * kNSlotStride;
        cs[c] = make_float2(sh, sl);
        cs[128 + c] = make_float2(qh, ql);
      }
    }
  } else if (warp >= 12) {
    // ---------------------------------------------------------------- epilogue (warpgroup 3)
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kNRegsEpi));
    const int quarter = warp & 3;
    const int m = 32 * quarter + lane;  // TMEM lane = operand row: h (m % 16 < 8) or l of column 8 (m / 16) + m % 8
    float acc[kNCols];
#pragma unroll
    for (int i = 0; i < kNCols; ++i) acc[i] = 0.f;
    int bd = 0;
    uint32_t phd = 0;
    bool live = true;
    for (int u = blockIdx.x; live && u < P.nunits; u += gridDim.x) {
      const NarrowUnit U = narrow_unit(P, u);
      float2* slot = reinterpret_cast<float2*>(P.slots) + static_cast<size_t>(U.slot) * kWideSlotPairs +
                     static_cast<size_t>(m) * kNSlotStride;
      bool fresh = true;
      int since = 0;
      auto flush = [&]() {
#pragma unroll
        for (int i0 = 0; i0 < kNCols; i0 += 8) {
          float2 hl[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) hl[k] = fresh ? make_float2(0.f, 0.f) : __ldcg(slot + i0 + k);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            two_sum(hl[k].x, hl[k].y, acc[i0 + k]);
            acc[i0 + k] = 0.f;
            __stcg(slot + i0 + k, hl[k]);
          }
          asm volatile("" ::: "memory");
        }
        fresh = false;
      };
      const int nchain = (U.nst + kNChain - 1) / kNChain;
      for (int k = 0; k < nchain; ++k) {
        const bool ok = __all_sync(0xffffffffu, wait_live(&d_full[bd], phd, &s_dead));  // .sync.aligned loads follow
        if (!ok) {
          if (lane == 0) record_timeout(&s_dead, P.status);
          live = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t taddr =
            tmem + (static_cast<uint32_t>(32 * quarter) << 16) + static_cast<uint32_t>(bd * 128);
        // 64 columns per round trip: four loads in flight, one wait
#pragma unroll
        for (int c0 = 0; c0 < NB; c0 += 64) {
          uint32_t v[4][16];
#pragma unroll
          for (int b = 0; b < 4; ++b) tmem_ld16_issue(taddr + c0 + 16 * b, v[b]);
          tmem_wait_ld();
#pragma unroll
          for (int b = 0; b < 4; ++b) tmem_hold16(v[b]);
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int cb = c0 + 16 * b;
            if (X4) {  // columns 16 g .. 16 g + 7: h of columns 8 g + i; the next 8: their l
#pragma unroll
              for (int i = 0; i < 8; ++i) acc[cb / 2 + i] += __uint_as_float(v[b][i]) + __uint_as_float(v[b][8 + i]);
            } else {
#pragma unroll
              for (int i = 0; i < 16; ++i) acc[cb + i] += __uint_as_float(v[b][i]);
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&d_empty[bd]);
        if (++bd == kNBufs) {
          bd = 0;
          phd ^= 1u;
        }
        since += kNChain;
        if (since >= P.flush_stages) {
          since = 0;
          flush();
        }
      }
      flush();  // every unit's slot is written, also when it had no stage
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kNTmemCols) : "memory");
  }
}

// Sum of slot entry idx over slots [q0, q1) into (h, l), eight loads in flight (consecutive
// slots are 133 KB apart: each load is its own L2 round trip).
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

// A table's unit slots into its context's double-double accumulators.  Block (t, m): table t,
// row m (< p) of S, or (m = p) the column sums; thread (n, quarter) adds a quarter of the
// table's slots and the quarters are then combined in order, so the result depends on the
// units only.
template <bool X4>
__global__ void __launch_bounds__(256) narrow_merge_kernel(const __grid_constant__ NarrowParams P) {
  __shared__ float2 part[4][kNCols];
  const int t = blockIdx.x;
  const NarrowTab& T = narrow_tab(P, t);
  const int p = T.p;
  const int m = blockIdx.y;
  if (m > p) return;  // the whole block
  const int u0 = P.tab_slot0 ? P.tab_slot0[t] : 0, u1 = P.tab_slot0 ? P.tab_slot0[t + 1] : P.nunits;
  const float2* slots = reinterpret_cast<const float2*>(P.slots);
  const int n = threadIdx.x & (kNCols - 1), qq = threadIdx.x / kNCols;
  const int q0 = u0 + qq * (u1 - u0) / 4, q1 = u0 + (qq + 1) * (u1 - u0) / 4;
  float h = 0.f, l = 0.f;
  if (m < p) {
    if (n >= m && n < p) {
      const int hm = 16 * (m / 8) + m % 8, hn = 16 * (n / 8) + n % 8;  // operand rows of h(m), h(n)
      sum_slots(slots, hm * kNSlotStride + n, q0, q1, h, l);          // H^T H (BF16x4: + H^T L)
      sum_slots(slots, (hm + 8) * kNSlotStride + n, q0, q1, h, l);    // L^T H (BF16x4: + L^T L)
      if (!X4) {
        sum_slots(slots, (hn + 8) * kNSlotStride + m, q0, q1, h, l);  // H^T L, from the transposed entry
        if (n == m) sum_slots(slots, 128 * kNSlotStride + 128 + m, q0, q1, h, l);  // + diag(L^T L)
      }
    }
  } else if (n < p) {
    sum_slots(slots, 128 * kNSlotStride + n, q0, q1, h, l);  // column sums
  }
  part[qq][n] = make_float2(h, l);
  __syncthreads();
  if (qq == 0) {
    for (int k = 1; k < 4; ++k) {
      two_sum(h, l, part[k][n].x);
      l += part[k][n].y;
    }
    if (m < p && n >= m && n < p)
      dd_add(T.acc_S, T.acc_S_lo, static_cast<int64_t>(m) * p - static_cast<int64_t>(m) * (m - 1) / 2 + (n - m), h, l);
    else if (m == p && n < p)
      dd_add(T.acc_s, T.acc_s_lo, n, h, l);
    if (m == p && n == 0) *T.acc_n += T.nrows;
  }
}

// pivot c_j = the mean of the table's first kPivotRows rows (or all, if fewer), rounded to FP32
__global__ void narrow_shift_kernel(const NarrowTab* __restrict__ tabs, const int* __restrict__ which) {
  const NarrowTab& T = tabs[which[blockIdx.x]];
  const int k = static_cast<int>(min(static_cast<int64_t>(kPivotRows), T.nrows));
  for (int j = threadIdx.x; j < T.p; j += blockDim.x) {
    double sum = 0.0;
    for (int i = 0; i < k; ++i) sum += static_cast<double>(T.base[static_cast<int64_t>(j) * T.ld + i]);
    const float v = static_cast<float>(sum / k);
    T.shift[j] = v;
    T.shift_d[j] = static_cast<double>(v);
  }
}

template <bool X4>
cudaError_t launch_n(const NarrowParams& P, int grid, cudaStream_t st) {
  const int smem = kNStages * kNStageBytes;
  cudaError_t e = cudaFuncSetAttribute(narrow_kernel<X4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  narrow_kernel<X4><<<grid, kNThreads, smem, st>>>(P);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  narrow_merge_kernel<X4><<<dim3(P.tabs ? P.ntabs : 1, kNCols + 1), 256, 0, st>>>(P);
  return cudaGetLastError();
}

}  // namespace

int narrow_cols() { return kNCols; }
int narrow_rows_per_stage() { return kNRows; }

cudaError_t launch_narrow(const NarrowParams& P, bool x4, int grid, cudaStream_t st) {
  if (grid < 1 || P.nunits < 1 || (P.tabs && (P.ntabs < 1 || !P.units || !P.tab_slot0))) return cudaErrorInvalidValue;
  return x4 ? launch_n<true>(P, grid, st) : launch_n<false>(P, grid, st);
}

cudaError_t launch_narrow_shift(const NarrowTab* tabs, const int* which, int count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  narrow_shift_kernel<<<count, 64, 0, st>>>(tabs, which);
  return cudaGetLastError();
}

}  // namespace ss
