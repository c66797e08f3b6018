// k_wide2.cu -- sufficient statistics of FP32 tables of 129 to 256 columns on pairs of SMs:
// tcgen05 MMAs of the cta_group::2 form, one 256 x 256 accumulator split over the two CTAs
// of a cluster.  arxiv 2604.23826, "Data Representation and Sufficient Statistics" (column
// sums and X^T X in one streaming pass, partials over row ranges combined), with the shift of
// "Numerical Considerations" (r = x - c, c = the mean of the table's first rows).
//
// The columns are two 128-column blocks; CTA rank r of a pair owns block r.  Each CTA reads
// and converts only its own block, so the table is read once and every value converted once.
// The pair's leader (rank 0) issues M = N = 256 MMAs whose A operand is the 256 operand rows
// (block 0 from the leader's shared memory, block 1 from the peer's, at the same offsets) and
// whose B operand is the same 256 columns (again 128 from each CTA); the accumulator D, 256 x
// 256 FP32, sits in tensor memory with rows 0..127 in the leader and 128..255 in the peer.
//   BF16x3: the converters store h and 2l; D = H^T H + H^T (2L), and (D + D^T) / 2 =
//           H^T H + H^T L + L^T H, formed by the merge (plus diag(L^T L) from the CUDA cores).
//   BF16x4: they store h and l; D = L^T L + 2 H^T L + H^T H (H^T L issued twice), and
//           (D + D^T) / 2 = H^T H + H^T L + L^T H + L^T L.
// The whole 256 x 256 block is formed, half of it twice, so the tensor pipe does a third more
// work than the upper triangle needs; it is not the bound.
//
// Each pair takes the 64-row stages q, q + pairs, ...; every two stages (128 rows) are one
// fresh MMA accumulation chain.
// In a CTA (512 threads, four warpgroups):
//   warp 0      producer: one 3D tensor copy of its block per stage (32 rows x 2 chunks x 128
//               columns, 128-byte swizzle, zeros past p) into a ring of six 32 KB stages;
//   warp 1      tensor memory (allocated by both CTAs together) and, in the leader, the MMA
//               issuer: it waits until both CTAs have converted the stage and drained the
//               accumulator buffer, issues the stage's MMAs, and commits to the stage-free and
//               (at a chain's end) chain-done barriers of both CTAs (multicast); in the peer,
//               one thread relays the epilogue's drained chains to the leader;
//   warps 2-3   in the peer, relays of converted stages (warp 2 the even stages, warp 3 the
//               odd): the converter warps arrive on local barriers, and a relay thread forwards
//               each completed phase to the leader with a single cluster-scope arrive (a release
//               at cluster scope stalls the arriving thread for about a stage's time under load,
//               so no converter pays it, and one thread alone could not keep up);
//   warps 4-7   converters: the stage's FP32 becomes, in place, the K-major core matrices of h
//               and l (or 2l), four 8-column groups per warp, two at a time; column sums of r
//               and (BF16x3) sums of l^2;
//   warps 8-15  epilogue: two warps per TMEM lane quarter, 128 columns each; every chain is
//               added into FP32 registers (round to nearest), and every flush into (hi, lo)
//               pairs in the CTA's slot.
// A second kernel adds the pairs' slots, in pair order, into the context's double-double
// accumulators.  Every wait is bounded; on expiry the CTA records STATS_ETIMEOUT and winds
// down; both CTAs always reach the final cluster barrier (no early exit).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tc05.cuh"

namespace ss {

namespace {

using tc05::bf_hi;
using tc05::bf_lo;
using tc05::fp32_piece;
using tc05::pack_bf16x2;
using tc05::record_timeout;
using tc05::tma_load_3d;
using tc05::two_sum;

constexpr int kPBlk = 128;                       // columns per block (per CTA)
constexpr int kPChunk = 32;                      // rows per 128-byte line of the tensor copy
constexpr int kPRows = 64;                       // rows per stage and per MMA chain
constexpr int kPStageBytes = kPBlk * kPRows * 4;  // 32 KB
constexpr int kPStages = 6;                      // 192 KB ring
constexpr int kPThreads = 512;
constexpr int kPConv = 4;                        // converter warps 4..7, four 8-column groups each
constexpr int kPEpi = 8;                         // epilogue warps 8..15
constexpr int kPRegsLow = 96, kPRegsEpi = 160;   // 2 x 128 x 96 + 2 x 128 x 160 = 65536
constexpr int kPGroupsAtOnce = 2;  // 8-column groups a converter warp loads before converting
constexpr uint32_t kPLbo = 256, kPSbo = 2048;    // next K group (8 rows), next 8 operand rows
constexpr int kPTmemCols = 512;                  // two 256-column accumulators
constexpr int kPChain = 2;                       // stages per MMA accumulation chain (128 rows)
constexpr uint32_t kPIdesc = tc05::idesc_bf16(256, 256);

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// the shared::cluster address of a local shared-memory object in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_addr(const void* local, uint32_t rank) {
  uint32_t a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_u32(local)), "r"(rank));
  return a;
}
__device__ __forceinline__ void arrive_cluster(uint32_t cluster_bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar) : "memory");
}
__device__ __forceinline__ bool try_wait_cluster(uint64_t* bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}
// bounded wait on a barrier that the other CTA of the pair also arrives on
__device__ __forceinline__ bool wait_cluster_live(uint64_t* bar, uint32_t parity, volatile unsigned int* dead) {
  if (try_wait_cluster(bar, parity, 0u)) return true;
  for (uint32_t i = 0; i < kSpinLimit; ++i) {
    if (try_wait_cluster(bar, parity, 1000u)) return true;
    if (*dead) return false;
  }
  return false;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void mma2(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(kPIdesc), "r"(accumulate)
      : "memory");
}
// arrive on the barrier at this offset in both CTAs once the issued MMAs complete
__device__ __forceinline__ void commit2(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(static_cast<uint16_t>(3))
      : "memory");
}
__device__ __forceinline__ uint64_t pdesc(uint32_t saddr) { return tc05::desc<kPLbo, kPSbo>(saddr); }

template <bool X4>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kPThreads, 1)
    wide2_kernel(const __grid_constant__ Wide2Params P) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t f_full[kPStages], c_full[kPStages], f_empty[kPStages], d_full[2], d_empty[2],
      fin, r_conv[kPStages], r_epi[2];
  __shared__ uint32_t s_tmem;
  __shared__ volatile unsigned int s_dead;
  __shared__ int s_rows[kPStages];
  __shared__ float s_piv[kPBlk];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
  const int64_t nst = (P.nrows + kPRows - 1) / kPRows;
  const int64_t my = pair < nst ? (nst - 1 - pair) / npairs + 1 : 0;  // stages of this pair
  const int64_t nchains = (my + kPChain - 1) / kPChain;                 // accumulation chains
  const int col0 = static_cast<int>(rank) * kPBlk;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kPStages; ++s) {
      mbar_init(&f_full[s], 1);
      mbar_init(&c_full[s], kPConv + 1);  // the leader's: its converter warps + the peer's relay
      mbar_init(&f_empty[s], 1);
      mbar_init(&r_conv[s], kPConv);      // the peer's: its converter warps, forwarded by the relay
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&d_full[b], 1);
      mbar_init(&d_empty[b], kPEpi + 1);  // the leader's: its epilogue warps + the peer's relay
      mbar_init(&r_epi[b], kPEpi);        // the peer's: its epilogue warps, forwarded by the relay
    }
    mbar_init(&fin, 1);
    s_dead = 0;
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < kPBlk; i += kPThreads) s_piv[i] = col0 + i < P.p ? P.shift[col0 + i] : 0.f;
  if (warp == 1) {  // both CTAs allocate the pair's tensor memory together
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(kPTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync();  // both CTAs' barriers initialised before any cross-CTA arrive
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  if (warp < 8) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kPRegsLow));
  if (warp == 0) {
    // ---------------------------------------------------------------- producer (both CTAs)
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      int64_t k = 0;
      for (; k < my; ++k) {
        const int64_t st = pair + k * npairs;
        if (k >= kPStages && !tc05::wait_live(&f_empty[s], ph ^ 1u, &s_dead)) {
          record_timeout(&s_dead, P.status);
          break;
        }
        s_rows[s] = static_cast<int>(min(static_cast<int64_t>(kPRows), P.nrows - st * kPRows));
        mbar_arrive_expect_tx(&f_full[s], static_cast<uint32_t>(kPStageBytes));
        tma_load_3d(smem + static_cast<size_t>(s) * kPStageBytes, P.tmap, 0, static_cast<int>(st * 2), col0,
                    &f_full[s]);
        if (++s == kPStages) {
          s = 0;
          ph ^= 1u;
        }
      }
      for (int d = 0; d < kPStages && d < k; ++d) {  // no copy in flight at exit
        int sk = s - 1 - d;
        uint32_t pk = ph;
        while (sk < 0) {
          sk += kPStages;
          pk ^= 1u;
        }
        mbar_wait_bounded(&f_full[sk], pk);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer (leader) / relay (peer)
    if (!leader && lane == 0) {
      // the peer's epilogue warps arrive on local barriers; this thread forwards each drained
      // chain to the leader (one cluster-scope arrive per chain)
      const uint32_t remote0 = cluster_addr(&d_empty[0], 0);
      int b = 0;
      uint32_t ph = 0;
      for (int64_t k = 0; k < nchains; ++k) {
        if (!tc05::wait_live(&r_epi[b], ph, &s_dead)) {
          record_timeout(&s_dead, P.status);
          break;
        }
        arrive_cluster(remote0 + static_cast<uint32_t>(b * sizeof(uint64_t)));
        if (++b == 2) {
          b = 0;
          ph ^= 1u;
        }
      }
    }
    if (leader) {
      int s = 0, bd = 0;
      uint32_t ph = 0, phd = 0;
      bool live = true;
      for (int64_t k = 0; live && k < my; ++k) {
        const int in_chain = static_cast<int>(k % kPChain);  // a chain starts on buffer bd at in_chain 0
        const int64_t chain = k / kPChain;
        const bool ok = __shfl_sync(
            0xffffffffu,
            lane == 0 ? (wait_cluster_live(&c_full[s], ph, &s_dead) &&
                         (in_chain != 0 || chain < 2 || wait_cluster_live(&d_empty[bd], phd ^ 1u, &s_dead)))
                      : false,
            0);
        if (!ok) {
          if (lane == 0) record_timeout(&s_dead, P.status);
          live = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base = smem_u32(smem + static_cast<size_t>(s) * kPStageBytes);
        const uint32_t dt = tmem + static_cast<uint32_t>(bd * 256);
        const bool last = in_chain == kPChain - 1 || k == my - 1;
        if (tc05::elect_one()) {
          // K step ks: K groups 2 ks, 2 ks + 1 of every 8-column group (h at +0, l at +128).  The
          // descriptors' address field is (address >> 4) in the low bits (no carry inside the
          // 227 KB of shared memory), so the others are the stage's h descriptor plus an offset.
          const uint64_t dh = pdesc(base), dl = dh + (128 >> 4);
          constexpr uint64_t kStep = 512 >> 4;
          uint32_t acc = in_chain != 0 ? 1u : 0u;
          if (X4) {
#pragma unroll 1
            for (int ks = 0; ks < kPRows / 16; ++ks, acc = 1) mma2(dt, dl + ks * kStep, dl + ks * kStep, acc);  // L^T L
#pragma unroll 1
            for (int ks = 0; ks < kPRows / 16; ++ks) mma2(dt, dh + ks * kStep, dl + ks * kStep, 1);  // H^T L
          }
#pragma unroll 1
          for (int ks = 0; ks < kPRows / 16; ++ks, acc = 1)
            mma2(dt, dh + ks * kStep, dl + ks * kStep, acc);  // H^T L (BF16x3: 2l)
#pragma unroll 1
          for (int ks = 0; ks < kPRows / 16; ++ks) mma2(dt, dh + ks * kStep, dh + ks * kStep, 1);  // H^T H
          commit2(&f_empty[s]);  // both CTAs' stage s is free once these MMAs have read it
          if (last) commit2(&d_full[bd]);
        }
        __syncwarp();
        if (last && ++bd == 2) {
          bd = 0;
          phd ^= 1u;
        }
        if (++s == kPStages) {
          s = 0;
          ph ^= 1u;
        }
      }
      if (tc05::elect_one()) commit2(&fin);  // every issued MMA completes before the memory is released
      __syncwarp();
    }
    if (lane == 0) mbar_wait_bounded(&fin, 0);
    __syncwarp();
  } else if (warp == 2 || warp == 3) {
    // ---------------------------------------------------------------- relays (peer CTA)
    // The peer's converter warps arrive on local barriers; one thread forwards each completed
    // phase to the leader with a single cluster-scope arrive, so the converters never wait on a
    // cluster-wide release themselves.  A release at cluster scope costs about a stage's time
    // under load, so two threads take alternate stages (warp 2 the even ones, warp 3 the odd).
    if (!leader && lane == 0) {
      const uint32_t remote0 = cluster_addr(&c_full[0], 0);
      for (int64_t k = warp - 2; k < my; k += 2) {
        const int b = static_cast<int>(k % kPStages);
        if (!tc05::wait_live(&r_conv[b], static_cast<uint32_t>((k / kPStages) & 1), &s_dead)) {
          record_timeout(&s_dead, P.status);
          break;
        }
        arrive_cluster(remote0 + static_cast<uint32_t>(b * sizeof(uint64_t)));
      }
    }
  } else if (warp >= 4 && warp < 4 + kPConv) {
    // ---------------------------------------------------------------- converters (in place)
    // Warp cw owns the 8-column groups 4 cw .. 4 cw + 3.  Group g's FP32 lines (columns 8g ..
    // 8g + 7, two 32-row chunks each) are the 2 KB at g * 2048; they become its core matrices:
    // K group kk (rows 8 kk .. 8 kk + 7) of h at g * 2048 + kk * 256 and of l at + 128.  Lane:
    // column sub = lane % 8 and, in step it, K group kk = 4 j + lane / 8 of chunk
    // j = (sub / 4) ^ it; every lane loads its pieces of the group before any lane stores.
    const int cw = warp - 4;
    const int sub = lane & 7, qd = lane >> 3;
    uint64_t* cbar = leader ? c_full : r_conv;  // the leader's own barrier, or the peer's relay
    float sh[4], sl[4], qh[4], ql[4];  // (hi, lo) column sums of r and of l^2
#pragma unroll
    for (int i = 0; i < 4; ++i) sh[i] = sl[i] = qh[i] = ql[i] = 0.f;
    const int64_t tail = P.nrows - P.nfull * kPChunk;  // rows after the last whole chunk (< 32)
    int s = 0;
    uint32_t ph = 0;
    for (int64_t k = 0; k < my; ++k) {
      const bool ok = __all_sync(0xffffffffu, tc05::wait_live(&f_full[s], ph, &s_dead));
      if (!ok) {
        if (lane == 0) record_timeout(&s_dead, P.status);
        break;
      }
      const int64_t st = pair + k * npairs;
      const int rows = s_rows[s];
      uint8_t* base = smem + static_cast<size_t>(s) * kPStageBytes;
      const int64_t jt = P.nfull - st * 2;  // chunk of the stage holding the tail, if 0 or 1
      if (tail > 0 && (jt == 0 || jt == 1)) {
        // the tail chunk is past the tensor map (zero-filled): this warp's 32 columns by plain loads
        const int c = 32 * cw + lane;
        const int L = 2 * c + static_cast<int>(jt);
        if (col0 + c < P.p) {
          const float* src = P.base + static_cast<int64_t>(col0 + c) * P.ld + P.nfull * kPChunk;
          for (int t = 0; t < static_cast<int>(tail); ++t)
            *reinterpret_cast<float*>(base + fp32_piece(L, t >> 2) + (t & 3) * 4) = src[t];
        }
        __syncwarp();
      }
#pragma unroll
      for (int g0 = 0; g0 < 4; g0 += kPGroupsAtOnce) {
        // the FP32 of kPGroupsAtOnce groups in registers first: independent conversions to overlap
        float4 x[kPGroupsAtOnce][2][2];
#pragma unroll
        for (int u = 0; u < kPGroupsAtOnce; ++u) {
          const int g = 4 * cw + g0 + u;
#pragma unroll
          for (int it = 0; it < 2; ++it) {
            const int L = 2 * (8 * g + sub) + ((sub >> 2) ^ it);
            x[u][it][0] = *reinterpret_cast<const float4*>(base + fp32_piece(L, 2 * qd));
            x[u][it][1] = *reinterpret_cast<const float4*>(base + fp32_piece(L, 2 * qd + 1));
          }
        }
        __syncwarp();  // the groups' FP32 is in registers before their h and l overwrite it
#pragma unroll
        for (int u = 0; u < kPGroupsAtOnce; ++u) {
          const int gi = g0 + u, g = 4 * cw + gi;
          const float ncp = -s_piv[8 * g + sub];
          const float2 np = make_float2(ncp, ncp), m1 = make_float2(-1.f, -1.f);
          // this lane's 16 values of the group in a depth-4 FP32 tree, its 16 squares of l in
          // FP32, each then once into its (hi, lo) pair
          float2 t = make_float2(0.f, 0.f), pq = make_float2(0.f, 0.f);
#pragma unroll
          for (int it = 0; it < 2; ++it) {
            const int j = (sub >> 2) ^ it;
            const int row = kPChunk * j + 8 * qd;
            float2 r[4] = {__fadd2_rn(make_float2(x[u][it][0].x, x[u][it][0].y), np),
                           __fadd2_rn(make_float2(x[u][it][0].z, x[u][it][0].w), np),
                           __fadd2_rn(make_float2(x[u][it][1].x, x[u][it][1].y), np),
                           __fadd2_rn(make_float2(x[u][it][1].z, x[u][it][1].w), np)};
            if (rows < kPRows) {
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
              l[q] = X4 ? pack_bf16x2(e[q].x, e[q].y) : pack_bf16x2(2.f * e[q].x, 2.f * e[q].y);
            }
            t = __fadd2_rn(t, __fadd2_rn(__fadd2_rn(r[0], r[1]), __fadd2_rn(r[2], r[3])));
            if (!X4)
#pragma unroll
              for (int q = 0; q < 4; ++q) pq = __ffma2_rn(e[q], e[q], pq);
            uint8_t* cm = base + g * 2048 + (4 * j + qd) * 256 + sub * 16;
            *reinterpret_cast<uint4*>(cm) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4*>(cm + 128) = make_uint4(l[0], l[1], l[2], l[3]);
          }
          two_sum(sh[gi], sl[gi], t.x + t.y);
          if (!X4) two_sum(qh[gi], ql[gi], pq.x + pq.y);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&cbar[s]);
      if (++s == kPStages) {
        s = 0;
        ph ^= 1u;
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      // the 4 lanes of a column (sub equal) add their pairs (fixed order), lanes 0-7 write
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
        const int c = 8 * (4 * cw + i) + lane;
        float2* cs = reinterpret_cast<float2*>(P.slots) + static_cast<size_t>(blockIdx.x) * kWide2SlotPairs +
                     kPBlk * 256;
        cs[c] = make_float2(sh[i], sl[i]);
        cs[kPBlk + c] = make_float2(qh[i], ql[i]);
      }
    }
  } else if (warp >= 8) {
    // ---------------------------------------------------------------- epilogue (warps 8-15)
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kPRegsEpi));
    const int quarter = warp & 3;                 // TMEM lanes 32 quarter .. 32 quarter + 31
    const int half = (warp - 8) >> 2;             // accumulator columns 128 half .. 128 half + 127
    const int m = 32 * quarter + lane;            // this thread's row of the CTA's 128 x 256 half
    uint64_t* ebar = leader ? d_empty : r_epi;  // the leader's own barrier, or the peer's relay
    float acc[128];
#pragma unroll
    for (int i = 0; i < 128; ++i) acc[i] = 0.f;
    float2* slot = reinterpret_cast<float2*>(P.slots) + static_cast<size_t>(blockIdx.x) * kWide2SlotPairs +
                   static_cast<size_t>(m) * 256 + 128 * half;
    bool fresh = true;
    int since = 0;
    auto flush = [&]() {  // four pairs at a time: the 128 sums leave little room
#pragma unroll
      for (int i0 = 0; i0 < 128; i0 += 4) {
        float2 hl[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) hl[k] = fresh ? make_float2(0.f, 0.f) : __ldcg(slot + i0 + k);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
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
    for (int64_t k = 0; k < nchains; ++k) {
      const bool ok = __all_sync(0xffffffffu, tc05::wait_live(&d_full[bd], phd, &s_dead));
      if (!ok) {
        if (lane == 0) record_timeout(&s_dead, P.status);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t taddr =
          tmem + (static_cast<uint32_t>(32 * quarter) << 16) + static_cast<uint32_t>(bd * 256 + 128 * half);
      // one 16-column load per wait (registers: 128 sums + 16); the warp sharing this SMSP
      // covers the load latency
#pragma unroll
      for (int c0 = 0; c0 < 128; c0 += 16) {
        uint32_t v[16];
        tc05::tmem_ld16_issue(taddr + c0, v);
        tc05::tmem_wait_ld();
        tc05::tmem_hold16(v);
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[c0 + i] += __uint_as_float(v[i]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&ebar[bd]);
      if (++bd == 2) {
        bd = 0;
        phd ^= 1u;
      }
      since += kPChain;
      if (since >= P.flush_stages) {
        since = 0;
        flush();
      }
    }
    flush();  // also writes the slot of a pair without stages
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kPTmemCols) : "memory");
  }
  cluster_sync();  // neither CTA leaves while the other may still arrive on its barriers
}

// Sum of slot entry idx over CTAs c = first, first + 2, ... (one CTA of each pair) in pair
// order, into (h, l), eight loads in flight.
__device__ __forceinline__ void sum_pairs(const float2* slots, int idx, int first, int q0, int q1, float& h, float& l) {
  for (int q = q0; q < q1; q += 8) {
    float2 x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      x[u] = q + u < q1 ? __ldcg(slots + static_cast<size_t>(2 * (q + u) + first) * kWide2SlotPairs + idx)
                        : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      two_sum(h, l, x[u].x);
      two_sum(h, l, x[u].y);
    }
  }
}

__device__ __forceinline__ void dd_add2(double* hi, double* lo, int64_t e, float h, float l) {
  const double v = static_cast<double>(h) + static_cast<double>(l);
  const double s = hi[e] + v;
  const double bp = s - hi[e];
  lo[e] += (hi[e] - (s - bp)) + (v - bp);
  hi[e] = s;
}

// The pairs' slots into the context's double-double accumulators.  Block i (< 256): row i of
// S, entries j >= i: (D_ij + D_ji) / 2, D_ij in the slot of CTA rank i / 128 (its row i % 128,
// column j), plus (BF16x3) sum l^2 on the diagonal; block 256: the column sums.  Thread
// (j, quarter) adds a quarter of the pairs and the quarters are combined in order.
template <bool X4>
__global__ void __launch_bounds__(1024) wide2_merge_kernel(const __grid_constant__ Wide2Params P, int npairs) {
  __shared__ float4 part[4][256];
  const int i = blockIdx.x;
  const int j = threadIdx.x & 255, qq = threadIdx.x >> 8;
  const int q0 = qq * npairs / 4, q1 = (qq + 1) * npairs / 4;
  const float2* slots = reinterpret_cast<const float2*>(P.slots);
  const int p = P.p;
  bool active;
  float h = 0.f, l = 0.f, qh = 0.f, ql = 0.f;
  if (i < 256) {
    active = i < p && j >= i && j < p;
    if (active) {
      sum_pairs(slots, (i % 128) * 256 + j, i / 128, q0, q1, h, l);  // D_ij
      sum_pairs(slots, (j % 128) * 256 + i, j / 128, q0, q1, h, l);  // D_ji
      if (!X4 && j == i) sum_pairs(slots, kPBlk * 256 + kPBlk + i % 128, i / 128, q0, q1, qh, ql);
    }
  } else {
    active = j < p;
    if (active) sum_pairs(slots, kPBlk * 256 + j % 128, j / 128, q0, q1, h, l);  // column sums
  }
  part[qq][j] = make_float4(h, l, qh, ql);
  __syncthreads();
  if (qq == 0 && active) {
    for (int k = 1; k < 4; ++k) {
      const float4 o = part[k][j];
      two_sum(h, l, o.x);
      l += o.y;
      two_sum(qh, ql, o.z);
      ql += o.w;
    }
    if (i < 256) {
      h *= 0.5f;  // (D_ij + D_ji) / 2, exact
      l *= 0.5f;
      two_sum(h, l, qh);
      l += ql;
      dd_add2(P.acc_S, P.acc_S_lo, static_cast<int64_t>(i) * p - static_cast<int64_t>(i) * (i - 1) / 2 + (j - i), h, l);
    } else {
      dd_add2(P.acc_s, P.acc_s_lo, j, h, l);
    }
  }
  if (i == 0 && threadIdx.x == 0) *P.acc_n += P.nrows;
}

template <bool X4>
cudaError_t launch_w2(const Wide2Params& P, int grid, cudaStream_t st) {
  const int smem = kPStages * kPStageBytes;
  cudaError_t e = cudaFuncSetAttribute(wide2_kernel<X4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  wide2_kernel<X4><<<grid, kPThreads, smem, st>>>(P);  // clusters of two (__cluster_dims__)
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  wide2_merge_kernel<X4><<<257, 1024, 0, st>>>(P, grid / 2);
  return cudaGetLastError();
}

}  // namespace

int wide2_grid(int sms) { return std::max(2, sms / 2 * 2); }

cudaError_t launch_wide2(const Wide2Params& P, bool x4, int grid, cudaStream_t st) {
  if (grid < 2 || (grid & 1) || P.p <= kPBlk || P.p > 2 * kPBlk) return cudaErrorInvalidValue;
  return x4 ? launch_w2<true>(P, grid, st) : launch_w2<false>(P, grid, st);
}

}  // namespace ss
