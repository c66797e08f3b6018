// k_gram32.cu -- sufficient statistics of FP32 tables of up to 64 columns on the
// tensor cores, register-fragment form of the bf16 split (BF16x3 / BF16x4):
// arxiv 2604.23826, "Data Representation and Sufficient Statistics" (column sums
// and X^T X in one streaming pass, partials over row ranges combined), with the
// shift of "Numerical Considerations" (r = x - c, c = the mean of the table's first
// rows, so that X^T X and n mu mu^T are never formed separately).
//
// Each value becomes r = h + l, h = bf16(r), l = bf16(r - h), and
//   S' = sum r r^T  ~  L^T H + H^T L + H^T H + diag(L^T L)   (BF16x3)
//                    + L^T L                                (BF16x4, issued first).
// The dropped L^T L is ~2^-16 of S'; its diagonal (sum of l^2 >= 0) is a bias that
// does not average out, so BF16x3 adds it from the CUDA cores (an FFMA per value);
// the off-diagonal terms are sums of products of rounding residuals and cancel.
//
// Data path.  The launch's tables are cut into stages of RS rows x P columns
// (P = 8, 16: 16384 / P rows, 64 KB; P = 32, 64: 240 rows); the stages of all
// tables, in order, are dealt in chunks of consecutive stages round-robin to the
// persistent CTAs (CTA b takes chunks b, b + G, ...; the chunk length comes from
// the call's size and the batch tuning), so that neighbouring CTAs read
// neighbouring row ranges of a large table and a small table stays in one CTA.
// In a CTA a producer warp streams its stages into a shared-memory ring (3 stages
// for P = 8, 16 and 64; 6 for P = 32): a table whose columns sit one 16-byte
// multiple apart, with P >= 32, takes one 2D tensor copy per stage (zeros past p);
// otherwise one bulk copy (cp.async.bulk, mbarrier completion) per column (4-8 KB
// for P <= 16), and columns sit RS + 16 floats apart, so that the consumers'
// 128-bit loads are free of bank conflicts.  Consumer warps (15 for up to 32 columns,
// 7 for 64) take the 16-row K blocks in turn.  Lane
// (g, t) reads rows 4t..4t+3 of columns g + 8m with one 128-bit load per m;
// those four rows fill the k slots (2t, 2t+1, 2t+8, 2t+9) of both the A
// fragment (m16n8k16, A = X^T: rows = columns of X) and the B fragment
// (B = X), so the operands never leave registers and no value is converted
// twice.  Any assignment of rows to k slots gives the same X^T X, as long as A
// and B use the same one.
//
// Accumulation.  The FP32 accumulation inside the tensor core truncates, with
// an error that grows with the magnitude already held in the accumulator.
// Every K block therefore starts a fresh MMA chain (C = 0, smallest products
// first) whose 16-row result is added, rounding to nearest, into per-lane FP32
// accumulators; every flush_kblocks K blocks of a warp those are added with
// TwoSum into (hi, lo) pairs kept per warp in global scratch.  Column sums of r
// come from the same registers.  When a CTA's run of stages in one table ends,
// its consumer warps add their partials, in warp order, through a shared buffer
// into the CTA's slot of that table; a second, small kernel then adds every
// table's slots, in slot order, into its double-double accumulators.  Every
// floating-point addition has a fixed order given by the grid and the table
// list: results do not depend on scheduling.
//
// A unit's ragged last K block is padded by the producer with the pivot (r = 0).
// Tables whose columns are not all 16-byte aligned are staged by the producer
// lanes with plain loads (correct, slower).  Every wait is bounded; on expiry
// the CTA records STATS_ETIMEOUT in the table's status word, stops waiting,
// lets its issued copies land and returns.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace ss {

namespace {

template <int P>
struct G32 {
  // P >= 32: 240-row stages, filled by one 2D tensor copy when the table's columns are
  // uniformly strided (a 960-byte column stride is free of bank conflicts as it is);
  // P <= 16: 64 KB stages of per-column bulk copies of 4 KB (P = 16) or 8 KB (P = 8); bulk
  // copies of 2 KB feed at ~75 % of HBM, 4 KB ones at ~97 %; columns RS + 16 apart
  static constexpr bool TMAP = P >= 32;
  static constexpr int STAGES = P == 64 ? 3 : P == 32 ? 6 : 3;
  static constexpr int RS = TMAP ? 240 : 16384 / P;  // rows per stage
  static constexpr int LDC = TMAP ? RS : RS + 16;   // column stride in floats (= 16 mod 32)
  static constexpr int SF = P * LDC;                // floats per stage
  static constexpr int KBS = RS / 16;
  // consumer warps (plus one producer warp): 15 for up to 32 columns, whose fragments fit the
  // 128 registers of a 512-thread block; 7 for 64 columns, which need ~255
  static constexpr int GC = P <= 32 ? kGram32Warps : 7;
  static constexpr int THREADS = 32 * (GC + 1);
  static constexpr int UNROLL = P <= 8 ? 4 : P <= 16 ? 2 : 1;  // independent K blocks in flight per warp
  static constexpr int NM = P / 8;            // column groups of a lane: columns g + 8m
  static constexpr int NI = P >= 16 ? P / 16 : 1;
  static constexpr int NJ = P / 8;
  static constexpr int tiles() {
    int n = 0;
    for (int I = 0; I < NI; ++I) n += NJ - 2 * I;
    return n;
  }
  static constexpr int TILES = tiles();
  static constexpr int E = 4 * TILES + 2 * NM;  // accumulator words per lane: tiles, sums, sums of l^2
};

__device__ __forceinline__ float4 lds128(const float* p) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(smem_u32(p)));
  return v;
}

// (lo, hi) -> bf16x2 with lo in the low half (the lower k index of a fragment pair)
__device__ __forceinline__ uint32_t pack_bf16x2(float2 v) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(v.y), "f"(v.x));
  return d;
}
__device__ __forceinline__ float2 unpack_bf16x2(uint32_t v) {
  return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xFFFF0000u));
}

__device__ __forceinline__ void two_sum(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (v - bp);
  hi = s;
}

// 2D tensor copy of a box (rows x columns of a column-major table) into shared memory
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const void* tmap, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(smem_dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// (h, l) += the (hi, lo) pairs at word `off` of slots 0..n-1 (slot stride `stride` pairs), in
// slot order; eight loads in flight at a time
__device__ __forceinline__ void add_slots(const float2* __restrict__ slots, int n, int stride, int off, float& h,
                                          float& l) {
  int v = 0;
  for (; v + 8 <= n; v += 8) {
    float2 x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = __ldcg(slots + static_cast<size_t>(v + k) * stride + off);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      two_sum(h, l, x[k].x);
      two_sum(h, l, x[k].y);
    }
  }
  for (; v < n; ++v) {
    const float2 x = __ldcg(slots + static_cast<size_t>(v) * stride + off);
    two_sum(h, l, x.x);
    two_sum(h, l, x.y);
  }
}

// consumer warps only (named barrier 1)
template <int GC>
__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(32 * GC) : "memory"); }

// bounded wait that also gives up once another warp of the CTA has recorded a failure
__device__ __forceinline__ bool wait_live(uint64_t* bar, uint32_t parity, volatile unsigned int* dead) {
  if (mbar_try_wait(bar, parity)) return true;
  for (uint32_t i = 0; i < kSpinLimit; ++i) {
    if (mbar_try_wait_sleep(bar, parity, 1000u)) return true;
    if (*dead) return false;
  }
  return false;
}

// A lane's fragments of one K block (m16n8k16): rows 4t, 4t+1 of column group m fill
// the k slots (2t, 2t+1), rows 4t+2, 4t+3 the k slots (2t+8, 2t+9).  B of the 8-column
// block J is the register pair (h[J][0], h[J][1]); A of the 16-column block I (rows g
// and g + 8 = column groups 2I and 2I + 1) is the quad (h[2I][0], h[2I+1][0], h[2I][1],
// h[2I+1][1]).
template <int P>
struct Frag {
  uint32_t h[G32<P>::NM][2], l[G32<P>::NM][2];    // B pairs
  uint32_t qh[G32<P>::NI][4], ql[G32<P>::NI][4];  // A quads
};

// Convert one 16-row K block of a stage into register fragments.
template <int P, bool X4>
__device__ __forceinline__ void convert_kblock(const float* __restrict__ st, int kb, int g, int t,
                                               const float2* __restrict__ npiv, float2 (&sum)[G32<P>::NM],
                                               float2 (&lsq)[G32<P>::NM], Frag<P>& F) {
  using C = G32<P>;
#pragma unroll
  for (int m = 0; m < C::NM; ++m) {
    const float4 v = lds128(st + (g + 8 * m) * C::LDC + 16 * kb + 4 * t);
    const float2 np = npiv[g + 8 * m];  // (-c, -c) of this lane's column, shared memory
    const float2 r01 = __fadd2_rn(make_float2(v.x, v.y), np);
    const float2 r23 = __fadd2_rn(make_float2(v.z, v.w), np);
    sum[m] = __fadd2_rn(sum[m], __fadd2_rn(r01, r23));
    const uint32_t h01 = pack_bf16x2(r01), h23 = pack_bf16x2(r23);
    const float2 m1 = make_float2(-1.f, -1.f);
    F.h[m][0] = h01;
    F.h[m][1] = h23;
    const float2 e01 = __ffma2_rn(unpack_bf16x2(h01), m1, r01);  // r - h, exact
    const float2 e23 = __ffma2_rn(unpack_bf16x2(h23), m1, r23);
    F.l[m][0] = pack_bf16x2(e01);
    F.l[m][1] = pack_bf16x2(e23);
    if (!X4) {  // BF16x3: the diagonal of L^T L on the CUDA cores
      lsq[m] = __ffma2_rn(e01, e01, lsq[m]);
      lsq[m] = __ffma2_rn(e23, e23, lsq[m]);
    }
  }
  constexpr bool kTwo = C::NM > 1;  // P = 8: the second row group of A is empty
#pragma unroll
  for (int I = 0; I < C::NI; ++I) {
    const int m0 = 2 * I, m1 = kTwo ? 2 * I + 1 : 0;
    F.qh[I][0] = F.h[m0][0];
    F.qh[I][1] = kTwo ? F.h[m1][0] : 0u;
    F.qh[I][2] = F.h[m0][1];
    F.qh[I][3] = kTwo ? F.h[m1][1] : 0u;
    F.ql[I][0] = F.l[m0][0];
    F.ql[I][1] = kTwo ? F.l[m1][0] : 0u;
    F.ql[I][2] = F.l[m0][1];
    F.ql[I][3] = kTwo ? F.l[m1][1] : 0u;
  }
}

// D = A B + Z (Z a register quad of zeros: a fresh chain) and D += A B, m16n8k16 bf16 -> f32
__device__ __forceinline__ void mma_z(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1,
                                      const float (&z)[4]) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%10,%11,%12,%13};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(z[0]), "f"(z[1]), "f"(z[2]),
        "f"(z[3]));
}
__device__ __forceinline__ void mma_acc(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The K block's products on every upper tile (smallest first), added into the FP32
// accumulators.
template <int P, bool X4>
__device__ __forceinline__ void mma_kblock(const Frag<P>& F, const float (&z)[4], float (&acc)[G32<P>::TILES][4]) {
  using C = G32<P>;
  int ti = 0;
#pragma unroll
  for (int I = 0; I < C::NI; ++I) {
#pragma unroll
    for (int J = 2 * I; J < C::NJ; ++J, ++ti) {
      float d[4];
      if (X4) {
        mma_z(d, F.ql[I], F.l[J][0], F.l[J][1], z);
        mma_acc(d, F.ql[I], F.h[J][0], F.h[J][1]);
      } else {
        mma_z(d, F.ql[I], F.h[J][0], F.h[J][1], z);
      }
      mma_acc(d, F.qh[I], F.l[J][0], F.l[J][1]);
      mma_acc(d, F.qh[I], F.h[J][0], F.h[J][1]);
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[ti][k] += d[k];
    }
  }
}

template <int P, bool X4>
__global__ void __launch_bounds__(G32<P>::THREADS, 1) gram32_kernel(const __grid_constant__ Gram32Launch L) {
  using C = G32<P>;
  constexpr int RS = C::RS, LDC = C::LDC, SF = C::SF, NJ = C::NJ, E = C::E, TILES = C::TILES;
  extern __shared__ __align__(128) float ring[];
  __shared__ __align__(8) uint64_t bars[2 * C::STAGES];
  __shared__ int s_rows[C::STAGES];
  __shared__ int s_stage0[kGram32MaxTables + 1];  // first global stage of every table, then the total
  __shared__ volatile unsigned int s_dead;
  __shared__ float2 s_npiv[P];  // (-c_j, -c_j) of the consumers' current table
  uint64_t* full = bars;
  uint64_t* empty = bars + C::STAGES;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x, b = blockIdx.x;
  for (int i = threadIdx.x; i < L.ntables; i += C::THREADS) s_stage0[i] = L.tabs[i].stage0;
  if (threadIdx.x == 0) {
    s_stage0[L.ntables] = L.total_stages;
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], C::GC);
    }
    s_dead = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == C::GC) {
    // ------------------------------------------------------------------ producer
    // the stages of all tables in order, dealt in chunks of L.chunk stages round-robin
    // to the CTAs: neighbouring CTAs read neighbouring row ranges of a large table,
    // and a small table stays in one CTA
    int s = 0;
    uint32_t ph = 0;
    int64_t issued = 0;
    bool dead = false;
    int ti = -1;
    const Gram32Table* T = nullptr;
    const float* c0 = nullptr;
    const float* c1 = nullptr;
    int slot_cols[C::STAGES];  // columns of a ring slot that may hold non-zero data
#pragma unroll
    for (int k = 0; k < C::STAGES; ++k) slot_cols[k] = P;
    // this CTA's stages: chunks b, b + G, ... of L.chunk consecutive stages
    for (int64_t ch = b, gs = static_cast<int64_t>(b) * L.chunk; gs < L.total_stages && !dead;
         (++gs == (ch + 1) * L.chunk) ? (ch += G, gs = ch * L.chunk) : 0) {
      if (ti < 0 || gs >= s_stage0[ti + 1]) {
        do {
          ++ti;
        } while (gs >= s_stage0[ti + 1]);
        T = &L.tabs[ti];
        c0 = lane < T->p ? T->cols[lane] : nullptr;
        c1 = lane + 32 < T->p ? T->cols[lane + 32] : nullptr;
      }
      const int p = T->p;
      const int64_t row0 = static_cast<int64_t>(gs - s_stage0[ti]) * RS;
      const int rows = static_cast<int>(min(static_cast<int64_t>(RS), T->nrows - row0));
      if (issued >= C::STAGES && !wait_live(&empty[s], ph ^ 1u, &s_dead)) {
        dead = true;
        break;
      }
      float* st = ring + s * SF;
      if (C::TMAP && T->tmap && rows == RS) {  // one tensor copy: all P columns, zeros past p
        if (lane == 0) {
          s_rows[s] = rows;
          mbar_arrive_expect_tx(&full[s], static_cast<uint32_t>(RS * P * 4));
          tma_load_2d(st, T->tmap, static_cast<int>(row0), 0, &full[s]);
        }
#pragma unroll
        for (int k = 0; k < C::STAGES; ++k)
          if (k == s) slot_cols[k] = p;
        __syncwarp();
        ++issued;
        if (++s == C::STAGES) {
          s = 0;
          ph ^= 1u;
        }
        continue;
      }
      bool generic = false;
      int sc = 0;
#pragma unroll
      for (int k = 0; k < C::STAGES; ++k)
        if (k == s) sc = slot_cols[k];
      if (sc > p) {  // columns p.. of this slot must read as zero
        for (int i = p * LDC + 4 * lane; i < sc * LDC; i += 128)
          *reinterpret_cast<float4*>(st + i) = make_float4(0.f, 0.f, 0.f, 0.f);
        generic = true;
      }
#pragma unroll
      for (int k = 0; k < C::STAGES; ++k)
        if (k == s) slot_cols[k] = p;
      const int bulk = T->aligned ? (rows & ~3) : 0;
      const int nr = rows - bulk;
      if (nr > 0) {  // rows not moved by bulk copies: plain loads by the producer lanes
        for (int idx = lane; idx < p * nr; idx += 32) {
          const int c = idx / nr, r = bulk + idx % nr;
          st[c * LDC + r] = __ldg(T->cols[c] + row0 + r);
        }
        generic = true;
      }
      const int pad = ((rows + 15) & ~15) - rows;
      if (pad > 0) {  // rows past the table's end up to the K block boundary hold the pivot: r = 0
        for (int idx = lane; idx < p * pad; idx += 32) {
          const int c = idx / pad, r = rows + idx % pad;
          st[c * LDC + r] = __ldg(T->shift + c);
        }
        generic = true;
      }
      if (generic) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        s_rows[s] = rows;
        mbar_arrive_expect_tx(&full[s], static_cast<uint32_t>(bulk) * 4u * static_cast<uint32_t>(p));
      }
      __syncwarp();
      if (bulk > 0) {
        if (c0) bulk_g2s(st + lane * LDC, c0 + row0, static_cast<uint32_t>(bulk) * 4u, &full[s]);
        if (c1) bulk_g2s(st + (lane + 32) * LDC, c1 + row0, static_cast<uint32_t>(bulk) * 4u, &full[s]);
      }
      ++issued;
      if (++s == C::STAGES) {
        s = 0;
        ph ^= 1u;
      }
    }
    if (dead) {
      s_dead = 1;
      if (lane == 0 && T) atomicOr(T->status, DEV_ETIMEOUT);
    }
    // no copy may be in flight when the CTA exits: wait for the last issued stages to land
    for (int k = 0; k < C::STAGES && k < issued; ++k) {
      int sk = s - 1 - k;
      uint32_t pk = ph;
      while (sk < 0) {
        sk += C::STAGES;
        pk ^= 1u;
      }
      mbar_wait_bounded(&full[sk], pk);
    }
    return;
  }

  // -------------------------------------------------------------------- consumers
  const int g = lane >> 2, t = lane & 3;
  float zq[4];  // a quad of zeros in registers: the C operand that starts each chain
#pragma unroll
  for (int i = 0; i < 4; ++i) asm volatile("mov.b32 %0, 0;" : "=f"(zq[i]));
  float2* scratch = reinterpret_cast<float2*>(L.warp_scratch) +
                    (static_cast<size_t>(b) * C::GC + warp) * (E * 32);
  int s = 0;
  uint32_t ph = 0;
  bool dead = false;
  int ti = -1;
  int64_t ch = b, gs = static_cast<int64_t>(b) * L.chunk;
  while (gs < L.total_stages) {
    // a run of this CTA's stages in one table
    do {
      ++ti;
    } while (gs >= s_stage0[ti + 1]);
    const Gram32Table& T = L.tabs[ti];
    const int p = T.p;
    for (int c = threadIdx.x; c < P; c += 32 * C::GC) {
      const float v = c < p ? -__ldg(T.shift + c) : 0.f;
      s_npiv[c] = make_float2(v, v);
    }
    consumers_sync<C::GC>();
    float acc[TILES][4];
    float2 sum[C::NM], lsq[C::NM];
#pragma unroll
    for (int i = 0; i < TILES; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
#pragma unroll
    for (int m = 0; m < C::NM; ++m) sum[m] = lsq[m] = make_float2(0.f, 0.f);
    bool fresh = true;
    int since = 0;

    // FP32 accumulators -> this warp's (hi, lo) pairs, eight words at a time (their loads in
    // flight together; the empty asm stops the compiler from hoisting every load ahead)
    auto flush = [&]() {
      constexpr int B = 8;
#pragma unroll
      for (int e0 = 0; e0 < E; e0 += B) {
        float2 hl[B];
#pragma unroll
        for (int k = 0; k < B; ++k)
          if (e0 + k < E) hl[k] = fresh ? make_float2(0.f, 0.f) : __ldcg(scratch + (e0 + k) * 32 + lane);
#pragma unroll
        for (int k = 0; k < B; ++k) {
          const int e = e0 + k;
          if (e >= E) continue;
          float w;
          if (e < 4 * TILES) {
            w = acc[e / 4][e % 4];
            acc[e / 4][e % 4] = 0.f;
          } else if (e < 4 * TILES + C::NM) {
            w = sum[e - 4 * TILES].x + sum[e - 4 * TILES].y;
            sum[e - 4 * TILES] = make_float2(0.f, 0.f);
          } else {
            w = lsq[e - 4 * TILES - C::NM].x + lsq[e - 4 * TILES - C::NM].y;
            lsq[e - 4 * TILES - C::NM] = make_float2(0.f, 0.f);
          }
          two_sum(hl[k].x, hl[k].y, w);
          __stcg(scratch + e * 32 + lane, hl[k]);
        }
        asm volatile("" ::: "memory");
      }
      fresh = false;
    };

    int rot = 0;  // K blocks of this run before the current stage, mod C::GC
    const int end = s_stage0[ti + 1];
    for (; gs < end && gs < L.total_stages; (++gs == (ch + 1) * L.chunk) ? (ch += G, gs = ch * L.chunk) : 0) {
      if (!dead && !wait_live(&full[s], ph, &s_dead)) {
        dead = true;
        s_dead = 1;
        if (lane == 0) atomicOr(T.status, DEV_ETIMEOUT);
      }
      if (!dead) {
        const int rows = s_rows[s];
        const float* st = ring + s * SF;
        // K blocks kb0, kb0 + C::GC, ...: the run's K block (stage * KBS + kb) = warp mod C::GC
        const int kb0 = (warp - rot + C::GC) % C::GC;
        const int nkb = (rows + 15) >> 4;  // a ragged last K block is padded with the pivot
        int done = 0, kb = kb0;
        constexpr int U = C::UNROLL;
#pragma unroll 1
        for (; kb + (U - 1) * C::GC < nkb; kb += U * C::GC, done += U) {
          Frag<P> F[U];
#pragma unroll
          for (int u = 0; u < U; ++u) convert_kblock<P, X4>(st, kb + u * C::GC, g, t, s_npiv, sum, lsq, F[u]);
#pragma unroll
          for (int u = 0; u < U; ++u) mma_kblock<P, X4>(F[u], zq, acc);
        }
#pragma unroll 1
        for (; kb < nkb; kb += C::GC, ++done) {
          Frag<P> F;
          convert_kblock<P, X4>(st, kb, g, t, s_npiv, sum, lsq, F);
          mma_kblock<P, X4>(F, zq, acc);
        }
        since += done;
        if (since >= L.flush_kblocks) {
          since = 0;
          flush();
        }
        rot = (rot + C::KBS) % C::GC;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
      if (++s == C::STAGES) {
        s = 0;
        ph ^= 1u;
      }
    }
    // this CTA's slot of the table: the consumer warps' partials (FP32 accumulators plus,
    // after mid-run flushes, the pairs in scratch) added in warp order through a shared
    // buffer, one warp at a time (eight words per step, their loads issued together)
    float2* __restrict__ red = reinterpret_cast<float2*>(ring + C::STAGES * SF) + lane;
    for (int w = 0; w < C::GC; ++w) {
      if (warp == w) {
        constexpr int B = 8;
#pragma unroll
        for (int e0 = 0; e0 < E; e0 += B) {
          float2 pr[B];
#pragma unroll
          for (int k = 0; k < B; ++k)
            if (e0 + k < E) pr[k] = w == 0 ? make_float2(0.f, 0.f) : red[(e0 + k) * 32];
          if (!fresh) {
#pragma unroll
            for (int k = 0; k < B; ++k)
              if (e0 + k < E) {
                const float2 q = __ldcg(scratch + (e0 + k) * 32 + lane);
                two_sum(pr[k].x, pr[k].y, q.x);
                two_sum(pr[k].x, pr[k].y, q.y);
              }
          }
#pragma unroll
          for (int k = 0; k < B; ++k) {
            const int e = e0 + k;
            if (e >= E) continue;
            float val;
            if (e < 4 * TILES)
              val = acc[e / 4][e % 4];
            else if (e < 4 * TILES + C::NM)
              val = sum[e - 4 * TILES].x + sum[e - 4 * TILES].y;
            else
              val = lsq[e - 4 * TILES - C::NM].x + lsq[e - 4 * TILES - C::NM].y;
            two_sum(pr[k].x, pr[k].y, val);
            red[e * 32] = pr[k];
          }
        }
      }
      consumers_sync<C::GC>();
    }
    const int sid = static_cast<int>(((b - s_stage0[ti] / L.chunk) % G + G) % G);
    float2* cslot = reinterpret_cast<float2*>(T.slots) + static_cast<size_t>(sid) * (E * 32);
    const float2* redb = reinterpret_cast<const float2*>(ring + C::STAGES * SF);
    for (int i = threadIdx.x; i < E * 32; i += 32 * C::GC) __stcg(cslot + i, redb[i]);
    consumers_sync<C::GC>();  // the buffer is free for the next run
  }
}

// The tables' slots, in slot order, into their double-double accumulators: block
// (t, part) takes every `parts`-th packed-upper entry and column sum of table t.
template <int P, bool X4>
__global__ void __launch_bounds__(256) gram32_merge_kernel(const Gram32Table* __restrict__ tabs, int parts) {
  using C = G32<P>;
  constexpr int E = C::E, TILES = C::TILES, NJ = C::NJ;
  const Gram32Table& T = tabs[blockIdx.x / parts];
  const int part = blockIdx.x % parts;
  const int p = T.p;
  const int Tn = p * (p + 1) / 2;
  const float2* slots = reinterpret_cast<const float2*>(T.slots);
  for (int e = part * 256 + threadIdx.x; e < Tn + p; e += parts * 256) {
    float h = 0.f, l = 0.f;
    if (e < Tn) {
      int j = 0, rm = e;
      while (rm >= p - j) {
        rm -= p - j;
        ++j;
      }
      const int k2 = j + rm;
      const int I = P >= 16 ? j / 16 : 0, J = k2 / 8;
      int tix = 0;
      for (int i = 0; i < I; ++i) tix += NJ - 2 * i;
      tix += J - 2 * I;
      const int lr = j - 16 * I, lc = k2 - 8 * J;
      const int ln = (lr & 7) * 4 + (lc >> 1);
      const int w = 4 * tix + 2 * (lr >> 3) + (lc & 1);
      add_slots(slots, T.nslots, E * 32, w * 32 + ln, h, l);
      if (!X4 && j == k2) {  // BF16x3: + the diagonal of L^T L
        const int wq = 4 * TILES + C::NM + (j >> 3), gq = j & 7;
        for (int tt = 0; tt < 4; ++tt) add_slots(slots, T.nslots, E * 32, wq * 32 + gq * 4 + tt, h, l);
      }
    } else {
      const int c = e - Tn, m = c >> 3, gg = c & 7;
      const int w = 4 * TILES + m;
      for (int tt = 0; tt < 4; ++tt) add_slots(slots, T.nslots, E * 32, w * 32 + gg * 4 + tt, h, l);
    }
    double* dh = e < Tn ? &T.acc_S[e] : &T.acc_s[e - Tn];
    double* dl = e < Tn ? &T.acc_S_lo[e] : &T.acc_s_lo[e - Tn];
    const double vv = static_cast<double>(h) + static_cast<double>(l);
    const double sd = *dh + vv;
    const double bp = sd - *dh;
    *dl += (*dh - (sd - bp)) + (vv - bp);
    *dh = sd;
  }
  if (part == 0 && threadIdx.x == 0) *T.acc_n += T.nrows;
}

template <int P, bool X4>
cudaError_t launch_p(const Gram32Launch& L, int grid, cudaStream_t st) {
  const int smem = G32<P>::STAGES * G32<P>::SF * 4 + G32<P>::E * 32 * 8;  // ring + reduction buffer
  cudaError_t e = cudaFuncSetAttribute(gram32_kernel<P, X4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  gram32_kernel<P, X4><<<grid, G32<P>::THREADS, smem, st>>>(L);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // merge: entries of a table spread over `parts` blocks, at least ~2 blocks per SM in all
  const int entries = P * (P + 1) / 2 + P;
  const int parts = std::max(1, std::min((entries + 255) / 256, (2 * grid + L.ntables - 1) / L.ntables));
  gram32_merge_kernel<P, X4><<<L.ntables * parts, 256, 0, st>>>(L.tabs, parts);
  return cudaGetLastError();
}

// pivot c_j = the mean of the table's first kPivotRows rows (or all, if fewer), rounded to FP32
__global__ void gram32_shift_kernel(const Gram32Table* __restrict__ tabs, const int* __restrict__ which) {
  const Gram32Table& T = tabs[which[blockIdx.x]];
  const int k = static_cast<int>(min(static_cast<int64_t>(kPivotRows), T.nrows));
  for (int j = threadIdx.x; j < T.p; j += blockDim.x) {
    double sum = 0.0;
    for (int i = 0; i < k; ++i) sum += static_cast<double>(T.cols[j][i]);
    const float v = static_cast<float>(sum / k);
    const_cast<float*>(T.shift)[j] = v;
    T.shift_d[j] = static_cast<double>(v);
  }
}

}  // namespace

cudaError_t launch_gram32_shift(const Gram32Table* tabs, const int* which, int count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  gram32_shift_kernel<<<count, 64, 0, st>>>(tabs, which);
  return cudaGetLastError();
}

int gram32_width(int p) { return p <= 8 ? 8 : p <= 16 ? 16 : p <= 32 ? 32 : 64; }

size_t gram32_slot_floats(int P) {
  int E = 0;
  switch (P) {
    case 8: E = G32<8>::E; break;
    case 16: E = G32<16>::E; break;
    case 32: E = G32<32>::E; break;
    default: E = G32<64>::E; break;
  }
  return static_cast<size_t>(E) * 32 * 2;
}

int gram32_rows_per_stage(int P) {
  switch (P) {
    case 8: return G32<8>::RS;
    case 16: return G32<16>::RS;
    case 32: return G32<32>::RS;
    default: return G32<64>::RS;
  }
}

cudaError_t launch_gram32(const Gram32Launch& L, int P, bool x4, int grid, cudaStream_t st) {
  if (L.total_stages <= 0) return cudaSuccess;
  switch (P) {
    case 8: return x4 ? launch_p<8, true>(L, grid, st) : launch_p<8, false>(L, grid, st);
    case 16: return x4 ? launch_p<16, true>(L, grid, st) : launch_p<16, false>(L, grid, st);
    case 32: return x4 ? launch_p<32, true>(L, grid, st) : launch_p<32, false>(L, grid, st);
    default: return x4 ? launch_p<64, true>(L, grid, st) : launch_p<64, false>(L, grid, st);
  }
}

}  // namespace ss
