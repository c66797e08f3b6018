// api.cu -- the C ABI of libsuffstats (declared in include/stats.h): context
// management, the digit plan of the exact pass, launches, host-streamed double
// buffering, merge, checkpoint.  Every step of the pass itself runs in the
// kernels of k_exact.cu / k_fp64.cu / k_finalize.cu; this file only validates
// arguments, owns device memory and orders work on streams.
#include <math.h>
#include <string.h>

#include <fcntl.h>
#include <sys/stat.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <unistd.h>

#include "../../include/stats.h"
#include "../../include/stats_csv.h"
#include "../../include/stats_file.h"
#include <cuda.h>

#include "file_format.h"
#include "kernels.h"

using namespace ss;

namespace {

constexpr uint64_t kMagic = 0x3130535441545353ull;  // "SSTATS01"
constexpr int64_t kDefaultChunkRows = int64_t(1) << 24;
// A call on a 33..64-column table of at least this many rows takes the tcgen05 pass; below it
// the pass's fixed costs (tensor-memory set-up, pipeline fill, per-CTA slots and their merge:
// tens of microseconds) outweigh its faster streaming.  Batches keep the register-fragment
// launch, which shares those costs across its tables.
constexpr int64_t kNarrowMinRows = int64_t(1) << 20;
// Tables of a batched call with 33..64 columns and at least this many rows share one
// persistent narrow launch; smaller ones stay with the register-fragment launch.
constexpr int64_t kNarrowBatchMinRows = 4096;

struct ColPlan {
  int k = 0;         // digit bytes
  int is_signed = 0;
  int is_real = 0;
  int shift = 0;     // real: q = RN(x * 2^shift)
  int emax = 0;      // real: largest allowed biased exponent field
  int off = 0;       // first digit slot
};

}  // namespace

struct stats_ctx {
  int device = 0;
  int p = 0;
  int pa = 0;
  int mode = 0;
  std::vector<int32_t> dtypes;
  std::vector<uint8_t> ident;
  std::vector<double> lo, hi;
  bool has_bounds = false;
  // exact plan
  std::vector<ColPlan> plan;
  int conv = CONV_GENERIC;
  ExactParams xp{};  // launch template (pointers of the call filled per launch)
  int stages = 3;
  // device state
  long long* d_g = nullptr;             // EXACT accumulator, kDigits^2
  unsigned long long* d_call = nullptr; // scratch: per-call accumulator
  unsigned int* d_ticket = nullptr;     // scratch
  unsigned int* d_err = nullptr;        // scratch
  unsigned int* d_status = nullptr;     // sticky device status bits
  double* d_fs = nullptr;               // FP64: s, s_lo, S, S_lo, shift (one allocation)
  double* d_fs_lo = nullptr;
  double* d_fS = nullptr;
  double* d_fS_lo = nullptr;
  double* d_shift = nullptr;
  long long* d_fn = nullptr;
  double* d_slots = nullptr;            // FP64 scratch: block slots + ticket
  int slot_grid = 0;
  double* d_core_slots = nullptr;       // CUDA-core comparators (wide FP64, FP32) scratch
  unsigned int* d_core_ticket = nullptr;
  int core_grid = 0;
  float* d_fshift = nullptr;            // BF16X3/X4: pivot as float
  float* d_wide_slots = nullptr;        // BF16X3/X4, p > 64 on tcgen05: per-CTA slots
  int wide_grid_alloc = 0;
  float* d_split_slots = nullptr;       // BF16X3/X4 scratch: warp slots
  unsigned int* d_split_ticket = nullptr;
  int split_grid = 0;
  int flush_rows = 0;                   // 0: by table width
  int exact_shape = -1;                 // EXACT launch shape (-1: the converter's default)
  int wide_pairs = 1;                   // 129..256 FP32 columns: the paired-CTA tcgen05 pass
  int64_t grid_wait_ns = 0;             // eigen-solver grid waits: limit (0: 2 s)
  int32_t grid_absent_block = -1;       // testing: a block of the eigen-solver that never arrives
  // the last 2D tensor map made for this ctx's FP32 columns (reused while the layout is the same)
  const void* tmap_base = nullptr;
  int64_t tmap_stride = 0, tmap_rows = 0;
  int tmap_box = 0;
  int tmap_cols = 0;  // columns per box of the cached map
  bool tmap_ok = false;
  alignas(64) CUtensorMap tmap{};
  void* d_tmap = nullptr;               // device copy of tmap for the wide kernel
  bool shift_set = false;
  double* d_out = nullptr;              // finalize result
  double* d_work = nullptr;             // finalize scratch
  double* d_jac = nullptr;              // grid-wide eigen-solver scratch (allocated on first use)
  int coop = 0;                         // the device takes cooperative launches
  double* h_out = nullptr;              // pinned host copy of the result
  FinalLayout lay{};
  // host streaming
  void* d_stage[2] = {nullptr, nullptr};
  int64_t stage_rows = 0;
  std::vector<size_t> stage_off;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr};
  cudaEvent_t ev_done[2] = {nullptr, nullptr};
  // file streaming: pinned host chunks (free again once ev_copied[b] has completed)
  void* h_stage[2] = {nullptr, nullptr};
  size_t h_stage_bytes = 0;
  cudaStream_t last = nullptr;
  int grid = 0;
  int sms = 0;
  // rows enqueued into the accumulator so far (host-side count; reset, merge and import keep it)
  int64_t rows_enqueued = 0;
  stats_status sticky = STATS_OK;
};

namespace {

stats_status cuda_fail(stats_ctx* c, cudaError_t e) {
  if (e == cudaSuccess) return STATS_OK;
  if (c) c->sticky = STATS_ECUDA;
  return STATS_ECUDA;
}

#define CK(c, expr)                                  \
  do {                                               \
    cudaError_t _e = (expr);                         \
    if (_e != cudaSuccess) return cuda_fail(c, _e);  \
  } while (0)

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int bitlen_u(unsigned long long v) { return v ? 64 - __builtin_clzll(v) : 0; }

// Digit field of an integer column with lo <= x <= hi (or the dtype's full range).
bool int_field(int32_t dt, bool bounded, double lo, double hi, ColPlan& cp) {
  if (!bounded) {
    cp.k = dtype_bytes(dt);
    cp.is_signed = 1;
    return true;
  }
  if (!(lo <= hi) || !isfinite(lo) || !isfinite(hi)) return false;
  const double ilo = ceil(lo), ihi = floor(hi);
  if (ilo >= 0) {
    if (ihi >= 18446744073709551616.0) return false;
    const int bits = bitlen_u(static_cast<unsigned long long>(std::max(ihi, 0.0)));
    cp.k = std::max(1, (bits + 7) / 8);
    cp.is_signed = 0;
  } else {
    const double m = std::max(-ilo - 1.0, ihi);
    if (m >= 9223372036854775808.0) return false;
    const int bits = bitlen_u(static_cast<unsigned long long>(std::max(m, 0.0))) + 1;
    cp.k = std::max(1, (bits + 7) / 8);
    cp.is_signed = 1;
  }
  cp.k = std::min(cp.k, dtype_bytes(dt));
  // An 8-byte field leaves no bits above it to range-check, so it is the dtype's own two's
  // complement.  A narrower full-width field with a non-negative range stays unsigned: the
  // sign-extended value of a negative entry then spills past the field and is rejected.
  if (cp.k == 8) cp.is_signed = 1;
  return true;
}

// Fixed-point field of a real column with |x| <= max(|lo|, |hi|) < 2^e.
bool real_field(bool bounded, double lo, double hi, ColPlan& cp) {
  if (!bounded || !isfinite(lo) || !isfinite(hi) || !(lo <= hi)) return false;
  const double m = std::max(fabs(lo), fabs(hi));
  if (!(m > 0)) return false;
  int e = 0;
  frexp(m, &e);  // m = f * 2^e, f in [0.5, 1): m < 2^e
  cp.is_real = 1;
  cp.k = 7;
  cp.is_signed = lo < 0 ? 1 : 0;
  const int P = cp.is_signed ? 8 * cp.k - 2 : 8 * cp.k - 1;
  cp.shift = P - e;
  cp.emax = 1022 + e;
  return true;
}

// The launch shape of the exact pass used unless a ctx asks for another (stats_set_exact_shape):
// per converter, the fastest measured on a GB300.
int exact_default_shape(int conv) {
  (void)conv;
  return 0;
}

// Whether a column plan is one of the Table 1 layouts that the specialised converters read
// (the dtypes of the layout, and digit fields no wider than the converter handles).
bool is_t1_plan(int p, const int32_t* dtypes, const ColPlan* cp, int layout) {
  if (p != 12) return false;
  static const int32_t l32[12] = {I64, I32, I32, I32, I32, I32, I32, I32, F64, I32, F64, I32};
  static const int32_t l16[12] = {I64, I16, I16, I16, I16, I32, I16, I16, F64, I16, F64, I16};
  const int32_t* want = layout ? l16 : l32;
  for (int j = 0; j < 12; ++j)
    if (dtypes[j] != want[j]) return false;
  for (int j : {1, 2, 3, 4, 6, 7, 11})
    if (cp[j].is_signed || cp[j].k != 1) return false;
  for (int j : {5, 9})
    if (cp[j].is_signed || cp[j].k > 2) return false;
  if (cp[0].is_signed || cp[0].k > 5) return false;
  if (!cp[8].is_real || !cp[8].is_signed) return false;
  if (!cp[10].is_real || cp[10].is_signed) return false;
  return true;
}

// The digit plan of STATS_EXACT for a configuration, in fixed-size arrays (no heap use), for
// stats_init and the no-allocation entry point alike: each column's digit field (bytes, sign,
// real scaling) and first digit slot; the converter (a Table 1 layout, whose slots are fixed,
// or the generic one with its table of digit pairs); and the pipeline's stage layout.
stats_status exact_plan(int p, const int32_t* dtypes, bool bounded, const double* lo, const double* hi,
                        ColPlan (&cp)[kMaxCols], ExactParams& xp, int& conv) {
  if (p < 1 || p > kMaxCols || !dtypes || (bounded && (!lo || !hi))) return STATS_EINVAL;
  for (int j = 0; j < p; ++j) {
    const int32_t dt = dtypes[j];
    if (dt < I16 || dt > F64) return STATS_EINVAL;
    cp[j] = ColPlan{};
    const double l = bounded ? lo[j] : 0.0, h = bounded ? hi[j] : 0.0;
    const bool ok = (dt == F32 || dt == F64) ? real_field(bounded, l, h, cp[j]) : int_field(dt, bounded, l, h, cp[j]);
    if (!ok) return STATS_EINVAL;
  }
  conv = CONV_GENERIC;
  for (int layout = 0; layout < 2; ++layout)
    if (is_t1_plan(p, dtypes, cp, layout)) {
      conv = layout ? CONV_T1_L16 : CONV_T1_L32;
      // slots: 0 ones | 1 B | 2 C | 3 D | 4 E | 5 G | 6 H | 7 K | 8-9 F | 10-11 I | 12-16 A | 17-23 cotC | 24-30 J
      static const int off[12] = {12, 1, 2, 3, 4, 8, 5, 6, 17, 10, 24, 7};
      static const int k[12] = {5, 1, 1, 1, 1, 2, 1, 1, 7, 2, 7, 1};
      for (int j = 0; j < 12; ++j) {
        cp[j].off = off[j];
        cp[j].k = k[j];
      }
      break;
    }
  if (conv == CONV_GENERIC) {
    int slot = 1;
    for (int j = 0; j < p; ++j) {
      cp[j].off = slot;
      slot += cp[j].k;
    }
    if (slot > kDigits) return STATS_EINVAL;
    // per digit slot: source column (-1 the ones column, -2 padding), byte, signed top byte
    int8_t col[kDigits], byt[kDigits], sg[kDigits];
    for (int q = 0; q < kDigits; ++q) {
      col[q] = -2;
      byt[q] = 0;
      sg[q] = 0;
    }
    col[0] = -1;
    for (int j = 0; j < p; ++j)
      for (int a = 0; a < cp[j].k; ++a) {
        col[cp[j].off + a] = static_cast<int8_t>(j);
        byt[cp[j].off + a] = static_cast<int8_t>(a);
        sg[cp[j].off + a] = (cp[j].is_signed && a == cp[j].k - 1) ? 1 : 0;
      }
    for (int q = 0; q < kDigitPairs; ++q) {
      xp.pc0[q] = col[2 * q];
      xp.pb0[q] = byt[2 * q];
      xp.ps0[q] = sg[2 * q];
      xp.pc1[q] = col[2 * q + 1];
      xp.pb1[q] = byt[2 * q + 1];
      xp.ps1[q] = sg[2 * q + 1];
    }
  }
  for (int j = 0; j < p; ++j) {
    xp.dtype[j] = dtypes[j];
    xp.col_bytes[j] = dtype_bytes(dtypes[j]);
    xp.real_shift[j] = cp[j].shift;
    xp.real_emax[j] = cp[j].emax;
    xp.kbytes[j] = cp[j].k;
    xp.is_signed[j] = cp[j].is_signed;
  }
  xp.p = p;
  if (!exact_layout(xp, exact_default_shape(conv))) return STATS_EINVAL;  // rows too wide for the pipeline
  return STATS_OK;
}

stats_status build_plan(stats_ctx* c) {
  ColPlan cp[kMaxCols];
  const stats_status s = exact_plan(c->p, c->dtypes.data(), c->has_bounds, c->lo.data(), c->hi.data(), cp, c->xp,
                                    c->conv);
  if (s != STATS_OK) return s;
  c->plan.assign(cp, cp + c->p);
  c->stages = c->xp.stages;
  return STATS_OK;
}

stats_status check_sticky(const stats_ctx* c) {
  if (!c) return STATS_EINVAL;
  return c->sticky != STATS_OK ? STATS_ESTATE : STATS_OK;
}

stats_status device_status(stats_ctx* c) {
  unsigned int bits = 0;
  CK(c, cudaMemcpy(&bits, c->d_status, sizeof(bits), cudaMemcpyDeviceToHost));
  if (bits & DEV_ETIMEOUT) return STATS_ETIMEOUT;
  if (bits & DEV_ERANGE) return STATS_ERANGE;
  if (bits & DEV_EOVERFLOW) return STATS_EOVERFLOW;
  return STATS_OK;
}

int default_grid(stats_ctx* c) {
  if (c->grid > 0) return c->grid;
  if (c->mode == STATS_EXACT) {
    int per = exact_max_active_blocks(c->conv, c->xp.shape, c->xp.stages, c->xp.stage_bytes);
    if (per < 1) per = 1;
    return c->sms * per;
  }
  return c->sms * 2;
}

stats_status ensure_slots(stats_ctx* c, int grid) {
  if (c->d_slots && c->slot_grid >= grid) return STATS_OK;
  if (c->d_slots) CK(c, cudaFree(c->d_slots));
  c->d_slots = nullptr;
  const size_t n = fp64_slot_doubles(grid);
  CK(c, cudaMalloc(&c->d_slots, n * sizeof(double)));
  CK(c, cudaMemset(c->d_slots, 0, n * sizeof(double)));
  c->slot_grid = grid;
  return STATS_OK;
}

// BF16x3 drops the off-diagonal products of the low halves, sum_i l_ij l_ik.  Their sum
// over n rows is a sum of products of rounding residuals (|l| <= 2^-9 |x - c|) with random
// signs: it grows as sqrt(n) while the covariance grows as n, so the relative Frobenius
// error it leaves is about 2.6e-6 * sqrt(p / n) for independent columns.  Until a context
// holds 64 p rows (error ~3e-7 there) its calls form all four products, as BF16x4 does;
// from then on the rows taken with three products are at least as many as would bring
// their own share of the error below that level.
constexpr int64_t kBf16x3RowsPerColumn = 64;

bool split_x4(const stats_ctx* c, int64_t nrows) {
  if (c->mode == STATS_BF16X4) return true;
  return c->mode == STATS_BF16X3 && c->rows_enqueued + nrows < kBf16x3RowsPerColumn * c->p;
}

// ---------------------------------------------------------------------------
// FP32 tables of up to 64 columns in BF16x3 / BF16x4 mode: register-fragment
// tensor-core pass over a list of (table, row range) units.  The launch's
// scratch (descriptors, unit list, tickets, unit and warp slots) lives in one
// per-device workspace; launches that share it are ordered through an event.
// ---------------------------------------------------------------------------
struct Gram32Job {
  stats_ctx* c;
  const void* const* cols;
  int64_t nrows;
  bool x4;  // all four products (BF16x4, or a BF16x3 context still below its row threshold)
};

// Tuning of the batched launches, per width class (P = 8, 16, 32, 64) and arithmetic (BF16x3,
// BF16x4): how a launch's stages are dealt to its persistent CTAs.  Set by stats_set_batch_tuning
// (the autotuner); the defaults were measured on the many-tables workload.
stats_batch_tuning g_batch_tuning[4][2];
std::once_flag g_batch_tuning_once;
std::mutex g_batch_tuning_mu;

int width_class(int P) { return P <= 8 ? 0 : P <= 16 ? 1 : P <= 32 ? 2 : 3; }

stats_batch_tuning batch_tuning(int P, bool x4) {
  std::call_once(g_batch_tuning_once, [] {
    for (auto& row : g_batch_tuning)
      for (auto& t : row) t = stats_batch_tuning{12, 32, 32};
  });
  std::lock_guard<std::mutex> lk(g_batch_tuning_mu);
  return g_batch_tuning[width_class(P)][x4 ? 1 : 0];
}

bool valid_tuning(const stats_batch_tuning& t) {
  return t.narrow_units_per_cta >= 1 && t.narrow_units_per_cta <= 256 && t.gram32_chunks_per_cta >= 1 &&
         t.gram32_chunks_per_cta <= 1024 && t.gram32_min_chunk >= 1 && t.gram32_min_chunk <= 65536;
}

struct Gram32Workspace {
  void* dev = nullptr;
  size_t bytes = 0;
  cudaEvent_t last = nullptr;
};
std::mutex g_g32_mu;
Gram32Workspace g_g32_ws[64];


size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  });
  return fn;
}

// A 2D tensor map over p FP32 columns that sit a fixed, 16-byte-multiple stride apart
// (column j at cols[0] + j * stride), box = rows x P columns; false when the columns
// are not laid out that way or the map cannot be made.
bool table_tensor_map(const void* const* cols, int p, int64_t nrows, int P, int rows, CUtensorMap* out,
                      bool swizzle128 = false) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn || nrows <= 0 || nrows >= (int64_t(1) << 31) || !aligned16(cols[0])) return false;
  const char* c0 = static_cast<const char*>(cols[0]);
  int64_t stride = p > 1 ? static_cast<const char*>(cols[1]) - c0 : (nrows * 4 + 15) / 16 * 16;
  if (stride <= 0 || stride % 16 != 0 || stride >= (int64_t(1) << 40)) return false;
  for (int j = 2; j < p; ++j)
    if (static_cast<const char*>(cols[j]) - c0 != j * stride) return false;
  const cuuint64_t dim[2] = {static_cast<cuuint64_t>(nrows), static_cast<cuuint64_t>(p)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(stride)};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(rows), static_cast<cuuint32_t>(P)};
  const cuuint32_t estr[2] = {1, 1};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<char*>(c0), dim, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// A 3D tensor map over p FP32 columns a fixed, 16-byte-multiple stride apart, each column's
// rows seen as (32 rows, nrows / 32 chunks): box (32, chunks, cols) with the 128-byte swizzle.
// Only whole 32-row chunks are mapped (the rest of a column may end the allocation).
bool table_tensor_map_chunks(const void* const* cols, int p, int64_t nrows, int cols_box, int chunks_box,
                             CUtensorMap* out) {
  EncodeTiledFn fn = encode_tiled();
  const int64_t nchunks = nrows / 32;
  if (!fn || nchunks < 1 || nchunks >= (int64_t(1) << 31) || !aligned16(cols[0])) return false;
  const char* c0 = static_cast<const char*>(cols[0]);
  int64_t stride = p > 1 ? static_cast<const char*>(cols[1]) - c0 : (nrows * 4 + 15) / 16 * 16;
  if (stride <= 0 || stride % 16 != 0 || stride >= (int64_t(1) << 40)) return false;
  for (int j = 2; j < p; ++j)
    if (static_cast<const char*>(cols[j]) - c0 != j * stride) return false;
  const cuuint64_t dim[3] = {32u, static_cast<cuuint64_t>(nchunks), static_cast<cuuint64_t>(p)};
  const cuuint64_t strides[2] = {128u, static_cast<cuuint64_t>(stride)};
  const cuuint32_t box[3] = {32u, static_cast<cuuint32_t>(chunks_box), static_cast<cuuint32_t>(cols_box)};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<char*>(c0), dim, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

stats_status run_gram32(const std::vector<Gram32Job>& jobs, cudaStream_t st) {
  if (jobs.empty()) return STATS_OK;
  stats_ctx* c0 = jobs[0].c;
  int dev = 0;
  CK(c0, cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return STATS_EINVAL;
  std::lock_guard<std::mutex> lk(g_g32_mu);
  Gram32Workspace& ws = g_g32_ws[dev];
  if (!ws.last) CK(c0, cudaEventCreateWithFlags(&ws.last, cudaEventDisableTiming));
  CK(c0, cudaStreamWaitEvent(st, ws.last, 0));  // the previous user of the workspace is done
  const int sms = std::max(1, c0->sms);
  // one launch per (P, x4) and per kGram32MaxTables tables
  for (int P : {8, 16, 32, 64}) {
    for (int x4 = 0; x4 < 2; ++x4) {
      std::vector<const Gram32Job*> all;
      for (const Gram32Job& j : jobs)
        if (gram32_width(j.c->p) == P && j.x4 == (x4 == 1) && j.nrows > 0) all.push_back(&j);
      for (size_t first = 0; first < all.size(); first += kGram32MaxTables) {
        const size_t nt = std::min<size_t>(kGram32MaxTables, all.size() - first);
        const int64_t rs = gram32_rows_per_stage(P);
        std::vector<Gram32Table> tabs(nt);
        std::vector<CUtensorMap> maps;
        std::vector<int> map_of(nt, -1);
        std::vector<const float*> colptrs;
        std::vector<int> need_shift;
        int64_t total = 0;
        for (size_t i = 0; i < nt; ++i) total += (all[first + i]->nrows + rs - 1) / rs;
        if (total >= (int64_t(1) << 31)) return STATS_EINVAL;  // over 2^31 stages in one call
        // chunks as long as possible while every CTA still gets >= chunks_per_cta of them (long
        // runs: few per-table partials; many chunks: balanced CTAs), and never below min_chunk
        const stats_batch_tuning tune = batch_tuning(P, x4 == 1);
        const int64_t K = std::max<int64_t>(tune.gram32_min_chunk, total / (int64_t(sms) * tune.gram32_chunks_per_cta));
        const int grid = static_cast<int>(std::min<int64_t>((total + K - 1) / K, sms));
        const size_t sf = gram32_slot_floats(P);
        size_t slot_floats_total = 0;
        int flush_kb = 16384 / 16;  // K blocks of a warp between FP32 -> (hi, lo) flushes
        int64_t stage0 = 0;
        for (size_t i = 0; i < nt; ++i) {
          const Gram32Job* j = all[first + i];
          stats_ctx* c = j->c;
          Gram32Table& T = tabs[i];
          T = Gram32Table{};
          T.p = c->p;
          T.nrows = j->nrows;
          const int64_t ns = (T.nrows + rs - 1) / rs;
          T.stage0 = static_cast<int32_t>(stage0);
          const int64_t nch = (stage0 + ns - 1) / K - stage0 / K + 1;  // chunks the table overlaps
          T.nslots = static_cast<int32_t>(std::min<int64_t>(grid, nch));
          stage0 += ns;
          T.shift = c->d_fshift;
          T.shift_d = c->d_shift;
          T.acc_s = c->d_fs;
          T.acc_s_lo = c->d_fs_lo;
          T.acc_S = c->d_fS;
          T.acc_S_lo = c->d_fS_lo;
          T.acc_n = c->d_fn;
          T.status = c->d_status;
          T.aligned = 1;
          for (int jj = 0; jj < c->p; ++jj) {
            const float* ptr = static_cast<const float*>(j->cols[jj]);
            colptrs.push_back(ptr);
            if (!aligned16(ptr)) T.aligned = 0;
          }
          slot_floats_total += static_cast<size_t>(T.nslots) * sf;
          if (P >= 32) {
            const int64_t stride = c->p > 1 ? static_cast<const char*>(j->cols[1]) - static_cast<const char*>(j->cols[0]) : 0;
            const bool same = c->tmap_base == j->cols[0] && c->tmap_stride == stride && c->tmap_rows == T.nrows &&
                              c->tmap_box == static_cast<int>(rs);
            bool ok = false;
            if (same) {
              // the cached map covers the same columns when they still sit one stride apart
              ok = c->tmap_ok;
              for (int jj = 2; ok && jj < c->p; ++jj)
                if (static_cast<const char*>(j->cols[jj]) - static_cast<const char*>(j->cols[0]) != jj * stride) ok = false;
            } else {
              ok = table_tensor_map(j->cols, c->p, T.nrows, P, static_cast<int>(rs), &c->tmap);
              c->tmap_base = j->cols[0];
              c->tmap_stride = stride;
              c->tmap_rows = T.nrows;
              c->tmap_box = static_cast<int>(rs);
              c->tmap_ok = ok;
            }
            if (ok) {
              map_of[i] = static_cast<int>(maps.size());
              maps.push_back(c->tmap);
            }
          }
          if (!c->shift_set) need_shift.push_back(static_cast<int>(i));
          if (c->flush_rows > 0) flush_kb = std::min(flush_kb, std::max(1, c->flush_rows / 16));
        }
        const size_t off_maps = round256(nt * sizeof(Gram32Table));
        const size_t off_cols = off_maps + round256(maps.size() * sizeof(CUtensorMap));
        const size_t off_which = off_cols + round256(colptrs.size() * sizeof(void*));
        const size_t off_slot = off_which + round256(need_shift.size() * sizeof(int));
        const size_t off_wslot = off_slot + round256(slot_floats_total * sizeof(float));
        const size_t need = off_wslot + round256(static_cast<size_t>(grid) * kGram32Warps * sf * sizeof(float));
        if (ws.bytes < need) {
          if (ws.dev) CK(c0, cudaFree(ws.dev));  // synchronises the device
          ws.dev = nullptr;
          ws.bytes = 0;
          CK(c0, cudaMalloc(&ws.dev, need));
          ws.bytes = need;
        }
        char* base = static_cast<char*>(ws.dev);
        size_t cp = 0, so = 0;
        for (size_t i = 0; i < nt; ++i) {
          tabs[i].cols = reinterpret_cast<const float* const*>(base + off_cols) + cp;
          tabs[i].slots = reinterpret_cast<float*>(base + off_slot) + so;
          tabs[i].tmap = map_of[i] >= 0 ? base + off_maps + static_cast<size_t>(map_of[i]) * sizeof(CUtensorMap) : nullptr;
          cp += tabs[i].p;
          so += static_cast<size_t>(tabs[i].nslots) * sf;
        }
        CK(c0, cudaMemcpyAsync(base, tabs.data(), nt * sizeof(Gram32Table), cudaMemcpyHostToDevice, st));
        CK(c0, cudaMemcpyAsync(base + off_cols, colptrs.data(), colptrs.size() * sizeof(void*),
                               cudaMemcpyHostToDevice, st));
        if (!maps.empty())
          CK(c0, cudaMemcpyAsync(base + off_maps, maps.data(), maps.size() * sizeof(CUtensorMap),
                                 cudaMemcpyHostToDevice, st));
        if (!need_shift.empty()) {
          CK(c0, cudaMemcpyAsync(base + off_which, need_shift.data(), need_shift.size() * sizeof(int),
                                 cudaMemcpyHostToDevice, st));
          CK(c0, launch_gram32_shift(reinterpret_cast<const Gram32Table*>(base),
                                     reinterpret_cast<const int*>(base + off_which),
                                     static_cast<int>(need_shift.size()), st));
          for (int i : need_shift) all[first + i]->c->shift_set = true;
        }
        Gram32Launch L{};
        L.tabs = reinterpret_cast<const Gram32Table*>(base);
        L.warp_scratch = reinterpret_cast<float*>(base + off_wslot);
        L.ntables = static_cast<int32_t>(nt);
        L.total_stages = static_cast<int32_t>(total);
        L.chunk = static_cast<int32_t>(K);
        L.flush_kblocks = flush_kb;
        CK(c0, launch_gram32(L, P, x4 == 1, grid, st));
        for (size_t i = 0; i < nt; ++i) all[first + i]->c->last = st;
      }
    }
  }
  CK(c0, cudaEventRecord(ws.last, st));
  return STATS_OK;
}

// Wide FP32 tables (p > 64) whose columns sit one 16-byte-multiple stride apart go to the
// tcgen05 kernel through a 2D tensor map (box 32 rows x 128 columns); others to the
// tiled split kernel.
bool wide_eligible(stats_ctx* c, const void* const* dcols, int64_t nrows) {
  if (c->p <= 64 || c->p > 1280 || nrows < wide_chunk_rows() || nrows >= (int64_t(1) << 35)) return false;
  const int rows = wide_rows_per_stage(), bcols = wide_block_cols();
  const int64_t stride = static_cast<const char*>(dcols[1]) - static_cast<const char*>(dcols[0]);
  if (c->tmap_base == dcols[0] && c->tmap_stride == stride && c->tmap_rows == nrows && c->tmap_box == -rows &&
      c->tmap_cols == bcols) {
    bool ok = c->tmap_ok;
    for (int j = 2; ok && j < c->p; ++j)
      if (static_cast<const char*>(dcols[j]) - static_cast<const char*>(dcols[0]) != j * stride) ok = false;
    return ok;
  }
  c->tmap_ok = table_tensor_map_chunks(dcols, c->p, nrows, bcols, rows / wide_chunk_rows(), &c->tmap);
  c->tmap_base = dcols[0];
  c->tmap_stride = stride;
  c->tmap_rows = nrows;
  c->tmap_box = -rows;  // negative: a chunked (3D) map
  c->tmap_cols = bcols;
  return c->tmap_ok;
}

// 33 to 64 columns, uniformly strided (one [p, ld] block): the tcgen05 pass of k_narrow.cu.
bool narrow_eligible(stats_ctx* c, const void* const* dcols, int64_t nrows) {
  if (c->p <= 32 || c->p > narrow_cols() || nrows < wide_chunk_rows() || nrows >= (int64_t(1) << 35)) return false;
  const int rows = narrow_rows_per_stage(), bcols = narrow_cols();
  const int64_t stride = static_cast<const char*>(dcols[1]) - static_cast<const char*>(dcols[0]);
  if (c->tmap_base == dcols[0] && c->tmap_stride == stride && c->tmap_rows == nrows && c->tmap_box == -rows &&
      c->tmap_cols == bcols) {
    bool ok = c->tmap_ok;
    for (int j = 2; ok && j < c->p; ++j)
      if (static_cast<const char*>(dcols[j]) - static_cast<const char*>(dcols[0]) != j * stride) ok = false;
    return ok;
  }
  c->tmap_ok = table_tensor_map_chunks(dcols, c->p, nrows, bcols, rows / wide_chunk_rows(), &c->tmap);
  c->tmap_base = dcols[0];
  c->tmap_stride = stride;
  c->tmap_rows = nrows;
  c->tmap_box = -rows;
  c->tmap_cols = bcols;
  return c->tmap_ok;
}

stats_status run_wide(stats_ctx* c, const void* const* dcols, int64_t nrows, cudaStream_t st) {
  if (!c->shift_set) {
    SplitParams S{};
    for (int j = 0; j < c->p; ++j) S.cols[j] = static_cast<const float*>(dcols[j]);
    S.p = c->p;
    S.shift = c->d_fshift;
    CK(c, launch_split_shift(S, nrows, c->d_shift, st));
    c->shift_set = true;
  }
  WideParams W{};
  const bool x4 = split_x4(c, nrows);
  const int grid = wide_plan(c->p, c->sms, x4, W);
  if (grid <= 0) return STATS_EINVAL;
  if (!c->d_wide_slots || c->wide_grid_alloc < grid) {
    if (c->d_wide_slots) CK(c, cudaFree(c->d_wide_slots));
    c->d_wide_slots = nullptr;
    CK(c, cudaMalloc(&c->d_wide_slots, static_cast<size_t>(grid) * kWideSlotPairs * 2 * sizeof(float)));
    c->wide_grid_alloc = grid;
  }
  // the tensor map travels in the kernel parameters' ctx-owned device copy
  if (!c->d_tmap) CK(c, cudaMalloc(&c->d_tmap, sizeof(CUtensorMap)));
  CK(c, cudaMemcpyAsync(c->d_tmap, &c->tmap, sizeof(CUtensorMap), cudaMemcpyHostToDevice, st));
  W.tmap = c->d_tmap;
  W.base = static_cast<const float*>(dcols[0]);
  W.ld = (static_cast<const char*>(dcols[1]) - static_cast<const char*>(dcols[0])) / 4;
  W.shift = c->d_fshift;
  W.slots = c->d_wide_slots;
  W.acc_s = c->d_fs;
  W.acc_s_lo = c->d_fs_lo;
  W.acc_S = c->d_fS;
  W.acc_S_lo = c->d_fS_lo;
  W.acc_n = c->d_fn;
  W.status = c->d_status;
  W.nrows = nrows;
  W.nfull = nrows / wide_chunk_rows();
  W.p = c->p;
  const int flush_rows = c->flush_rows > 0 ? c->flush_rows : 16384;
  W.flush_chains = std::max(1, flush_rows / wide_chunk_rows());
  CK(c, launch_wide(W, x4, grid, st));
  return STATS_OK;
}

// 129..256 columns of one [p, ld] block (tensor map current in c->tmap): the paired-CTA pass.
stats_status run_wide2(stats_ctx* c, const void* const* dcols, int64_t nrows, cudaStream_t st) {
  if (!c->shift_set) {
    SplitParams S{};
    for (int j = 0; j < c->p; ++j) S.cols[j] = static_cast<const float*>(dcols[j]);
    S.p = c->p;
    S.shift = c->d_fshift;
    CK(c, launch_split_shift(S, nrows, c->d_shift, st));
    c->shift_set = true;
  }
  const int grid = wide2_grid(c->sms);
  const size_t pairs = static_cast<size_t>(grid) * kWide2SlotPairs;
  if (!c->d_wide_slots || static_cast<size_t>(c->wide_grid_alloc) * kWideSlotPairs < pairs) {
    if (c->d_wide_slots) CK(c, cudaFree(c->d_wide_slots));
    c->d_wide_slots = nullptr;
    CK(c, cudaMalloc(&c->d_wide_slots, pairs * 2 * sizeof(float)));
    c->wide_grid_alloc = static_cast<int>((pairs + kWideSlotPairs - 1) / kWideSlotPairs);
  }
  if (!c->d_tmap) CK(c, cudaMalloc(&c->d_tmap, sizeof(CUtensorMap)));
  CK(c, cudaMemcpyAsync(c->d_tmap, &c->tmap, sizeof(CUtensorMap), cudaMemcpyHostToDevice, st));
  Wide2Params W{};
  W.tmap = c->d_tmap;
  W.base = static_cast<const float*>(dcols[0]);
  W.ld = (static_cast<const char*>(dcols[1]) - static_cast<const char*>(dcols[0])) / 4;
  W.shift = c->d_fshift;
  W.slots = c->d_wide_slots;
  W.acc_s = c->d_fs;
  W.acc_s_lo = c->d_fs_lo;
  W.acc_S = c->d_fS;
  W.acc_S_lo = c->d_fS_lo;
  W.acc_n = c->d_fn;
  W.status = c->d_status;
  W.nrows = nrows;
  W.nfull = nrows / wide_chunk_rows();
  W.p = c->p;
  const int flush_rows = c->flush_rows > 0 ? c->flush_rows : 16384;
  W.flush_stages = std::max(1, flush_rows / wide_rows_per_stage());
  CK(c, launch_wide2(W, split_x4(c, nrows), grid, st));
  return STATS_OK;
}

// The narrow-pass description of one table (its tensor map must be current in c->tmap).
NarrowTab narrow_table(stats_ctx* c, const void* const* dcols, int64_t nrows) {
  NarrowTab T{};
  T.tmap = c->d_tmap;
  T.base = static_cast<const float*>(dcols[0]);
  T.ld = (static_cast<const char*>(dcols[1]) - static_cast<const char*>(dcols[0])) / 4;
  T.shift = c->d_fshift;
  T.shift_d = c->d_shift;
  T.acc_s = c->d_fs;
  T.acc_s_lo = c->d_fs_lo;
  T.acc_S = c->d_fS;
  T.acc_S_lo = c->d_fS_lo;
  T.acc_n = c->d_fn;
  T.nrows = nrows;
  T.nfull = nrows / wide_chunk_rows();
  T.p = c->p;
  return T;
}

int narrow_flush_stages(const stats_ctx* c) {
  const int flush_rows = c->flush_rows > 0 ? c->flush_rows : 16384;
  return std::max(1, flush_rows / narrow_rows_per_stage());  // one chain per stage
}

stats_status run_narrow(stats_ctx* c, const void* const* dcols, int64_t nrows, cudaStream_t st) {
  if (!c->shift_set) {
    SplitParams S{};
    for (int j = 0; j < c->p; ++j) S.cols[j] = static_cast<const float*>(dcols[j]);
    S.p = c->p;
    S.shift = c->d_fshift;
    CK(c, launch_split_shift(S, nrows, c->d_shift, st));
    c->shift_set = true;
  }
  const int grid = std::max(1, c->sms);
  if (!c->d_wide_slots || c->wide_grid_alloc < grid) {
    if (c->d_wide_slots) CK(c, cudaFree(c->d_wide_slots));
    c->d_wide_slots = nullptr;
    CK(c, cudaMalloc(&c->d_wide_slots, static_cast<size_t>(grid) * kWideSlotPairs * 2 * sizeof(float)));
    c->wide_grid_alloc = grid;
  }
  if (!c->d_tmap) CK(c, cudaMalloc(&c->d_tmap, sizeof(CUtensorMap)));
  CK(c, cudaMemcpyAsync(c->d_tmap, &c->tmap, sizeof(CUtensorMap), cudaMemcpyHostToDevice, st));
  NarrowParams P{};
  P.tab0 = narrow_table(c, dcols, nrows);
  P.nunits = grid;  // the table's stages in grid consecutive ranges, one per CTA
  P.ntabs = 1;
  P.slots = c->d_wide_slots;
  P.status = c->d_status;
  P.flush_stages = narrow_flush_stages(c);
  CK(c, launch_narrow(P, split_x4(c, nrows), grid, st));
  return STATS_OK;
}

// Tables of 33..64 FP32 columns of one batched call, one mode: a single persistent narrow
// launch.  Each table is cut into units of at most U stages, U chosen so that the CTAs get
// about narrow_units_per_cta units each (a unit runs on one SM: large units would leave the
// last CTAs finishing alone); units are dealt to CTAs largest first (CTA b takes units b,
// b + grid, ...), and every unit has its own slot, merged per table in row order.
constexpr int64_t kNarrowUnitMinStages = 64, kNarrowUnitMaxStages = 16384;

struct NarrowJob {
  stats_ctx* c;
  const void* const* cols;
  int64_t nrows;
};

struct NarrowWorkspace {
  void* dev = nullptr;
  size_t bytes = 0;
  cudaEvent_t last = nullptr;
};
std::mutex g_narrow_mu;
NarrowWorkspace g_narrow_ws[64];

stats_status run_narrow_batch(const std::vector<NarrowJob>& jobs, bool x4, cudaStream_t st) {
  if (jobs.empty()) return STATS_OK;
  stats_ctx* c0 = jobs[0].c;
  int dev = 0;
  CK(c0, cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return STATS_EINVAL;
  const int rs = narrow_rows_per_stage();
  const size_t nt = jobs.size();
  std::vector<NarrowTab> tabs(nt);
  std::vector<CUtensorMap> maps(nt);
  std::vector<int32_t> slot0(nt + 1, 0);
  std::vector<NarrowUnit> units;
  std::vector<int> need_shift;
  int64_t total = 0;
  for (const NarrowJob& j : jobs) total += (j.nrows + rs - 1) / rs;
  const int64_t ustages =
      std::min(kNarrowUnitMaxStages, std::max(kNarrowUnitMinStages, total / (int64_t(std::max(1, c0->sms)) *
                                                                             batch_tuning(64, x4).narrow_units_per_cta)));
  for (size_t i = 0; i < nt; ++i) {
    const NarrowJob& j = jobs[i];
    tabs[i] = narrow_table(j.c, j.cols, j.nrows);
    maps[i] = j.c->tmap;
    if (!j.c->shift_set) need_shift.push_back(static_cast<int>(i));
    const int64_t nst = (j.nrows + rs - 1) / rs;
    const int64_t nu = (nst + ustages - 1) / ustages;
    slot0[i + 1] = slot0[i] + static_cast<int32_t>(nu);
    for (int64_t u = 0; u < nu; ++u) {
      NarrowUnit U{};
      U.st0 = u * nst / nu;
      U.nst = static_cast<int32_t>((u + 1) * nst / nu - U.st0);
      U.tab = static_cast<int32_t>(i);
      U.slot = slot0[i] + static_cast<int32_t>(u);
      units.push_back(U);
    }
  }
  std::stable_sort(units.begin(), units.end(), [](const NarrowUnit& a, const NarrowUnit& b) { return a.nst > b.nst; });
  const int nunits = static_cast<int>(units.size());
  const int grid = std::min(nunits, std::max(1, c0->sms));
  const size_t off_maps = ((nt * sizeof(NarrowTab) + 255) / 256) * 256;
  const size_t off_units = off_maps + nt * sizeof(CUtensorMap);  // 128-byte maps, 64-byte aligned
  const size_t off_slot0 = off_units + (((units.size() * sizeof(NarrowUnit)) + 255) / 256) * 256;
  const size_t off_which = off_slot0 + (((nt + 1) * sizeof(int32_t) + 255) / 256) * 256;
  const size_t off_slots = off_which + ((need_shift.size() * sizeof(int) + 255) / 256) * 256;
  const size_t need = off_slots + static_cast<size_t>(nunits) * kWideSlotPairs * 2 * sizeof(float);
  std::lock_guard<std::mutex> lk(g_narrow_mu);
  NarrowWorkspace& ws = g_narrow_ws[dev];
  if (!ws.last) CK(c0, cudaEventCreateWithFlags(&ws.last, cudaEventDisableTiming));
  CK(c0, cudaStreamWaitEvent(st, ws.last, 0));  // the previous user of the workspace is done
  if (ws.bytes < need) {
    if (ws.dev) CK(c0, cudaFree(ws.dev));  // synchronises the device
    ws.dev = nullptr;
    ws.bytes = 0;
    CK(c0, cudaMalloc(&ws.dev, need));
    ws.bytes = need;
  }
  char* base = static_cast<char*>(ws.dev);
  for (size_t i = 0; i < nt; ++i) tabs[i].tmap = base + off_maps + i * sizeof(CUtensorMap);
  CK(c0, cudaMemcpyAsync(base, tabs.data(), nt * sizeof(NarrowTab), cudaMemcpyHostToDevice, st));
  CK(c0, cudaMemcpyAsync(base + off_maps, maps.data(), nt * sizeof(CUtensorMap), cudaMemcpyHostToDevice, st));
  CK(c0, cudaMemcpyAsync(base + off_units, units.data(), units.size() * sizeof(NarrowUnit), cudaMemcpyHostToDevice,
                         st));
  CK(c0, cudaMemcpyAsync(base + off_slot0, slot0.data(), (nt + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  if (!need_shift.empty()) {
    CK(c0, cudaMemcpyAsync(base + off_which, need_shift.data(), need_shift.size() * sizeof(int),
                           cudaMemcpyHostToDevice, st));
    CK(c0, launch_narrow_shift(reinterpret_cast<const NarrowTab*>(base), reinterpret_cast<const int*>(base + off_which),
                               static_cast<int>(need_shift.size()), st));
    for (int i : need_shift) jobs[i].c->shift_set = true;
  }
  NarrowParams P{};
  P.tabs = reinterpret_cast<const NarrowTab*>(base);
  P.units = reinterpret_cast<const NarrowUnit*>(base + off_units);
  P.tab_slot0 = reinterpret_cast<const int32_t*>(base + off_slot0);
  P.slots = reinterpret_cast<float*>(base + off_slots);
  P.status = c0->d_status;
  P.nunits = nunits;
  P.ntabs = static_cast<int32_t>(nt);
  P.flush_stages = narrow_flush_stages(c0);
  for (const NarrowJob& j : jobs) P.flush_stages = std::min(P.flush_stages, narrow_flush_stages(j.c));
  CK(c0, launch_narrow(P, x4, grid, st));
  CK(c0, cudaEventRecord(ws.last, st));
  return STATS_OK;
}

stats_status launch_pass(stats_ctx* c, const void* const* dcols, int64_t nrows, cudaStream_t st) {
  if (nrows == 0) return STATS_OK;
  const int grid = default_grid(c);
  if (c->mode == STATS_EXACT) {
    ExactParams P = c->xp;
    if (c->exact_shape >= 0 && c->exact_shape != P.shape && !exact_layout(P, c->exact_shape)) return STATS_EINVAL;
    P.direct = 0;
    for (int j = 0; j < c->p; ++j) {
      P.cols[j] = dcols[j];
      if (!aligned16(dcols[j])) P.direct = 1;
    }
    P.nrows = nrows;
    P.nmain = P.direct ? nrows : (nrows & ~int64_t(7));
    int g = grid;
    if (c->grid <= 0 && P.shape != c->xp.shape)
      g = c->sms * std::max(1, exact_max_active_blocks(c->conv, P.shape, P.stages, P.stage_bytes));
    CK(c, launch_exact(P, c->conv, g, st));
  } else if ((c->mode == STATS_BF16X3 || c->mode == STATS_BF16X4) && c->p <= 64 && nrows >= kNarrowMinRows &&
             narrow_eligible(c, dcols, nrows)) {
    stats_status s = run_narrow(c, dcols, nrows, st);
    if (s != STATS_OK) return s;
  } else if ((c->mode == STATS_BF16X3 || c->mode == STATS_BF16X4) && c->p <= 64) {
    std::vector<Gram32Job> jobs{{c, dcols, nrows, split_x4(c, nrows)}};
    stats_status s = run_gram32(jobs, st);
    if (s != STATS_OK) return s;
  } else if ((c->mode == STATS_BF16X3 || c->mode == STATS_BF16X4) && wide_eligible(c, dcols, nrows)) {
    const bool pairs = c->wide_pairs && c->p > wide_block_cols() && c->p <= 2 * wide_block_cols() && c->sms >= 2;
    stats_status s = pairs ? run_wide2(c, dcols, nrows, st) : run_wide(c, dcols, nrows, st);
    if (s != STATS_OK) return s;
  } else if (c->mode == STATS_BF16X3 || c->mode == STATS_BF16X4) {
    SplitParams S{};
    for (int j = 0; j < c->p; ++j) S.cols[j] = static_cast<const float*>(dcols[j]);
    S.p = c->p;
    S.shift = c->d_fshift;
    if (!c->shift_set) {
      CK(c, launch_split_shift(S, nrows, c->d_shift, st));
      c->shift_set = true;
    }
    const int T = split_tile(c->p);
    S.nblk = (c->p + T - 1) / T;
    S.ntiles = S.nblk * (S.nblk + 1) / 2;
    const int64_t max_split = std::max<int64_t>(1, nrows / 4096);
    S.ksplit = static_cast<int>(std::min<int64_t>(max_split, (4 * c->sms + S.ntiles - 1) / S.ntiles));
    if (c->grid > 0) S.ksplit = std::max(1, c->grid / S.ntiles);
    const int g = S.ntiles * S.ksplit;
    if (!c->d_split_slots || c->split_grid < g) {
      if (c->d_split_slots) CK(c, cudaFree(c->d_split_slots));
      c->d_split_slots = nullptr;
      const size_t bytes = split_slot_floats(g) * sizeof(float) + 256;
      CK(c, cudaMalloc(&c->d_split_slots, bytes));
      CK(c, cudaMemset(c->d_split_slots, 0, bytes));
      c->split_grid = g;
      c->d_split_ticket = reinterpret_cast<unsigned int*>(c->d_split_slots + split_slot_floats(g));
    }
    // every 16-row K block is a fresh tensor chain; the FP32 accumulators go into (hi, lo)
    // pairs every 1024 rows of a warp
    S.flush_rows = c->flush_rows > 0 ? c->flush_rows : 1024;
    S.nrows = nrows;
    S.slots = c->d_split_slots;
    S.ticket = c->d_split_ticket;
    S.acc_s = c->d_fs;
    S.acc_s_lo = c->d_fs_lo;
    S.acc_S = c->d_fS;
    S.acc_S_lo = c->d_fS_lo;
    S.acc_n = c->d_fn;
    CK(c, launch_split(S, T, split_x4(c, nrows), g, st));
  } else if (c->mode == STATS_FP32 || c->p > 12) {
    // tiled CUDA-core pass: FP32-core, or FP64 for tables wider than the row kernel
    CoreParams C{};
    for (int j = 0; j < c->p; ++j) {
      C.cols[j] = dcols[j];
      C.dtype[j] = c->dtypes[j];
    }
    C.p = c->p;
    if (c->mode != STATS_FP64) {
      if (!c->shift_set) {
        CK(c, launch_set_shift(dcols, c->dtypes.data(), c->p, nrows, c->d_shift, st));
        c->shift_set = true;
      }
      C.shift = c->d_shift;
    }
    C.nblk = (c->p + 63) / 64;
    C.ntiles = C.nblk * (C.nblk + 1) / 2;
    const int64_t max_split = std::max<int64_t>(1, nrows / 4096);
    C.ksplit = static_cast<int>(std::min<int64_t>(max_split, (4 * c->sms + C.ntiles - 1) / C.ntiles));
    if (c->grid > 0) C.ksplit = std::max(1, c->grid / C.ntiles);
    const int g = C.ntiles * C.ksplit;
    if (!c->d_core_slots || c->core_grid < g) {
      if (c->d_core_slots) CK(c, cudaFree(c->d_core_slots));
      c->d_core_slots = nullptr;
      const size_t bytes = core_slot_doubles(g) * sizeof(double) + 256;
      CK(c, cudaMalloc(&c->d_core_slots, bytes));
      CK(c, cudaMemset(c->d_core_slots, 0, bytes));
      c->core_grid = g;
      c->d_core_ticket = reinterpret_cast<unsigned int*>(c->d_core_slots + core_slot_doubles(g));
    }
    C.flush_rows = c->flush_rows > 0 ? c->flush_rows : 64;
    C.nrows = nrows;
    C.slots = c->d_core_slots;
    C.ticket = c->d_core_ticket;
    C.acc_s = c->d_fs;
    C.acc_s_lo = c->d_fs_lo;
    C.acc_S = c->d_fS;
    C.acc_S_lo = c->d_fS_lo;
    C.acc_n = c->d_fn;
    CK(c, launch_core(C, c->mode == STATS_FP32, g, st));
  } else {
    Fp64Params P{};
    for (int j = 0; j < c->p; ++j) {
      P.cols[j] = dcols[j];
      P.dtype[j] = c->dtypes[j];
    }
    P.p = c->p;
    P.nrows = nrows;
    if (c->mode == STATS_FP64_SHIFTED) {
      if (!c->shift_set) {
        CK(c, launch_set_shift(dcols, c->dtypes.data(), c->p, nrows, c->d_shift, st));
        c->shift_set = true;
      }
      P.shift = c->d_shift;
    }
    stats_status s = ensure_slots(c, grid);
    if (s != STATS_OK) return s;
    P.slots = c->d_slots;
    P.acc_s = c->d_fs;
    P.acc_s_lo = c->d_fs_lo;
    P.acc_S = c->d_fS;
    P.acc_S_lo = c->d_fS_lo;
    P.acc_n = c->d_fn;
    CK(c, launch_fp64(P, grid, st));
  }
  c->rows_enqueued += nrows;
  c->last = st;
  return STATS_OK;
}

void build_final_params(const stats_ctx* c, int want_pca, int pca_on, FinalParams& F) {
  F = FinalParams{};
  F.p = c->p;
  F.mode = c->mode == STATS_EXACT ? 0 : 1;
  F.pca_on = pca_on;
  F.want_pca = want_pca;
  for (int j = 0; j < c->p; ++j) {
    F.col[j].off = c->plan.empty() ? 0 : c->plan[j].off;
    F.col[j].k = c->plan.empty() ? 0 : c->plan[j].k;
    F.col[j].shift = c->plan.empty() ? 0 : c->plan[j].shift;
    F.col[j].is_real = c->plan.empty() ? 0 : c->plan[j].is_real;
    F.col[j].is_ident = c->ident[j];
  }
  F.g = c->d_g;
  F.fs = c->d_fs;
  F.fs_lo = c->d_fs_lo;
  F.fS = c->d_fS;
  F.fS_lo = c->d_fS_lo;
  F.fn = c->d_fn;
  F.shift = ((c->mode == STATS_FP64_SHIFTED || c->mode == STATS_BF16X3 || c->mode == STATS_BF16X4 ||
              c->mode == STATS_FP32) &&
             c->shift_set)
                ? c->d_shift
                : nullptr;
  F.out = c->d_out;
  F.work = c->d_work;
}

// From this many analysis columns on, the eigen-solver runs over the whole GPU
// (jacobi_grid_kernel) instead of inside the one-block finalize kernel: GB300 has
// about 2 FP64 FMAs per SM clock, so one block is far too slow for p_a in the hundreds.
constexpr int kGridJacobiMinColumns = 24;

// Finalize on the ctx's stream.  With want_pca, the eigen-decomposition runs either in the
// finalize kernel (small p_a) or in the grid-wide solver, seeded by `seed` (host, p_a x p_a,
// rows = eigenvectors) when given.  Synchronises.
stats_status run_finalize(stats_ctx* c, int want_pca, int pca_on, const double* seed = nullptr) {
  FinalParams F;
  build_final_params(c, want_pca, pca_on, F);
  cudaStream_t st = c->last;
  const int pa = c->pa;
  const int grid = (want_pca && c->coop && pa >= 2 && (pa >= kGridJacobiMinColumns || seed)) ? jacobi_grid_blocks(pa, c->sms) : 0;
  JacobiParams J{};
  if (grid > 0) {
    if (!c->d_jac) CK(c, cudaMalloc(&c->d_jac, jacobi_scratch_doubles(pa) * sizeof(double)));
    const size_t m = (pa + 15) / 16 * 16;
    J.a = c->d_jac;
    J.b = J.a + m * m;
    J.v = J.b + m * m;
    J.w = J.v + m * m;
    double* basis = J.w + m * m;
    J.q = basis + static_cast<size_t>(pa) * pa;
    J.slots = J.q + (m / 16) * 256;
    J.bar = reinterpret_cast<unsigned int*>(J.slots + 1024);
    J.ctl = reinterpret_cast<const int32_t*>(J.bar + 4);
    J.basis = seed ? basis : nullptr;
    J.out = c->d_out;
    J.evals_off = c->lay.evals;
    J.evecs_off = c->lay.evecs;
    J.flags_off = c->lay.flags;
    J.pa = pa;
    J.m = static_cast<int32_t>(m);
    J.wait_ns = c->grid_wait_ns;
    J.absent_block = c->grid_absent_block;
    F.defer_A = J.a;
    F.defer_ctl = const_cast<int32_t*>(J.ctl);
    F.defer_m = J.m;
    if (seed) CK(c, cudaMemcpyAsync(basis, seed, sizeof(double) * pa * pa, cudaMemcpyHostToDevice, st));
    CK(c, cudaMemsetAsync(J.bar, 0, 8 * sizeof(unsigned int), st));
  }
  CK(c, launch_finalize(F, st));
  if (grid > 0) CK(c, launch_jacobi_grid(J, grid, st));
  CK(c, cudaMemcpyAsync(c->h_out, c->d_out, c->lay.total * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(c, cudaStreamSynchronize(st));
  if (c->h_out[c->lay.flags + 5] != 0.0) return STATS_ETIMEOUT;
  return STATS_OK;
}

void free_ctx(stats_ctx* c) {
  if (!c) return;
  cudaFree(c->d_g);
  cudaFree(c->d_call);
  cudaFree(c->d_fs);
  cudaFree(c->d_slots);
  cudaFree(c->d_fshift);
  cudaFree(c->d_core_slots);
  cudaFree(c->d_split_slots);
  cudaFree(c->d_wide_slots);
  cudaFree(c->d_tmap);
  cudaFree(c->d_out);
  cudaFree(c->d_work);
  cudaFree(c->d_jac);
  if (c->h_out) cudaFreeHost(c->h_out);
  for (int b = 0; b < 2; ++b) {
    cudaFree(c->d_stage[b]);
    if (c->h_stage[b]) cudaFreeHost(c->h_stage[b]);
    if (c->ev_copied[b]) cudaEventDestroy(c->ev_copied[b]);
    if (c->ev_done[b]) cudaEventDestroy(c->ev_done[b]);
  }
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  delete c;
}

stats_status create(stats_ctx** out, const stats_config* cfg) {
  if (!out || !cfg) return STATS_EINVAL;
  *out = nullptr;
  if (cfg->p < 1 || cfg->p > STATS_MAX_P || !cfg->dtypes) return STATS_EINVAL;
  if (cfg->mode < STATS_EXACT || cfg->mode > STATS_FP32) return STATS_EINVAL;
  if ((cfg->lo == nullptr) != (cfg->hi == nullptr)) return STATS_EINVAL;
  // modes not built yet: BF16X3 / BF16X4 / FP32
  if (cfg->mode == STATS_BF16X3 || cfg->mode == STATS_BF16X4)
    for (int j = 0; j < cfg->p; ++j)
      if (cfg->dtypes[j] != F32) return STATS_EINVAL;  // the split path takes FP32 columns
  stats_ctx* c = new (std::nothrow) stats_ctx();
  if (!c) return STATS_ENOMEM;
  c->p = cfg->p;
  c->mode = cfg->mode;
  c->dtypes.assign(cfg->dtypes, cfg->dtypes + cfg->p);
  for (int32_t dt : c->dtypes)
    if (dt < I16 || dt > F64) {
      delete c;
      return STATS_EINVAL;
    }
  c->ident.assign(cfg->p, 0);
  if (cfg->is_identifier)
    for (int j = 0; j < cfg->p; ++j) c->ident[j] = cfg->is_identifier[j] ? 1 : 0;
  c->has_bounds = cfg->lo != nullptr;
  if (c->has_bounds) {
    c->lo.assign(cfg->lo, cfg->lo + cfg->p);
    c->hi.assign(cfg->hi, cfg->hi + cfg->p);
  }
  c->pa = 0;
  for (int j = 0; j < c->p; ++j) c->pa += c->ident[j] ? 0 : 1;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return STATS_ECUDA;
  }
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  if (c->sms < 1) c->sms = 1;
  cudaDeviceGetAttribute(&c->coop, cudaDevAttrCooperativeLaunch, c->device);

  stats_status s = STATS_OK;
  if (c->mode == STATS_EXACT) {
    s = build_plan(c);  // digit plan, converter and stage layout
    if (s != STATS_OK) {
      delete c;
      return s;
    }
  }
  // device allocations
  cudaError_t e = cudaSuccess;
  const size_t T = static_cast<size_t>(c->p) * (c->p + 1) / 2;
  if (c->mode == STATS_EXACT) {
    e = cudaMalloc(&c->d_g, kDigits * kDigits * sizeof(long long));
    if (e == cudaSuccess) e = cudaMemset(c->d_g, 0, kDigits * kDigits * sizeof(long long));
    // scratch: per-call accumulator, ticket, error word, status word
    if (e == cudaSuccess) e = cudaMalloc(&c->d_call, kDigits * kDigits * sizeof(unsigned long long) + 256);
    if (e == cudaSuccess) e = cudaMemset(c->d_call, 0, kDigits * kDigits * sizeof(unsigned long long) + 256);
    if (e == cudaSuccess) {
      unsigned int* words = reinterpret_cast<unsigned int*>(c->d_call + kDigits * kDigits);
      c->d_ticket = words;
      c->d_err = words + 1;
      c->d_status = words + 2;
      c->xp.call_acc = c->d_call;
      c->xp.ticket = c->d_ticket;
      c->xp.err = c->d_err;
      c->xp.acc = c->d_g;
      c->xp.status = c->d_status;
    }
  } else {
    const size_t nd = 2 * c->p + 2 * T + c->p + 2;
    e = cudaMalloc(&c->d_fs, nd * sizeof(double) + 256);
    if (e == cudaSuccess) e = cudaMemset(c->d_fs, 0, nd * sizeof(double) + 256);
    if (e == cudaSuccess) {
      c->d_fs_lo = c->d_fs + c->p;
      c->d_fS = c->d_fs_lo + c->p;
      c->d_fS_lo = c->d_fS + T;
      c->d_shift = c->d_fS_lo + T;
      c->d_fn = reinterpret_cast<long long*>(c->d_shift + c->p);
      c->d_status = reinterpret_cast<unsigned int*>(c->d_fn + 1);
    }
    if (e == cudaSuccess && (c->mode == STATS_BF16X3 || c->mode == STATS_BF16X4))
      e = cudaMalloc(&c->d_fshift, c->p * sizeof(float));
  }
  c->lay = final_layout(c->p, c->pa);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_out, c->lay.total * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_work, (2 * static_cast<size_t>(c->pa) * c->pa + 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_out, c->lay.total * sizeof(double));
  if (e != cudaSuccess) {
    free_ctx(c);
    return e == cudaErrorMemoryAllocation ? STATS_ENOMEM : STATS_ECUDA;
  }
  *out = c;
  return STATS_OK;
}

}  // namespace

namespace {

// The two device staging buffers of the host- and file-streamed passes (each column of
// a chunk at stage_off[j], 256-byte aligned) and the copy stream with its events.
stats_status ensure_staging(stats_ctx* ctx, int64_t chunk_rows) {
  if (ctx->stage_rows < chunk_rows) {
    for (int b = 0; b < 2; ++b) {
      if (ctx->d_stage[b]) CK(ctx, cudaFree(ctx->d_stage[b]));
      ctx->d_stage[b] = nullptr;
    }
    ctx->stage_off.assign(ctx->p, 0);
    size_t off = 0;
    for (int j = 0; j < ctx->p; ++j) {
      ctx->stage_off[j] = off;
      off += ((static_cast<size_t>(chunk_rows) * dtype_bytes(ctx->dtypes[j]) + 255) / 256) * 256;
    }
    for (int b = 0; b < 2; ++b) {
      cudaError_t e = cudaMalloc(&ctx->d_stage[b], off);
      if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        ctx->stage_rows = 0;
        return STATS_ENOMEM;
      }
      CK(ctx, e);
    }
    ctx->stage_rows = chunk_rows;
  }
  if (!ctx->copy_stream) {
    CK(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
      CK(ctx, cudaEventCreateWithFlags(&ctx->ev_copied[b], cudaEventDisableTiming));
      CK(ctx, cudaEventCreateWithFlags(&ctx->ev_done[b], cudaEventDisableTiming));
    }
  }
  return STATS_OK;
}

// Copy one chunk (hc: p host column pointers at the chunk's first row) into staging
// buffer b on the copy stream and enqueue its pass on st.
stats_status enqueue_chunk(stats_ctx* ctx, int b, const void* const* hc, int64_t rows, cudaStream_t st) {
  std::vector<const void*> dcols(ctx->p);
  // the pass that last read buffer b must be done before it is overwritten
  CK(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_done[b], 0));
  for (int j = 0; j < ctx->p; ++j) {
    const size_t eb = dtype_bytes(ctx->dtypes[j]);
    char* dst = static_cast<char*>(ctx->d_stage[b]) + ctx->stage_off[j];
    CK(ctx, cudaMemcpyAsync(dst, hc[j], static_cast<size_t>(rows) * eb, cudaMemcpyHostToDevice, ctx->copy_stream));
    dcols[j] = dst;
  }
  CK(ctx, cudaEventRecord(ctx->ev_copied[b], ctx->copy_stream));
  CK(ctx, cudaStreamWaitEvent(st, ctx->ev_copied[b], 0));
  const stats_status s = launch_pass(ctx, dcols.data(), rows, st);
  if (s != STATS_OK) return s;
  CK(ctx, cudaEventRecord(ctx->ev_done[b], st));
  return STATS_OK;
}

}  // namespace

extern "C" {

stats_status stats_init(stats_ctx** out, const stats_config* cfg) { return create(out, cfg); }

stats_status stats_accumulate(stats_ctx* ctx, const void* const* dcols, int64_t nrows, void* stream) {
  stats_status s = check_sticky(ctx);
  if (s != STATS_OK) return s;
  if (nrows < 0 || (nrows > 0 && !dcols)) return STATS_EINVAL;
  for (int j = 0; j < ctx->p && nrows > 0; ++j)
    if (!dcols[j] || (reinterpret_cast<uintptr_t>(dcols[j]) % dtype_bytes(ctx->dtypes[j])) != 0)
      return STATS_EINVAL;
  return launch_pass(ctx, dcols, nrows, static_cast<cudaStream_t>(stream));
}

stats_status stats_accumulate_host(stats_ctx* ctx, const void* const* hcols, int64_t nrows, int64_t chunk_rows,
                                   void* stream) {
  stats_status s = check_sticky(ctx);
  if (s != STATS_OK) return s;
  if (nrows < 0 || chunk_rows < 0 || (nrows > 0 && !hcols)) return STATS_EINVAL;
  for (int j = 0; j < ctx->p && nrows > 0; ++j)
    if (!hcols[j]) return STATS_EINVAL;
  if (nrows == 0) return STATS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (chunk_rows == 0) chunk_rows = kDefaultChunkRows;
  chunk_rows = (chunk_rows + 7) & ~int64_t(7);
  if (chunk_rows > nrows) chunk_rows = (nrows + 7) & ~int64_t(7);
  s = ensure_staging(ctx, chunk_rows);
  if (s != STATS_OK) return s;
  std::vector<const void*> hc(ctx->p);
  int64_t chunk = 0;
  for (int64_t r0 = 0; r0 < nrows; r0 += chunk_rows, ++chunk) {
    const int64_t rows = std::min(chunk_rows, nrows - r0);
    for (int j = 0; j < ctx->p; ++j)
      hc[j] = static_cast<const char*>(hcols[j]) + static_cast<size_t>(r0) * dtype_bytes(ctx->dtypes[j]);
    s = enqueue_chunk(ctx, static_cast<int>(chunk & 1), hc.data(), rows, st);
    if (s != STATS_OK) return s;
  }
  return STATS_OK;
}

stats_status stats_accumulate_file(stats_ctx* ctx, const char* path, int64_t row0, int64_t nrows,
                                   int64_t chunk_rows, void* stream) {
  stats_status s = check_sticky(ctx);
  if (s != STATS_OK) return s;
  if (!path || row0 < 0 || chunk_rows < 0) return STATS_EINVAL;
  FileInfo info;
  int fd = -1;
  s = file_open_checked(path, info, &fd);
  if (s != STATS_OK) return s;
  struct Closer {
    int fd;
    ~Closer() { close(fd); }
  } closer{fd};
  if (info.p != ctx->p) return STATS_EINVAL;
  for (int j = 0; j < ctx->p; ++j)
    if (info.dtypes[j] != ctx->dtypes[j]) return STATS_EINVAL;
  if (row0 > info.nrows) return STATS_EINVAL;
  if (nrows < 0) nrows = info.nrows - row0;
  if (nrows > info.nrows - row0) return STATS_EINVAL;
  if (nrows == 0) return STATS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (chunk_rows == 0) chunk_rows = int64_t(1) << 22;
  chunk_rows = (chunk_rows + 7) & ~int64_t(7);
  if (chunk_rows > nrows) chunk_rows = (nrows + 7) & ~int64_t(7);
  s = ensure_staging(ctx, chunk_rows);
  if (s != STATS_OK) return s;
  // pinned host chunks laid out like the device staging buffers
  size_t bytes = 0;
  for (int j = 0; j < ctx->p; ++j)
    bytes = std::max(bytes, ctx->stage_off[j] + ((static_cast<size_t>(chunk_rows) * dtype_bytes(ctx->dtypes[j]) + 255) / 256) * 256);
  if (ctx->h_stage_bytes < bytes) {
    for (int b = 0; b < 2; ++b) {
      CK(ctx, cudaEventSynchronize(ctx->ev_copied[b]));  // no copy still reads the old chunk
      if (ctx->h_stage[b]) CK(ctx, cudaFreeHost(ctx->h_stage[b]));
      ctx->h_stage[b] = nullptr;
    }
    ctx->h_stage_bytes = 0;
    for (int b = 0; b < 2; ++b) {
      const cudaError_t e = cudaHostAlloc(&ctx->h_stage[b], bytes, cudaHostAllocDefault);
      if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return STATS_ENOMEM;
      }
      CK(ctx, e);
    }
    ctx->h_stage_bytes = bytes;
  }
  std::vector<void*> hc(ctx->p);
  int64_t chunk = 0;
  for (int64_t r = 0; r < nrows; r += chunk_rows, ++chunk) {
    const int b = static_cast<int>(chunk & 1);
    const int64_t rows = std::min(chunk_rows, nrows - r);
    // host chunk b is refilled once the copies that last read it have run; meanwhile the
    // device copies and reduces the other chunk
    CK(ctx, cudaEventSynchronize(ctx->ev_copied[b]));
    for (int j = 0; j < ctx->p; ++j) hc[j] = static_cast<char*>(ctx->h_stage[b]) + ctx->stage_off[j];
    s = file_read_rows(fd, info, row0 + r, rows, hc.data());
    if (s != STATS_OK) return s;
    s = enqueue_chunk(ctx, b, hc.data(), rows, st);
    if (s != STATS_OK) return s;
  }
  return STATS_OK;
}

stats_status stats_accumulate_csv(stats_ctx* ctx, const char* path, int64_t skip_lines, int64_t chunk_bytes,
                                  int64_t* nrows, int64_t* bad_line, void* stream) {
  if (nrows) *nrows = 0;
  if (bad_line) *bad_line = -1;
  stats_status s = check_sticky(ctx);
  if (s != STATS_OK) return s;
  if (!path || skip_lines < 0 || chunk_bytes < 0) return STATS_EINVAL;
  if (chunk_bytes == 0) chunk_bytes = int64_t(64) << 20;
  chunk_bytes = std::max<int64_t>(chunk_bytes, 64);
  const int fd = open(path, O_RDONLY);
  if (fd < 0) return STATS_EIO;
  struct Closer {
    int fd;
    ~Closer() { close(fd); }
  } closer{fd};
  struct stat sb;
  if (fstat(fd, &sb) != 0) return STATS_EIO;
  const int64_t fsize = sb.st_size;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int k = ctx->p;
  // a record of k fields takes at least 2k bytes with its newline: the rows one chunk can hold
  const int64_t row_cap = chunk_bytes / (2 * k) + 1;
  s = ensure_staging(ctx, row_cap);
  if (s != STATS_OK) return s;
  // device: two text buffers, the parse scratch (every line of a chunk indexable), two column-pointer arrays
  const int64_t ends_cap = chunk_bytes / 2 + 2;
  const size_t text_bytes = (static_cast<size_t>(chunk_bytes) + 1 + 255) / 256 * 256;
  const size_t scr = csv_scratch_bytes(chunk_bytes + 1, ends_cap, k);
  char* dev = nullptr;
  char* host = nullptr;
  struct Frees {
    char** d;
    char** h;
    ~Frees() {
      if (*d) cudaFree(*d);
      if (*h) cudaFreeHost(*h);
    }
  } frees{&dev, &host};
  cudaError_t e = cudaMalloc(&dev, 2 * text_bytes + scr + 2 * 256 * sizeof(void*));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return STATS_ENOMEM;
  }
  CK(ctx, e);
  e = cudaHostAlloc(&host, 2 * text_bytes + 256, cudaHostAllocDefault);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return STATS_ENOMEM;
  }
  CK(ctx, e);
  char* d_text[2] = {dev, dev + text_bytes};
  char* h_text[2] = {host, host + text_bytes};
  struct Out {
    int64_t total;
    uint32_t status;
    uint32_t pad;
    unsigned long long bad;
  }* out = reinterpret_cast<Out*>(host + 2 * text_bytes);
  CsvScratch S;
  csv_scratch_carve(dev + 2 * text_bytes, chunk_bytes + 1, ends_cap, k, S);
  void** d_cols[2] = {reinterpret_cast<void**>(dev + 2 * text_bytes + scr),
                      reinterpret_cast<void**>(dev + 2 * text_bytes + scr) + 256};
  std::vector<void*> hc(2 * k);
  for (int b = 0; b < 2; ++b)
    for (int j = 0; j < k; ++j) hc[b * k + j] = static_cast<char*>(ctx->d_stage[b]) + ctx->stage_off[j];
  CK(ctx, cudaMemcpy(d_cols[0], hc.data(), sizeof(void*) * k, cudaMemcpyHostToDevice));
  CK(ctx, cudaMemcpy(d_cols[1], hc.data() + k, sizeof(void*) * k, cudaMemcpyHostToDevice));
  CK(ctx, cudaMemcpy(S.dts, ctx->dtypes.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice));

  // parallel read of [off, off + len) into buf
  auto read_span = [&](char* buf, int64_t len, int64_t off) -> bool {
    const int64_t piece = int64_t(8) << 20;
    const int nt = static_cast<int>(std::min<int64_t>(16, (len + piece - 1) / piece));
    if (nt <= 1) {
      int64_t done = 0;
      while (done < len) {
        const ssize_t r = pread(fd, buf + done, static_cast<size_t>(len - done), off + done);
        if (r <= 0) return false;
        done += r;
      }
      return true;
    }
    std::vector<char> ok(nt, 1);
    std::vector<std::thread> th;
    const int64_t per = (len + nt - 1) / nt;
    for (int i = 0; i < nt; ++i)
      th.emplace_back([&, i] {
        const int64_t a = std::min(len, i * per), z = std::min(len, a + per);
        int64_t done = a;
        while (done < z) {
          const ssize_t r = pread(fd, buf + done, static_cast<size_t>(z - done), off + done);
          if (r <= 0) {
            ok[i] = 0;
            return;
          }
          done += r;
        }
      });
    for (auto& x : th) x.join();
    for (int i = 0; i < nt; ++i)
      if (!ok[i]) return false;
    return true;
  };

  int64_t foff = 0;          // next file byte to read
  int64_t carry = 0;         // bytes of a cut line, at carry_ptr in the previous buffer
  const char* carry_ptr = nullptr;
  int64_t lines_before = 0;  // file lines before the current chunk's first parsed line
  int64_t skip = skip_lines;
  int64_t added = 0;
  std::vector<const void*> dc(k);
  for (int64_t chunk = 0; foff < fsize || carry > 0; ++chunk) {
    const int b = static_cast<int>(chunk & 1);
    // the copy that last read h_text[b] has run (its parse was waited for)
    CK(ctx, cudaEventSynchronize(ctx->ev_copied[b]));
    char* buf = h_text[b];
    if (carry > 0) memcpy(buf, carry_ptr, static_cast<size_t>(carry));
    int64_t len = carry;
    const int64_t want = std::min(chunk_bytes - len, fsize - foff);
    if (want > 0) {
      if (!read_span(buf + len, want, foff)) return STATS_EIO;
      foff += want;
      len += want;
    }
    int64_t whole;
    if (foff >= fsize) {  // the end of the file closes the last line
      if (len > 0 && buf[len - 1] != '\n') buf[len++] = '\n';
      whole = len;
      carry = 0;
    } else {
      whole = len;
      while (whole > 0 && buf[whole - 1] != '\n') --whole;
      if (whole == 0) {  // a line longer than a chunk
        if (bad_line) *bad_line = lines_before;
        return STATS_EFORMAT;
      }
      carry = len - whole;
      carry_ptr = buf + whole;
    }
    int64_t start = 0;
    while (skip > 0 && start < whole) {  // header lines
      const char* nl = static_cast<const char*>(memchr(buf + start, '\n', static_cast<size_t>(whole - start)));
      start = nl - buf + 1;
      --skip;
      ++lines_before;
    }
    if (start >= whole) continue;
    const int64_t nb = whole - start;
    CK(ctx, cudaMemcpyAsync(d_text[b], buf + start, static_cast<size_t>(nb), cudaMemcpyHostToDevice,
                            ctx->copy_stream));
    CK(ctx, cudaEventRecord(ctx->ev_copied[b], ctx->copy_stream));
    CK(ctx, cudaStreamWaitEvent(st, ctx->ev_copied[b], 0));
    CK(ctx, cudaStreamWaitEvent(st, ctx->ev_done[b], 0));  // the pass that last read staging buffer b
    S.cols = d_cols[b];
    CK(ctx, cudaMemsetAsync(S.status, 0, sizeof(uint32_t), st));
    CK(ctx, cudaMemsetAsync(S.bad, 0xFF, sizeof(unsigned long long), st));
    CK(ctx, launch_csv_lines(d_text[b], nb, S, st));
    CK(ctx, launch_csv_parse(d_text[b], S, k, row_cap, ctx->sms, st));
    CK(ctx, cudaMemcpyAsync(&out->total, S.total, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaMemcpyAsync(&out->status, S.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaMemcpyAsync(&out->bad, S.bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaStreamSynchronize(st));
    if (out->status) {
      if (bad_line) *bad_line = lines_before + static_cast<int64_t>(out->bad >> 2);
      if (nrows) *nrows = added;
      return (out->bad & kCsvFormat) ? STATS_EFORMAT : STATS_ERANGE;
    }
    if (out->total > row_cap) return STATS_EFORMAT;  // unreachable: some line would be too short
    for (int j = 0; j < k; ++j) dc[j] = hc[b * k + j];
    s = launch_pass(ctx, dc.data(), out->total, st);
    if (s != STATS_OK) return s;
    CK(ctx, cudaEventRecord(ctx->ev_done[b], st));
    lines_before += out->total;
    added += out->total;
  }
  if (nrows) *nrows = added;
  return STATS_OK;
}

}  // extern "C"

namespace {

// Device workspace of batched launches (table descriptors, column-pointer arrays,
// work units), grown as needed, one per device; batched calls are stream-ordered.
struct BatchWorkspace {
  void* dev = nullptr;
  size_t bytes = 0;
};
std::mutex g_batch_mu;
BatchWorkspace g_batch_ws[64];

constexpr int64_t kBatchRowsPerUnit = int64_t(1) << 20;  // rows one block takes in a batched launch

}  // namespace

extern "C" {

stats_status stats_accumulate_batched(stats_ctx* const* ctxs, int32_t ntables, const void* const* const* dcols,
                                      const int64_t* nrows, void* stream) {
  if (ntables < 0 || (ntables > 0 && (!ctxs || !dcols || !nrows))) return STATS_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // tables not on the split path go one by one through stats_accumulate; split tables of
  // up to 64 columns share the register-fragment launch, wider ones the tiled launch
  std::vector<int> split_idx;
  std::vector<Gram32Job> g32;
  std::vector<NarrowJob> narrow[2];  // by mode: BF16x3, BF16x4
  for (int t = 0; t < ntables; ++t) {
    stats_ctx* c = ctxs[t];
    stats_status s = check_sticky(c);
    if (s != STATS_OK) return s;
    if (nrows[t] < 0 || (nrows[t] > 0 && !dcols[t])) return STATS_EINVAL;
    if (nrows[t] == 0) continue;
    if (c->mode == STATS_BF16X3 || c->mode == STATS_BF16X4) {
      for (int j = 0; j < c->p; ++j)
        if (!dcols[t][j] || (reinterpret_cast<uintptr_t>(dcols[t][j]) & 3u)) return STATS_EINVAL;
      const bool x4 = split_x4(c, nrows[t]);
      if (c->p > 32 && c->p <= 64 && nrows[t] >= kNarrowBatchMinRows && narrow_eligible(c, dcols[t], nrows[t])) {
        narrow[x4 ? 1 : 0].push_back({c, dcols[t], nrows[t]});
        c->rows_enqueued += nrows[t];
      } else if (c->p <= 64) {
        g32.push_back({c, dcols[t], nrows[t], x4});
        c->rows_enqueued += nrows[t];
      } else if (wide_eligible(c, dcols[t], nrows[t])) {
        s = launch_pass(c, dcols[t], nrows[t], st);  // one tcgen05 launch per wide table
        if (s != STATS_OK) return s;
      } else {
        split_idx.push_back(t);
      }
    } else {
      s = stats_accumulate(c, dcols[t], nrows[t], stream);
      if (s != STATS_OK) return s;
    }
  }
  if (!g32.empty()) {
    stats_status s = run_gram32(g32, st);
    if (s != STATS_OK) return s;
  }
  for (int x4 = 0; x4 < 2; ++x4) {
    stats_status s = run_narrow_batch(narrow[x4], x4 == 1, st);
    if (s != STATS_OK) return s;
  }
  if (split_idx.empty()) return STATS_OK;
  int dev = 0;
  CK(ctxs[split_idx[0]], cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return STATS_EINVAL;
  // host image: descriptors, then column-pointer arrays, then units
  const size_t nt = split_idx.size();
  size_t ncolptr = 0;
  for (int t : split_idx) ncolptr += ctxs[t]->p;
  std::vector<SplitParams> descs(nt);
  std::vector<const float*> colptrs(ncolptr);
  std::vector<int2> units[2][2];  // [T == 64][x4]
  std::vector<int64_t> unit_rows[2][2];
  const size_t off_cols = ((nt * sizeof(SplitParams) + 255) / 256) * 256;
  const size_t off_units = off_cols + ((ncolptr * sizeof(void*) + 255) / 256) * 256;
  std::vector<int> need_shift;  // descriptors whose table gets its pivot in this call
  std::lock_guard<std::mutex> lk(g_batch_mu);
  BatchWorkspace& ws = g_batch_ws[dev];
  size_t total_units = 0;
  size_t cp = 0;
  for (size_t i = 0; i < nt; ++i) {
    const int t = split_idx[i];
    stats_ctx* c = ctxs[t];
    SplitParams& S = descs[i];
    S = SplitParams{};
    S.p = c->p;
    S.shift = c->d_fshift;
    const int T = split_tile(c->p);
    S.nblk = (c->p + T - 1) / T;
    S.ntiles = S.nblk * (S.nblk + 1) / 2;
    S.ksplit = static_cast<int>(std::max<int64_t>(1, (nrows[t] + kBatchRowsPerUnit - 1) / kBatchRowsPerUnit));
    const int g = S.ntiles * S.ksplit;
    if (!c->d_split_slots || c->split_grid < g) {
      if (c->d_split_slots) CK(c, cudaFree(c->d_split_slots));
      c->d_split_slots = nullptr;
      const size_t bytes = split_slot_floats(g) * sizeof(float) + 256;
      CK(c, cudaMalloc(&c->d_split_slots, bytes));
      CK(c, cudaMemset(c->d_split_slots, 0, bytes));
      c->split_grid = g;
      c->d_split_ticket = reinterpret_cast<unsigned int*>(c->d_split_slots + split_slot_floats(g));
    }
    S.flush_rows = c->flush_rows > 0 ? c->flush_rows : 1024;
    S.nrows = nrows[t];
    S.slots = c->d_split_slots;
    S.ticket = c->d_split_ticket;
    S.acc_s = c->d_fs;
    S.acc_s_lo = c->d_fs_lo;
    S.acc_S = c->d_fS;
    S.acc_S_lo = c->d_fS_lo;
    S.acc_n = c->d_fn;
    S.shift_d = c->d_shift;
    if (!c->shift_set) need_shift.push_back(static_cast<int>(i));
    for (int j = 0; j < c->p; ++j) colptrs[cp + j] = static_cast<const float*>(dcols[t][j]);
    cp += c->p;
    const int a = T == 64 ? 1 : 0, b = split_x4(c, nrows[t]) ? 1 : 0;
    c->rows_enqueued += nrows[t];
    for (int u = 0; u < g; ++u) {
      units[a][b].push_back(make_int2(static_cast<int>(i), u));
      unit_rows[a][b].push_back(nrows[t] / S.ksplit);
    }
    total_units += g;
  }
  const size_t off_which = off_units + ((total_units * sizeof(int2) + 255) / 256) * 256;
  const size_t need = off_which + need_shift.size() * sizeof(int) + 256;
  if (ws.bytes < need) {
    if (ws.dev) CK(ctxs[split_idx[0]], cudaFree(ws.dev));
    ws.dev = nullptr;
    ws.bytes = 0;
    CK(ctxs[split_idx[0]], cudaMalloc(&ws.dev, need));
    ws.bytes = need;
  }
  char* base = static_cast<char*>(ws.dev);
  // device column-pointer arrays, then descriptors pointing at them
  cp = 0;
  for (size_t i = 0; i < nt; ++i) {
    descs[i].col_ptrs = reinterpret_cast<const float* const*>(base + off_cols) + cp;
    cp += descs[i].p;
  }
  // units, grouped by (T, mode), larger row ranges first
  std::vector<int2> all_units;
  size_t group_off[2][2], group_n[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      std::vector<size_t> order(units[a][b].size());
      for (size_t k = 0; k < order.size(); ++k) order[k] = k;
      std::stable_sort(order.begin(), order.end(),
                       [&](size_t x, size_t y) { return unit_rows[a][b][x] > unit_rows[a][b][y]; });
      group_off[a][b] = all_units.size();
      group_n[a][b] = order.size();
      for (size_t k : order) all_units.push_back(units[a][b][k]);
    }
  stats_ctx* c0 = ctxs[split_idx[0]];
  CK(c0, cudaMemcpyAsync(base, descs.data(), nt * sizeof(SplitParams), cudaMemcpyHostToDevice, st));
  CK(c0, cudaMemcpyAsync(base + off_cols, colptrs.data(), ncolptr * sizeof(void*), cudaMemcpyHostToDevice, st));
  CK(c0, cudaMemcpyAsync(base + off_units, all_units.data(), all_units.size() * sizeof(int2), cudaMemcpyHostToDevice,
                         st));
  // pivots of tables seen for the first time: one launch for all of them
  if (!need_shift.empty()) {
    CK(c0, cudaMemcpyAsync(base + off_which, need_shift.data(), need_shift.size() * sizeof(int),
                           cudaMemcpyHostToDevice, st));
    CK(c0, launch_split_shift_batched(reinterpret_cast<const SplitParams*>(base),
                                      reinterpret_cast<const int*>(base + off_which),
                                      static_cast<int>(need_shift.size()), st));
    for (int i : need_shift) ctxs[split_idx[i]]->shift_set = true;
  }
  const SplitParams* dtabs = reinterpret_cast<const SplitParams*>(base);
  const int2* dunits = reinterpret_cast<const int2*>(base + off_units);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      if (group_n[a][b])
        CK(c0, launch_split_batched(dtabs, dunits + group_off[a][b], static_cast<int>(group_n[a][b]), a ? 64 : 32,
                                    b == 1, st));
  for (int t : split_idx) ctxs[t]->last = st;
  return STATS_OK;
}

stats_status stats_merge(stats_ctx* dst, const stats_ctx* src) {
  stats_status s = check_sticky(dst);
  if (s != STATS_OK) return s;
  if (!src || src->sticky != STATS_OK) return src ? STATS_ESTATE : STATS_EINVAL;
  if (dst->p != src->p || dst->mode != src->mode || dst->dtypes != src->dtypes || dst->ident != src->ident)
    return STATS_EINVAL;
  if (dst->mode == STATS_EXACT) {
    for (int j = 0; j < dst->p; ++j)
      if (dst->plan[j].off != src->plan[j].off || dst->plan[j].k != src->plan[j].k ||
          dst->plan[j].shift != src->plan[j].shift || dst->plan[j].is_signed != src->plan[j].is_signed)
        return STATS_EINVAL;
  }
  const bool shifted = dst->mode == STATS_FP64_SHIFTED || dst->mode == STATS_BF16X3 || dst->mode == STATS_BF16X4 ||
                       dst->mode == STATS_FP32;
  if (src->last) CK(dst, cudaStreamSynchronize(src->last));
  stats_ctx* srcm = const_cast<stats_ctx*>(src);
  // carry src's device error bits over
  unsigned int bits = 0;
  CK(dst, cudaMemcpy(&bits, srcm->d_status, sizeof(bits), cudaMemcpyDeviceToHost));
  if (bits) {
    unsigned int mine = 0;
    CK(dst, cudaMemcpy(&mine, dst->d_status, sizeof(mine), cudaMemcpyDeviceToHost));
    mine |= bits;
    CK(dst, cudaMemcpy(dst->d_status, &mine, sizeof(mine), cudaMemcpyHostToDevice));
  }
  cudaStream_t st = dst->last;
  dst->rows_enqueued += src->rows_enqueued;
  if (shifted && !src->shift_set) return STATS_OK;  // src holds no rows
  if (shifted && dst->shift_set) {
    // the two ctxs generally have different pivots: re-express src about dst's pivot
    CK(dst, launch_merge_shifted(dst->d_fs, dst->d_fs_lo, dst->d_fS, dst->d_fS_lo, dst->d_shift, src->d_fs,
                                 src->d_fs_lo, src->d_fS, src->d_fS_lo, src->d_shift, src->d_fn, dst->p, st));
    CK(dst, launch_merge_i64(dst->d_fn, src->d_fn, 1, st));
    return STATS_OK;
  }
  if (shifted) {  // dst holds no rows yet: take src's pivot
    CK(dst, cudaMemcpyAsync(dst->d_shift, src->d_shift, dst->p * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (dst->d_fshift && src->d_fshift)
      CK(dst, cudaMemcpyAsync(dst->d_fshift, src->d_fshift, dst->p * sizeof(float), cudaMemcpyDeviceToDevice, st));
    dst->shift_set = true;
  }
  if (dst->mode == STATS_EXACT) {
    CK(dst, launch_merge_i64(dst->d_g, src->d_g, kDigits * kDigits, st));
  } else {
    const int T = dst->p * (dst->p + 1) / 2;
    CK(dst, launch_merge_dd(dst->d_fs, dst->d_fs_lo, src->d_fs, src->d_fs_lo, dst->p, st));
    CK(dst, launch_merge_dd(dst->d_fS, dst->d_fS_lo, src->d_fS, src->d_fS_lo, T, st));
    CK(dst, launch_merge_i64(dst->d_fn, src->d_fn, 1, st));
  }
  return STATS_OK;
}

stats_status stats_sync(stats_ctx* ctx) {
  stats_status s = check_sticky(ctx);
  if (s != STATS_OK) return s;
  CK(ctx, cudaStreamSynchronize(ctx->last));
  if (ctx->copy_stream) CK(ctx, cudaStreamSynchronize(ctx->copy_stream));
  return device_status(ctx);
}

stats_status stats_reset(stats_ctx* ctx) {
  stats_status s = check_sticky(ctx);
  if (s != STATS_OK) return s;
  // stream-ordered: work already enqueued on the ctx's stream completes first
  cudaStream_t st = ctx->last;
  if (ctx->mode == STATS_EXACT) {
    CK(ctx, cudaMemsetAsync(ctx->d_g, 0, kDigits * kDigits * sizeof(long long), st));
  } else {
    const size_t T = static_cast<size_t>(ctx->p) * (ctx->p + 1) / 2;
    CK(ctx, cudaMemsetAsync(ctx->d_fs, 0, (2 * ctx->p + 2 * T + ctx->p + 2) * sizeof(double), st));
    ctx->shift_set = false;
  }
  CK(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned int), st));
  ctx->rows_enqueued = 0;
  return STATS_OK;
}

stats_status stats_raw(stats_ctx* ctx, int64_t* n, double* s, double* S_upper, stats_i128* s_exact,
                       stats_i128* S_exact_upper) {
  stats_status st = stats_sync(ctx);
  if (st != STATS_OK) return st;
  st = run_finalize(ctx, 0, 0);
  if (st != STATS_OK) return st;
  const FinalLayout& L = ctx->lay;
  const double* h = ctx->h_out;
  const int p = ctx->p;
  const int T = p * (p + 1) / 2;
  if (n) memcpy(n, h + L.n, sizeof(int64_t));
  if (s) memcpy(s, h + L.s, sizeof(double) * p);
  if (S_upper) memcpy(S_upper, h + L.S, sizeof(double) * T);
  if (s_exact) memcpy(s_exact, h + L.s_ex, sizeof(stats_i128) * p);
  if (S_exact_upper) memcpy(S_exact_upper, h + L.S_ex, sizeof(stats_i128) * T);
  return h[L.flags] != 0.0 ? STATS_EOVERFLOW : STATS_OK;
}

stats_status stats_finalize(stats_ctx* ctx, double* mean, double* cov, double* corr, double* evals, double* evecs,
                            int32_t pca_on) {
  return stats_finalize_warm(ctx, mean, cov, corr, evals, evecs, pca_on, nullptr, nullptr);
}

stats_status stats_finalize_warm(stats_ctx* ctx, double* mean, double* cov, double* corr, double* evals,
                                 double* evecs, int32_t pca_on, const double* evecs_prev, int32_t* sweeps) {
  if (sweeps) *sweeps = -1;
  stats_status st = stats_sync(ctx);
  if (st != STATS_OK) return st;
  if (pca_on != 0 && pca_on != 1) return STATS_EINVAL;
  // the row count decides whether a covariance exists
  int64_t n = 0;
  if (ctx->mode == STATS_EXACT) {
    CK(ctx, cudaMemcpy(&n, ctx->d_g, sizeof(n), cudaMemcpyDeviceToHost));
  } else {
    CK(ctx, cudaMemcpy(&n, ctx->d_fn, sizeof(n), cudaMemcpyDeviceToHost));
  }
  if (n < 2) return STATS_EINVAL;
  st = run_finalize(ctx, (evals || evecs) ? 1 : 0, pca_on, (evals || evecs) ? evecs_prev : nullptr);
  if (st != STATS_OK) return st;
  const FinalLayout& L = ctx->lay;
  const double* h = ctx->h_out;
  const size_t pa = ctx->pa;
  if (sweeps && h[L.flags + 3] != 0.0) *sweeps = static_cast<int32_t>(h[L.flags + 2]);
  if (mean) memcpy(mean, h + L.mean, sizeof(double) * pa);
  if (cov) memcpy(cov, h + L.cov, sizeof(double) * pa * pa);
  if (corr) memcpy(corr, h + L.corr, sizeof(double) * pa * pa);
  if (evals) memcpy(evals, h + L.evals, sizeof(double) * pa);
  if (evecs) memcpy(evecs, h + L.evecs, sizeof(double) * pa * pa);
  return STATS_OK;
}

stats_status stats_finalize_batched(stats_ctx* const* ctxs, int32_t count, int32_t pca_on, double* const* mean,
                                    double* const* cov, double* const* corr, double* const* evals,
                                    double* const* evecs) {
  if (count < 0 || (count > 0 && !ctxs) || (pca_on != 0 && pca_on != 1)) return STATS_EINVAL;
  if (count == 0) return STATS_OK;
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i]) return STATS_EINVAL;
    stats_status st = stats_sync(ctxs[i]);
    if (st != STATS_OK) return st;
  }
  const bool want_pca = evals || evecs;
  std::vector<FinalParams> params(count);
  std::vector<size_t> off(count);
  size_t total = 0;
  for (int i = 0; i < count; ++i) {
    off[i] = total;
    total += static_cast<size_t>(ctxs[i]->lay.total);
  }
  stats_ctx* c0 = ctxs[0];
  const size_t pbytes = round256(count * sizeof(FinalParams));
  void* dbuf = nullptr;
  CK(c0, cudaMalloc(&dbuf, pbytes + total * sizeof(double)));
  double* dout = reinterpret_cast<double*>(static_cast<char*>(dbuf) + pbytes);
  for (int i = 0; i < count; ++i) {
    build_final_params(ctxs[i], want_pca ? 1 : 0, pca_on, params[i]);
    params[i].out = dout + off[i];  // the work scratch stays per context
  }
  std::vector<double> h(total);
  cudaError_t e = cudaMemcpy(dbuf, params.data(), count * sizeof(FinalParams), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_finalize_batched(reinterpret_cast<const FinalParams*>(dbuf), count, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(h.data(), dout, total * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(dbuf);
  if (e != cudaSuccess) return cuda_fail(c0, e);
  stats_status ret = STATS_OK;
  for (int i = 0; i < count; ++i) {
    const stats_ctx* c = ctxs[i];
    const double* r = h.data() + off[i];
    const FinalLayout& L = c->lay;
    const size_t pa = c->pa;
    int64_t nrows = 0;
    memcpy(&nrows, r + L.n, sizeof(nrows));  // the row count is stored as an integer
    if (nrows < 2) {  // no covariance for fewer than two rows
      ret = STATS_EINVAL;
      continue;
    }
    if (mean && mean[i]) memcpy(mean[i], r + L.mean, sizeof(double) * pa);
    if (cov && cov[i]) memcpy(cov[i], r + L.cov, sizeof(double) * pa * pa);
    if (corr && corr[i]) memcpy(corr[i], r + L.corr, sizeof(double) * pa * pa);
    if (evals && evals[i]) memcpy(evals[i], r + L.evals, sizeof(double) * pa);
    if (evecs && evecs[i]) memcpy(evecs[i], r + L.evecs, sizeof(double) * pa * pa);
  }
  return ret;
}

// Checkpoint image: magic, version, p, mode, has_bounds, dtypes, ident, lo, hi,
// shift_set, then the accumulator words.
stats_status stats_export(stats_ctx* ctx, void* buf, size_t* len) {
  if (!len) return STATS_EINVAL;
  stats_status st = stats_sync(ctx);
  if (st != STATS_OK) return st;
  const int p = ctx->p;
  const size_t T = static_cast<size_t>(p) * (p + 1) / 2;
  const size_t acc_bytes = ctx->mode == STATS_EXACT ? kDigits * kDigits * sizeof(long long)
                                                    : (2 * p + 2 * T + p + 1) * sizeof(double);
  const size_t need = 8 + 4 * 4 + p * 4 + p + 2 * p * 8 + 4 + acc_bytes;
  if (!buf || *len < need) {
    *len = need;
    return buf ? STATS_EINVAL : STATS_OK;
  }
  char* w = static_cast<char*>(buf);
  auto put = [&](const void* src, size_t n) {
    memcpy(w, src, n);
    w += n;
  };
  const int32_t version = 1, mode = ctx->mode, hb = ctx->has_bounds ? 1 : 0, ss = ctx->shift_set ? 1 : 0;
  put(&kMagic, 8);
  put(&version, 4);
  put(&p, 4);
  put(&mode, 4);
  put(&hb, 4);
  put(ctx->dtypes.data(), 4 * p);
  put(ctx->ident.data(), p);
  std::vector<double> lo(p, 0.0), hi(p, 0.0);
  if (ctx->has_bounds) {
    lo = ctx->lo;
    hi = ctx->hi;
  }
  put(lo.data(), 8 * p);
  put(hi.data(), 8 * p);
  put(&ss, 4);
  if (ctx->mode == STATS_EXACT) {
    CK(ctx, cudaMemcpy(w, ctx->d_g, acc_bytes, cudaMemcpyDeviceToHost));
  } else {
    CK(ctx, cudaMemcpy(w, ctx->d_fs, acc_bytes, cudaMemcpyDeviceToHost));
  }
  *len = need;
  return STATS_OK;
}

stats_status stats_import(stats_ctx** out, const void* buf, size_t len) {
  if (!out || !buf || len < 28) return STATS_EINVAL;
  const char* r = static_cast<const char*>(buf);
  const char* end = r + len;
  auto get = [&](void* dst, size_t n) -> bool {
    if (r + n > end) return false;
    memcpy(dst, r, n);
    r += n;
    return true;
  };
  uint64_t magic = 0;
  int32_t version = 0, p = 0, mode = 0, hb = 0, ss = 0;
  if (!get(&magic, 8) || magic != kMagic || !get(&version, 4) || version != 1 || !get(&p, 4) || !get(&mode, 4) ||
      !get(&hb, 4))
    return STATS_EINVAL;
  if (p < 1 || p > STATS_MAX_P) return STATS_EINVAL;
  std::vector<int32_t> dt(p);
  std::vector<uint8_t> id(p);
  std::vector<double> lo(p), hi(p);
  if (!get(dt.data(), 4 * p) || !get(id.data(), p) || !get(lo.data(), 8 * p) || !get(hi.data(), 8 * p) ||
      !get(&ss, 4))
    return STATS_EINVAL;
  stats_config cfg{p, dt.data(), id.data(), hb ? lo.data() : nullptr, hb ? hi.data() : nullptr, mode};
  stats_ctx* c = nullptr;
  stats_status st = stats_init(&c, &cfg);
  if (st != STATS_OK) return st;
  const size_t T = static_cast<size_t>(p) * (p + 1) / 2;
  const size_t acc_bytes = mode == STATS_EXACT ? kDigits * kDigits * sizeof(long long)
                                               : (2 * p + 2 * T + p + 1) * sizeof(double);
  if (r + acc_bytes > end) {
    stats_destroy(c);
    return STATS_EINVAL;
  }
  cudaError_t e = cudaMemcpy(mode == STATS_EXACT ? static_cast<void*>(c->d_g) : static_cast<void*>(c->d_fs), r,
                             acc_bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    stats_destroy(c);
    return STATS_ECUDA;
  }
  if (mode != STATS_EXACT) memcpy(&c->rows_enqueued, r + (2 * p + 2 * T + p) * sizeof(double), sizeof(int64_t));
  c->shift_set = ss != 0;
  if (c->shift_set && c->d_fshift) {  // the split kernels' float copy of the pivot
    e = launch_pivot_to_float(c->d_shift, c->d_fshift, p, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      stats_destroy(c);
      return STATS_ECUDA;
    }
  }
  *out = c;
  return STATS_OK;
}

void stats_destroy(stats_ctx* ctx) {
  if (!ctx) return;
  if (ctx->last) cudaStreamSynchronize(ctx->last);
  if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
  free_ctx(ctx);
}

const char* stats_strerror(stats_status st) {
  switch (st) {
    case STATS_OK: return "ok";
    case STATS_EINVAL: return "invalid argument or configuration";
    case STATS_ENOMEM: return "out of memory";
    case STATS_ECUDA: return "CUDA runtime error";
    case STATS_EOVERFLOW: return "exact result does not fit its output type";
    case STATS_ETIMEOUT: return "a bounded device-side wait expired";
    case STATS_ESTATE: return "context failed earlier or call out of order";
    case STATS_ERANGE: return "a value lay outside its declared range or column type";
    case STATS_EIO: return "a file could not be opened, read or written";
    case STATS_EFORMAT: return "malformed input (table file header, layout or size; or CSV text)";
    case STATS_EMISMATCH: return "a sampled file row differs from its source";
    default: return "unknown status";
  }
}

int32_t stats_num_analysis_columns(const stats_ctx* ctx) { return ctx ? ctx->pa : -1; }

stats_status stats_set_batch_tuning(int32_t width, int32_t mode, const stats_batch_tuning* t) {
  if (!t || width < 1 || width > 64 || (mode != STATS_BF16X3 && mode != STATS_BF16X4) || !valid_tuning(*t))
    return STATS_EINVAL;
  (void)batch_tuning(width, mode == STATS_BF16X4);  // defaults in place first
  std::lock_guard<std::mutex> lk(g_batch_tuning_mu);
  g_batch_tuning[width_class(width)][mode == STATS_BF16X4 ? 1 : 0] = *t;
  return STATS_OK;
}

stats_status stats_get_batch_tuning(int32_t width, int32_t mode, stats_batch_tuning* t) {
  if (!t || width < 1 || width > 64 || (mode != STATS_BF16X3 && mode != STATS_BF16X4)) return STATS_EINVAL;
  *t = batch_tuning(width, mode == STATS_BF16X4);
  return STATS_OK;
}

stats_status stats_set_grid_wait(stats_ctx* ctx, int64_t wait_ns, int32_t absent_block) {
  if (!ctx || wait_ns < 0 || wait_ns > int64_t(60) * 1000000000 || absent_block < -1) return STATS_EINVAL;
  ctx->grid_wait_ns = wait_ns;
  ctx->grid_absent_block = absent_block;
  return STATS_OK;
}

stats_status stats_set_wide_pairs(stats_ctx* ctx, int32_t pairs) {
  if (!ctx || (pairs != 0 && pairs != 1)) return STATS_EINVAL;
  ctx->wide_pairs = pairs;
  return STATS_OK;
}

stats_status stats_set_exact_shape(stats_ctx* ctx, int32_t shape) {
  if (!ctx || shape < -1 || shape >= kExactShapes) return STATS_EINVAL;
  if (ctx->mode == STATS_EXACT && shape >= 0) {
    ExactParams P = ctx->xp;
    if (!exact_layout(P, shape)) return STATS_EINVAL;
  }
  ctx->exact_shape = shape;
  return STATS_OK;
}

stats_status stats_set_grid(stats_ctx* ctx, int32_t blocks) {
  if (!ctx || blocks < 0) return STATS_EINVAL;
  ctx->grid = blocks;
  return STATS_OK;
}

stats_status stats_set_flush_rows(stats_ctx* ctx, int32_t rows) {
  if (!ctx || rows < 16 || rows > 4096 || (rows & 15)) return STATS_EINVAL;
  ctx->flush_rows = rows;
  return STATS_OK;
}

int32_t stats_table1_row_bytes(int32_t layout) {
  return layout == STATS_T1_L32 ? 60 : layout == STATS_T1_L16 ? 44 : 0;
}

stats_status stats_table1_config(int32_t layout, int64_t max_rows, int32_t* dtypes, uint8_t* is_identifier,
                                 double* lo, double* hi) {
  if (layout != STATS_T1_L32 && layout != STATS_T1_L16) return STATS_EINVAL;
  if (max_rows < 1 || max_rows >= (int64_t(1) << 40)) return STATS_EINVAL;
  static const int32_t l32[12] = {I64, I32, I32, I32, I32, I32, I32, I32, F64, I32, F64, I32};
  static const int32_t l16[12] = {I64, I16, I16, I16, I16, I32, I16, I16, F64, I16, F64, I16};
  // value ranges produced by the Table 1 formulas: |cotC| <= |cot 3| = 7.0153, J <= |tan 11| = 225.951
  const double rlo[12] = {1, 3, 1, 1, 0, 0, 0, 0, -7.1, 0, 0, 0};
  const double rhi[12] = {static_cast<double>(max_rows), 8, 10, 100, 255, 65535, 100, 100, 7.1, 65535, 226, 100};
  for (int j = 0; j < 12; ++j) {
    if (dtypes) dtypes[j] = layout == STATS_T1_L32 ? l32[j] : l16[j];
    if (is_identifier) is_identifier[j] = j == 0 ? 1 : 0;
    if (lo) lo[j] = rlo[j];
    if (hi) hi[j] = rhi[j];
  }
  return STATS_OK;
}

stats_status stats_gen_table1(uint64_t seed, uint64_t row0, int64_t nrows, int32_t layout, void* const* dcols,
                              void* stream) {
  if (layout != STATS_T1_L32 && layout != STATS_T1_L16) return STATS_EINVAL;
  if (nrows < 0 || (nrows > 0 && !dcols)) return STATS_EINVAL;
  if (nrows == 0) return STATS_OK;
  for (int j = 0; j < 12; ++j)
    if (!dcols[j] || !aligned16(dcols[j])) return STATS_EINVAL;
  cudaError_t e = launch_gen_table1(seed, row0, nrows, layout, dcols, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? STATS_OK : STATS_ECUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The no-allocation entry point.
//
// Some callers cannot allocate device memory.  A serving process or framework that
// takes the GPU's memory up front into its own pool forbids libraries to call
// cudaMalloc behind its back (an allocation outside the pool can fail, or steal
// memory the pool has promised elsewhere); code that must not block, such as a
// latency-critical loop, cannot afford cudaMalloc / cudaFree either, since
// cudaFree synchronises the device.  Such callers can still run the exact pass
// through stats_pass_noalloc: it takes no context, and its scratch -- the digit
// Gram of one call, the per-call staging accumulator and the ticket / error /
// status words -- lives in the file-scope device array below (16,640 bytes, held
// by every GPU that loads the library until the process exits).  The caller
// passes the inputs and the result buffer.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoallocWords = 2 * kDigits * kDigits + 32;  // 16,640 bytes
// A digit pair sums at most 2^46 products of two digits below 256: 2^46 * 255^2 < 2^62
constexpr int64_t kNoallocMaxRows = int64_t(1) << 46;

__device__ __align__(256) unsigned long long g_noalloc_scratch[kNoallocWords];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};

// Device address of the scratch array on the current device, looked up once per
// device (a host-side reference to the array is not a device address).  The address
// belongs to the device's primary context: after cudaDeviceReset it is stale, as are
// every context and device pointer of this library on that device.
cudaError_t noalloc_scratch(unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = p;
  }
  *out = static_cast<unsigned long long*>(g_noalloc_addr[dev]);
  return cudaSuccess;
}

}  // namespace

extern "C" stats_status stats_pass_noalloc(const stats_config* cfg, const void* const* dcols, int64_t nrows,
                                           void* d_result, void* stream) {
  if (!cfg || !cfg->dtypes || cfg->mode != STATS_EXACT || cfg->p < 1 || cfg->p > kMaxCols) return STATS_EINVAL;
  if ((cfg->lo == nullptr) != (cfg->hi == nullptr)) return STATS_EINVAL;
  if (nrows < 0 || nrows > kNoallocMaxRows) return STATS_EINVAL;
  if (!d_result || (reinterpret_cast<uintptr_t>(d_result) & 7u)) return STATS_EINVAL;
  if (nrows > 0 && !dcols) return STATS_EINVAL;
  for (int j = 0; j < cfg->p && nrows > 0; ++j)
    if (!dcols[j] || (reinterpret_cast<uintptr_t>(dcols[j]) % dtype_bytes(cfg->dtypes[j])) != 0)
      return STATS_EINVAL;
  ColPlan cp[kMaxCols];
  ExactParams P{};
  int conv = CONV_GENERIC;
  stats_status s = exact_plan(cfg->p, cfg->dtypes, cfg->lo != nullptr, cfg->lo, cfg->hi, cp, P, conv);
  if (s != STATS_OK) return s;
  unsigned long long* scratch = nullptr;
  if (noalloc_scratch(&scratch) != cudaSuccess) return STATS_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // every call shares the array: clear the accumulators and words that must start at zero
  if (cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * kNoallocWords, st) != cudaSuccess) return STATS_ECUDA;
  unsigned int* words = reinterpret_cast<unsigned int*>(scratch + 2 * kDigits * kDigits);
  P.call_acc = scratch;
  P.acc = reinterpret_cast<long long*>(scratch + kDigits * kDigits);
  P.ticket = words;
  P.err = words + 1;
  P.status = words + 2;
  if (nrows > 0) {
    P.direct = 0;
    for (int j = 0; j < cfg->p; ++j) {
      P.cols[j] = dcols[j];
      if (!aligned16(dcols[j])) P.direct = 1;
    }
    P.nrows = nrows;
    P.nmain = P.direct ? nrows : (nrows & ~int64_t(7));
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess) return STATS_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return STATS_ECUDA;
    const int per = std::max(1, exact_max_active_blocks(conv, P.shape, P.stages, P.stage_bytes));
    if (launch_exact(P, conv, std::max(sms, 1) * per, st) != cudaSuccess) return STATS_ECUDA;
  }
  // recombination into the caller's buffer (all columns flagged identifiers: raw outputs only)
  FinalParams F{};
  F.p = cfg->p;
  F.mode = 0;
  for (int j = 0; j < cfg->p; ++j) {
    F.col[j].off = cp[j].off;
    F.col[j].k = cp[j].k;
    F.col[j].shift = cp[j].shift;
    F.col[j].is_real = cp[j].is_real;
    F.col[j].is_ident = 1;
  }
  F.g = P.acc;
  F.out = static_cast<double*>(d_result);
  if (launch_finalize(F, st) != cudaSuccess) return STATS_ECUDA;
  const FinalLayout L = final_layout(cfg->p, 0);
  double* status_slot = static_cast<double*>(d_result) + L.flags + 4;
  if (cudaMemsetAsync(status_slot, 0, sizeof(double), st) != cudaSuccess) return STATS_ECUDA;
  if (cudaMemcpyAsync(status_slot, P.status, sizeof(unsigned int), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return STATS_ECUDA;
  return STATS_OK;
}
