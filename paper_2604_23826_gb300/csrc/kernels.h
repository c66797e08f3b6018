// kernels.h -- host-side launch interface between the C-ABI layer (api.cu) and
// the kernel translation units.  Internal to libsuffstats.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ss {

// Status bits written by kernels into a device status word; the host maps them
// to stats_status codes at the next synchronising call.
enum : uint32_t {
  DEV_ERANGE = 1u,    // a value lay outside the digit field of its declared range
  DEV_ETIMEOUT = 2u,  // a bounded wait (mbarrier) expired
  DEV_EOVERFLOW = 4u  // an exact result does not fit its output type
};

constexpr int kPivotRows = 64;  // shifted modes: the pivot is the mean of a table's first rows
constexpr int kMaxCols = 16;     // columns of the EXACT pass
constexpr int kDigits = 32;      // digit slots of the EXACT pass (ones column included)
constexpr int kDigitPairs = kDigits / 2;

enum Dtype : int32_t { I16 = 0, I32 = 1, I64 = 2, F32 = 3, F64 = 4 };

inline int dtype_bytes(int32_t dt) { return dt == I16 ? 2 : (dt == I32 || dt == F32) ? 4 : 8; }

// Which converter the EXACT pass uses for a row.
enum ExactConv : int32_t { CONV_GENERIC = 0, CONV_T1_L32 = 1, CONV_T1_L16 = 2 };

// Parameters of one launch of the EXACT pass (passed by value as a kernel parameter).
struct ExactParams {
  const void* cols[kMaxCols];  // device column pointers, element 0 = first row of the call
  int32_t dtype[kMaxCols];
  int32_t col_off[kMaxCols];   // byte offset of each column inside a pipeline stage
  int32_t col_bytes[kMaxCols];
  int32_t real_shift[kMaxCols];  // real columns: q = RN(x * 2^shift)
  int32_t real_emax[kMaxCols];   // real columns: largest allowed biased exponent field
  int32_t kbytes[kMaxCols];      // digit bytes of the column's field
  int32_t is_signed[kMaxCols];   // field is two's complement (top byte signed)
  // Generic plan, per digit pair q: source column of the low / high digit
  // (-1 = the ones column, -2 = zero padding), its byte index, and whether it is
  // the signed top byte of its field.
  int8_t pc0[kDigitPairs], pb0[kDigitPairs], ps0[kDigitPairs];
  int8_t pc1[kDigitPairs], pb1[kDigitPairs], ps1[kDigitPairs];
  int32_t p;
  int32_t direct;       // 1: some column is not 16-byte aligned -- consumers read global memory directly
  int32_t shape;        // launch shape (0 .. kExactShapes - 1)
  int32_t stages;       // pipeline depth (2..kExactMaxStages)
  int32_t stage_bytes;  // bytes of one stage (multiple of 128)
  int64_t nrows;        // rows of this call
  int64_t nmain;        // rows moved by bulk copies (nrows rounded down to a multiple of 8)
  unsigned long long* call_acc;  // scratch: kDigits*kDigits int64, zero between calls
  unsigned int* ticket;          // scratch: block counter, zero between calls
  unsigned int* err;             // scratch: error bits of this call, zero between calls
  long long* acc;                // ctx accumulator: kDigits*kDigits int64 (entries r <= c valid)
  unsigned int* status;          // ctx sticky device status bits
};

// Launch shapes of the EXACT pass: converting warps (plus one producer warp) and rows each
// takes per stage (a multiple of 32).  One block per SM; the register budget falls with the
// thread count (128, 96 and 80 per thread for 16, 20 and 24 warps).  Shapes 0-2 multiply on
// the converting warps (mma.sync); shape 3 hands the digits to tcgen05 MMAs issued by one
// thread (plus an MMA warp and four tensor-memory reader warps: 20 warps, 96 registers).
constexpr int kExactShapes = 4;
__host__ __device__ constexpr int exact_shape_warps(int shape) {
  return shape == 0 ? 15 : shape == 1 ? 19 : shape == 2 ? 23 : 14;
}
__host__ __device__ constexpr int exact_shape_rpw(int shape) { return (shape == 0 || shape == 3) ? 64 : 32; }
__host__ __device__ constexpr bool exact_shape_tc(int shape) { return shape == 3; }
constexpr int kExactMaxStages = 6;
__host__ __device__ constexpr int exact_tile_rows(int shape) { return exact_shape_warps(shape) * exact_shape_rpw(shape); }
// Bytes one column of `elem_bytes`-byte values takes in a stage of `tile` rows (128-byte granules).
__host__ __device__ constexpr int stage_col_bytes(int elem_bytes, int tile) { return ((tile * elem_bytes + 127) / 128) * 128; }
size_t exact_smem_bytes(int shape, int stages, int stage_bytes);
// Deepest pipeline (2..kExactMaxStages stages) whose shared memory fits one block, or 0.
int exact_pick_stages(int shape, int stage_bytes);
// Stage layout of P's columns for a shape: col_off, stage_bytes, stages, shape (needs p and
// col_bytes); false when the shape does not fit.
bool exact_layout(ExactParams& P, int shape);
// Launch with at most max_grid blocks (fewer when the rows have fewer stages).
cudaError_t launch_exact(const ExactParams& P, int conv, int max_grid, cudaStream_t stream);
int exact_max_active_blocks(int conv, int shape, int stages, int stage_bytes);

// ---------------------------------------------------------------------------
// FP64 CUDA-core passes (raw or shifted), fixed-order merge of block slots.
// ---------------------------------------------------------------------------
struct Fp64Params {
  const void* cols[256];
  int32_t dtype[256];
  int32_t p;
  int64_t nrows;
  const double* shift;  // p values or nullptr (raw moments)
  double* slots;        // scratch: grid * (T(p) + p) doubles
  double* acc_s;        // ctx: p doubles (column sums, shifted when shift != nullptr)
  double* acc_S;        // ctx: T(p) doubles, packed upper
  double* acc_s_lo;     // ctx: p low parts (double-double)
  double* acc_S_lo;     // ctx: T(p) low parts
  long long* acc_n;     // ctx: row count
};
cudaError_t launch_fp64(const Fp64Params& P, int grid, cudaStream_t stream);
size_t fp64_slot_doubles(int grid);  // slots + ticket word, zeroed once at allocation
cudaError_t launch_set_shift(const void* const* cols, const int32_t* dtypes, int p, int64_t rows, double* shift,
                             cudaStream_t stream);

// ---------------------------------------------------------------------------
// FP32 tables on the tensor cores with a bf16 two-term split (BF16x3 / BF16x4).
// ---------------------------------------------------------------------------
struct SplitParams {
  const float* cols[256];          // single-table launches: the column pointers
  const float* const* col_ptrs;    // batched launches: device array of the column pointers
  const float* shift;   // p floats (device): pivot c_j
  int32_t p;
  int32_t nblk;         // ceil(p / T)
  int32_t ntiles;       // nblk (nblk + 1) / 2
  int32_t ksplit;       // row ranges per tile
  int32_t flush_rows;   // rows of a warp between FP32 -> (hi, lo) flushes
  int64_t nrows;
  float* slots;         // scratch: split_slot_floats(grid) floats
  unsigned int* ticket; // scratch: block counter, zero between calls
  double* acc_s;        // ctx accumulators (shifted sums), double-double
  double* acc_s_lo;
  double* acc_S;
  double* acc_S_lo;
  long long* acc_n;
  double* shift_d;      // batched launches: p doubles (device), the pivot as double for finalize
};
size_t split_slot_floats(int grid);
int split_tile(int p);  // T = 32 or 64
cudaError_t launch_split(const SplitParams& P, int T, bool x4, int grid, cudaStream_t stream);
// Pivot of a shifted context from its first call: the mean of its first min(rows, kPivotRows)
// rows (FP32 data: rounded to FP32, so that x - c is exact wherever Sterbenz's lemma holds).
cudaError_t launch_split_shift(const SplitParams& P, int64_t rows, double* shift_d, cudaStream_t stream);
// pivots of tabs[which[i]] for i < count, one block per table (batched launches)
cudaError_t launch_split_shift_batched(const SplitParams* tabs, const int* which, int count, cudaStream_t stream);
// units[i] = (index into tabs, local block of that table); all tables share T and the mode
cudaError_t launch_split_batched(const SplitParams* tabs, const int2* units, int nunits, int T, bool x4,
                                 cudaStream_t stream);

// ---------------------------------------------------------------------------
// FP32 tables of up to 64 columns, bf16 split on the tensor cores with register
// fragments (k_gram32.cu).  One launch (one CTA per SM, persistent) streams the
// stages of a list of tables; a small second launch adds each table's per-CTA
// slots, in slot order, into its accumulators.
// ---------------------------------------------------------------------------
constexpr int kGram32Warps = 15;        // most consumer warps per CTA (plus one producer warp)
constexpr int kGram32MaxTables = 4096;  // tables per launch
struct Gram32Table {
  const float* const* cols;  // device array of p column pointers
  const float* shift;        // p pivots (device)
  float* slots;              // nslots * gram32_slot_floats(P) floats of scratch
  double* acc_s;             // ctx accumulators (shifted), double-double
  double* acc_s_lo;
  double* acc_S;
  double* acc_S_lo;
  long long* acc_n;
  double* shift_d;           // p pivots as double (device), for finalize
  unsigned int* status;      // the ctx's device status word (DEV_* bits)
  const void* tmap;          // 2D tensor map of the columns (uniform stride), or null
  int64_t nrows;
  int32_t p;
  int32_t stage0;            // the table's first stage in the launch's stage list
  int32_t nslots;            // CTAs that take stages of the table: min(grid, chunks it overlaps)
  int32_t aligned;           // every column pointer 16-byte aligned
};
struct Gram32Launch {
  const Gram32Table* tabs;
  float* warp_scratch;       // grid * kGram32Warps * gram32_slot_floats(P) floats
  int32_t ntables;
  int32_t total_stages;
  int32_t chunk;             // consecutive stages dealt to one CTA (chunk c goes to CTA c % grid)
  int32_t flush_kblocks;     // 16-row K blocks between FP32 -> (hi, lo) flushes
};
int gram32_width(int p);                 // P = 8, 16, 32 or 64
size_t gram32_slot_floats(int P);        // floats of one warp / unit slot
int gram32_rows_per_stage(int P);
cudaError_t launch_gram32(const Gram32Launch& L, int P, bool x4, int grid, cudaStream_t st);
// pivots (means of the first kPivotRows rows) of tabs[which[i]], i < count
cudaError_t launch_gram32_shift(const Gram32Table* tabs, const int* which, int count, cudaStream_t st);

// ---------------------------------------------------------------------------
// Wide FP32 tables (p > 64) on tcgen05 (k_wide.cu): 128 x 128 column-block units of
// the upper block triangle, one unit per CTA, CTAs per unit in proportion to the unit's
// work, a 3D tensor map over the columns (32-row lines, 64-row stages).
// ---------------------------------------------------------------------------
constexpr int kWideSlotPairs = 128 * 128 + 2 * 128;  // (hi, lo) pairs of a CTA's slot
constexpr int kWideMaxUnits = 64;                    // p <= 1280
struct WideParams {
  const void* tmap;          // 3D tensor map: dims (32, nrows / 32, p), box (32, 2, 128), 128-byte swizzle
  const float* base;         // column 0; column j at base + j * ld
  const float* shift;        // p pivots (device)
  float* slots;              // grid * kWideSlotPairs pairs of scratch
  double* acc_s;             // ctx accumulators (shifted), double-double
  double* acc_s_lo;
  double* acc_S;
  double* acc_S_lo;
  long long* acc_n;
  unsigned int* status;      // the ctx's device status word (DEV_* bits)
  int64_t nrows;
  int64_t ld;                // floats between consecutive columns (a multiple of 4)
  int64_t nfull;             // whole 32-row chunks (nrows / 32); the rest is read with plain loads
  int32_t p;
  int32_t nunits;
  int32_t flush_chains;      // 32-row MMA chains between FP32 -> (hi, lo) flushes
  int32_t unit_i[kWideMaxUnits], unit_j[kWideMaxUnits];
  int32_t unit_first[kWideMaxUnits], unit_ctas[kWideMaxUnits];  // CTAs [first, first + ctas) of each unit
};
// Units of the upper block triangle and their CTAs (in proportion to each unit's measured
// time per stage in the mode); returns the grid (at most sms), or 0 when p has more units
// than kWideMaxUnits or sms.
int wide_plan(int p, int sms, bool x4, WideParams& W);
int wide_rows_per_stage();
int wide_chunk_rows();
int wide_block_cols();
cudaError_t launch_wide(const WideParams& P, bool x4, int grid, cudaStream_t st);
// 129..256 columns on pairs of SMs (k_wide2.cu): cluster of two CTAs, CTA rank r converts
// column block r, the pair's leader issues cta_group::2 MMAs of M = N = 256.
constexpr int kWide2SlotPairs = 128 * 256 + 2 * 128;  // (hi, lo) pairs of a CTA's slot
struct Wide2Params {
  const void* tmap;          // 3D tensor map: dims (32, nrows / 32, p), box (32, 2, 128), 128-byte swizzle
  const float* base;         // column 0; column j at base + j * ld
  const float* shift;        // p pivots (device)
  float* slots;              // grid * kWide2SlotPairs pairs of scratch
  double* acc_s;             // ctx accumulators (shifted), double-double
  double* acc_s_lo;
  double* acc_S;
  double* acc_S_lo;
  long long* acc_n;
  unsigned int* status;      // the ctx's device status word (DEV_* bits)
  int64_t nrows;
  int64_t ld;                // floats between consecutive columns (a multiple of 4)
  int64_t nfull;             // whole 32-row chunks (nrows / 32); the rest is read with plain loads
  int32_t p;
  int32_t flush_stages;      // 64-row stages between FP32 -> (hi, lo) flushes
};
int wide2_grid(int sms);  // an even number of CTAs, at most sms
cudaError_t launch_wide2(const Wide2Params& P, bool x4, int grid, cudaStream_t st);
// 33..64 columns (k_narrow.cu): one 64-column block, h and l stacked into an M = 128 operand;
// WideParams with a single unit (0, 0) of `grid` CTAs, tmap boxed (32, 2, 64).
int narrow_cols();
int narrow_rows_per_stage();
// A table of a narrow launch: a [p, ld] block of FP32 columns, 33 <= p <= 64.
struct NarrowTab {
  const void* tmap;          // device copy of its 3D tensor map: dims (32, nrows / 32, p), box (32, 2, 64)
  const float* base;         // column 0; column j at base + j * ld
  float* shift;              // p pivots (FP32, device)
  double* shift_d;           // the same in FP64 (the ctx's shift vector)
  double* acc_s;             // ctx accumulators (shifted), double-double
  double* acc_s_lo;
  double* acc_S;
  double* acc_S_lo;
  long long* acc_n;
  int64_t nrows, ld, nfull;  // nfull: whole 32-row chunks; the rest is read with plain loads
  int32_t p, pad;
};
// A unit of work: 64-row stages [st0, st0 + nst) of table tab, reduced into slot `slot`
// (a table's units own consecutive slots, in row order).
struct NarrowUnit {
  int64_t st0;
  int32_t nst, tab, slot, pad;
};
struct NarrowParams {
  NarrowTab tab0;            // the table of a single-table launch (tabs == nullptr)
  const NarrowTab* tabs;     // ntabs tables (device), or nullptr
  const NarrowUnit* units;   // nunits units in launch order (device), or nullptr: tab0's stages cut
                             // into nunits consecutive ranges, unit u in slot u
  const int32_t* tab_slot0;  // ntabs + 1 entries: table t's slots are [tab_slot0[t], tab_slot0[t + 1])
  float* slots;              // one slot of kWideSlotPairs pairs per unit
  unsigned int* status;      // device status word (one per launch: the first table's ctx)
  int32_t nunits, ntabs;
  int32_t flush_stages;      // 64-row stages between FP32 -> (hi, lo) flushes
};
// CTA b takes units b, b + grid, ...; then one merge block per (row of S or column sums, table).
cudaError_t launch_narrow(const NarrowParams& P, bool x4, int grid, cudaStream_t st);
// Pivots (the means of the first kPivotRows rows) of tables which[0 .. count) of a device table list.
cudaError_t launch_narrow_shift(const NarrowTab* tabs, const int* which, int count, cudaStream_t st);

// ---------------------------------------------------------------------------
// CUDA-core comparators for any width: FP64 (raw / shifted) and FP32-core.
// ---------------------------------------------------------------------------
constexpr int kCoreSlotDoubles = 2 * (32 * 32 + 32);
struct CoreParams {
  const void* cols[256];
  int32_t dtype[256];
  const double* shift;  // p pivots or nullptr (raw moments)
  int32_t p;
  int32_t nblk;         // ceil(p / 64)
  int32_t ntiles;
  int32_t ksplit;
  int32_t flush_rows;   // FP32 only: rows between flushes into (hi, lo) pairs
  int64_t nrows;
  double* slots;        // scratch: core_slot_doubles(grid)
  unsigned int* ticket;
  double* acc_s;
  double* acc_s_lo;
  double* acc_S;
  double* acc_S_lo;
  long long* acc_n;
};
size_t core_slot_doubles(int grid);
cudaError_t launch_core(const CoreParams& P, bool fp32, int grid, cudaStream_t stream);

// ---------------------------------------------------------------------------
// Finalize (one block): recombination, exact centering, cov / corr, Jacobi.
// ---------------------------------------------------------------------------
struct FinalPlanCol {
  int32_t off;      // first digit slot of the column
  int32_t k;        // digit bytes
  int32_t shift;    // real columns: fixed-point shift (value = q * 2^-shift); 0 for integers
  int32_t is_real;
  int32_t is_ident;
};
struct FinalParams {
  int32_t p;
  int32_t mode;      // stats_mode
  int32_t pca_on;    // 0 cov, 1 corr
  int32_t want_pca;
  FinalPlanCol col[256];
  const long long* g;          // EXACT: digit gram kDigits x kDigits
  const double* fs;            // FP64: sums (hi), p
  const double* fs_lo;
  const double* fS;            // FP64: packed upper (hi)
  const double* fS_lo;
  const long long* fn;         // FP64: count
  const double* shift;         // FP64 shifted: shift vector or nullptr
  double* out;                 // device result buffer (layout: final_layout())
  double* work;                // device scratch: 2 * pa * pa doubles
  // When set, the eigen-decomposition is left to jacobi_grid_kernel: the matrix goes to
  // defer_A (defer_m x defer_m, zero-padded to an even order) and *defer_ctl = 1 when the
  // eigenpairs are wanted and defined (0 otherwise).
  double* defer_A;
  int32_t* defer_ctl;
  int32_t defer_m;
};
// Offsets (in doubles) of the finalize result buffer.
struct FinalLayout {
  int64_t n, s, S, s_ex, S_ex, mean, cov, corr, evals, evecs, flags, total;
};
__host__ __device__ inline FinalLayout final_layout(int p, int pa) {
  FinalLayout L;
  const int64_t T = static_cast<int64_t>(p) * (p + 1) / 2;
  L.n = 0;
  L.s = 1;
  L.S = L.s + p;
  L.s_ex = L.S + T;            // p int128 values as (lo, hi) int64 pairs
  L.S_ex = L.s_ex + 2 * p;     // T int128 values
  L.mean = L.S_ex + 2 * T;
  L.cov = L.mean + pa;
  L.corr = L.cov + static_cast<int64_t>(pa) * pa;
  L.evals = L.corr + static_cast<int64_t>(pa) * pa;
  L.evecs = L.evals + pa;
  L.flags = L.evecs + static_cast<int64_t>(pa) * pa;
  L.total = L.flags + 8;
  return L;
}
// flags: [0] an exact integer entry did not fit 128 bits, [1] zero-variance columns,
//        [2] Jacobi sweeps, [3] eigenpairs computed (1) or not (0),
//        [5] a grid-wide wait of jacobi_grid_kernel ran out (1), [6] its seed basis was used (1)
cudaError_t launch_finalize(const FinalParams& P, cudaStream_t stream);
// d_params: count FinalParams in device memory, one block each
cudaError_t launch_finalize_batched(const FinalParams* d_params, int count, cudaStream_t stream);

// Block-cyclic Jacobi spread over a cooperative grid.  The indices are cut into blocks
// of 8; in each block round (the round-robin ordering over blocks) every pair of blocks
// solves its 16 x 16 diagonal problem with one cyclic Jacobi sweep (the one-block
// solver's rotation formula) in shared memory, then all 16 x 16 blocks of A and V are
// updated with the pairs' accumulated rotations: two grid-wide barriers per block round.
// A is double buffered (a round reads a and writes b).
struct JacobiParams {
  double* a;                // m x m, holds the matrix on entry (written by the finalize kernel)
  double* b;                // m x m
  double* v;                // m x m eigenvector accumulator
  double* w;                // m x m, warm start product
  double* q;                // (m / 16) x 16 x 16: the rotation of every block pair of a round
  const double* basis;      // pa x pa, row k = a previous eigenvector k, or nullptr (cold start)
  double* slots;            // >= grid partial sums
  unsigned int* bar;        // [0] arrivals, [1] generation, [2] error; zero before each launch
  const int32_t* ctl;       // written by the finalize kernel: 1 = decompose
  double* out;              // finalize result buffer
  int64_t evals_off, evecs_off, flags_off;
  int32_t pa, m;            // analysis columns; m = pa rounded up to a multiple of 16
  int64_t wait_ns;          // limit of one grid-wide wait (<= 0: 2 s)
  int32_t absent_block;     // testing: this block leaves before its first arrival (-1: none)
};
// Doubles of scratch jacobi_grid_kernel needs for pa analysis columns (the five arrays above).
size_t jacobi_scratch_doubles(int pa);
// Blocks of the cooperative grid for pa columns on a device of `sms` SMs (0: not possible).
int jacobi_grid_blocks(int pa, int sms);
cudaError_t launch_jacobi_grid(const JacobiParams& J, int grid, cudaStream_t stream);

// ---------------------------------------------------------------------------
// CSV text on the device (csv.cu): line index and field parse.
// ---------------------------------------------------------------------------
constexpr int kCsvTile = 4096;  // bytes per line-counting tile
// error bits of CsvScratch::status
constexpr uint32_t kCsvFormat = 1u, kCsvRange = 2u;
struct CsvScratch {
  uint32_t* counts;          // newlines per tile
  int64_t* offs;             // exclusive prefix of counts
  int64_t* ends;             // ends[i]: offset of line i's '\n' (or the text's end), i < ends_cap
  int64_t ends_cap;
  int64_t* total;            // number of lines
  uint32_t* status;          // kCsvFormat | kCsvRange
  unsigned long long* bad;   // (first offending line << 2) | its error bit (all ones: none)
  void** cols;               // k device column pointers
  int32_t* dts;              // k stats_dtype values
};
// Bytes of scratch for texts of up to nbytes bytes, ends_cap lines and k fields; carve
// lays the arrays out in base (256-byte aligned pieces).
size_t csv_scratch_bytes(int64_t nbytes, int64_t ends_cap, int k);
void csv_scratch_carve(void* base, int64_t nbytes, int64_t ends_cap, int k, CsvScratch& s);
// Counts the lines of d_text[0, nbytes) and writes their ends (no host synchronisation).
cudaError_t launch_csv_lines(const char* d_text, int64_t nbytes, const CsvScratch& s, cudaStream_t st);
// Parses the first k fields of lines [0, min(*total, ends_cap)) into s.cols (rows below
// row_cap are stored; every line is checked); status and bad must be reset before.
cudaError_t launch_csv_parse(const char* d_text, const CsvScratch& s, int k, int64_t row_cap, int sms,
                             cudaStream_t st);

// ---------------------------------------------------------------------------
// Table 1 generator and misc.
// ---------------------------------------------------------------------------
cudaError_t t1_upload_lut();  // builds the lookup tables with libm on the host, once per device
cudaError_t launch_gen_table1(uint64_t seed, uint64_t row0, int64_t nrows, int layout, void* const* cols,
                              cudaStream_t stream);
cudaError_t launch_merge_i64(long long* dst, const long long* src, int count, cudaStream_t stream);
cudaError_t launch_merge_dd(double* dst_hi, double* dst_lo, const double* src_hi, const double* src_lo, int count,
                            cudaStream_t stream);
// shifted moments of src (pivot c_s, n_s rows) re-expressed about c_d, added to dst (double-double)
cudaError_t launch_merge_shifted(double* s, double* s_lo, double* S, double* S_lo, const double* c_d,
                                 const double* ss, const double* ss_lo, const double* Ss, const double* Ss_lo,
                                 const double* c_s, const long long* n_s, int p, cudaStream_t stream);
// float copy of p double pivots (the split kernels' shift), exact for pivots taken from FP32 data
cudaError_t launch_pivot_to_float(const double* src, float* dst, int p, cudaStream_t stream);

}  // namespace ss
