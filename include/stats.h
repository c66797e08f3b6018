/*
 * stats.h -- C ABI of the GB300 sufficient-statistics library (libsuffstats.so).
 *
 * One streaming pass over a tall-skinny n x p table X, stored column by
 * column on the device, produces the row count n, the column sums s = X^T 1
 * and the upper triangle of S = X^T X.  Mean, covariance, correlation and the
 * PCA eigenpairs are then computed from (n, s, S) alone, without revisiting
 * the data (arxiv 2604.23826, "Data Representation and Sufficient
 * Statistics": column sums and the cross-product matrix accumulated in one
 * pass; "Principal Component Analysis Results": PCA from the aggregated
 * matrices only).
 *
 * Conventions that hold for every call:
 *   - Return codes only; nothing is thrown across the ABI.  stats_strerror()
 *     names a code.
 *   - Device pointers are plain CUDA device addresses of the current device;
 *     host pointers are ordinary process memory.  The library never frees or
 *     retains caller memory beyond the documented lifetime.
 *   - A stream argument is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream).  Work is enqueued asynchronously; device buffers passed
 *     in must stay valid until the stream reaches the work (stats_sync()).
 *   - A ctx is used from one stream at a time: calls on one ctx that overlap
 *     on the GPU race on its accumulator.
 *   - A CUDA error inside the library makes the ctx sticky-failed: every later
 *     call on it returns STATS_ESTATE until it is destroyed.
 *   - Device-side errors (a value outside its declared range, an expired
 *     bounded wait) are recorded in the ctx and reported by the next call that
 *     synchronises with the device (stats_sync, stats_raw, stats_finalize,
 *     stats_export).  An accumulate call whose kernel detected such an error
 *     leaves the accumulator unchanged.
 *   - Packed upper triangle: entry (j, k), j <= k, of a p x p symmetric matrix
 *     is at index j*p - j*(j-1)/2 + (k - j); T(p) = p*(p+1)/2 entries.
 *   - Matrices returned by stats_finalize are full, row-major, over the
 *     "analysis columns": the columns not flagged as identifiers, in order.
 */
#ifndef SUFFSTATS_STATS_H
#define SUFFSTATS_STATS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stats_ctx stats_ctx;

typedef enum {
  STATS_OK = 0,
  STATS_EINVAL = 1,     /* bad argument or configuration                           */
  STATS_ENOMEM = 2,     /* a device or host allocation failed                      */
  STATS_ECUDA = 3,      /* a CUDA runtime call failed (ctx is now sticky-failed)   */
  STATS_EOVERFLOW = 4,  /* an exact result does not fit its output type            */
  STATS_ETIMEOUT = 5,   /* a bounded device-side wait expired                      */
  STATS_ESTATE = 6,     /* ctx is sticky-failed, or the call is out of order       */
  STATS_ERANGE = 7,     /* a value lay outside the digit field of its declared range,
                           or (stats_csv.h) outside its column type                  */
  STATS_EIO = 8,        /* a file could not be opened, read or written (stats_file.h) */
  STATS_EFORMAT = 9,    /* a file is not a valid table file (stats_file.h), or CSV
                           text is malformed (stats_csv.h)                           */
  STATS_EMISMATCH = 10  /* a sampled file row differs from its source (stats_file.h) */
} stats_status;

/* Column storage types. */
typedef enum { STATS_I16 = 0, STATS_I32 = 1, STATS_I64 = 2, STATS_F32 = 3, STATS_F64 = 4 } stats_dtype;

/* Arithmetic of the pass.
 *   STATS_EXACT        integer-valued columns exact (bit-exact s and S), real-valued
 *                      columns as 56-bit fixed point of their declared range; tensor
 *                      cores on 8-bit digits with FP32 accumulation flushed to int64
 *                      before it can round (all products and partial sums are exact
 *                      integers below 2^24).  Centering in exact integer arithmetic.
 *   STATS_FP64         the plain FP64 CUDA-core kernel with raw moments, as in the
 *                      paper (covariance = (S - s s^T / n) / (n - 1) in FP64); a
 *                      row-parallel kernel for p <= 12, a tiled one above.
 *   STATS_FP64_SHIFTED FP64 CUDA cores on x - c, c = the mean of the first rows accumulated
 *                      (the first 64 rows of the first call, or all of them if fewer; for
 *                      FP32 data in the BF16 and FP32 modes rounded to FP32).  A pivot near the
 *                      mean keeps the shifted cross products small, so rounding in their
 *                      accumulation does not survive the centering.
 *   STATS_BF16X3       FP32 data: x - c split into bf16 h + l; S ~ H^T H + H^T L + L^T H
 *                      on tensor cores (each 16-row block a fresh FP32 chain, added in
 *                      round-to-nearest FP32, then double-double); for p <= 64 plus the
 *                      diagonal of L^T L from the CUDA cores (its missing positive bias).
 *                      While a ctx holds fewer than 64 p rows (this call's included) its
 *                      calls form all four products, as STATS_BF16X4 does: the off-diagonal
 *                      L^T L terms that BF16X3 drops cancel only as 1/sqrt(n) and would leave
 *                      about 2.6e-6 sqrt(p / n) of relative error at small n.
 *   STATS_BF16X4       as BF16X3 plus all of L^T L on the tensor cores.
 *   STATS_FP32         FP32 CUDA-core FMA on x - c, flushed into FP32 (hi, lo) pairs.
 * The BF16 modes take FP32 columns only; the others take any dtype.             */
typedef enum {
  STATS_EXACT = 0,
  STATS_FP64 = 1,
  STATS_FP64_SHIFTED = 2,
  STATS_BF16X3 = 3,
  STATS_BF16X4 = 4,
  STATS_FP32 = 5
} stats_mode;

/* Table configuration (arrays are read during stats_init only).
 *   p             number of columns, 1..STATS_MAX_P
 *   dtypes        p stats_dtype values
 *   is_identifier p flags (1 = identifier: kept in s and S, left out of mean, cov,
 *                 corr and PCA, as the paper drops its row index A); may be NULL
 *   lo, hi        p declared value bounds, lo <= x <= hi for every value of the
 *                 column; may be NULL.  STATS_EXACT only: they fix each column's
 *                 digit field (integers: the bytes needed for [lo, hi]; reals: the
 *                 binary exponent e with max(|lo|,|hi|) < 2^e, fixed point
 *                 q = round(x * 2^(P - e)) with 56 bits).  NULL means the full
 *                 range of the integer dtype; real columns need bounds in STATS_EXACT.
 *   mode          a stats_mode value                                              */
typedef struct {
  int32_t p;
  const int32_t* dtypes;
  const uint8_t* is_identifier;
  const double* lo;
  const double* hi;
  int32_t mode;
} stats_config;

#define STATS_MAX_P 256
/* Widest digit plan of STATS_EXACT: the ones column plus all digit fields. */
#define STATS_EXACT_MAX_DIGITS 32

/* A 128-bit two's complement integer: value = hi * 2^64 + lo. */
typedef struct {
  uint64_t lo;
  int64_t hi;
} stats_i128;

/* Create a ctx on the current device: validates cfg, builds the digit plan
 * (STATS_EXACT), allocates the device accumulator and the per-call scratch.
 * *out receives the ctx, owned by the caller until stats_destroy().
 * Errors: EINVAL (bad p, dtype, mode, bounds; plan wider than
 * STATS_EXACT_MAX_DIGITS), ENOMEM, ECUDA. */
stats_status stats_init(stats_ctx** out, const stats_config* cfg);

/* Add nrows rows held on the device to the accumulator: dcols is a HOST array of
 * p DEVICE pointers, column j holding nrows values of dtypes[j], each pointer
 * aligned to its element size.  When every pointer is 16-byte aligned the rows
 * stream through the bulk-copy pipeline; otherwise the same kernel reads them
 * with plain loads (same results, lower throughput).  nrows may be 0.
 * Asynchronous on stream.
 * The single fused pass of the paper's "Data Representation and Sufficient
 * Statistics" section; partial results of the thread blocks are combined on the
 * device in a fixed order.  Errors: EINVAL (NULL or misaligned pointer, nrows < 0),
 * ESTATE, ECUDA; range errors are reported at the next synchronising call. */
stats_status stats_accumulate(stats_ctx* ctx, const void* const* dcols, int64_t nrows, void* stream);

/* Same from HOST memory: hcols is a host array of p HOST pointers (page-locked
 * memory gives overlapped copies; pageable memory works but serialises).
 * Rows are copied in chunks of chunk_rows (0 = library default) into two
 * library-owned device buffers, the copy of one chunk overlapping the pass over
 * the previous one (one cudaMemcpyAsync per column per chunk on an internal copy
 * stream, ordered with events).  Returns once everything is enqueued; the host
 * buffers must stay valid until stats_sync().  Errors as stats_accumulate, plus
 * ENOMEM for the staging buffers. */
stats_status stats_accumulate_host(stats_ctx* ctx, const void* const* hcols, int64_t nrows, int64_t chunk_rows,
                                   void* stream);

/* Many independent tables in one pass: table t (ctx ctxs[t], nrows[t] rows, dcols[t]
 * a host array of ctxs[t]'s p device column pointers) is added to ctxs[t].  Tables
 * of STATS_BF16X3 / STATS_BF16X4 contexts with p <= 64 run together in one
 * persistent launch per padded width (8, 16, 32, 64) and mode (up to 4096 tables per
 * launch): their 32-64 KB stages are dealt in chunks to one CTA per SM, and a second
 * small launch adds each table's per-CTA partials in a fixed order (results depend
 * only on the call, not on scheduling).  Tables whose columns sit one 16-byte-multiple
 * stride apart (a [p, ld] block) are read with 2D tensor copies, others with one bulk
 * copy per column.  Exception: tables of 33..64 columns stored as such a block, with at
 * least 4096 rows, share one persistent tcgen05 launch per mode instead (ranges of
 * 64-row stages of any table, each range reduced into its own partial and the partials
 * of a table added in row order).  Wider split tables use the tiled launch; contexts in
 * other modes go through stats_accumulate one by one.  The descriptors go to per-device
 * workspaces inside the library (grown on demand; use from one stream at a time).  A
 * context appears at most once per call; a device-side timeout of the shared tcgen05
 * launch is recorded in the first of its tables' contexts.
 * Errors: as stats_accumulate. */
stats_status stats_accumulate_batched(stats_ctx* const* ctxs, int32_t ntables, const void* const* const* dcols,
                                      const int64_t* nrows, void* stream);

/* dst += src for two ctxs with identical configuration: the combination of
 * partial results from disjoint row subsets that the paper does across its GPUs
 * ("Data Representation and Sufficient Statistics").  Exact for STATS_EXACT;
 * STATS_FP64 adds in double-double.  The shifted modes (STATS_FP64_SHIFTED,
 * STATS_BF16X3, STATS_BF16X4, STATS_FP32) hold moments about each ctx's own pivot
 * (the mean of its first rows): src's are re-expressed about dst's pivot, in double-double,
 *   sum (x - c_d) = s'_src + n_src d,
 *   sum (x - c_d)(x - c_d)^T = S'_src + d s'_src^T + s'_src d^T + n_src d d^T,
 * with d = c_src - c_dst; an empty dst takes src's pivot.  Enqueued on dst's last
 * stream; src must be idle.  Errors: EINVAL (configs differ), ESTATE. */
stats_status stats_merge(stats_ctx* dst, const stats_ctx* src);

/* Wait for all work of ctx and return its sticky device status. */
stats_status stats_sync(stats_ctx* ctx);

/* Zero the accumulator and clear recorded device errors (configuration kept).
 * Stream-ordered on the ctx's last stream. */
stats_status stats_reset(stats_ctx* ctx);

/* The sufficient statistics.  Synchronises.  Any output may be NULL.
 *   n              row count
 *   s              p column sums, rounded once to double
 *   S_upper        T(p) entries of X^T X (packed upper), rounded once to double
 *   s_exact        p exact sums; valid for integer-valued columns in STATS_EXACT
 *                  (zero elsewhere)
 *   S_exact_upper  T(p) exact entries; valid where both columns are integer-valued
 *                  in STATS_EXACT (zero elsewhere)
 * Errors: EOVERFLOW if an exact integer entry does not fit 128 bits (the double
 * outputs are still written), ERANGE/ETIMEOUT/ECUDA recorded by earlier work. */
stats_status stats_raw(stats_ctx* ctx, int64_t* n, double* s, double* S_upper, stats_i128* s_exact,
                       stats_i128* S_exact_upper);

/* Mean, covariance (divisor n - 1), correlation and eigenpairs over the analysis
 * columns (p_a = number of columns without the identifier flag), computed on the
 * device from (n, s, S) only.  Synchronises.  Caller-owned HOST outputs, any may
 * be NULL: mean[p_a], cov[p_a*p_a], corr[p_a*p_a], evals[p_a] (descending),
 * evecs[p_a*p_a] (row k = eigenvector k, sign chosen so that its largest-magnitude
 * component is positive).  pca_on: 0 = eigenpairs of cov, 1 = of corr.  A zero
 * variance gives NaN correlations in its row and column (the paper's "undefined
 * correlation values"); eigenpairs of corr are then not computed (NaN).
 * STATS_EXACT centres exactly (n S - s s^T in integer arithmetic) and rounds once;
 * STATS_FP64 uses the paper's raw-moment formula in FP64.
 * Errors: EINVAL (n < 2), and those of stats_raw. */
stats_status stats_finalize(stats_ctx* ctx, double* mean, double* cov, double* corr, double* evals, double* evecs,
                            int32_t pca_on);

/* Streaming analysis (finalize after every chunk of a growing table): stats_finalize with
 * the eigen-solver seeded by an earlier result.  The paper's method re-derives every
 * quantity from (n, s, S) alone ("Data Representation and Sufficient Statistics"), so a
 * snapshot can be taken between any two accumulate calls; this call makes a snapshot's
 * PCA ("Principal Component Analysis Results") cheap when the matrix has moved little.
 *   evecs_prev: HOST, p_a*p_a doubles, row k = eigenvector k, as written by an earlier
 *     stats_finalize / stats_finalize_warm (any ctx with the same p_a), or NULL (cold
 *     start).  The matrix M (cov, or corr with pca_on = 1) is rotated into that basis,
 *     V^T M V, before the cyclic Jacobi sweeps.  A seed whose columns are not orthonormal
 *     (max |V^T V - I| > 1e-9, or NaN) is ignored.  The eigenpairs are those of M
 *     whatever the seed, up to rounding; inside a cluster of equal eigenvalues the
 *     eigenvectors may be another basis of the same subspace.
 *   sweeps: may be NULL; receives the number of Jacobi sweeps taken, -1 when no
 *     eigenpairs were computed.
 * The other arguments are those of stats_finalize.  With more than 23 analysis columns,
 * or with a seed, the eigen-solver is a cooperative launch over the GPU's SMs.
 * Errors: those of stats_finalize; ETIMEOUT when a grid-wide wait of the eigen-solver
 * ran out (after 2 s; the ctx stays usable, the eigenpairs are not written). */
stats_status stats_finalize_warm(stats_ctx* ctx, double* mean, double* cov, double* corr, double* evals,
                                 double* evecs, int32_t pca_on, const double* evecs_prev, int32_t* sweeps);

/* stats_finalize for many contexts in one launch (one thread block per context; the
 * FP64 eigen-solver of each block is what a single call costs, so many contexts cost
 * about one call per SM-load instead of one call each).  Synchronises every context.
 * mean, cov and corr are those of stats_finalize bit for bit; the eigenpairs too below 24
 * analysis columns, while from 24 columns (where stats_finalize runs its eigen-solver
 * over the whole GPU) they agree with stats_finalize's to rounding.
 * For context i the caller-owned HOST outputs mean[i], cov[i], corr[i], evals[i],
 * evecs[i] are laid out as in stats_finalize; any of the five arrays may be NULL, and
 * so may any entry.  Outputs of contexts with fewer than two rows are left untouched.
 * Errors: EINVAL (bad arguments, or some context has n < 2: the others are still
 * written), the errors of stats_sync for any context. */
stats_status stats_finalize_batched(stats_ctx* const* ctxs, int32_t count, int32_t pca_on, double* const* mean,
                                    double* const* cov, double* const* corr, double* const* evals,
                                    double* const* evecs);

/* Checkpoint: serialise the accumulator and configuration into buf (len bytes).
 * With buf == NULL, *len receives the size needed.  Synchronises.
 * Errors: EINVAL (buffer too small: *len set to the size needed). */
stats_status stats_export(stats_ctx* ctx, void* buf, size_t* len);

/* Create a ctx on the current device from a stats_export() image.
 * Errors: EINVAL (not an image of this library / version), ENOMEM, ECUDA. */
stats_status stats_import(stats_ctx** out, const void* buf, size_t len);

/* Release the ctx and its device memory (synchronises first). NULL is a no-op. */
void stats_destroy(stats_ctx* ctx);

/* Static string naming a status code. */
const char* stats_strerror(stats_status st);

/* Number of analysis columns of ctx (columns without the identifier flag). */
int32_t stats_num_analysis_columns(const stats_ctx* ctx);

/* Tuning knob for tests and measurement: the number of thread blocks of the
 * pass kernels (0 = library default, a multiple of the SM count).  Results of
 * STATS_EXACT do not depend on it.  Errors: EINVAL (negative). */
stats_status stats_set_grid(stats_ctx* ctx, int32_t blocks);

/* How stats_accumulate_batched deals the stages of its split-mode tables to the persistent
 * CTAs of a launch, per width class (tables of 1-8, 9-16, 17-32 and 33-64 columns) and mode
 * (STATS_BF16X3, STATS_BF16X4).  The autotuner in paper_2604_23826_gb300/tune.py measures
 * candidate settings on a batch and sets the fastest.
 *   narrow_units_per_cta   33-64 columns in [p, ld] blocks (the persistent tcgen05 launch):
 *                          tables are cut into units of 64-row stages, sized so that each CTA
 *                          gets about this many units (1..256; default 12)
 *   gram32_chunks_per_cta  the register-fragment launch: stages are dealt in chunks, as long
 *                          as possible while each CTA gets at least this many (1..1024;
 *                          default 32)
 *   gram32_min_chunk       ... and never shorter than this many stages (1..65536; default 32)
 * The setting changes how rows are grouped into per-CTA partial sums, so results move within
 * rounding (the stated tolerance holds for every setting); a fixed setting reproduces its
 * bits.  Process-wide, for every device.  Errors: EINVAL (bad width, mode or values). */
typedef struct {
  int32_t narrow_units_per_cta;
  int32_t gram32_chunks_per_cta;
  int32_t gram32_min_chunk;
} stats_batch_tuning;
stats_status stats_set_batch_tuning(int32_t width, int32_t mode, const stats_batch_tuning* t);
stats_status stats_get_batch_tuning(int32_t width, int32_t mode, stats_batch_tuning* t);

/* Testing knob of the bounded grid-wide waits of the eigen-solver that stats_finalize and
 * stats_finalize_warm run over the whole GPU (more than 23 analysis columns, or a seed).
 *   wait_ns       how long a block waits at a grid barrier before the call gives up with
 *                 STATS_ETIMEOUT (0 = the default 2 s; at most 60 s)
 *   absent_block  -1 (normal), or the index of a block of the eigen-solver's grid that leaves
 *                 before its first arrival: every other block's wait at that barrier then
 *                 runs out after wait_ns, the eigenpairs are not written, and the call
 *                 returns STATS_ETIMEOUT.  This exercises the stalled-block failure path
 *                 (the error word, every block leaving, the host reading the status) with no
 *                 device fault; the ctx stays usable.  A block index past the grid has no
 *                 effect.
 * Applies to later finalize calls on ctx.  Errors: EINVAL. */
stats_status stats_set_grid_wait(stats_ctx* ctx, int64_t wait_ns, int32_t absent_block);

/* Kernel of STATS_BF16X3 / STATS_BF16X4 for tables of 129..256 FP32 columns stored as one
 * [p, ld] block: 1 (default) = pairs of SMs, each CTA of a pair converting one 128-column block
 * and the pair's 256 x 256 product formed by tcgen05 MMAs spanning both (the table is read
 * once); 0 = one CTA per 128 x 128 output block (blocks shared by two outputs are read twice).
 * Results agree to rounding.  Errors: EINVAL. */
stats_status stats_set_wide_pairs(stats_ctx* ctx, int32_t pairs);

/* Launch shape of the STATS_EXACT pass (-1 = the library's default for the ctx's converter):
 *   0  15 consumer warps, 64 rows each per stage (960-row stages), mma.sync on those warps
 *   1  19 consumer warps, 32 rows each (608-row stages), mma.sync
 *   2  23 consumer warps, 32 rows each (736-row stages), mma.sync
 *   3  14 converting warps, 64 rows each (896-row stages); the digit Gram on tcgen05 MMAs
 *      issued by one thread, accumulated in tensor memory and read by four more warps
 * More warps hide more latency per SM but get fewer registers and smaller stages.  Results
 * do not depend on the shape (integer accumulation).  Errors: EINVAL (unknown shape, or the
 * ctx's rows do not fit that shape's pipeline). */
stats_status stats_set_exact_shape(stats_ctx* ctx, int32_t shape);

/* Tuning knob of STATS_BF16X3 / STATS_BF16X4 (16..4096, a multiple of 16): rows of
 * round-to-nearest FP32 accumulation of a warp before its (hi, lo) pairs (default
 * 1024 for p > 64, 16384 for p <= 64).  Every 16-row block is a fresh tensor-core
 * chain whatever the knob.  Errors: EINVAL. */
stats_status stats_set_flush_rows(stats_ctx* ctx, int32_t rows);

/* ---------------------------------------------------------------------------
 * The paper's Table 1 workload (section "Background and Motivation", Table 1
 * "Dataset used in this study"): twelve columns
 *   A = row identifier 1..n, B = randBetween(3,8), C = randBetween(1,10),
 *   D = randBetween(1,100), E = int(log C / log B * 100),
 *   F = round(log D / log B * 10000), G = int(|cos C| * 100),
 *   H = int(|sin D| * 100), cotC = 1.0 / tan C, I = round(|cotC| * 1000),
 *   J = |tan D|, K = D / C (integer division)
 * in this column order.  Row i (0-based) draws its three uniforms with
 * Philox4x32-10 (Salmon et al., SC'11) at counter (i_lo, i_hi, 0, 0) under key
 * (seed_lo, seed_hi) and maps a 32-bit word u to lo + floor(u * (hi - lo + 1) / 2^32).
 * ------------------------------------------------------------------------- */

/* Column storage layouts of the Table 1 table.
 *   STATS_T1_L32: A int64; B C D E F G H I K int32; cotC J float64 (60 B/row)
 *   STATS_T1_L16: A int64; F int32; B C D E G H I K int16; cotC J float64 (44 B/row) */
typedef enum { STATS_T1_L32 = 0, STATS_T1_L16 = 1 } stats_t1_layout;

#define STATS_T1_P 12

/* Fill a stats_config's arrays for Table 1 in the given layout, for tables of at
 * most max_rows rows (sizes the identifier's digit field): dtypes[12],
 * is_identifier[12] (A only), lo[12], hi[12] (the ranges the Table 1 formulas
 * produce).  The caller sets p = 12 and the mode.  Errors: EINVAL. */
stats_status stats_table1_config(int32_t layout, int64_t max_rows, int32_t* dtypes, uint8_t* is_identifier,
                                 double* lo, double* hi);

/* Generate rows [row0, row0 + nrows) of Table 1 on the device into dcols (host
 * array of 12 device pointers in the layout's dtypes, 16-byte aligned; element 0
 * of each column receives row row0).  Counter-based: the values of a row depend
 * only on (seed, row index), never on chunking.  Asynchronous on stream.
 * Errors: EINVAL, ECUDA. */
stats_status stats_gen_table1(uint64_t seed, uint64_t row0, int64_t nrows, int32_t layout, void* const* dcols,
                              void* stream);

/* Bytes per row of a Table 1 layout (60 or 44), or 0 for an unknown layout. */
int32_t stats_table1_row_bytes(int32_t layout);

/* ---------------------------------------------------------------------------
 * No-allocation variant of the exact pass.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory -- a serving
 * process or framework that reserves the GPU's memory up front in its own pool
 * and lets no library call cudaMalloc outside it, or code that must not block
 * the device (cudaFree synchronises it).
 *
 * It computes (n, s, S) of nrows rows (dcols: host array of cfg->p device
 * pointers, as for stats_accumulate) with the exact pass and writes them to the
 * caller's DEVICE buffer d_result of STATS_NOALLOC_RESULT_BYTES(p) bytes
 * (8-byte aligned), laid out in 8-byte slots:
 *   [0]                 n (int64)
 *   [1, 1+p)            s, rounded once to double
 *   [1+p, 1+p+T)        S packed upper, rounded once to double      (T = p(p+1)/2)
 *   next 2p slots       s exact as stats_i128 (integer-valued columns; 0 for reals)
 *   next 2T slots       S exact as stats_i128 (both columns integer-valued; 0 otherwise)
 *   next 8 slots        flags: slot 0 = 1.0 if an exact entry does not fit 128 bits;
 *                       slot 4 (low 32 bits) = device status bits of the pass:
 *                       1 = a value outside its digit field (the sums are invalid),
 *                       2 = a bounded wait expired.
 * cfg must be STATS_EXACT with p <= 16 columns and a digit plan of at most
 * STATS_EXACT_MAX_DIGITS digits; nrows <= 2^46.  Larger sizes return STATS_EINVAL.
 * Each call computes the statistics of its own rows (no accumulation across calls).
 *
 * Scratch: a file-scope device array of 16,640 bytes inside the library, present
 * on every GPU that loads the library until the process exits.  No cudaMalloc,
 * cudaFree or allocating library routine is called.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) once; make that
 * first call before any stream capture begins.  The address stays valid until the
 * device is reset (cudaDeviceReset), which invalidates it together with every
 * other context and pointer of this library on that device.  All calls share the one array:
 * each call clears it first, and calls whose work overlaps on the GPU (for
 * example on two streams) race on it and must be serialised by the caller.
 * Asynchronous on stream; results are valid once the stream reaches them.
 * Errors: EINVAL (configuration, sizes beyond the maximum, NULL or misaligned
 * pointers), ECUDA. */
#define STATS_NOALLOC_RESULT_BYTES(p) (8 * (9 + 3 * (p) + 3 * ((p) * ((p) + 1) / 2)))
stats_status stats_pass_noalloc(const stats_config* cfg, const void* const* dcols, int64_t nrows, void* d_result,
                                void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SUFFSTATS_STATS_H */
