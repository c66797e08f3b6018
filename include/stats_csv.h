/*
 * stats_csv.h -- text tables (comma-separated values) for libsuffstats: a writer, a
 * parser that runs on the GPU, and a streaming pass from a CSV file into a context.
 *
 * The paper's first validation program streamed its CSV file in fixed-size chunks,
 * parsed only the first column (the row index, whose sum is known in closed form) and
 * reduced it on the GPUs; it then found that parsing text dominated the run time and
 * converted the table to binary once ("Validation and Infrastructure Verification";
 * "Data Representation and Sufficient Statistics").  These calls provide that text
 * path on the GPU, for the first k fields of every line, so that its cost can be set
 * against the binary path (stats_file.h) on the same table.
 *
 * Text format (both directions):
 *   - one record per line, fields separated by ',', lines ended by '\n' (a '\r' just
 *     before the '\n' is accepted when parsing); the last line may lack its '\n';
 *   - integer fields: an optional sign and 1 to 19 decimal digits;
 *   - real fields: an optional sign, digits with an optional '.', optionally 'e' or 'E'
 *     and a signed decimal exponent (at most 4 digits); at least one mantissa digit.
 *     At most 19 significant digits (further digits must be zeros), and the value
 *     must be M * 10^E for some integer M < 10^19 and -38 <= E <= 19 (magnitudes from
 *     1e-38 to about 1e38) and lie in the normal range of the column type, or be zero.  The writer prints FP64
 *     values with 17 and FP32 values with 9 significant digits (round-trip exact).
 *   - Conversion is exact: the parser forms M * 10^E or M / 10^-E in integer
 *     arithmetic (up to 128-bit) and rounds once to nearest, ties to even, straight
 *     to the column type, so every accepted field gives the correctly rounded value.
 * Parsing errors are reported per call with the first offending line (0-based, counted
 * from the start of the text or file, header lines included):
 *   STATS_EFORMAT  a malformed field, a missing field (fewer than k on a line), an empty
 *                  line, more significant digits or a wider exponent than supported;
 *   STATS_ERANGE   an integer outside its column type, a real that overflows it or
 *                  would be subnormal.
 * Conventions of stats.h hold; STATS_EIO as in stats_file.h.
 */
#ifndef SUFFSTATS_STATS_CSV_H
#define SUFFSTATS_STATS_CSV_H

#include "stats.h"

#ifdef __cplusplus
extern "C" {
#endif

#define STATS_CSV_MAX_DIGITS 19

/* Write an n x p table from host columns (hcols: p host pointers, column j of
 * dtypes[j]) as CSV text to a new file at path (replaced if it exists), after an
 * optional header line (header: the line's text without its '\n', or NULL).  Rows are
 * formatted by parallel host threads.  Real values outside the parser's range (above)
 * are written but cannot be parsed back.  Errors: EINVAL (also: a NaN or infinite
 * value), ENOMEM, EIO. */
stats_status stats_csv_write(const char* path, int32_t p, const int32_t* dtypes, int64_t nrows,
                             const void* const* hcols, const char* header);

/* Write rows [row0, row0 + nrows) of Table 1 (seed, layout) as CSV with the header line
 * "A,B,C,D,E,F,G,H,cotC,I,J,K", generating them on the current device in chunks of
 * chunk_rows rows (0 = 2^22).  Errors: EINVAL, ENOMEM, ECUDA, EIO. */
stats_status stats_csv_write_table1(const char* path, uint64_t seed, uint64_t row0, int64_t nrows,
                                    int32_t layout, int64_t chunk_rows);

/* Parse CSV text in device memory (d_text, nbytes bytes, whole lines; the last may
 * lack its '\n') into device columns: field j of line i goes to row i of d_cols[j]
 * (dtypes[j]), for the first k fields of every line (later fields are not read).
 * Every line is a record (no header handling here).  Synchronises the stream; on
 * success *nrows (if not NULL) receives the number of lines.  max_rows is the room
 * of every column; more lines than that is EINVAL with nothing written beyond it.
 * On a parse error *bad_line (if not NULL) receives the first offending line, else -1.
 * Scratch is allocated stream-ordered on the current device.
 * Errors: EINVAL, ENOMEM, ECUDA, EFORMAT, ERANGE. */
stats_status stats_csv_parse(const char* d_text, int64_t nbytes, int32_t k, const int32_t* dtypes,
                             void* const* d_cols, int64_t max_rows, int64_t* nrows, int64_t* bad_line,
                             void* stream);

/* Stream a CSV file into ctx: the first ctx->p fields of every line after skip_lines
 * header lines are parsed on the device into the ctx's column types and added by the
 * ctx's pass.  The file is read in chunks of chunk_bytes (0 = 64 MB; a line may not be
 * longer) by the host into one of two pinned buffers while the device copies, parses
 * and reduces the previous chunk; a line cut by a chunk boundary is carried into the
 * next chunk.  *nrows (if not NULL) receives the records added.  A chunk that fails to
 * parse is not added (chunks before it are): the call returns the error with
 * *bad_line (if not NULL) the file line, else -1.
 * Errors: EINVAL, ENOMEM, ECUDA, EIO, EFORMAT (also: a line longer than a chunk), ERANGE,
 * ESTATE. */
stats_status stats_accumulate_csv(stats_ctx* ctx, const char* path, int64_t skip_lines, int64_t chunk_bytes,
                                  int64_t* nrows, int64_t* bad_line, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SUFFSTATS_STATS_CSV_H */
