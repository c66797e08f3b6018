/*
 * stats_file.h -- columnar binary table files for libsuffstats: writing, validation,
 * sampled-row checks and a streaming pass from file into a context.
 *
 * The paper converts its CSV table once to a fixed-width binary file and checks the
 * conversion before any statistics are computed: the file's size, row count and
 * column layout against the known dimensions, and records from its beginning,
 * middle and end against the source (arxiv 2604.23826, "Validation and
 * Infrastructure Verification"; the binary file is the canonical input of the
 * single streaming pass, "Data Representation and Sufficient Statistics").  Here
 * the binary file is columnar (the same compact column types the device pass
 * reads), and the source a sampled row is compared with is the Table 1 generator,
 * whose rows depend only on (seed, row index).
 *
 * File layout (little-endian):
 *   bytes [0, 4096)   header
 *       0    char     magic[8]     "SSCOL01" and a NUL
 *       8    uint32   version      1
 *      12    int32    p            1 .. STATS_FILE_MAX_P
 *      16    int64    nrows        >= 0
 *      24    uint64   file_bytes   total size of the file
 *      32    int32    dtypes[256]  stats_dtype of column j (entries >= p are 0)
 *    1056    uint64   offsets[256] byte offset of column j (entries >= p are 0)
 *    3104    uint64   header_hash  FNV-1a 64 of bytes [0, 3104)
 *    3112             zero to 4096
 *   column j: nrows * sizeof(dtypes[j]) bytes at offsets[j], a multiple of 4096;
 *   the columns follow one another in order, each starting on the next 4096-byte
 *   boundary, and file_bytes is the end of the last one (4096 when p columns are
 *   empty).
 *
 * Conventions of stats.h hold.  Additional return codes: STATS_EIO (open, read or
 * write failed), STATS_EFORMAT (the file is not a valid table file: a header field,
 * the header hash, the column layout or the file size is wrong), STATS_EMISMATCH
 * (a sampled row differs from its source).
 */
#ifndef SUFFSTATS_STATS_FILE_H
#define SUFFSTATS_STATS_FILE_H

#include "stats.h"

#ifdef __cplusplus
extern "C" {
#endif

#define STATS_FILE_HEADER_BYTES 4096
#define STATS_FILE_ALIGN 4096
#define STATS_FILE_MAX_P 256
#define STATS_FILE_VERSION 1

/* Write an n x p table from host columns (hcols: p host pointers, column j of
 * dtypes[j]) to a new file at path (replaced if it exists).  Columns are written in
 * parallel.  Errors: EINVAL (p, dtypes, nrows or a NULL column), EIO. */
stats_status stats_file_write(const char* path, int32_t p, const int32_t* dtypes, int64_t nrows,
                              const void* const* hcols);

/* Write rows [row0, row0 + nrows) of Table 1 (seed, layout) to a new table file,
 * generating them on the current device in chunks of chunk_rows rows (0 = 2^24)
 * and copying each chunk through pinned host memory; file row r holds table row
 * row0 + r.  Errors: EINVAL, ENOMEM, ECUDA, EIO. */
stats_status stats_file_write_table1(const char* path, uint64_t seed, uint64_t row0, int64_t nrows,
                                     int32_t layout, int64_t chunk_rows);

/* Validate the file's header, column layout and size; on success fill *p, *nrows
 * and dtypes[0 .. p) (dtypes: room for STATS_FILE_MAX_P entries; any output may be
 * NULL).  Errors: EINVAL (NULL path), EIO, EFORMAT. */
stats_status stats_file_info(const char* path, int32_t* p, int64_t* nrows, int32_t* dtypes);

/* Read rows [row0, row0 + nrows) of every column of a validated file into host
 * buffers (hcols: p host pointers, each with room for nrows values of its dtype).
 * Errors: EINVAL (range outside the file, NULL buffer), EIO, EFORMAT. */
stats_status stats_file_read_rows(const char* path, int64_t row0, int64_t nrows, void* const* hcols);

/* The paper's conversion check for a Table 1 file: the header must describe 12
 * columns of the layout's dtypes; then rows_per_region rows from the beginning,
 * the middle and the end of the file (fewer when the file is shorter) are read and
 * compared bit for bit with the same rows regenerated on the current device from
 * (seed, row0 + r), row0 being the table row of file row 0.  On a difference,
 * *first_bad_row (if not NULL) receives the file row and STATS_EMISMATCH is
 * returned; otherwise *first_bad_row = -1.  Errors: EINVAL, ENOMEM, ECUDA, EIO,
 * EFORMAT, EMISMATCH. */
stats_status stats_file_check_table1(const char* path, uint64_t seed, uint64_t row0, int32_t layout,
                                     int64_t rows_per_region, int64_t* first_bad_row);

/* Add file rows [row0, row0 + nrows) (nrows < 0: to the end of the file) to ctx: the
 * file's columns must match the ctx's p and dtypes.  Chunks of chunk_rows rows
 * (0 = 2^22; rounded up to a multiple of 8) are read by parallel host threads into
 * one of two ctx-owned pinned buffers while the device copies and reduces the
 * previous chunk (the double-buffered pipeline of stats_accumulate_host).  Returns
 * once every chunk has been read and its copies and pass are enqueued on stream.
 * Rows of one file can be split across calls, contexts or processes by row range
 * and recombined with stats_merge.  Errors: EINVAL, ENOMEM, ECUDA, EIO, EFORMAT,
 * ESTATE. */
stats_status stats_accumulate_file(stats_ctx* ctx, const char* path, int64_t row0, int64_t nrows,
                                   int64_t chunk_rows, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SUFFSTATS_STATS_FILE_H */
