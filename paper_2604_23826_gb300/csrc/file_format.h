// file_format.h -- internal helpers for the columnar table files of stats_file.h:
// header encoding and validation, parallel positional reads and writes.
#pragma once

#include <stdint.h>

#include "stats_file.h"

namespace ss {

// Header field offsets (stats_file.h documents the layout).
constexpr int kFileMagicOff = 0, kFileVersionOff = 8, kFilePOff = 12, kFileRowsOff = 16, kFileBytesOff = 24,
              kFileDtypesOff = 32, kFileOffsetsOff = 1056, kFileHashOff = 3104;
constexpr char kFileMagic[8] = {'S', 'S', 'C', 'O', 'L', '0', '1', '\0'};

struct FileInfo {
  int32_t p = 0;
  int64_t nrows = 0;
  uint64_t file_bytes = 0;
  int32_t dtypes[STATS_FILE_MAX_P] = {};
  uint64_t offsets[STATS_FILE_MAX_P] = {};
};

int file_dtype_bytes(int32_t dt);  // 2, 4 or 8; 0 for an unknown dtype
uint64_t file_fnv1a(const unsigned char* p, size_t n);

// The layout a writer produces for (p, dtypes, nrows): offsets and file size.
bool file_plan(int32_t p, const int32_t* dtypes, int64_t nrows, FileInfo& out);
// Serialize info into a STATS_FILE_HEADER_BYTES buffer (hash included).
void file_encode_header(const FileInfo& info, unsigned char* hdr);

// Open path read-only and validate it; *fd receives the open descriptor on success.
stats_status file_open_checked(const char* path, FileInfo& info, int* fd);
// Read rows [row0, row0 + nrows) of every column into hcols (parallel over pieces).
stats_status file_read_rows(int fd, const FileInfo& info, int64_t row0, int64_t nrows, void* const* hcols);
// Write rows [row0, row0 + nrows) of every column from hcols (parallel over pieces).
stats_status file_write_rows(int fd, const FileInfo& info, int64_t row0, int64_t nrows, const void* const* hcols);
// Create (truncate) path, sized and with its header written; *fd stays open for writing.
stats_status file_create(const char* path, const FileInfo& info, int* fd);

}  // namespace ss
