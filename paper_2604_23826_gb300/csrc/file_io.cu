// file_io.cu -- columnar table files (stats_file.h): writing, validation of size, row
// count and column layout, sampled-row checks against the Table 1 generator
// (arxiv 2604.23826, "Validation and Infrastructure Testing": the converted binary
// file checked for size, row count and layout, and records from its beginning,
// middle and end compared with the source), parallel positional reads for the
// streaming pass from file (stats_accumulate_file, api.cu).
#include <errno.h>
#include <fcntl.h>
#include <sched.h>
#include <string.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "file_format.h"

namespace ss {

namespace {

constexpr uint64_t kPieceBytes = 32ull << 20;  // unit of parallel I/O
constexpr int kMaxIoThreads = 16;

// Threads for parallel reads and writes: the cores this process may run on, 4 .. 16.
int io_threads() {
  cpu_set_t set;
  int n = 0;
  if (sched_getaffinity(0, sizeof(set), &set) == 0) n = CPU_COUNT(&set);
  if (n <= 0) n = static_cast<int>(std::thread::hardware_concurrency());
  return std::max(4, std::min(kMaxIoThreads, n));
}

uint64_t align_up(uint64_t x) { return (x + STATS_FILE_ALIGN - 1) / STATS_FILE_ALIGN * STATS_FILE_ALIGN; }

template <class T>
void put(unsigned char* h, int off, T v) {
  memcpy(h + off, &v, sizeof(T));
}
template <class T>
T get(const unsigned char* h, int off) {
  T v;
  memcpy(&v, h + off, sizeof(T));
  return v;
}

bool pread_all(int fd, void* buf, uint64_t len, uint64_t off) {
  char* b = static_cast<char*>(buf);
  while (len > 0) {
    const ssize_t r = pread(fd, b, static_cast<size_t>(std::min<uint64_t>(len, 1ull << 30)), static_cast<off_t>(off));
    if (r < 0 && errno == EINTR) continue;
    if (r <= 0) return false;
    b += r;
    off += static_cast<uint64_t>(r);
    len -= static_cast<uint64_t>(r);
  }
  return true;
}

bool pwrite_all(int fd, const void* buf, uint64_t len, uint64_t off) {
  const char* b = static_cast<const char*>(buf);
  while (len > 0) {
    const ssize_t r = pwrite(fd, b, static_cast<size_t>(std::min<uint64_t>(len, 1ull << 30)), static_cast<off_t>(off));
    if (r < 0 && errno == EINTR) continue;
    if (r <= 0) return false;
    b += r;
    off += static_cast<uint64_t>(r);
    len -= static_cast<uint64_t>(r);
  }
  return true;
}

struct Piece {
  int col;
  uint64_t file_off;  // where in the file
  uint64_t mem_off;   // where in the column's host buffer
  uint64_t len;
};

// The (column, byte range) pieces of rows [row0, row0 + nrows).
std::vector<Piece> pieces_of(const FileInfo& info, int64_t row0, int64_t nrows) {
  std::vector<Piece> out;
  for (int j = 0; j < info.p; ++j) {
    const uint64_t eb = static_cast<uint64_t>(file_dtype_bytes(info.dtypes[j]));
    const uint64_t total = static_cast<uint64_t>(nrows) * eb;
    for (uint64_t done = 0; done < total; done += kPieceBytes)
      out.push_back(Piece{j, info.offsets[j] + static_cast<uint64_t>(row0) * eb + done, done,
                          std::min<uint64_t>(kPieceBytes, total - done)});
  }
  return out;
}

// Run fn(piece) over all pieces on up to io_threads() threads; false if any call failed.
template <class Fn>
bool run_pieces(const std::vector<Piece>& ps, Fn fn) {
  if (ps.empty()) return true;
  std::atomic<size_t> next{0};
  std::atomic<bool> ok{true};
  auto worker = [&]() {
    for (size_t i = next.fetch_add(1); i < ps.size(); i = next.fetch_add(1))
      if (!fn(ps[i])) ok = false;
  };
  const int nt = static_cast<int>(std::min<size_t>(static_cast<size_t>(io_threads()), ps.size()));
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(worker);
  worker();
  for (auto& t : th) t.join();
  return ok;
}

}  // namespace

int file_dtype_bytes(int32_t dt) {
  switch (dt) {
    case STATS_I16: return 2;
    case STATS_I32: return 4;
    case STATS_F32: return 4;
    case STATS_I64: return 8;
    case STATS_F64: return 8;
    default: return 0;
  }
}

uint64_t file_fnv1a(const unsigned char* p, size_t n) {
  uint64_t h = 14695981039346656037ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

bool file_plan(int32_t p, const int32_t* dtypes, int64_t nrows, FileInfo& out) {
  if (p < 1 || p > STATS_FILE_MAX_P || nrows < 0 || !dtypes) return false;
  out = FileInfo{};
  out.p = p;
  out.nrows = nrows;
  uint64_t off = STATS_FILE_HEADER_BYTES;
  for (int j = 0; j < p; ++j) {
    const int eb = file_dtype_bytes(dtypes[j]);
    if (!eb) return false;
    out.dtypes[j] = dtypes[j];
    off = align_up(off);
    out.offsets[j] = off;
    off += static_cast<uint64_t>(nrows) * static_cast<uint64_t>(eb);
  }
  out.file_bytes = off;
  return true;
}

void file_encode_header(const FileInfo& info, unsigned char* hdr) {
  memset(hdr, 0, STATS_FILE_HEADER_BYTES);
  memcpy(hdr + kFileMagicOff, kFileMagic, 8);
  put<uint32_t>(hdr, kFileVersionOff, STATS_FILE_VERSION);
  put<int32_t>(hdr, kFilePOff, info.p);
  put<int64_t>(hdr, kFileRowsOff, info.nrows);
  put<uint64_t>(hdr, kFileBytesOff, info.file_bytes);
  for (int j = 0; j < info.p; ++j) {
    put<int32_t>(hdr, kFileDtypesOff + 4 * j, info.dtypes[j]);
    put<uint64_t>(hdr, kFileOffsetsOff + 8 * j, info.offsets[j]);
  }
  put<uint64_t>(hdr, kFileHashOff, file_fnv1a(hdr, kFileHashOff));
}

stats_status file_open_checked(const char* path, FileInfo& info, int* fd_out) {
  if (!path) return STATS_EINVAL;
  const int fd = open(path, O_RDONLY | O_CLOEXEC);
  if (fd < 0) return STATS_EIO;
  unsigned char hdr[STATS_FILE_HEADER_BYTES];
  struct stat sb;
  stats_status st = STATS_OK;
  if (fstat(fd, &sb) != 0) {
    st = STATS_EIO;
  } else if (static_cast<uint64_t>(sb.st_size) < STATS_FILE_HEADER_BYTES || !pread_all(fd, hdr, sizeof(hdr), 0)) {
    st = STATS_EFORMAT;  // shorter than a header
  } else {
    // the header's own fields
    info = FileInfo{};
    info.p = get<int32_t>(hdr, kFilePOff);
    info.nrows = get<int64_t>(hdr, kFileRowsOff);
    info.file_bytes = get<uint64_t>(hdr, kFileBytesOff);
    bool ok = memcmp(hdr + kFileMagicOff, kFileMagic, 8) == 0 &&
              get<uint32_t>(hdr, kFileVersionOff) == STATS_FILE_VERSION &&
              get<uint64_t>(hdr, kFileHashOff) == file_fnv1a(hdr, kFileHashOff) && info.p >= 1 &&
              info.p <= STATS_FILE_MAX_P && info.nrows >= 0 && info.nrows < (int64_t(1) << 48);
    // column layout: known dtypes, each column on the next 4096-byte boundary after the last
    uint64_t end = STATS_FILE_HEADER_BYTES;
    for (int j = 0; ok && j < info.p; ++j) {
      info.dtypes[j] = get<int32_t>(hdr, kFileDtypesOff + 4 * j);
      info.offsets[j] = get<uint64_t>(hdr, kFileOffsetsOff + 8 * j);
      const int eb = file_dtype_bytes(info.dtypes[j]);
      ok = eb > 0 && info.offsets[j] == align_up(end);  // the writer's layout, exactly
      end = info.offsets[j] + static_cast<uint64_t>(info.nrows) * static_cast<uint64_t>(eb);
    }
    for (int j = info.p; ok && j < STATS_FILE_MAX_P; ++j)
      ok = get<int32_t>(hdr, kFileDtypesOff + 4 * j) == 0 && get<uint64_t>(hdr, kFileOffsetsOff + 8 * j) == 0;
    // size: the header's total, the end of the last column and the file agree
    ok = ok && info.file_bytes == end && static_cast<uint64_t>(sb.st_size) == info.file_bytes;
    if (!ok) st = STATS_EFORMAT;
  }
  if (st != STATS_OK) {
    close(fd);
    return st;
  }
  *fd_out = fd;
  return STATS_OK;
}

stats_status file_read_rows(int fd, const FileInfo& info, int64_t row0, int64_t nrows, void* const* hcols) {
  if (row0 < 0 || nrows < 0 || row0 + nrows > info.nrows || (nrows > 0 && !hcols)) return STATS_EINVAL;
  for (int j = 0; nrows > 0 && j < info.p; ++j)
    if (!hcols[j]) return STATS_EINVAL;
  const bool ok = run_pieces(pieces_of(info, row0, nrows), [&](const Piece& q) {
    return pread_all(fd, static_cast<char*>(hcols[q.col]) + q.mem_off, q.len, q.file_off);
  });
  return ok ? STATS_OK : STATS_EIO;
}

stats_status file_write_rows(int fd, const FileInfo& info, int64_t row0, int64_t nrows, const void* const* hcols) {
  if (row0 < 0 || nrows < 0 || row0 + nrows > info.nrows || (nrows > 0 && !hcols)) return STATS_EINVAL;
  for (int j = 0; nrows > 0 && j < info.p; ++j)
    if (!hcols[j]) return STATS_EINVAL;
  const bool ok = run_pieces(pieces_of(info, row0, nrows), [&](const Piece& q) {
    return pwrite_all(fd, static_cast<const char*>(hcols[q.col]) + q.mem_off, q.len, q.file_off);
  });
  return ok ? STATS_OK : STATS_EIO;
}

stats_status file_create(const char* path, const FileInfo& info, int* fd_out) {
  if (!path) return STATS_EINVAL;
  const int fd = open(path, O_WRONLY | O_CREAT | O_TRUNC | O_CLOEXEC, 0644);
  if (fd < 0) return STATS_EIO;
  unsigned char hdr[STATS_FILE_HEADER_BYTES];
  file_encode_header(info, hdr);
  if (ftruncate(fd, static_cast<off_t>(info.file_bytes)) != 0 || !pwrite_all(fd, hdr, sizeof(hdr), 0)) {
    close(fd);
    return STATS_EIO;
  }
  *fd_out = fd;
  return STATS_OK;
}

}  // namespace ss

using namespace ss;

namespace {

// Table 1 dtypes of a layout (as stats_table1_config reports them).
bool table1_dtypes(int32_t layout, int32_t* dt) {
  double lo[STATS_T1_P], hi[STATS_T1_P];
  uint8_t ident[STATS_T1_P];
  return stats_table1_config(layout, 1, dt, ident, lo, hi) == STATS_OK;
}

}  // namespace

extern "C" {

stats_status stats_file_write(const char* path, int32_t p, const int32_t* dtypes, int64_t nrows,
                              const void* const* hcols) {
  FileInfo info;
  if (!path || !file_plan(p, dtypes, nrows, info)) return STATS_EINVAL;
  for (int j = 0; nrows > 0 && j < p; ++j)
    if (!hcols || !hcols[j]) return STATS_EINVAL;
  int fd = -1;
  stats_status st = file_create(path, info, &fd);
  if (st != STATS_OK) return st;
  st = file_write_rows(fd, info, 0, nrows, hcols);
  if (close(fd) != 0 && st == STATS_OK) st = STATS_EIO;
  return st;
}

stats_status stats_file_write_table1(const char* path, uint64_t seed, uint64_t row0, int64_t nrows,
                                     int32_t layout, int64_t chunk_rows) {
  int32_t dt[STATS_T1_P];
  if (!path || nrows < 0 || chunk_rows < 0 || !table1_dtypes(layout, dt)) return STATS_EINVAL;
  FileInfo info;
  if (!file_plan(STATS_T1_P, dt, nrows, info)) return STATS_EINVAL;
  if (chunk_rows == 0) chunk_rows = int64_t(1) << 24;
  chunk_rows = std::max<int64_t>(1, std::min<int64_t>(chunk_rows, std::max<int64_t>(nrows, 1)));
  chunk_rows = (chunk_rows + 3) & ~int64_t(3);
  // device and pinned host columns of one chunk
  std::vector<size_t> off(STATS_T1_P);
  size_t bytes = 0;
  for (int j = 0; j < STATS_T1_P; ++j) {
    off[j] = bytes;
    bytes += (static_cast<size_t>(chunk_rows) * file_dtype_bytes(dt[j]) + 255) / 256 * 256;
  }
  void* d = nullptr;
  void* h = nullptr;
  if (cudaMalloc(&d, bytes) != cudaSuccess) {
    cudaGetLastError();
    return STATS_ENOMEM;
  }
  if (cudaHostAlloc(&h, bytes, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d);
    return STATS_ENOMEM;
  }
  int fd = -1;
  stats_status st = file_create(path, info, &fd);
  std::vector<void*> dcols(STATS_T1_P);
  std::vector<const void*> hcols(STATS_T1_P);
  for (int j = 0; j < STATS_T1_P; ++j) {
    dcols[j] = static_cast<char*>(d) + off[j];
    hcols[j] = static_cast<char*>(h) + off[j];
  }
  for (int64_t r = 0; st == STATS_OK && r < nrows; r += chunk_rows) {
    const int64_t m = std::min(chunk_rows, nrows - r);
    st = stats_gen_table1(seed, row0 + static_cast<uint64_t>(r), m, layout, dcols.data(), nullptr);
    if (st == STATS_OK && (cudaMemcpy(h, d, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)) st = STATS_ECUDA;
    if (st == STATS_OK) st = file_write_rows(fd, info, r, m, hcols.data());  // rows [r, r + m)
  }
  if (fd >= 0 && close(fd) != 0 && st == STATS_OK) st = STATS_EIO;
  cudaFreeHost(h);
  cudaFree(d);
  return st;
}

stats_status stats_file_info(const char* path, int32_t* p, int64_t* nrows, int32_t* dtypes) {
  FileInfo info;
  int fd = -1;
  const stats_status st = file_open_checked(path, info, &fd);
  if (st != STATS_OK) return st;
  close(fd);
  if (p) *p = info.p;
  if (nrows) *nrows = info.nrows;
  if (dtypes)
    for (int j = 0; j < info.p; ++j) dtypes[j] = info.dtypes[j];
  return STATS_OK;
}

stats_status stats_file_read_rows(const char* path, int64_t row0, int64_t nrows, void* const* hcols) {
  FileInfo info;
  int fd = -1;
  stats_status st = file_open_checked(path, info, &fd);
  if (st != STATS_OK) return st;
  st = file_read_rows(fd, info, row0, nrows, hcols);
  close(fd);
  return st;
}

stats_status stats_file_check_table1(const char* path, uint64_t seed, uint64_t row0, int32_t layout,
                                     int64_t rows_per_region, int64_t* first_bad_row) {
  if (first_bad_row) *first_bad_row = -1;
  int32_t dt[STATS_T1_P];
  if (!path || rows_per_region < 1 || !table1_dtypes(layout, dt)) return STATS_EINVAL;
  FileInfo info;
  int fd = -1;
  stats_status st = file_open_checked(path, info, &fd);
  if (st != STATS_OK) return st;
  if (info.p != STATS_T1_P) st = STATS_EFORMAT;
  for (int j = 0; st == STATS_OK && j < STATS_T1_P; ++j)
    if (info.dtypes[j] != dt[j]) st = STATS_EFORMAT;
  const int64_t n = info.nrows, k = std::min(rows_per_region, n);
  // regions: beginning, middle, end (overlapping ones checked twice)
  const int64_t starts[3] = {0, std::max<int64_t>(0, n / 2 - k / 2), n - k};
  size_t bytes = 0;
  std::vector<size_t> off(STATS_T1_P);
  for (int j = 0; j < STATS_T1_P; ++j) {
    off[j] = bytes;
    bytes += (static_cast<size_t>(std::max<int64_t>(k, 1)) * file_dtype_bytes(dt[j]) + 255) / 256 * 256;
  }
  std::vector<char> from_file(bytes), from_gen(bytes);
  void* d = nullptr;
  if (st == STATS_OK && k > 0 && cudaMalloc(&d, bytes) != cudaSuccess) {
    cudaGetLastError();
    st = STATS_ENOMEM;
  }
  std::vector<void*> fcols(STATS_T1_P), dcols(STATS_T1_P);
  for (int j = 0; j < STATS_T1_P; ++j) {
    fcols[j] = from_file.data() + off[j];
    if (d) dcols[j] = static_cast<char*>(d) + off[j];
  }
  for (int r = 0; st == STATS_OK && k > 0 && r < 3; ++r) {
    st = file_read_rows(fd, info, starts[r], k, fcols.data());
    if (st == STATS_OK) st = stats_gen_table1(seed, row0 + static_cast<uint64_t>(starts[r]), k, layout, dcols.data(), nullptr);
    if (st == STATS_OK && cudaMemcpy(from_gen.data(), d, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
      st = STATS_ECUDA;
    for (int64_t i = 0; st == STATS_OK && i < k; ++i)
      for (int j = 0; j < STATS_T1_P; ++j) {
        const int eb = file_dtype_bytes(dt[j]);
        if (memcmp(from_file.data() + off[j] + i * eb, from_gen.data() + off[j] + i * eb, eb) != 0) {
          if (first_bad_row) *first_bad_row = starts[r] + i;
          st = STATS_EMISMATCH;
          break;
        }
      }
  }
  if (d) cudaFree(d);
  close(fd);
  return st;
}

}  // extern "C"
