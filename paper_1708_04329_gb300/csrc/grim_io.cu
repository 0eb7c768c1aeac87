// Index persistence (§GRIM-Filter: the bit vectors are generated once for a
// reference and stored, so that every later run only loads them).
//
// File layout (little-endian, as written by this library):
//   FileHeader (256 bytes): magic, version, the build parameters (reference
//   length, B, q, max_read_len, coarse factor), the layouts stored, the byte
//   size of each stored table and a checksum of the table bytes;
//   then the tables back to back in the order token-major, bin-major
//   (including the zero vectors that pad it to whole super-bins), coarse
//   token-major -- each exactly as it sits in device memory.
// The per-token presence counts are not stored: loading recomputes them
// from the loaded tables, as a build would.
//
// Copies go through two pinned staging buffers so that the disk and the
// host<->device copies overlap.
#include <stdio.h>
#include <string.h>

#include "grim_internal.cuh"

namespace grim {
namespace {

constexpr char kMagic[8] = {'G', 'R', 'I', 'M', 'I', 'D', 'X', '1'};
constexpr uint32_t kVersion = 1;
constexpr uint64_t kChunk = 64ull << 20;

struct FileHeader {
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  uint64_t ref_len;
  uint32_t B, q, max_read_len, coarse_factor;
  uint32_t layouts;  // tables present in the file
  uint32_t pad0;
  uint64_t num_bins;
  uint64_t bytes[3];  // token-major, bin-major, coarse token-major (0 if absent)
  uint64_t checksum;  // over the table bytes in file order
  uint8_t pad[256 - 88];
};
static_assert(sizeof(FileHeader) == 256, "header is 256 bytes");

// Order-dependent checksum of 8-byte words: sum over words w_i of
// (w_i + i) * 0x9E3779B97F4A7C15 (mod 2^64), with i the word's position in
// the file's table section.  The tables are multiples of 8 bytes.
struct Checksum {
  uint64_t h = 0, pos = 0;
  void add(const void* p, uint64_t n) {
    const uint64_t* w = static_cast<const uint64_t*>(p);
    for (uint64_t i = 0; i < n / 8; ++i) h += (w[i] + pos + i) * 0x9E3779B97F4A7C15ull;
    pos += n / 8;
  }
};

struct Staging {
  char* buf[2] = {nullptr, nullptr};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaStream_t st = nullptr;
  cudaError_t init() {
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
      e = cudaMallocHost(&buf[i], kChunk);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    }
    return e;
  }
  ~Staging() {
    if (st) cudaStreamSynchronize(st);
    for (int i = 0; i < 2; ++i) {
      if (buf[i]) cudaFreeHost(buf[i]);
      if (ev[i]) cudaEventDestroy(ev[i]);
    }
    if (st) cudaStreamDestroy(st);
  }
};

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

// device table -> file, chunk k+1 copied down while chunk k is written
int write_table(Staging& sg, FILE* f, const void* dev, uint64_t n, Checksum& ck) {
  const char* src = static_cast<const char*>(dev);
  uint64_t nchunks = (n + kChunk - 1) / kChunk;
  for (uint64_t k = 0; k < nchunks + 1; ++k) {
    if (k < nchunks) {
      const uint64_t o = k * kChunk, m = n - o < kChunk ? n - o : kChunk;
      cudaError_t e = cudaMemcpyAsync(sg.buf[k & 1], src + o, m, cudaMemcpyDeviceToHost, sg.st);
      if (e == cudaSuccess) e = cudaEventRecord(sg.ev[k & 1], sg.st);
      if (e != cudaSuccess) return record_cuda_error(e);
    }
    if (k > 0) {
      const uint64_t j = k - 1, o = j * kChunk, m = n - o < kChunk ? n - o : kChunk;
      const cudaError_t e = cudaEventSynchronize(sg.ev[j & 1]);
      if (e != cudaSuccess) return record_cuda_error(e);
      ck.add(sg.buf[j & 1], m);
      if (fwrite(sg.buf[j & 1], 1, m, f) != m) return GRIM_E_IO;
    }
  }
  return GRIM_OK;
}

// file -> device table (or skipped with dev == nullptr), chunk k read while
// chunk k-1 is copied up
int read_table(Staging& sg, FILE* f, void* dev, uint64_t n, Checksum& ck, bool verify) {
  if (!dev && !verify) return fseeko(f, (off_t)n, SEEK_CUR) == 0 ? GRIM_OK : GRIM_E_IO;
  char* dst = static_cast<char*>(dev);
  const uint64_t nchunks = (n + kChunk - 1) / kChunk;
  for (uint64_t k = 0; k < nchunks; ++k) {
    const uint64_t o = k * kChunk, m = n - o < kChunk ? n - o : kChunk;
    char* b = sg.buf[k & 1];
    if (k >= 2) {  // the buffer's previous copy must have left it
      const cudaError_t e = cudaEventSynchronize(sg.ev[k & 1]);
      if (e != cudaSuccess) return record_cuda_error(e);
    }
    if (fread(b, 1, m, f) != m) return GRIM_E_IO;
    if (verify) ck.add(b, m);
    if (dst) {
      cudaError_t e = cudaMemcpyAsync(dst + o, b, m, cudaMemcpyHostToDevice, sg.st);
      if (e == cudaSuccess) e = cudaEventRecord(sg.ev[k & 1], sg.st);
      if (e != cudaSuccess) return record_cuda_error(e);
    }
  }
  const cudaError_t e = cudaStreamSynchronize(sg.st);
  return e == cudaSuccess ? GRIM_OK : record_cuda_error(e);
}

uint64_t table_bytes(const grim_index* ix, int t) {
  const IndexView& v = ix->v;
  const IndexView& cv = ix->cv;
  switch (t) {
    case 0: return ix->tm ? (uint64_t)v.r4 * v.wpad * sizeof(uint32_t) : 0;
    case 1: return ix->bm ? cv.num_bins * ix->factor * v.wpb * sizeof(uint32_t) : 0;
    default: return ix->ctm ? (uint64_t)cv.r4 * cv.wpad * sizeof(uint32_t) : 0;
  }
}

const void* table_ptr(const grim_index* ix, int t) {
  return t == 0 ? (const void*)ix->tm : t == 1 ? (const void*)ix->bm : (const void*)ix->ctm;
}

}  // namespace
}  // namespace grim

using namespace grim;

extern "C" {

int grim_save(const grim_index* idx, const char* path) {
  if (!idx || !path) return GRIM_E_ARG;
  File out;
  out.f = fopen(path, "wb");
  if (!out.f) return GRIM_E_IO;
  FileHeader h{};
  memcpy(h.magic, kMagic, sizeof(kMagic));
  h.version = kVersion;
  h.header_bytes = sizeof(FileHeader);
  h.ref_len = idx->v.n;
  h.B = idx->v.B;
  h.q = idx->v.q;
  h.max_read_len = idx->v.max_read_len;
  h.coarse_factor = idx->factor;
  h.layouts = idx->layouts;
  h.num_bins = idx->v.num_bins;
  for (int t = 0; t < 3; ++t) h.bytes[t] = table_bytes(idx, t);
  // header first (checksum filled in at the end)
  if (fwrite(&h, sizeof(h), 1, out.f) != 1) return GRIM_E_IO;
  Staging sg;
  const cudaError_t e = sg.init();
  if (e != cudaSuccess) return record_cuda_error(e);
  Checksum ck;
  for (int t = 0; t < 3; ++t) {
    if (!h.bytes[t]) continue;
    const int rc = write_table(sg, out.f, table_ptr(idx, t), h.bytes[t], ck);
    if (rc != GRIM_OK) return rc;
  }
  h.checksum = ck.h;
  if (fseeko(out.f, 0, SEEK_SET) != 0 || fwrite(&h, sizeof(h), 1, out.f) != 1) return GRIM_E_IO;
  if (fflush(out.f) != 0) return GRIM_E_IO;
  return GRIM_OK;
}

int grim_load(const char* path, uint32_t layouts, uint32_t flags, grim_index** out) {
  if (!out) return GRIM_E_ARG;
  *out = nullptr;
  if (!path || (layouts & ~GRIM_LAYOUT_ALL) || (flags & ~GRIM_LOAD_VERIFY)) return GRIM_E_ARG;
  File in;
  in.f = fopen(path, "rb");
  if (!in.f) return GRIM_E_IO;
  FileHeader h{};
  if (fread(&h, sizeof(h), 1, in.f) != 1) return GRIM_E_FORMAT;
  if (memcmp(h.magic, kMagic, sizeof(kMagic)) != 0 || h.version != kVersion ||
      h.header_bytes != sizeof(FileHeader) || (h.layouts & ~GRIM_LAYOUT_ALL) || h.layouts == 0)
    return GRIM_E_FORMAT;
  if (layouts == 0) layouts = h.layouts;
  if (layouts & ~h.layouts) return GRIM_E_NO_LAYOUT;
  grim_index* ix = nullptr;
  int rc = index_alloc(h.ref_len, h.B, h.q, h.max_read_len, layouts, h.coarse_factor, &ix);
  if (rc != GRIM_OK) return rc == GRIM_E_ARG || rc == GRIM_E_UNSUPPORTED ? GRIM_E_FORMAT : rc;
  // the file's table sizes must be those its parameters give
  const uint32_t bits[3] = {GRIM_LAYOUT_TOKEN_MAJOR, GRIM_LAYOUT_BIN_MAJOR, GRIM_LAYOUT_COARSE};
  bool ok = ix->v.num_bins == h.num_bins;
  for (int t = 0; t < 3 && ok; ++t) {
    // a table's size follows from the parameters; absent tables have size 0
    const uint64_t want =
        (h.layouts & bits[t]) == 0 ? 0
        : t == 0 ? (uint64_t)ix->v.r4 * ix->v.wpad * sizeof(uint32_t)
        : t == 1 ? ix->cv.num_bins * ix->factor * ix->v.wpb * sizeof(uint32_t)
                 : (uint64_t)ix->cv.r4 * ix->cv.wpad * sizeof(uint32_t);
    ok = h.bytes[t] == want && h.bytes[t] % 8 == 0;
  }
  if (!ok) {
    grim_free(ix);
    return GRIM_E_FORMAT;
  }
  Staging sg;
  cudaError_t e = sg.init();
  if (e != cudaSuccess) {
    grim_free(ix);
    return record_cuda_error(e);
  }
  const bool verify = (flags & GRIM_LOAD_VERIFY) != 0;
  Checksum ck;
  void* dst[3] = {ix->tm, ix->bm, ix->ctm};
  for (int t = 0; t < 3; ++t) {
    if (!h.bytes[t]) continue;
    rc = read_table(sg, in.f, (layouts & bits[t]) ? dst[t] : nullptr, h.bytes[t], ck, verify);
    if (rc != GRIM_OK) {
      grim_free(ix);
      return rc == GRIM_E_IO ? GRIM_E_FORMAT : rc;
    }
  }
  if (verify && ck.h != h.checksum) {
    grim_free(ix);
    return GRIM_E_FORMAT;
  }
  // presence counts from the table the all-bins filter sweeps first, as in a build
  if (ix->ctm) launch_row_popcount(ix->ctm, ix->cv.r4, ix->cv.wpad, ix->presence, sg.st);
  else if (ix->tm) launch_row_popcount(ix->tm, ix->v.r4, ix->v.wpad, ix->presence, sg.st);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(sg.st);
  prof_collect();
  if (e != cudaSuccess) {
    grim_free(ix);
    return record_cuda_error(e);
  }
  *out = ix;
  return GRIM_OK;
}

}  // extern "C"
