// Checkpoint and restore of a finished setup: the test vectors, P = R^dag and
// the coarse operator D_c, the products of the setup phase (Sec. 2, Alg. 1/2)
// that every later solve reuses. Restoring one skips the whole setup.
//
// File layout (host byte order): a fixed header, then the raw device images
// of the test vectors, of P and of D_c, then a 64-bit checksum of the header
// (padding zeroed) and the three payloads. The images are in the library's device site order, so the header
// carries a hash of that order (the canonical -> device site permutation) and
// a file only loads into a context of the same geometry, N_tv and precision.
// The gauge field and the clover term are not part of it: they are inputs,
// set by the caller as for any setup.
//
// Host code only: bounded copies between the context's buffers and a pinned
// host staging buffer, and stdio.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"

using namespace mrhs;

namespace {

constexpr char kMagic[8] = {'M', 'R', 'H', 'S', 'S', 'E', 'T', 'P'};
constexpr int kVersion = 2;  // 2: the checksum covers the header too
constexpr size_t kChunk = size_t(64) << 20;  // host staging per copy

struct Header {
  char magic[8];
  int version;
  int L[4], a[4];
  int ntv, prec, tv_dtype, work_dtype;
  unsigned long long order_hash;  // of the canonical -> device site permutation
  double tv_scale;
  unsigned long long tv_bytes, P_bytes, Dc_bytes;
};

// 64-bit running hash of a byte stream, eight bytes at a time (xor, multiply
// by an odd constant, fold the high bits down): detects truncated or damaged
// files, not deliberate tampering
struct Hash64 {
  unsigned long long h = 0x6a09e667f3bcc909ULL;
  void words(const unsigned char* p, size_t n) {
    size_t i = 0;
    for (; i + 8 <= n; i += 8) {
      unsigned long long w;
      std::memcpy(&w, p + i, 8);
      mix(w);
    }
    if (i < n) {
      unsigned long long w = 0;
      std::memcpy(&w, p + i, n - i);
      mix(w ^ ((unsigned long long)(n - i) << 56));
    }
  }
  void mix(unsigned long long w) {
    h ^= w;
    h *= 0x9e3779b97f4a7c15ULL;
    h ^= h >> 29;
  }
};

size_t tv_bytes(mrhs_ctx c) { return fine_elems(c, c->ntv) * dtype_size(c->tv_dtype); }
size_t dc_bytes(mrhs_ctx c) {
  const size_t nc = 2 * (size_t)c->ntv;
  return (size_t)c->g.nagg * 9 * nc * nc * 2 * dtype_size(c->work_dtype);
}

unsigned long long order_hash(mrhs_ctx c) {
  std::vector<int> perm(c->g.V);
  MRHS_CUDA(cudaMemcpyAsync(perm.data(), c->perm, sizeof(int) * perm.size(), cudaMemcpyDeviceToHost, c->stream));
  MRHS_CUDA(cudaStreamSynchronize(c->stream));
  Hash64 h;
  h.words((const unsigned char*)perm.data(), sizeof(int) * perm.size());
  return h.h;
}

struct File {
  std::FILE* f = nullptr;
  ~File() {
    if (f) std::fclose(f);
  }
};

// device buffer -> file through the pinned staging buffer, one chunk at a time
void write_buffer(mrhs_ctx c, std::FILE* f, const void* dev, size_t bytes, Hash64& h) {
  if (bytes == 0) return;
  unsigned char* st = (unsigned char*)host_scratch(c, std::min(bytes, kChunk));
  for (size_t off = 0; off < bytes; off += kChunk) {
    const size_t n = std::min(kChunk, bytes - off);
    MRHS_CUDA(cudaMemcpyAsync(st, (const unsigned char*)dev + off, n, cudaMemcpyDeviceToHost, c->stream));
    MRHS_CUDA(cudaStreamSynchronize(c->stream));
    h.words(st, n);
    MRHS_REQUIRE(std::fwrite(st, 1, n, f) == n, MRHS_ERR_ARG, "checkpoint: write failed");
  }
}

// file -> device buffer; the staging buffer is reused only after its copy ended
void read_buffer(mrhs_ctx c, std::FILE* f, void* dev, size_t bytes, Hash64& h) {
  if (bytes == 0) return;
  unsigned char* st = (unsigned char*)host_scratch(c, std::min(bytes, kChunk));
  for (size_t off = 0; off < bytes; off += kChunk) {
    const size_t n = std::min(kChunk, bytes - off);
    MRHS_REQUIRE(std::fread(st, 1, n, f) == n, MRHS_ERR_ARG, "checkpoint: file is truncated");
    h.words(st, n);
    MRHS_CUDA(cudaMemcpyAsync((unsigned char*)dev + off, st, n, cudaMemcpyHostToDevice, c->stream));
    MRHS_CUDA(cudaStreamSynchronize(c->stream));
  }
}

}  // namespace

extern "C" {

int mrhs_save_setup(mrhs_ctx c, const char* path) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && path, MRHS_ERR_ARG, "null argument");
    MRHS_REQUIRE(c->have_tv && c->have_P && c->have_Dc, MRHS_ERR_STATE, "mrhs_save_setup before the setup has run");
    Header hd;
    std::memset(&hd, 0, sizeof hd);
    std::memcpy(hd.magic, kMagic, sizeof kMagic);
    hd.version = kVersion;
    for (int m = 0; m < 4; ++m) {
      hd.L[m] = c->g.L[m];
      hd.a[m] = c->g.a[m];
    }
    hd.ntv = c->ntv;
    hd.prec = c->prec;
    hd.tv_dtype = c->tv_dtype;
    hd.work_dtype = c->work_dtype;
    hd.order_hash = order_hash(c);  // also waits for the work queued on the stream
    hd.tv_scale = c->tv_scale;
    hd.tv_bytes = hd.P_bytes = tv_bytes(c);
    hd.Dc_bytes = dc_bytes(c);
    const std::string part = std::string(path) + ".part";
    try {
      File out;
      out.f = std::fopen(part.c_str(), "wb");
      MRHS_REQUIRE(out.f, MRHS_ERR_ARG, "checkpoint: cannot open " + part + " for writing");
      MRHS_REQUIRE(std::fwrite(&hd, sizeof hd, 1, out.f) == 1, MRHS_ERR_ARG, "checkpoint: write failed");
      Hash64 h;
      h.words((const unsigned char*)&hd, sizeof hd);  // fields the load does not compare (tv_scale)
      write_buffer(c, out.f, c->tv, hd.tv_bytes, h);
      write_buffer(c, out.f, c->P, hd.P_bytes, h);
      write_buffer(c, out.f, c->Dc, hd.Dc_bytes, h);
      MRHS_REQUIRE(std::fwrite(&h.h, sizeof h.h, 1, out.f) == 1, MRHS_ERR_ARG, "checkpoint: write failed");
      const int rc = std::fclose(out.f);
      out.f = nullptr;
      MRHS_REQUIRE(rc == 0, MRHS_ERR_ARG, "checkpoint: write failed");
      MRHS_REQUIRE(std::rename(part.c_str(), path) == 0, MRHS_ERR_ARG,
                   std::string("checkpoint: cannot rename the finished file to ") + path);
    } catch (...) {
      std::remove(part.c_str());
      throw;
    }
  });
}

int mrhs_load_setup(mrhs_ctx c, const char* path) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && path, MRHS_ERR_ARG, "null argument");
    File in;
    in.f = std::fopen(path, "rb");
    MRHS_REQUIRE(in.f, MRHS_ERR_ARG, std::string("checkpoint: cannot open ") + path);
    Header hd;
    MRHS_REQUIRE(std::fread(&hd, sizeof hd, 1, in.f) == 1, MRHS_ERR_ARG, "checkpoint: file is truncated");
    MRHS_REQUIRE(std::memcmp(hd.magic, kMagic, sizeof kMagic) == 0, MRHS_ERR_ARG, "checkpoint: not a setup checkpoint");
    MRHS_REQUIRE(hd.version == kVersion, MRHS_ERR_ARG, "checkpoint: unsupported format version");
    bool same = hd.ntv == c->ntv && hd.prec == c->prec && hd.tv_dtype == c->tv_dtype && hd.work_dtype == c->work_dtype;
    for (int m = 0; m < 4; ++m) same = same && hd.L[m] == c->g.L[m] && hd.a[m] == c->g.a[m];
    MRHS_REQUIRE(same, MRHS_ERR_SHAPE, "checkpoint: lattice, aggregates, ntv or precision differ from the context's");
    MRHS_REQUIRE(hd.tv_bytes == tv_bytes(c) && hd.P_bytes == tv_bytes(c) && hd.Dc_bytes == dc_bytes(c),
                 MRHS_ERR_SHAPE, "checkpoint: payload sizes differ from the context's");
    MRHS_REQUIRE(hd.order_hash == order_hash(c), MRHS_ERR_SHAPE,
                 "checkpoint: written with a different device site order");
    MRHS_REQUIRE(std::isfinite(hd.tv_scale) && hd.tv_scale > 0, MRHS_ERR_ARG, "checkpoint: bad test-vector scale");
    if (!c->tv) c->tv = dalloc(c, tv_bytes(c));
    if (!c->P) c->P = dalloc(c, tv_bytes(c));
    if (!c->Dc) c->Dc = dalloc(c, dc_bytes(c));
    // the context holds no setup until the whole file has been read and checked
    c->have_tv = c->have_P = c->have_Dc = false;
    Hash64 h;
    h.words((const unsigned char*)&hd, sizeof hd);
    read_buffer(c, in.f, c->tv, hd.tv_bytes, h);
    read_buffer(c, in.f, c->P, hd.P_bytes, h);
    read_buffer(c, in.f, c->Dc, hd.Dc_bytes, h);
    unsigned long long sum = 0;
    MRHS_REQUIRE(std::fread(&sum, sizeof sum, 1, in.f) == 1, MRHS_ERR_ARG, "checkpoint: file is truncated");
    MRHS_REQUIRE(sum == h.h, MRHS_ERR_ARG, "checkpoint: checksum mismatch (damaged file)");
    c->tv_scale = hd.tv_scale;
    c->have_tv = c->have_P = c->have_Dc = true;
    ++c->dc_version;  // operand images of an earlier D_c are stale
    dc_images_build(c);
    MRHS_CUDA(cudaStreamSynchronize(c->stream));
  });
}

}  // extern "C"
