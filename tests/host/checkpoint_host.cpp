// Host-only test of the setup checkpoint (paper_1601_03184_gb300/csrc/
// checkpoint.cu) without a GPU. checkpoint.cu is compiled as plain C++ and
// linked against the stand-ins below: its three CUDA runtime calls become
// host memcpy (the "device" buffers are host memory) and the four library
// internals it uses are replaced by host versions. What is tested is the
// file logic: header checks, chunked copies, checksum, .part handling and
// every refusal. Usage: checkpoint_host <scratch directory>; exit status 0
// when every check passes.
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

extern "C" cudaError_t cudaMemcpyAsync(void* dst, const void* src, size_t n, cudaMemcpyKind, cudaStream_t) {
  std::memcpy(dst, src, n);
  return cudaSuccess;
}
extern "C" cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
extern "C" const char* cudaGetErrorString(cudaError_t) { return "host stand-in"; }

namespace mrhs {
std::string& create_error_slot() {
  static std::string s;
  return s;
}
void* dalloc(mrhs_ctx c, size_t bytes) {
  void* p = std::calloc(1, bytes ? bytes : 16);
  c->allocs.push_back(p);
  return p;
}
double* host_scratch(mrhs_ctx c, size_t bytes) {
  if (c->hbuf_bytes < bytes) {
    std::free(c->hbuf);
    c->hbuf = (double*)std::malloc(bytes);
    c->hbuf_bytes = bytes;
  }
  return c->hbuf;
}
int images_built = 0;
void dc_images_build(mrhs_ctx) { ++images_built; }
}  // namespace mrhs

using namespace mrhs;

namespace {

int failures = 0;
#define CHECK(cond)                                                      \
  do {                                                                   \
    if (!(cond)) {                                                       \
      std::printf("FAILED line %d: %s\n", __LINE__, #cond);             \
      ++failures;                                                        \
    }                                                                    \
  } while (0)

size_t tv_size(mrhs_ctx c) { return fine_elems(c, c->ntv) * dtype_size(c->tv_dtype); }
size_t dc_size(mrhs_ctx c) { return (size_t)c->g.nagg * 9 * 4 * c->ntv * c->ntv * 2 * dtype_size(c->work_dtype); }

mrhs_ctx make_ctx(const int L[4], const int a[4], int ntv, int prec, int order_shift = 0) {
  mrhs_ctx c = new mrhs_ctx_s();
  c->g.V = c->g.Va = c->g.nagg = 1;
  for (int m = 0; m < 4; ++m) {
    c->g.L[m] = L[m];
    c->g.a[m] = a[m];
    c->g.nb[m] = L[m] / a[m];
    c->g.V *= L[m];
    c->g.Va *= a[m];
    c->g.nagg *= L[m] / a[m];
  }
  c->ntv = ntv;
  c->prec = prec;
  c->tv_dtype = prec == MRHS_PREC_FP64 ? MRHS_F64 : prec == MRHS_PREC_FP32 ? MRHS_F32
                : prec == MRHS_PREC_MIX_BF16 ? MRHS_BF16 : MRHS_F16;
  c->work_dtype = prec == MRHS_PREC_FP64 ? MRHS_F64 : MRHS_F32;
  c->perm = (int*)dalloc(c, sizeof(int) * c->g.V);
  for (int s = 0; s < c->g.V; ++s) c->perm[s] = (s + order_shift) % c->g.V;
  return c;
}

void fill(void* p, size_t n, unsigned long long seed) {
  unsigned char* b = (unsigned char*)p;
  for (size_t i = 0; i < n; ++i) {
    seed = seed * 6364136223846793005ULL + 1442695040888963407ULL;
    b[i] = (unsigned char)(seed >> 56);
  }
}

void make_setup(mrhs_ctx c, unsigned long long seed, double scale) {
  c->tv = dalloc(c, tv_size(c));
  c->P = dalloc(c, tv_size(c));
  c->Dc = dalloc(c, dc_size(c));
  fill(c->tv, tv_size(c), seed);
  fill(c->P, tv_size(c), seed + 1);
  fill(c->Dc, dc_size(c), seed + 2);
  c->tv_scale = scale;
  c->have_tv = c->have_P = c->have_Dc = true;
}

void destroy(mrhs_ctx c) {
  for (void* p : c->allocs) std::free(p);
  std::free(c->hbuf);
  delete c;
}

bool exists(const std::string& p) {
  std::FILE* f = std::fopen(p.c_str(), "rb");
  if (f) std::fclose(f);
  return f != nullptr;
}

std::vector<unsigned char> read_all(const std::string& p) {
  std::vector<unsigned char> d;
  std::FILE* f = std::fopen(p.c_str(), "rb");
  if (!f) return d;
  int ch;
  while ((ch = std::fgetc(f)) != EOF) d.push_back((unsigned char)ch);
  std::fclose(f);
  return d;
}

void write_all(const std::string& p, const unsigned char* d, size_t n) {
  std::FILE* f = std::fopen(p.c_str(), "wb");
  std::fwrite(d, 1, n, f);
  std::fclose(f);
}

// the file header as checkpoint.cu writes it (for offsets of its fields)
struct HeaderView {
  char magic[8];
  int version;
  int L[4], a[4];
  int ntv, prec, tv_dtype, work_dtype;
  unsigned long long order_hash;
  double tv_scale;
  unsigned long long tv_bytes, P_bytes, Dc_bytes;
};

bool same_setup(mrhs_ctx a, mrhs_ctx b) {
  return std::memcmp(a->tv, b->tv, tv_size(a)) == 0 && std::memcmp(a->P, b->P, tv_size(a)) == 0 &&
         std::memcmp(a->Dc, b->Dc, dc_size(a)) == 0 && a->tv_scale == b->tv_scale;
}

// save, restore bit for bit, and every refusal, for one shape
void run_case(const std::string& dir, const int L[4], const int a[4], int ntv, int prec, double scale) {
  const std::string path = dir + "/setup.bin";
  std::remove(path.c_str());
  mrhs_ctx src = make_ctx(L, a, ntv, prec);
  // no setup yet: refused, nothing written
  CHECK(mrhs_save_setup(src, path.c_str()) == MRHS_ERR_STATE);
  CHECK(!exists(path) && !exists(path + ".part"));
  make_setup(src, 12345 + prec, scale);
  CHECK(mrhs_save_setup(src, path.c_str()) == MRHS_OK);
  CHECK(exists(path) && !exists(path + ".part"));

  // restore into a fresh context of the same shape
  mrhs_ctx dst = make_ctx(L, a, ntv, prec);
  const int built = images_built;
  const long long version = dst->dc_version;
  CHECK(mrhs_load_setup(dst, path.c_str()) == MRHS_OK);
  CHECK(dst->have_tv && dst->have_P && dst->have_Dc);
  CHECK(same_setup(src, dst));
  CHECK(images_built == built + 1 && dst->dc_version == version + 1);

  // another ntv or another device site order: refused, context untouched
  mrhs_ctx other = make_ctx(L, a, ntv / 2, prec);
  CHECK(mrhs_load_setup(other, path.c_str()) == MRHS_ERR_SHAPE);
  CHECK(!other->have_P && other->tv == nullptr);
  mrhs_ctx shuffled = make_ctx(L, a, ntv, prec, 1);
  CHECK(mrhs_load_setup(shuffled, path.c_str()) == MRHS_ERR_SHAPE);

  // damaged payload: checksum mismatch, and no setup afterwards
  std::vector<unsigned char> data = read_all(path);
  CHECK(data.size() > 200);
  std::vector<unsigned char> bad(data);
  bad[bad.size() / 2] ^= 0x5A;
  const std::string damaged = dir + "/damaged.bin";
  write_all(damaged, bad.data(), bad.size());
  mrhs_ctx d2 = make_ctx(L, a, ntv, prec);
  CHECK(mrhs_load_setup(d2, damaged.c_str()) == MRHS_ERR_ARG);
  CHECK(!d2->have_tv && !d2->have_P && !d2->have_Dc);
  // a damaged header field that the load does not compare with the context
  // (the fp16 scale, still finite and positive): checksum mismatch
  {
    std::vector<unsigned char> hb(data);
    const size_t off = offsetof(HeaderView, tv_scale);
    double sc;
    std::memcpy(&sc, hb.data() + off, sizeof sc);
    sc *= 1.5;
    std::memcpy(hb.data() + off, &sc, sizeof sc);
    const std::string hdr = dir + "/header.bin";
    write_all(hdr, hb.data(), hb.size());
    CHECK(mrhs_load_setup(d2, hdr.c_str()) == MRHS_ERR_ARG);
    CHECK(!d2->have_tv && !d2->have_P && !d2->have_Dc);
  }
  // truncated, one byte short
  const std::string shortf = dir + "/short.bin";
  write_all(shortf, data.data(), data.size() - 1);
  CHECK(mrhs_load_setup(d2, shortf.c_str()) == MRHS_ERR_ARG);
  // not a checkpoint, no file at all
  std::vector<unsigned char> zeros(256, 0);
  const std::string junk = dir + "/junk.bin";
  write_all(junk, zeros.data(), zeros.size());
  CHECK(mrhs_load_setup(d2, junk.c_str()) == MRHS_ERR_ARG);
  CHECK(mrhs_load_setup(d2, (dir + "/missing.bin").c_str()) == MRHS_ERR_ARG);
  // the intact file still loads into the same context
  CHECK(mrhs_load_setup(d2, path.c_str()) == MRHS_OK);
  CHECK(same_setup(src, d2));
  // a file that cannot be written: refused, no .part left behind
  const std::string nodir = dir + "/no/such/dir/setup.bin";
  CHECK(mrhs_save_setup(src, nodir.c_str()) == MRHS_ERR_ARG);
  CHECK(!exists(nodir + ".part"));
  // null arguments
  CHECK(mrhs_save_setup(src, nullptr) == MRHS_ERR_ARG);
  CHECK(mrhs_load_setup(nullptr, path.c_str()) == MRHS_ERR_ARG);
  for (mrhs_ctx c : {src, dst, other, shuffled, d2}) destroy(c);
}

}  // namespace

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  const std::string dir = argv[1];
  // FP64 with buffers above the 64 MiB copy chunk: 100.7 MB of test vectors
  // and P, 75.5 MB of D_c, so every copy takes two chunks
  const int L1[4] = {8, 8, 8, 16}, a1[4] = {4, 4, 4, 4};
  run_case(dir, L1, a1, 64, MRHS_PREC_FP64, 1.0);
  // fp16 test vectors with their storage scale, a ragged shape
  const int L2[4] = {4, 6, 4, 8}, a2[4] = {2, 3, 2, 2};
  run_case(dir, L2, a2, 6, MRHS_PREC_MIX_FP16, 78.38367176906169);
  std::printf("%s (%d failed checks)\n", failures ? "FAILED" : "ok", failures);
  return failures ? 1 : 0;
}
