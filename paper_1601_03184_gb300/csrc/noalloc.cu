// Coarse solve that allocates nothing.
//
// Some callers cannot let the library call cudaMalloc: a host application
// whose device memory is handed out entirely by its own pool or caching
// allocator, code that must not take the device-wide synchronisation that
// cudaMalloc/cudaFree can cause in the middle of a solve, or an embedding
// that forbids allocation after start-up. For them the coarse GMRES keeps its
// Krylov basis, GMRES state and reduction partials in one file-scope device
// array of fixed size (every GPU that loads the library holds it until the
// process exits) instead of the context's scratch buffers.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kNoAllocBytes = size_t(64) << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the array on `device`. The name g_noalloc_scratch in host
// code is only a host-side stand-in, so the address is looked up once per
// device, with that device current.
void* noalloc_address(int device) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  MRHS_REQUIRE(device >= 0 && device < kMaxDevices, MRHS_ERR_ARG, "device ordinal out of range");
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    MRHS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_addr[device] = p;
  }
  return g_noalloc_addr[device];
}

}  // namespace

using namespace mrhs;

extern "C" int mrhs_coarse_solve_noalloc(mrhs_ctx c, const void* bc, void* xc, int nrhs, int dtype, double tol,
                                         int restart, int maxit, int* iters) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && bc && xc, MRHS_ERR_ARG, "null argument");
    require_dev(c, bc, "mrhs_coarse_solve_noalloc bc");
    require_dev(c, xc, "mrhs_coarse_solve_noalloc xc");
    MRHS_REQUIRE(nrhs >= 1 && nrhs <= 256 && restart >= 1 && restart <= 64, MRHS_ERR_ARG,
                 "coarse solve: need 1 <= nrhs <= 256, 1 <= restart <= 64");
    MRHS_REQUIRE(dtype == MRHS_F64 || dtype == MRHS_F32, MRHS_ERR_ARG, "coarse fields are F64 or F32");
    int cur = -1;
    MRHS_CUDA(cudaGetDevice(&cur));
    MRHS_REQUIRE(cur == c->device, MRHS_ERR_ARG, "the context's device must be the current device");
    const size_t need = coarse_solve_ws_bytes(c, nrhs, dtype, restart);
    MRHS_REQUIRE(need <= kNoAllocBytes, MRHS_ERR_SHAPE,
                 "mrhs_coarse_solve_noalloc: this problem needs " + std::to_string(need) +
                     " bytes of workspace, more than the fixed " + std::to_string(kNoAllocBytes) +
                     " (reduce nrhs or restart, or use mrhs_coarse_solve)");
    void* ws = noalloc_address(c->device);
    coarse_solve_ws(c, bc, xc, nrhs, dtype, tol, restart, maxit, iters, ws, kNoAllocBytes);
  });
}
