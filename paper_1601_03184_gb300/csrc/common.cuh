// Shared definitions of the CUDA library: context, types, complex helpers,
// error handling and the internal launch interfaces between translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/mrhs.h"

namespace mrhs {

// ------------------------------------------------------------- errors -----
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define MRHS_CUDA(call)                                                                              \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess)                                                                           \
      throw ::mrhs::Error(e_ == cudaErrorMemoryAllocation ? MRHS_ERR_OOM : MRHS_ERR_CUDA,           \
                          std::string(#call) + ": " + cudaGetErrorString(e_));                       \
  } while (0)

#define MRHS_LAUNCH_CHECK(name)                                                                      \
  do {                                                                                               \
    cudaError_t e_ = cudaGetLastError();                                                             \
    if (e_ != cudaSuccess) throw ::mrhs::Error(MRHS_ERR_CUDA, std::string(name) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define MRHS_REQUIRE(cond, code, msg)                                                                \
  do {                                                                                               \
    if (!(cond)) throw ::mrhs::Error(code, msg);                                                     \
  } while (0)

// ------------------------------------------------------------ complex -----
template <class R>
struct cx {
  R re, im;
};

template <class R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) {
  cx<R> r;
  r.re = a;
  r.im = b;
  return r;
}
template <class R>
__host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk(a.re + b.re, a.im + b.im); }
template <class R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk(a.re - b.re, a.im - b.im); }
template <class R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class R>
__host__ __device__ __forceinline__ cx<R> scale(cx<R> a, R s) { return mk(a.re * s, a.im * s); }
template <class R>
__host__ __device__ __forceinline__ cx<R> cnj(cx<R> a) { return mk(a.re, -a.im); }
// i*a and -i*a
template <class R>
__host__ __device__ __forceinline__ cx<R> ti(cx<R> a) { return mk(-a.im, a.re); }
template <class R>
__host__ __device__ __forceinline__ cx<R> tmi(cx<R> a) { return mk(a.im, -a.re); }
// acc += a*b ; acc += conj(a)*b
template <class R>
__host__ __device__ __forceinline__ void fma_(cx<R>& acc, cx<R> a, cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
template <class R>
__host__ __device__ __forceinline__ void fmac_(cx<R>& acc, cx<R> a, cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}

// ------------------------------------------------------ storage types -----
template <class S>
struct Real {
  using type = float;
};
template <>
struct Real<double> {
  using type = double;
};

__device__ __forceinline__ double to_r(double v) { return v; }
__device__ __forceinline__ float to_r(float v) { return v; }
__device__ __forceinline__ float to_r(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_r(__half v) { return __half2float(v); }

// storage conversions; the float overloads keep FP32 data off the FP64 pipe
// (conversions to and from double run at the FP64 rate, which is low here)
template <class S>
__device__ __forceinline__ S from_r(double v);
template <class S>
__device__ __forceinline__ S from_r(float v);
template <>
__device__ __forceinline__ double from_r<double>(double v) { return v; }
template <>
__device__ __forceinline__ float from_r<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_r<__nv_bfloat16>(double v) { return __float2bfloat16((float)v); }
template <>
__device__ __forceinline__ __half from_r<__half>(double v) { return __float2half((float)v); }
template <>
__device__ __forceinline__ double from_r<double>(float v) { return (double)v; }
template <>
__device__ __forceinline__ float from_r<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_r<__nv_bfloat16>(float v) { return __float2bfloat16(v); }
template <>
__device__ __forceinline__ __half from_r<__half>(float v) { return __float2half(v); }

inline size_t dtype_size(int dt) {
  switch (dt) {
    case MRHS_F64: return 8;
    case MRHS_F32: return 4;
    case MRHS_BF16:
    case MRHS_F16: return 2;
  }
  throw Error(MRHS_ERR_ARG, "unknown dtype " + std::to_string(dt));
}

#define MRHS_DISPATCH(dt, S, ...)                                                                    \
  switch (dt) {                                                                                      \
    case MRHS_F64: { using S = double; __VA_ARGS__; } break;                                        \
    case MRHS_F32: { using S = float; __VA_ARGS__; } break;                                         \
    case MRHS_BF16: { using S = __nv_bfloat16; __VA_ARGS__; } break;                                \
    case MRHS_F16: { using S = __half; __VA_ARGS__; } break;                                        \
    default: throw ::mrhs::Error(MRHS_ERR_ARG, "unknown dtype " + std::to_string(dt));              \
  }

// interleaved field element index
__host__ __device__ __forceinline__ size_t fidx(size_t row, int reim, int N, int r) {
  return (row * 2 + reim) * (size_t)N + r;
}

// ------------------------------------------------------------ context -----
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Geometry {
  int L[4], a[4], nb[4];
  int V, Va, nagg;
};

struct NNState;  // nn.cu

}  // namespace mrhs

struct mrhs_ctx_s {
  mrhs::Geometry g;
  int ntv = 0, prec = 0;
  int dc_engine = 0;    // mrhs_dc_engine
  int block_len = 0;    // N_b of Alg. 2 for the setup phases (0: all ntv at once)
  int tv_dtype = 0;     // storage of test vectors and P
  int work_dtype = 0;   // storage/compute of smoother work fields, D_c, coarse fields (F64 or F32)
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 0;
  std::string err;
  size_t held_bytes = 0;
  std::vector<void*> allocs;

  // tables (device)
  int* nbr = nullptr;        // [V][8] device-order neighbours, bit 30 = t-boundary sign
  int* perm = nullptr;       // canonical site -> device site
  int* iperm = nullptr;      // device site -> canonical site
  int* aggnbr = nullptr;     // [nagg][8]
  int* blocks_col = nullptr; // [2][nagg/2] aggregate ids of colour 0, then colour 1
  int ncol[2] = {0, 0};
  int* colpos = nullptr;     // [nagg] position of every aggregate in its colour's list

  // gauge field and clover, device order
  double* U64 = nullptr;  // [V][4][9] complex
  float* U32 = nullptr;
  float* U20 = nullptr;   // [V][4][20]: FP32 links padded to 80 bytes (float4-aligned records)
  double* A64 = nullptr;  // [V][2][36]
  float* A32 = nullptr;
  double* Ainv64 = nullptr;  // [V][2][36] inverse clover term (even-odd smoother), built on first use
  float* Ainv32 = nullptr;
  bool have_clover_inv = false;
  int even_odd = 0;          // 1: SAP domain solves on the Schur complement of the even sites
  bool have_gauge = false, have_clover = false;

  // setup state
  void* tv = nullptr;   // [V][12][2][ntv] in tv_dtype
  void* P = nullptr;    // same
  void* Dc = nullptr;   // [nagg][9][2ntv][2ntv] complex in work dtype
  long long dc_version = 0;        // bumped by every build of D_c
  void* dc_img = nullptr;          // D_c as tensor-core operand images (coarse_tc.cu)
  long long dc_img_version = -1;   // the D_c version the images hold
  int dc_img_split = -1;           // 1: tf32 hi + lo images, 0: tf32 only
  void* dc_inv = nullptr;          // [nagg/2][2ntv][2ntv] inverse self blocks of the odd aggregates (list order)
  long long dc_inv_version = -1;   // the D_c version dc_inv holds
  int coarse_eo = 0;               // 1: coarse GMRES on the Schur complement of the even aggregates
  bool have_tv = false, have_P = false, have_Dc = false;
  // the setup stores its (unit-norm) test vectors multiplied by tv_scale:
  // sqrt(12 V) for fp16 storage (entries of order 1, inside the fp16 range),
  // 1 otherwise; every use of the stored vectors is invariant under scaling
  double tv_scale = 1.0;

  float* coef32 = nullptr;   // [65][256][2] float copy of BLAS coefficients
  int* dflag = nullptr;      // device error flag
  int* hflag = nullptr;      // pinned host mirror
  double* hbuf = nullptr;    // pinned host scratch
  size_t hbuf_bytes = 0;

  // named scratch buffers, grown on demand
  mrhs::DevBuf scratch[20];

  mrhs::NNState* nn = nullptr;  // learned test-vector generator (nn.cu)

  // per-kernel CUDA-event timing (off unless enabled through mrhs_profile)
  bool prof = false;
  std::vector<std::string> prof_names;        // kernel class names
  std::vector<long long> prof_launches;       // per name
  std::vector<double> prof_ms;                // per name, folded totals
  std::vector<cudaEvent_t> prof_events;       // pool, used in (start, stop) pairs
  std::vector<int> prof_rec_name;             // name of every recorded pair
  size_t prof_used = 0;                       // events of the pool in use
};

namespace mrhs {

enum Scratch {
  SC_STAGE = 0,   // host<->device staging
  SC_X,           // smoother iterate / work field
  SC_R,           // residual / rho
  SC_Q,           // q = D_B rho
  SC_ALPHA,       // per block per rhs MR coefficients
  SC_RED,         // reduction partials
  SC_GS,          // Gram-Schmidt workspace
  SC_KRYLOV,      // coarse Krylov basis
  SC_COARSE,      // coarse vectors for the refinement
  SC_HESS,        // Hessenberg and rotation data
  SC_FINE1,       // FGMRES work
  SC_FINE2,
  SC_FINE3,
  SC_KRYLOV_F,    // FGMRES basis
  SC_MISC,
  SC_BLOCK,       // one block of test vectors (block length N_b < ntv)
  SC_EO1,         // even-odd domain solves: rho (even sites) / A^-1 H rho (odd sites)
  SC_EO2,         // q (even) and e (both parities), interleaved as two fields
  SC_COARSE_EO,   // even-odd coarse solve: two operator work fields and bhat
  SC_COUNT
};

void* scratch(mrhs_ctx c, int which, size_t bytes);
// refuse (MRHS_ERR_ARG) a caller pointer of the wrong memory type before any
// launch or copy touches it: require_dev wants device memory of the
// context's GPU (or managed memory), require_host host memory (pageable,
// pinned or managed); a null pointer passes (optional arguments)
void require_dev(mrhs_ctx c, const void* p, const char* what);
void require_host(mrhs_ctx c, const void* p, const char* what);
void* dalloc(mrhs_ctx c, size_t bytes);
double* host_scratch(mrhs_ctx c, size_t bytes);

inline size_t fine_elems(const mrhs_ctx c, int nrhs) { return (size_t)c->g.V * 24 * nrhs; }
inline size_t coarse_elems(const mrhs_ctx c, int nrhs) { return (size_t)c->g.nagg * 2 * c->ntv * 2 * nrhs; }
inline int compute_dtype(int dtype) { return dtype == MRHS_F64 ? MRHS_F64 : MRHS_F32; }

inline int grid_for(size_t work, int block) { return (int)((work + block - 1) / block); }

// --------------------------------------------------- internal interfaces --
// dslash.cu
enum DslashMode { DS_FULL = 0, DS_BLOCK = 1, DS_RESID = 2 };
void dslash(mrhs_ctx c, const void* x, void* y, const void* b, int nrhs, int dtype, int mode, int colour);
void sap(mrhs_ctx c, const void* b, void* x, int nrhs, int dtype, int n_sweeps, int n_mr);
// gs.cu
void build_P(mrhs_ctx c);
// coarse.cu
void build_Dc(mrhs_ctx c);
// operand formats of the tensor-core contraction (tcgen05 instruction-descriptor codes)
constexpr int tc_fmt_f16 = 0, tc_fmt_bf16 = 1, tc_fmt_tf32 = 2;
bool build_Dc_tc(mrhs_ctx c, int fmt, bool split);
// A part of the coarse stencil y = D_c x: the aggregates alist[0..na) in
// that order (all aggregates in order when alist is null), the blocks
// kb <= k < ke of each (k = 0 the self block, 1+mu / 5+mu the hops); block 0
// reads x0 and the hop blocks xh, the row block of aggregate B at pos[B] (B
// when pos is null); row block b of y (and of add, y = stencil + add, when
// add is given) belongs to alist[b]. The plain stencil is {null, nagg, null,
// 0, 9, x, x, null}.
struct DcPart {
  const int* alist;
  int na;
  const int* pos;
  int kb, ke;
  const void* x0;
  const void* xh;
  const void* add;
};
// coarse stencil on the tensor cores; sets dflag[3] if a pipeline wait ran out
bool apply_Dc_tc(mrhs_ctx c, const DcPart& part, void* yc, int nrhs, bool split);
void apply_Dc_part(mrhs_ctx c, const DcPart& part, void* yc, int nrhs, int dtype);
// nn_tc.cu: one network layer for inference with bf16 tensor-core mixing
// (false: shape outside the kernel's); sets dflag[6] if a wait ran out
bool covconv_tc(mrhs_ctx c, const float* h, float* z, const float* W, int cin, int cout, int N);
void check_nn_tc_timeout(mrhs_ctx c);
void dc_images_build(mrhs_ctx c);
void check_tc_timeout(mrhs_ctx c);
void restrict_(mrhs_ctx c, const void* v, void* vc, int nrhs, int dtype);
void prolong(mrhs_ctx c, const void* uc, void* u, int nrhs, int dtype);
void apply_Dc(mrhs_ctx c, const void* xc, void* yc, int nrhs, int dtype);
void coarse_solve(mrhs_ctx c, const void* bc, void* xc, int nrhs, int dtype, double tol, int restart, int maxit,
                  int* iters);
// blas.cu: per right-hand-side reductions and updates on interleaved arrays of
// `rows` complex rows, each [2][N]
void multi_dot(mrhs_ctx c, const void* X, size_t stride, int K, const void* Y, size_t rows, int N, int dtype,
               double* out /* device [K][N][2] */);
void norms(mrhs_ctx c, const void* X, size_t rows, int N, int dtype, double* out /* device [N] (squared) */);
void convert(mrhs_ctx c, const void* x, int dx, void* y, int dy, size_t n);
void convert_scaled(mrhs_ctx c, const void* x, int dx, void* y, int dy, size_t n, float scale);
// blas.cu: T = X[., r] / |X[., r]| * scale in T's storage type, one pass after the norms
void normalise_into(mrhs_ctx c, const void* X, int dx, void* T, int dt, size_t rows, int N, float scale);
// columns k0 .. k0+nb-1 of a fine field of ntv right-hand sides to a field of
// nb (same storage type), and back with conversion and a scale factor
void gather_cols(mrhs_ctx c, const void* src, int ntv, void* dst, int nb, int k0, int dtype);
void scatter_cols(mrhs_ctx c, const void* src, int ds, int nb, void* dst, int dd, int ntv, int k0, float scale);
// x0_zero: the caller promises x = 0 on entry (the first domain solves then
// skip the product with the starting guess)
void sap_mixed(mrhs_ctx c, const void* b, int bdtype, void* x, int nrhs, int dtype, int n_sweeps, int n_mr,
               bool x0_zero = false);
void ensure_clover_inverse(mrhs_ctx c);
// sap.cu: the on-chip SAP (FP32 work fields)
bool sap_fused_ok(mrhs_ctx c, int dtype);
void sap_fused(mrhs_ctx c, const void* b, int bdtype, void* x, int nrhs, int n_sweeps, int n_mr, bool x0_zero = false);
bool sap_tm_ok(mrhs_ctx c, int nrhs);
bool sap_pk_ok(mrhs_ctx c, int nrhs);
void sap_pk(mrhs_ctx c, const void* b, int bdtype, void* x, int nrhs, int n_sweeps, int n_mr, bool x0_zero = false);
void sap_tm(mrhs_ctx c, const void* b, int bdtype, void* x, int nrhs, int n_sweeps, int n_mr);
// blas.cu: y[row][r] += sign * sum_k coef[k][r] * X_k[row][r], X_k = X + k*stride elements
void multi_axpy(mrhs_ctx c, const void* X, size_t stride, int K, void* Y, size_t rows, int N, int dtype,
                const double* coef /* device [K][N][2] */, double sign);
void normalise_rhs(mrhs_ctx c, void* X, size_t rows, int N, int dtype);
size_t multi_dot_partials_bytes(size_t rows, int N, int K);
void multi_dot_ws(mrhs_ctx c, const void* X, size_t stride, int K, const void* Y, size_t rows, int N, int dtype,
                  double* out, double* part);
// coarse.cu: the coarse solve on a caller-supplied workspace (no allocation)
size_t coarse_solve_ws_bytes(mrhs_ctx c, int nrhs, int dtype, int restart);
void coarse_solve_ws(mrhs_ctx c, const void* bc, void* xc, int nrhs, int dtype, double tol, int restart, int maxit,
                     int* iters, void* ws, size_t ws_bytes);

// RAII timer of one launch (or a group of launches) on the context stream
struct Prof {
  mrhs_ctx c;
  size_t idx = (size_t)-1;
  Prof(mrhs_ctx ctx, const char* name);
  ~Prof();
};

// nn.cu
void nn_forward(mrhs_ctx c, const float* in, float* out, int N);
void nn_infer(mrhs_ctx c, const float* in, float* out, int N);
void nn_destroy(mrhs_ctx c);

// every extern "C" entry point runs its body through this guard
std::string& create_error_slot();
template <class F>
int guarded(mrhs_ctx c, F&& f) {
  try {
    f();
    return MRHS_OK;
  } catch (const Error& e) {
    (c ? c->err : create_error_slot()) = e.what();
    return e.code;
  } catch (const std::exception& e) {
    (c ? c->err : create_error_slot()) = e.what();
    return MRHS_ERR_ARG;
  }
}

}  // namespace mrhs
