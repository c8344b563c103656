// BLAS-like operations on interleaved multi-RHS arrays (Sec. 5 of the paper:
// with the right-hand sides innermost these are elementwise per RHS; the
// global sums are taken for all right-hand sides in one pass).
// Arrays are `rows` complex rows of [2][N]: element (row, re/im, rhs).
// Reductions use a fixed two-level tree (per-CTA partials, then a fixed-order
// sum), so results are bitwise reproducible.
#include <algorithm>
#include <cstdint>

#include "common.cuh"

namespace mrhs {
namespace {

constexpr int kBlock = 256;

int n_chunks(size_t rows, int N) {
  size_t work = rows * (size_t)N;
  size_t ch = work / (kBlock * 64);
  if (ch < 1) ch = 1;
  if (ch > 2048) ch = 2048;
  return (int)ch;
}

// partial[k][chunk][r] = sum over the chunk's rows of conj(X_k) * Y, for the
// group of up to kKG vectors k = kKG*blockIdx.y + j: every element of Y read
// serves the whole group
constexpr int kKG = 8;

template <class S>
__global__ void __launch_bounds__(kBlock) k_multi_dot(const S* X, size_t stride, int K, const S* Y, size_t rows, int N,
                                                      int nchunk, double* part) {
  using R = typename Real<S>::type;
  __shared__ double sre[kBlock], sim[kBlock];
  const int k0 = blockIdx.y * kKG, ch = blockIdx.x;
  const int nk = min(kKG, K - k0);
  const size_t r0 = rows * ch / nchunk, r1 = rows * (ch + 1) / nchunk;
  const int lanes = blockDim.x / N;
  const int tid = threadIdx.x, r = tid % N, lane = tid / N;
  double are[kKG], aim[kKG];
  R pre[kKG], pim[kKG];
#pragma unroll
  for (int j = 0; j < kKG; ++j) are[j] = aim[j] = 0, pre[j] = pim[j] = 0;
  if (lane < lanes) {
    int cnt = 0;
    for (size_t row = r0 + lane; row < r1; row += lanes) {
      const R yr = to_r(Y[fidx(row, 0, N, r)]), yi = to_r(Y[fidx(row, 1, N, r)]);
#pragma unroll
      for (int j = 0; j < kKG; ++j) {
        if (j < nk) {
          const S* Xk = X + (size_t)(k0 + j) * stride;
          const R xr = to_r(Xk[fidx(row, 0, N, r)]), xi = to_r(Xk[fidx(row, 1, N, r)]);
          pre[j] = fma(xr, yr, fma(xi, yi, pre[j]));
          pim[j] = fma(xr, yi, fma(-xi, yr, pim[j]));
        }
      }
      if (++cnt == 32) {
#pragma unroll
        for (int j = 0; j < kKG; ++j) are[j] += pre[j], aim[j] += pim[j], pre[j] = pim[j] = 0;
        cnt = 0;
      }
    }
#pragma unroll
    for (int j = 0; j < kKG; ++j) are[j] += pre[j], aim[j] += pim[j];
  }
  for (int j = 0; j < nk; ++j) {
    sre[tid] = are[j];
    sim[tid] = aim[j];
    __syncthreads();
    if (tid < N) {
      double a = 0, b = 0;
      for (int l = 0; l < lanes; ++l) {
        a += sre[l * N + tid];
        b += sim[l * N + tid];
      }
      double* o = part + (((size_t)(k0 + j) * nchunk + ch) * N + tid) * 2;
      o[0] = a;
      o[1] = b;
    }
    __syncthreads();
  }
}

// The same for FP32 arrays with N % 4 == 0: a thread takes four right-hand
// sides (16-byte loads of the real and the imaginary row) and sums its rows
// of the chunk in FP32 before the CTA adds the threads' sums in FP64. Used
// when a thread has at most kMaxRows4 rows of the chunk (the coarse fields).
constexpr int kMaxRows4 = 128;

constexpr int kKG4 = 4;  // vectors per group (register budget of 16 FP32 sums each)

__global__ void __launch_bounds__(kBlock, 2) k_multi_dot4(const float* __restrict__ X, size_t stride, int K,
                                                          const float* __restrict__ Y, size_t rows, int N, int nchunk,
                                                          double* __restrict__ part) {
  constexpr int kKG = kKG4;
  __shared__ double sre[4 * kBlock], sim[4 * kBlock];  // [lanes][N]
  const int k0 = blockIdx.y * kKG, ch = blockIdx.x;
  const int nk = min(kKG, K - k0);
  const size_t r0 = rows * ch / nchunk, r1 = rows * (ch + 1) / nchunk;
  const int Q = N / 4, lanes = kBlock / Q;
  const int tid = threadIdx.x, q = tid % Q, lane = tid / Q;
  float pre[kKG][4], pim[kKG][4];
#pragma unroll
  for (int j = 0; j < kKG; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) pre[j][e] = pim[j][e] = 0.f;
  if (lane < lanes) {
    for (size_t row = r0 + lane; row < r1; row += lanes) {
      const float4 yr = *reinterpret_cast<const float4*>(Y + fidx(row, 0, N, 4 * q));
      const float4 yi = *reinterpret_cast<const float4*>(Y + fidx(row, 1, N, 4 * q));
#pragma unroll
      for (int j = 0; j < kKG; ++j) {
        if (j < nk) {
          const float* Xk = X + (size_t)(k0 + j) * stride;
          const float4 xr = *reinterpret_cast<const float4*>(Xk + fidx(row, 0, N, 4 * q));
          const float4 xi = *reinterpret_cast<const float4*>(Xk + fidx(row, 1, N, 4 * q));
          const float xre[4] = {xr.x, xr.y, xr.z, xr.w}, xim[4] = {xi.x, xi.y, xi.z, xi.w};
          const float yre[4] = {yr.x, yr.y, yr.z, yr.w}, yim[4] = {yi.x, yi.y, yi.z, yi.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            pre[j][e] = fmaf(xre[e], yre[e], fmaf(xim[e], yim[e], pre[j][e]));
            pim[j][e] = fmaf(xre[e], yim[e], fmaf(-xim[e], yre[e], pim[j][e]));
          }
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kKG; ++j) {
    if (j >= nk) break;
    if (lane < lanes) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        sre[lane * N + 4 * q + e] = (double)pre[j][e];
        sim[lane * N + 4 * q + e] = (double)pim[j][e];
      }
    }
    __syncthreads();
    if (tid < N) {
      double a = 0, b = 0;
      for (int l = 0; l < lanes; ++l) {
        a += sre[l * N + tid];
        b += sim[l * N + tid];
      }
      double* o = part + (((size_t)(k0 + j) * nchunk + ch) * N + tid) * 2;
      o[0] = a;
      o[1] = b;
    }
    __syncthreads();
  }
}

// out[k][r] = sum over the chunks of part[k][chunk][r]: one warp per (k, r),
// lane l adds chunks l, l+32, ... and the lanes are joined by a fixed
// butterfly, so the order of the sum does not depend on timing
__global__ void k_sum_chunks(const double* part, int K, int nchunk, int N, double* out) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (t >= K * N) return;
  const int k = t / N, r = t % N;
  double a = 0, b = 0;
  for (int ch = lane; ch < nchunk; ch += 32) {
    a += part[(((size_t)k * nchunk + ch) * N + r) * 2];
    b += part[(((size_t)k * nchunk + ch) * N + r) * 2 + 1];
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) {
    out[2 * t] = a;
    out[2 * t + 1] = b;
  }
}

// coefficients sign*coef in the compute precision, once per (k, r)
__global__ void k_coef_to_float(const double* coef, double sign, float* out, int n) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = (float)(sign * coef[t]);
}

template <class S, class C>
__global__ void k_multi_axpy(const S* X, size_t stride, int K, S* Y, size_t rows, int N, const C* coef, C sign) {
  using R = typename Real<S>::type;
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= rows * N) return;
  int r = (int)(t % N);
  size_t row = t / N;
  R yr = to_r(Y[fidx(row, 0, N, r)]), yi = to_r(Y[fidx(row, 1, N, r)]);
  for (int k = 0; k < K; ++k) {
    R cr = (R)(sign * coef[((size_t)k * N + r) * 2]), ci = (R)(sign * coef[((size_t)k * N + r) * 2 + 1]);
    const S* Xk = X + (size_t)k * stride;
    R xr = to_r(Xk[fidx(row, 0, N, r)]), xi = to_r(Xk[fidx(row, 1, N, r)]);
    yr = fma(cr, xr, fma(-ci, xi, yr));
    yi = fma(cr, xi, fma(ci, xr, yi));
  }
  Y[fidx(row, 0, N, r)] = from_r<S>(yr);
  Y[fidx(row, 1, N, r)] = from_r<S>(yi);
}

// FP32, N % 4 == 0: four right-hand sides per thread, 16-byte loads and
// stores (the scalar kernel's operations in its order: the same bits)
__global__ void k_multi_axpy4(const float* __restrict__ X, size_t stride, int K, float* __restrict__ Y, size_t rows,
                              int N, const float* __restrict__ coef) {
  const int Q = N / 4;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= rows * Q) return;
  const int q = (int)(t % Q);
  const size_t row = t / Q;
  float4* py = reinterpret_cast<float4*>(Y + fidx(row, 0, N, 4 * q));
  float4* pyi = reinterpret_cast<float4*>(Y + fidx(row, 1, N, 4 * q));
  const float4 y0 = *py, y1 = *pyi;
  float yr[4] = {y0.x, y0.y, y0.z, y0.w}, yi[4] = {y1.x, y1.y, y1.z, y1.w};
  for (int k = 0; k < K; ++k) {
    const float4 c01 = *reinterpret_cast<const float4*>(coef + ((size_t)k * N + 4 * q) * 2);
    const float4 c23 = *reinterpret_cast<const float4*>(coef + ((size_t)k * N + 4 * q) * 2 + 4);
    const float cr[4] = {c01.x, c01.z, c23.x, c23.z}, ci[4] = {c01.y, c01.w, c23.y, c23.w};
    const float* Xk = X + (size_t)k * stride;
    const float4 x0 = *reinterpret_cast<const float4*>(Xk + fidx(row, 0, N, 4 * q));
    const float4 x1 = *reinterpret_cast<const float4*>(Xk + fidx(row, 1, N, 4 * q));
    const float xr[4] = {x0.x, x0.y, x0.z, x0.w}, xi[4] = {x1.x, x1.y, x1.z, x1.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      yr[e] = fmaf(cr[e], xr[e], fmaf(-ci[e], xi[e], yr[e]));
      yi[e] = fmaf(cr[e], xi[e], fmaf(ci[e], xr[e], yi[e]));
    }
  }
  *py = make_float4(yr[0], yr[1], yr[2], yr[3]);
  *pyi = make_float4(yi[0], yi[1], yi[2], yi[3]);
}

// s[r] = 1/sqrt(nrm2[r]) (0 for a zero vector), once per right-hand side
__global__ void k_inv_sqrt(const double* nrm2, double* s, int N) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  double n = nrm2[2 * r];
  s[r] = n > 0 ? 1.0 / sqrt(n) : 0.0;
}

// X[., r] *= s[r]
template <class S>
__global__ void k_scale_by(S* X, size_t rows, int N, const double* s) {
  using R = typename Real<S>::type;
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= rows * N) return;
  int r = (int)(t % N);
  size_t row = t / N;
  R f = (R)s[r];
  X[fidx(row, 0, N, r)] = from_r<S>(to_r(X[fidx(row, 0, N, r)]) * f);
  X[fidx(row, 1, N, r)] = from_r<S>(to_r(X[fidx(row, 1, N, r)]) * f);
}

// the four-RHS kernels need FP32, N % 4 == 0 and 16-byte aligned rows
bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }
bool use_dot4(const void* X, size_t stride, const void* Y, size_t rows, int N, int dtype, int nch) {
  if (dtype != MRHS_F32 || N % 4 != 0 || N > 4 * kBlock || !aligned16(X) || !aligned16(Y) || stride % 4 != 0)
    return false;
  const size_t lanes = kBlock / (N / 4);
  return (rows / nch + lanes - 1) / lanes <= (size_t)kMaxRows4;
}

}  // namespace

void multi_dot(mrhs_ctx c, const void* X, size_t stride, int K, const void* Y, size_t rows, int N, int dtype,
               double* out) {
  MRHS_REQUIRE(N >= 1 && N <= kBlock && K >= 1, MRHS_ERR_ARG, "multi_dot: bad sizes");
  int nch = n_chunks(rows, N);
  double* part = (double*)scratch(c, SC_RED, sizeof(double) * 2 * (size_t)K * nch * N);
  dim3 grid(nch, (K + kKG - 1) / kKG);
  Prof pr(c, "multi_dot");
  if (use_dot4(X, stride, Y, rows, N, dtype, nch))
    k_multi_dot4<<<dim3(nch, (K + kKG4 - 1) / kKG4), kBlock, 0, c->stream>>>((const float*)X, stride, K,
                                                                             (const float*)Y, rows, N, nch, part);
  else
    MRHS_DISPATCH(dtype, S, (k_multi_dot<S><<<grid, kBlock, 0, c->stream>>>((const S*)X, stride, K, (const S*)Y, rows, N, nch, part)));
  MRHS_LAUNCH_CHECK("multi_dot");
  k_sum_chunks<<<grid_for((size_t)K * N * 32, 256), 256, 0, c->stream>>>(part, K, nch, N, out);
  MRHS_LAUNCH_CHECK("sum_chunks");
}

// multi_dot with the per-CTA partials in a caller-supplied buffer of at
// least multi_dot_partials_bytes(rows, N, K) bytes (no allocation)
size_t multi_dot_partials_bytes(size_t rows, int N, int K) {
  return sizeof(double) * 2 * (size_t)K * n_chunks(rows, N) * N;
}

void multi_dot_ws(mrhs_ctx c, const void* X, size_t stride, int K, const void* Y, size_t rows, int N, int dtype,
                  double* out, double* part) {
  MRHS_REQUIRE(N >= 1 && N <= kBlock && K >= 1, MRHS_ERR_ARG, "multi_dot: bad sizes");
  int nch = n_chunks(rows, N);
  dim3 grid(nch, (K + kKG - 1) / kKG);
  Prof pr(c, "multi_dot");
  if (use_dot4(X, stride, Y, rows, N, dtype, nch))
    k_multi_dot4<<<dim3(nch, (K + kKG4 - 1) / kKG4), kBlock, 0, c->stream>>>((const float*)X, stride, K,
                                                                             (const float*)Y, rows, N, nch, part);
  else
    MRHS_DISPATCH(dtype, S, (k_multi_dot<S><<<grid, kBlock, 0, c->stream>>>((const S*)X, stride, K, (const S*)Y, rows, N, nch, part)));
  MRHS_LAUNCH_CHECK("multi_dot");
  k_sum_chunks<<<grid_for((size_t)K * N * 32, 256), 256, 0, c->stream>>>(part, K, nch, N, out);
  MRHS_LAUNCH_CHECK("sum_chunks");
}

// out[r] (as [N][2], imaginary part 0) = |X_r|^2
void norms(mrhs_ctx c, const void* X, size_t rows, int N, int dtype, double* out) {
  multi_dot(c, X, 0, 1, X, rows, N, dtype, out);
}

void multi_axpy(mrhs_ctx c, const void* X, size_t stride, int K, void* Y, size_t rows, int N, int dtype,
                const double* coef, double sign) {
  size_t work = rows * N;
  Prof pr(c, "multi_axpy");
  if (dtype == MRHS_F64) {
    k_multi_axpy<double, double><<<grid_for(work, kBlock), kBlock, 0, c->stream>>>((const double*)X, stride, K, (double*)Y, rows, N, coef, sign);
  } else {
    MRHS_REQUIRE(K <= 65 && N <= 256, MRHS_ERR_ARG, "multi_axpy: K <= 65 and N <= 256");
    const int n = 2 * K * N;
    k_coef_to_float<<<grid_for(n, 256), 256, 0, c->stream>>>(coef, sign, c->coef32, n);
    if (dtype == MRHS_F32 && N % 4 == 0 && aligned16(X) && aligned16(Y) && stride % 4 == 0)
      k_multi_axpy4<<<grid_for(rows * (N / 4), kBlock), kBlock, 0, c->stream>>>((const float*)X, stride, K, (float*)Y,
                                                                                rows, N, (const float*)c->coef32);
    else
      MRHS_DISPATCH(dtype, S, (k_multi_axpy<S, float><<<grid_for(work, kBlock), kBlock, 0, c->stream>>>((const S*)X, stride, K, (S*)Y, rows, N, (const float*)c->coef32, 1.0f)));
  }
  MRHS_LAUNCH_CHECK("multi_axpy");
}

// normalise every right-hand side of X to unit 2-norm
namespace {
// |X[., r]|^2 of a fine FP32 field (N / 4 divides 256, 16-byte aligned rows):
// thread (quad of right-hand sides, lane) over a grid-stride range of rows,
// FP32 sums over 64 rows at a time added into FP64; the lanes of a quad summed
// in a fixed order, then the CTAs (k_norm2_sum)
constexpr int kNormCtas = 608;
__global__ void __launch_bounds__(kBlock) k_norm2_4(const float* __restrict__ X, size_t rows, int N,
                                                    double* __restrict__ part) {
  __shared__ double sh[kBlock * 4];
  const int nq = N / 4, lanes = kBlock / nq;
  const int q = threadIdx.x % nq, lane = threadIdx.x / nq;
  double acc[4] = {0, 0, 0, 0};
  float f[4] = {0.f, 0.f, 0.f, 0.f};
  int cnt = 0;
  for (size_t row = (size_t)blockIdx.x * lanes + lane; row < rows; row += (size_t)gridDim.x * lanes) {
    const float4 re = __ldg(reinterpret_cast<const float4*>(X + row * 2 * N + 4 * q));
    const float4 im = __ldg(reinterpret_cast<const float4*>(X + row * 2 * N + N + 4 * q));
    f[0] = fmaf(re.x, re.x, fmaf(im.x, im.x, f[0]));
    f[1] = fmaf(re.y, re.y, fmaf(im.y, im.y, f[1]));
    f[2] = fmaf(re.z, re.z, fmaf(im.z, im.z, f[2]));
    f[3] = fmaf(re.w, re.w, fmaf(im.w, im.w, f[3]));
    if (++cnt == 64) {
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[e] += f[e], f[e] = 0.f;
      cnt = 0;
    }
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) sh[lane * N + 4 * q + e] = acc[e] + f[e];
  __syncthreads();
  if (threadIdx.x < N) {
    double t = 0;
    for (int l = 0; l < lanes; ++l) t += sh[l * N + threadIdx.x];
    part[(size_t)blockIdx.x * N + threadIdx.x] = t;
  }
}
__global__ void k_norm2_sum(const double* part, int nblk, int N, double* out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  double t = 0;
  for (int b = 0; b < nblk; ++b) t += part[(size_t)b * N + r];
  out[2 * r] = t;
  out[2 * r + 1] = 0;
}

// tv = (X[., r] * s[r]) * scale in the storage type of tv: the normalised
// vectors converted in one pass (the same two roundings as scaling X in
// place and converting it)
template <class SI, class SO>
__global__ void k_scale_convert(const SI* __restrict__ X, SO* __restrict__ T, size_t rows, int N,
                                const double* __restrict__ s, float scale) {
  using R = typename Real<SI>::type;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= rows * 2 * N) return;
  const int r = (int)(t % N);
  const R v = (R)(to_r(X[t]) * (R)s[r]);
  T[t] = from_r<SO>(v * (R)scale);
}

// the same four values at a time for FP32 X (N % 4 == 0, 16-byte aligned)
template <class SO>
__device__ __forceinline__ void store4(SO* p, float a, float b, float c, float d);
template <>
__device__ __forceinline__ void store4<float>(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
template <>
__device__ __forceinline__ void store4<double>(double* p, float a, float b, float c, float d) {
  p[0] = a, p[1] = b, p[2] = c, p[3] = d;
}
template <>
__device__ __forceinline__ void store4<__nv_bfloat16>(__nv_bfloat16* p, float a, float b, float c, float d) {
  __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
  *reinterpret_cast<uint2*>(p) = make_uint2(*reinterpret_cast<uint32_t*>(&lo), *reinterpret_cast<uint32_t*>(&hi));
}
template <>
__device__ __forceinline__ void store4<__half>(__half* p, float a, float b, float c, float d) {
  __half2 lo = __floats2half2_rn(a, b), hi = __floats2half2_rn(c, d);
  *reinterpret_cast<uint2*>(p) = make_uint2(*reinterpret_cast<uint32_t*>(&lo), *reinterpret_cast<uint32_t*>(&hi));
}
// resident CTAs per SM of k_scale_convert4 (256 threads each)
constexpr int kScaleCtasPerSm = 8;
// loads in flight per thread in k_scale_convert4
constexpr int kScaleUnroll = 4;

// the same four values at a time for FP32 X on a persistent grid: the
// grid-stride step is a multiple of N/4 float4, so a thread keeps the same
// four right-hand sides (and their factors) throughout, and it keeps
// kScaleUnroll loads in flight; the products are those of k_scale_convert
template <class SO>
__global__ void __launch_bounds__(kBlock) k_scale_convert4(const float* __restrict__ X, SO* __restrict__ T, size_t n4,
                                                           int N, const double* __restrict__ s, float scale) {
  const int nq = N / 4;
  const size_t G = (size_t)gridDim.x * blockDim.x;
  const size_t step = G - G % (size_t)nq;
  const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t0 >= step) return;
  const int r = 4 * (int)(t0 % (size_t)nq);
  const float s0 = (float)s[r], s1 = (float)s[r + 1], s2 = (float)s[r + 2], s3 = (float)s[r + 3];
  const float4* X4 = reinterpret_cast<const float4*>(X);
  size_t t = t0;
  for (; t + (kScaleUnroll - 1) * step < n4; t += kScaleUnroll * step) {
    float4 v[kScaleUnroll];
#pragma unroll
    for (int u = 0; u < kScaleUnroll; ++u) v[u] = __ldg(X4 + t + u * step);
#pragma unroll
    for (int u = 0; u < kScaleUnroll; ++u)
      store4<SO>(T + 4 * (t + u * step), (v[u].x * s0) * scale, (v[u].y * s1) * scale, (v[u].z * s2) * scale,
                 (v[u].w * s3) * scale);
  }
  for (; t < n4; t += step) {
    const float4 v = __ldg(X4 + t);
    store4<SO>(T + 4 * t, (v.x * s0) * scale, (v.y * s1) * scale, (v.z * s2) * scale, (v.w * s3) * scale);
  }
}

void norms_of_field(mrhs_ctx c, const void* X, size_t rows, int N, int dtype, double* nrm) {
  if (dtype == MRHS_F32 && N % 4 == 0 && kBlock % (N / 4) == 0 && aligned16(X)) {
    double* part = (double*)scratch(c, SC_RED, sizeof(double) * kNormCtas * (size_t)N);
    Prof pr(c, "norms");
    k_norm2_4<<<kNormCtas, kBlock, 0, c->stream>>>((const float*)X, rows, N, part);
    MRHS_LAUNCH_CHECK("norm2_4");
    k_norm2_sum<<<grid_for(N, 64), 64, 0, c->stream>>>(part, kNormCtas, N, nrm);
    MRHS_LAUNCH_CHECK("norm2_sum");
    return;
  }
  norms(c, X, rows, N, dtype, nrm);
}
}  // namespace

// T = X / |X[., r]| * scale in T's storage type (X unchanged)
void normalise_into(mrhs_ctx c, const void* X, int dx, void* T, int dt, size_t rows, int N, float scale) {
  double* nrm = (double*)scratch(c, SC_MISC, sizeof(double) * 3 * N);
  norms_of_field(c, X, rows, N, dx, nrm);
  k_inv_sqrt<<<grid_for(N, 64), 64, 0, c->stream>>>(nrm, nrm + 2 * N, N);
  MRHS_LAUNCH_CHECK("inv_sqrt");
  const size_t work = rows * 2 * N;
  Prof pr(c, "normalise");
  const size_t n4 = work / 4;
  const int grid = (int)std::min<size_t>((size_t)std::max(c->num_sms, 1) * kScaleCtasPerSm, (n4 + kBlock - 1) / kBlock);
  // (the persistent form needs a grid of at least N/4 threads)
  if (dx == MRHS_F32 && dt != MRHS_F64 && N % 4 == 0 && aligned16(X) && aligned16(T) &&
      (size_t)grid * kBlock >= (size_t)(N / 4)) {
    MRHS_DISPATCH(dt, SO, (k_scale_convert4<SO><<<grid, kBlock, 0, c->stream>>>((const float*)X, (SO*)T, n4, N, nrm + 2 * N, scale)));
    MRHS_LAUNCH_CHECK("scale_convert4");
    return;
  }
  MRHS_DISPATCH(dx, SI, MRHS_DISPATCH(dt, SO, (k_scale_convert<SI, SO><<<grid_for(work, kBlock), kBlock, 0, c->stream>>>((const SI*)X, (SO*)T, rows, N, nrm + 2 * N, scale))));
  MRHS_LAUNCH_CHECK("scale_convert");
}

void normalise_rhs(mrhs_ctx c, void* X, size_t rows, int N, int dtype) {
  double* nrm = (double*)scratch(c, SC_MISC, sizeof(double) * 3 * N);
  norms_of_field(c, X, rows, N, dtype, nrm);
  k_inv_sqrt<<<grid_for(N, 64), 64, 0, c->stream>>>(nrm, nrm + 2 * N, N);
  MRHS_LAUNCH_CHECK("inv_sqrt");
  size_t work = rows * N;
  Prof pr(c, "normalise");
  MRHS_DISPATCH(dtype, S, (k_scale_by<S><<<grid_for(work, kBlock), kBlock, 0, c->stream>>>((S*)X, rows, N, nrm + 2 * N)));
  MRHS_LAUNCH_CHECK("normalise");
}

}  // namespace mrhs
