// Aggregate-wise orthonormalisation of the test vectors: P = R^dag.
//
// For every aggregate A and chirality h the ntv test vectors restricted to
// (sites of A) x (the 6 spin-colour components of chirality h) form an
// L x ntv matrix V (L = 6 |A|). P restricted there is the Q factor of the thin
// QR decomposition V = Q R with R upper triangular and positive real diagonal;
// that factor is unique, so any stable orthonormalisation in the order
// v_1, v_2, ... gives it. Here: Cholesky-QR applied twice (CholQR2):
//   G = V^dag V (double accumulation), G = L L^dag (Cholesky), Q = V L^-dag,
// then the same on Q. One CTA per (aggregate, chirality); the second pass
// repairs the loss of orthogonality of the first.
#include "common.cuh"

namespace mrhs {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 128;  // rows staged in shared memory at a time

// field row of row l (0 <= l < 6|A|) of group (A, h)
__device__ __forceinline__ size_t gs_row(int A, int h, int Va, int l) {
  return ((size_t)A * Va + l / 6) * 12 + 6 * h + (l % 6);
}

template <class S, class R>
__global__ void k_cholqr2(const S* V, S* Q, int N, int Va, int* flag) {
  extern __shared__ double smem[];
  const int A = blockIdx.x >> 1, h = blockIdx.x & 1;
  const int L = 6 * Va;
  const int ld = N + 1;  // padded row stride of the staged chunk
  cx<double>* G = (cx<double>*)smem;                 // [N][N]
  cx<R>* Lr = (cx<R>*)(G + N * N);                   // [N][N] Cholesky factor in R
  cx<R>* buf = Lr + N * N;                           // [kChunk][ld]
  double* dg = (double*)(buf + kChunk * ld);         // [N] diagonal of G before factorising
  const int tid = threadIdx.x;
  // a pivot below this fraction of its original diagonal (squared sine of the
  // angle between v_k and span(v_1..v_k-1)) is treated as linear dependence
  const double rel_pivot = 16.0 * (sizeof(R) == 8 ? 1.1102230246251565e-16 : 5.960464477539063e-08);
  for (int pass = 0; pass < 2; ++pass) {
    const S* src = pass == 0 ? V : Q;
    // ---- Gram matrix
    cx<double> acc[16];
    const int ne = (N * N + kThreads - 1) / kThreads;
    for (int e = 0; e < ne; ++e) acc[e] = mk(0.0, 0.0);
    for (int l0 = 0; l0 < L; l0 += kChunk) {
      int nl = min(kChunk, L - l0);
      for (int w = tid; w < nl * N; w += kThreads) {
        int l = w / N, j = w % N;
        size_t row = gs_row(A, h, Va, l0 + l);
        buf[l * ld + j] = mk<R>(to_r(src[fidx(row, 0, N, j)]), to_r(src[fidx(row, 1, N, j)]));
      }
      __syncthreads();
      for (int e = 0; e < ne; ++e) {
        int idx = tid + e * kThreads;
        if (idx >= N * N) break;
        int i = idx / N, j = idx % N;
        cx<R> p = mk<R>(0, 0);
        for (int l = 0; l < nl; ++l) fmac_(p, buf[l * ld + i], buf[l * ld + j]);
        acc[e].re += (double)p.re;
        acc[e].im += (double)p.im;
      }
      __syncthreads();
    }
    for (int e = 0; e < ne; ++e) {
      int idx = tid + e * kThreads;
      if (idx < N * N) G[idx] = acc[e];
    }
    __syncthreads();
    for (int k = tid; k < N; k += kThreads) dg[k] = G[k * N + k].re;
    __syncthreads();
    // ---- Cholesky G = L L^dag in place (lower triangle), double precision
    for (int k = 0; k < N; ++k) {
      if (tid == 0) {
        double d = G[k * N + k].re;
        if (!(d > rel_pivot * dg[k]) || !isfinite(d)) {
          atomicExch(flag, 1);
          d = 1;
        }
        G[k * N + k] = mk(sqrt(d), 0.0);
      }
      __syncthreads();
      double dk = G[k * N + k].re;
      for (int i = k + 1 + tid; i < N; i += kThreads) G[i * N + k] = scale(G[i * N + k], 1.0 / dk);
      __syncthreads();
      // trailing update G[i][j] -= L[i][k] conj(L[j][k]) for k < j <= i
      int m = N - k - 1;
      for (int w = tid; w < m * m; w += kThreads) {
        int i = k + 1 + w / m, j = k + 1 + w % m;
        if (j <= i) G[i * N + j] = G[i * N + j] - G[i * N + k] * cnj(G[j * N + k]);
      }
      __syncthreads();
    }
    for (int w = tid; w < N * N; w += kThreads) {
      int i = w / N, j = w % N;
      Lr[w] = j <= i ? mk<R>((R)G[w].re, (R)G[w].im) : mk<R>(0, 0);
    }
    __syncthreads();
    // ---- Q = V L^-dag: per row, q_j = (v_j - sum_{i<j} q_i conj(L_ji)) / L_jj
    for (int l0 = 0; l0 < L; l0 += kChunk) {
      int nl = min(kChunk, L - l0);
      for (int w = tid; w < nl * N; w += kThreads) {
        int l = w / N, j = w % N;
        size_t row = gs_row(A, h, Va, l0 + l);
        buf[l * ld + j] = mk<R>(to_r(src[fidx(row, 0, N, j)]), to_r(src[fidx(row, 1, N, j)]));
      }
      __syncthreads();
      for (int l = tid; l < nl; l += kThreads) {
        cx<R>* q = buf + l * ld;
        for (int j = 0; j < N; ++j) {
          cx<R> v = q[j];
          for (int i = 0; i < j; ++i) {
            cx<R> t = mk<R>(-q[i].re, -q[i].im);
            fmac_(v, Lr[j * N + i], t);  // v -= q_i * conj(L_ji)
          }
          q[j] = scale(v, (R)1 / Lr[j * N + j].re);
        }
      }
      __syncthreads();
      for (int w = tid; w < nl * N; w += kThreads) {
        int l = w / N, j = w % N;
        size_t row = gs_row(A, h, Va, l0 + l);
        Q[fidx(row, 0, N, j)] = from_r<S>(buf[l * ld + j].re);
        Q[fidx(row, 1, N, j)] = from_r<S>(buf[l * ld + j].im);
      }
      __syncthreads();
    }
  }
}

// Tiled Cholesky-QR twice for ntv <= 32. Gram matrix: every thread owns a
// 2x2 tile of G; the factor is inverted explicitly (M = L^-dag, upper
// triangular) and Q = X M is formed with 4-column tiles per row.
template <class S, class R>
__global__ void __launch_bounds__(256) k_cholqr2_tiled(const S* V, S* Q, int N, int Va, int* flag) {
  extern __shared__ double smem[];
  const int A = blockIdx.x >> 1, h = blockIdx.x & 1;
  const int L = 6 * Va;
  const int ld = N + 1;
  cx<double>* G = (cx<double>*)smem;                 // [N][N]
  cx<double>* Md = G + N * N;                        // [N][N] L^-dag in double
  cx<R>* Mr = (cx<R>*)(Md + N * N);                  // [N][N] L^-dag in R
  cx<R>* buf = Mr + N * N;                           // [kChunk][ld]
  double* dg = (double*)(buf + kChunk * ld);         // [N]
  const int tid = threadIdx.x;
  const double rel_pivot = 16.0 * (sizeof(R) == 8 ? 1.1102230246251565e-16 : 5.960464477539063e-08);
  const int nt2 = (N + 1) / 2;
  const int ti = tid / nt2, tj = tid % nt2;
  const bool gon = tid < nt2 * nt2;
  const int gi = 2 * ti, gj = 2 * tj;
  const int nct = (N + 3) / 4;
  for (int pass = 0; pass < 2; ++pass) {
    const S* src = pass == 0 ? V : Q;
    // ---- Gram matrix, 2x2 tiles
    cx<double> acc[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a) acc[a][0] = acc[a][1] = mk(0.0, 0.0);
    for (int l0 = 0; l0 < L; l0 += kChunk) {
      const int nl = min(kChunk, L - l0);
      for (int w = tid; w < nl * N; w += blockDim.x) {
        int l = w / N, j = w % N;
        size_t row = gs_row(A, h, Va, l0 + l);
        buf[l * ld + j] = mk<R>(to_r(src[fidx(row, 0, N, j)]), to_r(src[fidx(row, 1, N, j)]));
      }
      __syncthreads();
      if (gon) {
        cx<R> p[2][2];
#pragma unroll
        for (int a = 0; a < 2; ++a) p[a][0] = p[a][1] = mk<R>(0, 0);
        const int i1 = min(gi + 1, N - 1), j1 = min(gj + 1, N - 1);
        for (int l = 0; l < nl; ++l) {
          cx<R> xi0 = buf[l * ld + gi], xi1 = buf[l * ld + i1];
          cx<R> xj0 = buf[l * ld + gj], xj1 = buf[l * ld + j1];
          fmac_(p[0][0], xi0, xj0);
          fmac_(p[0][1], xi0, xj1);
          fmac_(p[1][0], xi1, xj0);
          fmac_(p[1][1], xi1, xj1);
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 2; ++b) {
            acc[a][b].re += (double)p[a][b].re;
            acc[a][b].im += (double)p[a][b].im;
          }
      }
      __syncthreads();
    }
    if (gon) {
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
          if (gi + a < N && gj + b < N) G[(gi + a) * N + gj + b] = acc[a][b];
    }
    __syncthreads();
    for (int k = tid; k < N; k += blockDim.x) dg[k] = G[k * N + k].re;
    __syncthreads();
    // ---- Cholesky G = L L^dag (lower triangle, in place)
    for (int k = 0; k < N; ++k) {
      if (tid == 0) {
        double d = G[k * N + k].re;
        if (!(d > rel_pivot * dg[k]) || !isfinite(d)) {
          atomicExch(flag, 1);
          d = 1;
        }
        G[k * N + k] = mk(sqrt(d), 0.0);
      }
      __syncthreads();
      const double dk = G[k * N + k].re;
      for (int i = k + 1 + tid; i < N; i += blockDim.x) G[i * N + k] = scale(G[i * N + k], 1.0 / dk);
      __syncthreads();
      const int m = N - k - 1;
      for (int w = tid; w < m * m; w += blockDim.x) {
        int i = k + 1 + w / m, j = k + 1 + w % m;
        if (j <= i) G[i * N + j] = G[i * N + j] - G[i * N + k] * cnj(G[j * N + k]);
      }
      __syncthreads();
    }
    // ---- M = L^-dag (upper triangular): L^dag M = 1, column j by back substitution
    for (int j = tid; j < N; j += blockDim.x) {
      for (int i = N - 1; i >= 0; --i) {
        if (i > j) {
          Md[i * N + j] = mk(0.0, 0.0);
          continue;
        }
        cx<double> sacc = i == j ? mk(1.0, 0.0) : mk(0.0, 0.0);
        for (int k2 = i + 1; k2 <= j; ++k2) sacc = sacc - cnj(G[k2 * N + i]) * Md[k2 * N + j];
        Md[i * N + j] = scale(sacc, 1.0 / G[i * N + i].re);
      }
    }
    __syncthreads();
    for (int w = tid; w < N * N; w += blockDim.x) Mr[w] = mk<R>((R)Md[w].re, (R)Md[w].im);
    __syncthreads();
    // ---- Q = X M, rows staged in chunks, 4 output columns per item
    for (int l0 = 0; l0 < L; l0 += kChunk) {
      const int nl = min(kChunk, L - l0);
      for (int w = tid; w < nl * N; w += blockDim.x) {
        int l = w / N, j = w % N;
        size_t row = gs_row(A, h, Va, l0 + l);
        buf[l * ld + j] = mk<R>(to_r(src[fidx(row, 0, N, j)]), to_r(src[fidx(row, 1, N, j)]));
      }
      __syncthreads();
      for (int w = tid; w < nl * nct; w += blockDim.x) {
        const int l = w / nct, j0 = 4 * (w % nct);
        cx<R> o[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) o[b] = mk<R>(0, 0);
        const int iend = min(N, j0 + 4);
        for (int i = 0; i < iend; ++i) {
          cx<R> xv = buf[l * ld + i];
#pragma unroll
          for (int b = 0; b < 4; ++b)
            if (j0 + b < N) fma_(o[b], xv, Mr[i * N + j0 + b]);
        }
        size_t row = gs_row(A, h, Va, l0 + l);
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if (j0 + b < N) {
            Q[fidx(row, 0, N, j0 + b)] = from_r<S>(o[b].re);
            Q[fidx(row, 1, N, j0 + b)] = from_r<S>(o[b].im);
          }
      }
      __syncthreads();
    }
  }
}

}  // namespace

void build_P(mrhs_ctx c) {
  MRHS_REQUIRE(c->have_tv, MRHS_ERR_STATE, "mrhs_build_P before test vectors exist");
  const int N = c->ntv;
  MRHS_REQUIRE(N * N <= 16 * kThreads, MRHS_ERR_SHAPE, "ntv too large for the Gram-Schmidt kernel");
  if (!c->P) c->P = dalloc(c, fine_elems(c, N) * dtype_size(c->tv_dtype));
  MRHS_CUDA(cudaMemsetAsync(c->dflag, 0, sizeof(int), c->stream));
  MRHS_DISPATCH(c->tv_dtype, S, {
    Prof pr(c, "gs_cholqr2");
    using R = typename Real<S>::type;
    if (N <= 32) {
      size_t smem = 2 * sizeof(cx<double>) * N * N + sizeof(cx<R>) * (N * N + (size_t)kChunk * (N + 1)) +
                    sizeof(double) * N;
      MRHS_CUDA(cudaFuncSetAttribute(k_cholqr2_tiled<S, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_cholqr2_tiled<S, R><<<2 * c->g.nagg, kThreads, smem, c->stream>>>((const S*)c->tv, (S*)c->P, N, c->g.Va,
                                                                          c->dflag);
    } else {
      size_t smem = sizeof(cx<double>) * N * N + sizeof(cx<R>) * (N * N + (size_t)kChunk * (N + 1)) + sizeof(double) * N;
      MRHS_CUDA(cudaFuncSetAttribute(k_cholqr2<S, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_cholqr2<S, R><<<2 * c->g.nagg, kThreads, smem, c->stream>>>((const S*)c->tv, (S*)c->P, N, c->g.Va, c->dflag);
    }
  });
  MRHS_LAUNCH_CHECK("cholqr2");
  MRHS_CUDA(cudaMemcpyAsync(c->hflag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MRHS_CUDA(cudaStreamSynchronize(c->stream));
  c->have_P = false;
  c->have_Dc = false;
  MRHS_REQUIRE(c->hflag[0] == 0, MRHS_ERR_NONFINITE,
               "Gram-Schmidt: test vectors are linearly dependent or not finite on some aggregate");
  c->have_P = true;
}

}  // namespace mrhs

using namespace mrhs;

extern "C" int mrhs_build_P(mrhs_ctx c) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c, MRHS_ERR_ARG, "null context");
    build_P(c);
  });
}
