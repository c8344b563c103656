// Aggregate-wise orthonormalisation of the test vectors: P = R^dag (Sec. 2
// of the paper; split by chirality as in Algorithm 3, Sec. 5).
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

// ---------------------------------------------------------------------------
// Cholesky-QR twice for ntv = NC, NC % 4 == 0, NC <= 32, with the work in
// register tiles:
//  - Gram matrix: only the lower triangle (the Cholesky factorisation reads
//    nothing else), 4x4 tiles of G, the rows of the group split over
//    kThreads / (#tiles) slices; each thread sums its rows in R and the
//    slices are added into the double G in slice order (deterministic);
//  - Q = X M with M = L^-dag upper triangular: a thread owns two rows and
//    the column groups c and NC/4-1-c, so every thread does the same work;
//  - rows staged with 16-byte loads into a [kChunk][NC+2] tile (even stride:
//    16-byte aligned rows, conflict-free column reads);
//  - the trailing update of the Cholesky factorisation on a fixed 2-D map
//    of threads to entries (no division by a runtime size).
template <class S>
__device__ __forceinline__ void ld4s(const S* p, float v[4]) {
  if constexpr (sizeof(S) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
  } else {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    S h[4];
    *reinterpret_cast<uint2*>(h) = t;
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = to_r(h[i]);
  }
}
__device__ __forceinline__ void ld4s(const double* p, double v[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}
template <class S>
__device__ __forceinline__ void st4s(S* p, const float v[4]) {
  if constexpr (sizeof(S) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    S h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = from_r<S>(v[i]);
    *reinterpret_cast<uint2*>(p) = *reinterpret_cast<const uint2*>(h);
  }
}
__device__ __forceinline__ void st4s(double* p, const double v[4]) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}

// Cholesky factorisation G = L L^dag of the Hermitian positive definite
// N x N matrix G (lower triangle, in place, type T) and the upper triangular
// M = L^-dag (L^dag M = 1, one column per thread by back substitution), by the
// threads of the CTA; a pivot at or below rel_pivot times the diagonal dg[k]
// of the original Gram matrix, or not finite, raises *flag (the vectors are
// numerically dependent) and is replaced by 1 to finish safely
template <class T, int N>
__device__ __forceinline__ void chol_inv(cx<T>* G, cx<T>* M, const double* dg, double rel_pivot, int* flag,
                                         int tid) {
  __shared__ T s_rdiag[N];  // 1 / L_kk
  for (int k = 0; k < N; ++k) {
    if (tid == 0) {
      T d = G[k * N + k].re;
      if (!((double)d > rel_pivot * dg[k]) || !isfinite(d)) {
        atomicExch(flag, 1);
        d = 1;
      }
      const T l = sqrt(d);
      G[k * N + k] = mk<T>(l, 0);
      s_rdiag[k] = (T)1 / l;
    }
    __syncthreads();
    if (tid > k && tid < N) G[tid * N + k] = scale(G[tid * N + k], s_rdiag[k]);
    __syncthreads();
    {
      // thread -> column j = tid % N of rows i = tid / N + (kThreads / N) m
      const int j = tid % N;
      if (j > k && tid < N * (kThreads / N)) {
        const cx<T> gjk = cnj(G[j * N + k]);
        for (int i = tid / N; i < N; i += kThreads / N)
          if (i >= j) G[i * N + j] = G[i * N + j] - G[i * N + k] * gjk;
      }
    }
    __syncthreads();
  }
  for (int j = tid; j < N; j += kThreads) {
    for (int i = N - 1; i >= 0; --i) {
      if (i > j) {
        M[i * N + j] = mk<T>(0, 0);
        continue;
      }
      cx<T> sacc = i == j ? mk<T>(1, 0) : mk<T>(0, 0);
      for (int k2 = i + 1; k2 <= j; ++k2) sacc = sacc - cnj(G[k2 * N + i]) * M[k2 * N + j];
      M[i * N + j] = scale(sacc, s_rdiag[i]);
    }
  }
  __syncthreads();
}

template <class S, class R, int NC, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_cholqr2_reg(const S* V, S* Q, int Va, int* flag) {
  constexpr int N = NC;
  constexpr int NT = N / 4;                  // tiles per side
  constexpr int NLOW = NT * (NT + 1) / 2;    // lower-triangle tiles
  constexpr int KS = kThreads / NLOW;        // row slices
  constexpr int LD = N + 2;                  // staged row stride (complex)
  extern __shared__ double smem[];
  const int A = blockIdx.x >> 1, h = blockIdx.x & 1;
  const int L = 6 * Va;
  cx<double>* G = (cx<double>*)smem;         // [N][N]
  cx<R>* Mr = (cx<R>*)(G + N * N);           // [N][N] L^-dag in R
  cx<R>* buf = Mr + N * N;                   // [kChunk][LD]
  cx<double>* Md = (cx<double>*)buf;         // [N][N] L^-dag in double, while buf is unused
  double* dg = (double*)(buf + kChunk * LD); // [N]
  static_assert(sizeof(cx<R>) * kChunk * LD >= sizeof(cx<double>) * N * N, "L^-dag must fit in the staging tile");
  const int tid = threadIdx.x;
  const double rel_pivot = 16.0 * (sizeof(R) == 8 ? 1.1102230246251565e-16 : 5.960464477539063e-08);
  // Gram tile of this thread: lower-triangle tile index -> (ti >= tj)
  const bool gon = tid < NLOW * KS;
  const int tile = tid % NLOW, slice = tid / NLOW;
  int ti = 0;
  while ((ti + 1) * (ti + 2) / 2 <= tile) ++ti;
  const int tj = tile - ti * (ti + 1) / 2;
  // Q = X M items: rows 2 rp, 2 rp + 1 of the chunk, column groups cA and
  // NT-1-cA (cA < ceil(NT/2))
  const int rp = tid >> 2;
  const int cA = tid & 3;
  static_assert(kChunk == 2 * (kThreads / 4), "two rows per thread quarter");
  for (int pass = 0; pass < 2; ++pass) {
    const S* src = pass == 0 ? V : Q;
    auto stage = [&](int l0, int nl) {
      for (int u = tid; u < nl * NT; u += kThreads) {
        const int l = u / NT, q = u % NT;  // NT is a compile-time constant
        const size_t row = gs_row(A, h, Va, l0 + l);
        R re[4], im[4];
        ld4s(src + fidx(row, 0, N, 4 * q), re);
        ld4s(src + fidx(row, 1, N, 4 * q), im);
        cx<R>* d = buf + l * LD + 4 * q;
#pragma unroll
        for (int b = 0; b < 4; ++b) d[b] = mk<R>(re[b], im[b]);
      }
    };
    // ---- lower triangle of G = X^dag X
    cx<R> acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = mk<R>(0, 0);
    for (int l0 = 0; l0 < L; l0 += kChunk) {
      const int nl = min(kChunk, L - l0);
      stage(l0, nl);
      __syncthreads();
      if (gon) {
        for (int l = slice; l < nl; l += KS) {
          const cx<R>* xr = buf + l * LD;
          cx<R> xi[4], xj[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) xi[a] = xr[4 * ti + a];
#pragma unroll
          for (int b = 0; b < 4; ++b) xj[b] = xr[4 * tj + b];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) fmac_(acc[a][b], xi[a], xj[b]);
        }
      }
      __syncthreads();
    }
    for (int sl = 0; sl < KS; ++sl) {
      if (gon && slice == sl) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            cx<double>& g = G[(4 * ti + a) * N + 4 * tj + b];
            const cx<double> v = mk((double)acc[a][b].re, (double)acc[a][b].im);
            g = sl == 0 ? v : g + v;
          }
      }
      __syncthreads();
    }
    for (int k = tid; k < N; k += kThreads) dg[k] = G[k * N + k].re;
    __syncthreads();
    // ---- Cholesky G = L L^dag and M = L^-dag in the compute type R: FP64
    // for FP64 data; FP32 for FP32 and reduced storage, where FP64 runs at a
    // small fraction of the FP32 rate and the vectors accepted by the pivot
    // test (pivot above 16 u32 of its diagonal, kappa below ~1/(4 sqrt(u32)))
    // give a first-pass Q that the second pass brings to FP32 orthogonality
    cx<R>* Gf;
    cx<R>* Mc;
    if constexpr (sizeof(R) == 8) {
      Gf = reinterpret_cast<cx<R>*>(G);
      Mc = reinterpret_cast<cx<R>*>(Md);
    } else {
      Gf = buf;          // the staging tile is free between the passes over the rows
      Mc = buf + N * N;
      for (int w = tid; w < N * N; w += kThreads) Gf[w] = mk<R>((R)G[w].re, (R)G[w].im);
      __syncthreads();
    }
    chol_inv<R, N>(Gf, Mc, dg, rel_pivot, flag, tid);
    for (int w = tid; w < N * N; w += kThreads) Mr[w] = Mc[w];
    __syncthreads();
    // ---- Q = X M
    for (int l0 = 0; l0 < L; l0 += kChunk) {
      const int nl = min(kChunk, L - l0);
      stage(l0, nl);
      __syncthreads();
      if (2 * rp < nl && cA < (NT + 1) / 2) {
        const int cB = NT - 1 - cA;
        const bool twoB = cB != cA;
        const int endA = 4 * cA + 4, endB = 4 * cB + 4;  // M[i][j] = 0 for i > j
        cx<R> oA[2][4], oB[2][4];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) oA[a][b] = oB[a][b] = mk<R>(0, 0);
        const int r1 = min(2 * rp + 1, nl - 1);
        const int e1 = max(endA, endB);
        for (int i = 0; i < e1; ++i) {
          const cx<R> x0 = buf[(2 * rp) * LD + i], x1 = buf[r1 * LD + i];
          if (i < endA) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const cx<R> m = Mr[i * N + 4 * cA + b];
              fma_(oA[0][b], x0, m);
              fma_(oA[1][b], x1, m);
            }
          }
          if (twoB && i < endB) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const cx<R> m = Mr[i * N + 4 * cB + b];
              fma_(oB[0][b], x0, m);
              fma_(oB[1][b], x1, m);
            }
          }
        }
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          if (2 * rp + a >= nl) break;
          const size_t row = gs_row(A, h, Va, l0 + 2 * rp + a);
          R re[4], im[4];
#pragma unroll
          for (int b = 0; b < 4; ++b) re[b] = oA[a][b].re, im[b] = oA[a][b].im;
          st4s(Q + fidx(row, 0, N, 4 * cA), re);
          st4s(Q + fidx(row, 1, N, 4 * cA), im);
          if (twoB) {
#pragma unroll
            for (int b = 0; b < 4; ++b) re[b] = oB[a][b].re, im[b] = oB[a][b].im;
            st4s(Q + fidx(row, 0, N, 4 * cB), re);
            st4s(Q + fidx(row, 1, N, 4 * cB), im);
          }
        }
      }
      __syncthreads();
    }
  }
}

// three CTAs per SM (at most 85 registers, 60 KB shared memory each at
// ntv = 32): measured 1.6x faster than two CTAs with the registers unbounded
template <class S, class R, int NC, int MINB = 3>
void launch_cholqr2_reg(mrhs_ctx c) {
  const size_t smem = sizeof(cx<double>) * NC * NC + sizeof(cx<R>) * (NC * NC + (size_t)kChunk * (NC + 2)) +
                      sizeof(double) * NC;
  MRHS_CUDA(cudaFuncSetAttribute(k_cholqr2_reg<S, R, NC, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_cholqr2_reg<S, R, NC, MINB><<<2 * c->g.nagg, kThreads, smem, c->stream>>>((const S*)c->tv, (S*)c->P, c->g.Va, c->dflag);
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
    if (N % 4 == 0 && N <= 32) {
      switch (N) {
        case 4: launch_cholqr2_reg<S, R, 4>(c); break;
        case 8: launch_cholqr2_reg<S, R, 8>(c); break;
        case 12: launch_cholqr2_reg<S, R, 12>(c); break;
        case 16: launch_cholqr2_reg<S, R, 16>(c); break;
        case 20: launch_cholqr2_reg<S, R, 20>(c); break;
        case 24: launch_cholqr2_reg<S, R, 24>(c); break;
        case 28: launch_cholqr2_reg<S, R, 28>(c); break;
        default: launch_cholqr2_reg<S, R, 32>(c); break;
      }
    } else if (N <= 32) {
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
