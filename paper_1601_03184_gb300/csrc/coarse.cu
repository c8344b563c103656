// Coarse grid: D_c = P^dag D P assembly, restriction R = P^dag (Algorithm 3
// of the paper, all right-hand sides at once), prolongation, the coarse
// 9-point stencil and the multi-RHS coarse GMRES.
#include <cstdint>
#include <cstdlib>

#include "coarse_common.cuh"

namespace mrhs {
namespace {

constexpr int kSites = 8;  // sites staged per chunk in the contractions

// One CTA per (aggregate A, stencil entry k). Columns (h', j), rows (h, i):
//   k = 0:      sum_{x in A} P_(h,i)(x)^dag [A(x) + hops inside A] P_(h',j)
//   k = 1+mu:   sum over the +mu face of A of P_(h,i)(x)^dag hop_{+mu} P_(h',j)(x+mu)
//   k = 5+mu:   the same for the -mu face and hop_{-mu}
template <class SP, class R, int EPT>
__global__ void k_coarse_op(const SP* __restrict__ P, const cx<R>* __restrict__ U, const R* __restrict__ Acl,
                            const int* __restrict__ nbr, int Nt, Agg4 ag, int Va, cx<R>* __restrict__ Dc) {
  extern __shared__ double smem_d[];
  const int A = blockIdx.x / 9, k = blockIdx.x % 9;
  const int nc = 2 * Nt;
  cx<R>* W = (cx<R>*)smem_d;               // [kSites][12][nc]
  cx<R>* Pc = W + kSites * 12 * nc;        // [kSites][12][Nt]
  const int mu = k == 0 ? -1 : (k - 1) % 4;
  const int nsite = k == 0 ? Va : Va / ag.a[mu];
  const int lmu = k == 0 ? 0 : (k <= 4 ? ag.a[mu] - 1 : 0);
  const int dir = k <= 4 ? +1 : -1;
  cx<R> acc[EPT];
#pragma unroll
  for (int m = 0; m < EPT; ++m) acc[m] = mk<R>(0, 0);
  for (int q0 = 0; q0 < nsite; q0 += kSites) {
    const int nq = min(kSites, nsite - q0);
    for (int w = threadIdx.x; w < nq * nc; w += blockDim.x) {
      int q = w / nc, col = w % nc;
      int l = k == 0 ? q0 + q : face_site(ag, mu, lmu, q0 + q);
      int s = A * Va + l;
      cx<R> out[12];
#pragma unroll
      for (int c = 0; c < 12; ++c) out[c] = mk<R>(0, 0);
      if (k == 0) {
        cx<R> psi[12];
        load_pcol<SP, R>(psi, P, s, Nt, col);
        clover_apply_reg<R>(out, psi, Acl + (size_t)s * 72);
        for (int d = -1; d <= 1; d += 2) {
          hop_pcol<0, SP, R>(out, P, U, nbr, s, d, Nt, col, true, Va);
          hop_pcol<1, SP, R>(out, P, U, nbr, s, d, Nt, col, true, Va);
          hop_pcol<2, SP, R>(out, P, U, nbr, s, d, Nt, col, true, Va);
          hop_pcol<3, SP, R>(out, P, U, nbr, s, d, Nt, col, true, Va);
        }
      } else {
        switch (mu) {
          case 0: hop_pcol<0, SP, R>(out, P, U, nbr, s, dir, Nt, col, false, Va); break;
          case 1: hop_pcol<1, SP, R>(out, P, U, nbr, s, dir, Nt, col, false, Va); break;
          case 2: hop_pcol<2, SP, R>(out, P, U, nbr, s, dir, Nt, col, false, Va); break;
          default: hop_pcol<3, SP, R>(out, P, U, nbr, s, dir, Nt, col, false, Va); break;
        }
      }
#pragma unroll
      for (int c = 0; c < 12; ++c) W[(q * 12 + c) * nc + col] = out[c];
    }
    for (int w = threadIdx.x; w < nq * 12 * Nt; w += blockDim.x) {
      int q = w / (12 * Nt), c = (w / Nt) % 12, i = w % Nt;
      int l = k == 0 ? q0 + q : face_site(ag, mu, lmu, q0 + q);
      Pc[w] = ld<SP, R>(P, ((size_t)A * Va + l) * 12 + c, Nt, i);
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < EPT; ++m) {
      int e = threadIdx.x + m * blockDim.x;
      if (e < nc * nc) {
        int row = e / nc, col = e % nc;
        int h = row / Nt, i = row % Nt;
        for (int q = 0; q < nq; ++q)
#pragma unroll
          for (int cc = 0; cc < 6; ++cc) {
            int c = 6 * h + cc;
            fmac_(acc[m], Pc[(q * 12 + c) * Nt + i], W[(q * 12 + c) * nc + col]);
          }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < EPT; ++m) {
    int e = threadIdx.x + m * blockDim.x;
    if (e < nc * nc) Dc[((size_t)A * 9 + k) * nc * nc + e] = acc[m];
  }
}

// Tiled form for ntv % 4 == 0 and 2*ntv <= 64. One CTA per (aggregate A,
// k in 0..4): k = 0 the self block, k = 1+mu the forward block (A+mu). Per
// chunk of sites Y[q][c][col] = (D_k P_col)(x_q, c) is built in shared memory
// (one (site, column) per thread), then every thread accumulates a 4x4 tile
// of P^dag Y (rows (h,i0..i0+3), columns col0..col0+3) over the chunk.
// The backward blocks follow from gamma_5-hermiticity (k_coarse_backward).
constexpr int kTileSites = 8;

template <class SP, class R>
__global__ void __launch_bounds__(256) k_coarse_op_tiled(const SP* __restrict__ P, const cx<R>* __restrict__ U,
                                                         const R* __restrict__ Acl, const int* __restrict__ nbr, int Nt,
                                                         Agg4 ag, int Va, cx<R>* __restrict__ Dc) {
  extern __shared__ double smem_d[];
  const int A = blockIdx.x / 5, k = blockIdx.x % 5;
  const int nc = 2 * Nt;
  cx<R>* Y = (cx<R>*)smem_d;                 // [kTileSites][12][nc]
  cx<R>* Pc = Y + kTileSites * 12 * nc;      // [kTileSites][12][Nt]
  const int mu = k - 1;
  const int nsite = k == 0 ? Va : Va / ag.a[mu];
  const int lmu = k == 0 ? 0 : ag.a[mu] - 1;
  const int ntile = nc / 4;
  const int rt = threadIdx.x / ntile, ct = threadIdx.x % ntile;
  const bool tile_on = threadIdx.x < ntile * ntile;
  const int r0 = 4 * rt, c0 = 4 * ct;
  const int h = r0 / Nt, i0 = r0 % Nt;
  cx<R> acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = mk<R>(0, 0);
  for (int q0 = 0; q0 < nsite; q0 += kTileSites) {
    const int nq = min(kTileSites, nsite - q0);
    for (int w = threadIdx.x; w < nq * nc; w += blockDim.x) {
      int q = w / nc, col = w % nc;
      int l = k == 0 ? q0 + q : face_site(ag, mu, lmu, q0 + q);
      int s = A * Va + l;
      cx<R> out[12];
      if (col < Nt) dk_pcol<0, SP, R>(out, P, U, Acl, nbr, s, k, Nt, col, A * Va, Va);
      else dk_pcol<1, SP, R>(out, P, U, Acl, nbr, s, k, Nt, col - Nt, A * Va, Va);
#pragma unroll
      for (int c = 0; c < 12; ++c) Y[(q * 12 + c) * nc + col] = out[c];
    }
    for (int w = threadIdx.x; w < nq * 12 * Nt; w += blockDim.x) {
      int q = w / (12 * Nt), c = (w / Nt) % 12, i = w % Nt;
      int l = k == 0 ? q0 + q : face_site(ag, mu, lmu, q0 + q);
      Pc[w] = ld<SP, R>(P, ((size_t)A * Va + l) * 12 + c, Nt, i);
    }
    __syncthreads();
    if (tile_on) {
      for (int q = 0; q < nq; ++q)
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) {
          const int c = 6 * h + cc;
          cx<R> pv[4], yv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) pv[a] = Pc[(q * 12 + c) * Nt + i0 + a];
#pragma unroll
          for (int b = 0; b < 4; ++b) yv[b] = Y[(q * 12 + c) * nc + c0 + b];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) fmac_(acc[a][b], pv[a], yv[b]);
        }
    }
    __syncthreads();
  }
  if (tile_on) {
    const int kk = k;  // self and forward blocks keep their stencil index
    cx<R>* out = Dc + ((size_t)A * 9 + kk) * nc * nc;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) out[(size_t)(r0 + a) * nc + c0 + b] = acc[a][b];
  }
}

// D_c[A][5+mu][r][c] = eta(r) eta(c) conj(D_c[A-mu][1+mu][c][r]), eta = +1 for
// chirality 0 rows/columns and -1 for chirality 1 (gamma_5-hermiticity of D
// and the chirality-split P).
template <class R>
__global__ void k_coarse_backward(cx<R>* Dc, const int* __restrict__ aggnbr, int nagg, int Nt) {
  const int nc = 2 * Nt;
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t tot = (size_t)nagg * 4 * nc * nc;
  if (t >= tot) return;
  int c = (int)(t % nc);
  int r = (int)((t / nc) % nc);
  int mu = (int)((t / ((size_t)nc * nc)) % 4);
  int A = (int)(t / ((size_t)4 * nc * nc));
  int B = aggnbr[A * 8 + 4 + mu];
  cx<R> v = Dc[(((size_t)B * 9 + 1 + mu) * nc + c) * nc + r];
  R sgn = ((r / Nt) == (c / Nt)) ? (R)1 : (R)-1;
  Dc[(((size_t)A * 9 + 5 + mu) * nc + r) * nc + c] = mk<R>(sgn * v.re, -sgn * v.im);
}

// vc[A][(h,i)][r] = sum_{x in A, c in h} conj(P_i(x,c)) v(x,c,r)
template <class SP, class SV, class SC, int EPT>
__global__ void k_restrict(const SP* __restrict__ P, const SV* __restrict__ v, SC* __restrict__ vc, int Nt, int N,
                           int Va) {
  using R = typename Real<SC>::type;
  extern __shared__ double smem_d[];
  const int A = blockIdx.x;
  const int nc = 2 * Nt;
  cx<R>* Pc = (cx<R>*)smem_d;          // [kSites][12][Nt]
  cx<R>* Xc = Pc + kSites * 12 * Nt;   // [kSites][12][N]
  cx<R> acc[EPT];
#pragma unroll
  for (int m = 0; m < EPT; ++m) acc[m] = mk<R>(0, 0);
  for (int q0 = 0; q0 < Va; q0 += kSites) {
    const int nq = min(kSites, Va - q0);
    for (int w = threadIdx.x; w < nq * 12 * Nt; w += blockDim.x) {
      int q = w / (12 * Nt), c = (w / Nt) % 12, i = w % Nt;
      Pc[w] = ld<SP, R>(P, ((size_t)A * Va + q0 + q) * 12 + c, Nt, i);
    }
    for (int w = threadIdx.x; w < nq * 12 * N; w += blockDim.x) {
      int q = w / (12 * N), c = (w / N) % 12, r = w % N;
      Xc[w] = ld<SV, R>(v, ((size_t)A * Va + q0 + q) * 12 + c, N, r);
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < EPT; ++m) {
      int e = threadIdx.x + m * blockDim.x;
      if (e < nc * N) {
        int row = e / N, r = e % N;
        int h = row / Nt, i = row % Nt;
        for (int q = 0; q < nq; ++q)
#pragma unroll
          for (int cc = 0; cc < 6; ++cc) {
            int c = 6 * h + cc;
            fmac_(acc[m], Pc[(q * 12 + c) * Nt + i], Xc[(q * 12 + c) * N + r]);
          }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < EPT; ++m) {
    int e = threadIdx.x + m * blockDim.x;
    if (e < nc * N) {
      int row = e / N, r = e % N;
      st<SC, R>(vc, (size_t)A * nc + row, N, r, acc[m]);
    }
  }
}

// Tiled restriction for ntv % 4 == 0 and an even number of right-hand
// sides: each thread accumulates 4 rows (h, i0..i0+3) x 2 right-hand sides.
template <class SP, class SV, class SC>
__global__ void __launch_bounds__(256) k_restrict_tiled(const SP* __restrict__ P, const SV* __restrict__ v,
                                                        SC* __restrict__ vc, int Nt, int N, int Va) {
  using R = typename Real<SC>::type;
  extern __shared__ double smem_d[];
  const int A = blockIdx.x;
  const int nc = 2 * Nt;
  cx<R>* Pc = (cx<R>*)smem_d;                 // [kSites][12][Nt]
  cx<R>* Xc = Pc + kSites * 12 * Nt;          // [kSites][12][N]
  const int nrt = nc / 4, nct = N / 2;
  const int rt = threadIdx.x / nct, ct = threadIdx.x % nct;
  const bool on = threadIdx.x < nrt * nct;
  const int r0 = 4 * rt, j0 = 2 * ct;
  const int h = r0 / Nt, i0 = r0 % Nt;
  cx<R> acc[4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = mk<R>(0, 0);
  for (int q0 = 0; q0 < Va; q0 += kSites) {
    const int nq = min(kSites, Va - q0);
    for (int w = threadIdx.x; w < nq * 12 * Nt; w += blockDim.x) {
      int q = w / (12 * Nt), c = (w / Nt) % 12, i = w % Nt;
      Pc[w] = ld<SP, R>(P, ((size_t)A * Va + q0 + q) * 12 + c, Nt, i);
    }
    for (int w = threadIdx.x; w < nq * 12 * N; w += blockDim.x) {
      int q = w / (12 * N), c = (w / N) % 12, r = w % N;
      Xc[w] = ld<SV, R>(v, ((size_t)A * Va + q0 + q) * 12 + c, N, r);
    }
    __syncthreads();
    if (on) {
      for (int q = 0; q < nq; ++q)
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) {
          const int c = 6 * h + cc;
          cx<R> pv[4], xv[2];
#pragma unroll
          for (int a = 0; a < 4; ++a) pv[a] = Pc[(q * 12 + c) * Nt + i0 + a];
          xv[0] = Xc[(q * 12 + c) * N + j0];
          xv[1] = Xc[(q * 12 + c) * N + j0 + 1];
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            fmac_(acc[a][0], pv[a], xv[0]);
            fmac_(acc[a][1], pv[a], xv[1]);
          }
        }
    }
    __syncthreads();
  }
  if (on) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) st<SC, R>(vc, (size_t)A * nc + r0 + a, N, j0 + b, acc[a][b]);
  }
}

// FP32 restriction streamed through registers: one thread per (aggregate A,
// chirality h, four rows i0..i0+3, four right-hand sides r0..r0+3), the sum
// over the aggregate's sites and the chirality's six components in the
// thread's registers (no staging, no barrier): every 16-byte load of P or v
// feeds 16 complex products. Nt % 4 = 0, N % 4 = 0.
__global__ void __launch_bounds__(128) k_restrict_stream(const float* __restrict__ P, const float* __restrict__ v,
                                                         float* __restrict__ vc, int Nt, int N, int Va) {
  const int A = blockIdx.x;
  const int nq = N / 4, ni = Nt / 4;
  const int t = threadIdx.x;
  if (t >= 2 * ni * nq) return;
  const int r0 = 4 * (t % nq), i0 = 4 * ((t / nq) % ni), h = t / (nq * ni);
  float are[4][4], aim[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) are[a][b] = aim[a][b] = 0.f;
  const size_t row0 = (size_t)A * Va * 12 + 6 * h;
#pragma unroll 2
  for (int q = 0; q < Va * 6; ++q) {
    const size_t row = row0 + (size_t)(q / 6) * 12 + q % 6;
    const float4 pr = __ldg(reinterpret_cast<const float4*>(P + row * 2 * Nt + i0));
    const float4 pi = __ldg(reinterpret_cast<const float4*>(P + (row * 2 + 1) * Nt + i0));
    const float4 xr = __ldg(reinterpret_cast<const float4*>(v + row * 2 * N + r0));
    const float4 xi = __ldg(reinterpret_cast<const float4*>(v + (row * 2 + 1) * N + r0));
    const float Pr[4] = {pr.x, pr.y, pr.z, pr.w}, Pi[4] = {pi.x, pi.y, pi.z, pi.w};
    const float Xr[4] = {xr.x, xr.y, xr.z, xr.w}, Xi[4] = {xi.x, xi.y, xi.z, xi.w};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        // conj(p) x: re = pr xr + pi xi, im = pr xi - pi xr
        are[a][b] = fmaf(Pi[a], Xi[b], fmaf(Pr[a], Xr[b], are[a][b]));
        aim[a][b] = fmaf(-Pi[a], Xr[b], fmaf(Pr[a], Xi[b], aim[a][b]));
      }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const size_t crow = (size_t)A * 2 * Nt + h * Nt + i0 + a;
    *reinterpret_cast<float4*>(vc + fidx(crow, 0, N, r0)) = make_float4(are[a][0], are[a][1], are[a][2], are[a][3]);
    *reinterpret_cast<float4*>(vc + fidx(crow, 1, N, r0)) = make_float4(aim[a][0], aim[a][1], aim[a][2], aim[a][3]);
  }
}

// u(x,c,r) = sum_j P_j(x,c) uc[A(x)][(h(c), j)][r]
template <class SP, class SC, class SU>
__global__ void k_prolong(const SP* __restrict__ P, const SC* __restrict__ uc, SU* __restrict__ u, int Nt, int N,
                          int Va, size_t nwork) {
  using R = typename Real<SC>::type;
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= nwork) return;
  int r = (int)(t % N);
  size_t row = t / N;  // s*12 + c
  int c = (int)(row % 12);
  size_t s = row / 12;
  size_t A = s / Va;
  int h = c / 6;
  cx<R> acc = mk<R>(0, 0);
  for (int j = 0; j < Nt; ++j)
    fma_(acc, ld<SP, R>(P, row, Nt, j), ld<SC, R>(uc, A * 2 * Nt + h * Nt + j, N, r));
  st<SU, R>(u, row, N, r, acc);
}

// the launch arguments of a part of the stencil (DcPart, typed)
template <class SC>
struct DcPartArgs {
  const int* alist;
  const int* pos;
  int kb, ke;
  const SC* x0;
  const SC* xh;
  const SC* add;
};

// y[b][row][r] = sum_{kb<=k<ke} sum_col Dc[A][k][row][col] x[nbr_k(A)][col][r]
// (+ add[b][row][r]) for A = alist[b]
template <class SC>
__global__ void k_apply_dc(const cx<typename Real<SC>::type>* __restrict__ Dc, DcPartArgs<SC> pa,
                           SC* __restrict__ y, const int* __restrict__ aggnbr, int nc, int N, size_t nwork) {
  using R = typename Real<SC>::type;
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= nwork) return;
  int r = (int)(t % N);
  size_t q = t / N;
  int row = (int)(q % nc);
  const int b = (int)(q / nc);
  const int A = pa.alist ? pa.alist[b] : b;
  cx<R> acc = pa.add ? ld<SC, R>(pa.add, (size_t)b * nc + row, N, r) : mk<R>(0, 0);
  for (int k = pa.kb; k < pa.ke; ++k) {
    const int B = k == 0 ? A : aggnbr[A * 8 + k - 1];
    const SC* x = k == 0 ? pa.x0 : pa.xh;
    const size_t rb = pa.pos ? pa.pos[B] : B;
    const cx<R>* d = Dc + (((size_t)A * 9 + k) * nc + row) * nc;
    for (int col = 0; col < nc; ++col) fma_(acc, d[col], ld<SC, R>(x, rb * nc + col, N, r));
  }
  st<SC, R>(y, (size_t)b * nc + row, N, r, acc);
}

// 8 rows x 1 right-hand side per thread; pairs of columns read as one
// 16-byte (FP32) load per row; requires 2*ntv % 8 == 0.
template <class SC>
__global__ void k_apply_dc_tiled(const cx<typename Real<SC>::type>* __restrict__ Dc, DcPartArgs<SC> pa,
                                 SC* __restrict__ y, const int* __restrict__ aggnbr, int nc, int N, size_t nwork) {
  using R = typename Real<SC>::type;
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= nwork) return;
  const int r = (int)(t % N);
  const size_t q = t / N;
  const int nrt = nc / 8;
  const int row0 = 8 * (int)(q % nrt);
  const int b = (int)(q / nrt);
  const int A = pa.alist ? pa.alist[b] : b;
  cx<R> acc[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) acc[a] = pa.add ? ld<SC, R>(pa.add, (size_t)b * nc + row0 + a, N, r) : mk<R>(0, 0);
  for (int k = pa.kb; k < pa.ke; ++k) {
    const int B = k == 0 ? A : aggnbr[A * 8 + k - 1];
    const SC* x = k == 0 ? pa.x0 : pa.xh;
    const size_t rb = pa.pos ? pa.pos[B] : B;
    const cx<R>* d = Dc + (((size_t)A * 9 + k) * nc + row0) * nc;
    for (int col = 0; col < nc; col += 2) {
      cx<R> x0 = ld<SC, R>(x, rb * nc + col, N, r);
      cx<R> x1 = ld<SC, R>(x, rb * nc + col + 1, N, r);
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        fma_(acc[a], d[(size_t)a * nc + col], x0);
        fma_(acc[a], d[(size_t)a * nc + col + 1], x1);
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) st<SC, R>(y, (size_t)b * nc + row0 + a, N, r, acc[a]);
}

// u = P uc with one thread per (site, chirality, right-hand side): 6 outputs
// share every load of uc
template <class SP, class SC, class SU>
__global__ void k_prolong6(const SP* __restrict__ P, const SC* __restrict__ uc, SU* __restrict__ u, int Nt, int N,
                           int Va, size_t nwork) {
  using R = typename Real<SC>::type;
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= nwork) return;
  const int r = (int)(t % N);
  const size_t q = t / N;
  const int h = (int)(q % 2);
  const size_t s = q / 2;
  const size_t A = s / Va;
  cx<R> acc[6];
#pragma unroll
  for (int cc = 0; cc < 6; ++cc) acc[cc] = mk<R>(0, 0);
  for (int j = 0; j < Nt; ++j) {
    cx<R> w = ld<SC, R>(uc, A * 2 * Nt + h * Nt + j, N, r);
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) fma_(acc[cc], ld<SP, R>(P, s * 12 + 6 * h + cc, Nt, j), w);
  }
#pragma unroll
  for (int cc = 0; cc < 6; ++cc) st<SU, R>(u, s * 12 + 6 * h + cc, N, r, acc[cc]);
}

// The same for FP32 coarse and fine fields with N % 4 == 0: four right-hand
// sides per thread (16-byte loads of uc and stores of u), so every P entry
// loaded serves 4 x 6 complex products; the scalar kernel's operations in
// its order (the same bits).
template <class SP>
__global__ void k_prolong6x4(const SP* __restrict__ P, const float* __restrict__ uc, float* __restrict__ u, int Nt,
                             int N, int Va, size_t nwork) {
  const int Q = N / 4;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= nwork) return;
  const int r0 = 4 * (int)(t % Q);
  const size_t q = t / Q;
  const int h = (int)(q % 2);
  const size_t s = q / 2;
  const size_t A = s / Va;
  float are[6][4], aim[6][4];
#pragma unroll
  for (int cc = 0; cc < 6; ++cc)
#pragma unroll
    for (int e = 0; e < 4; ++e) are[cc][e] = aim[cc][e] = 0.f;
  for (int j = 0; j < Nt; ++j) {
    const size_t crow = A * 2 * Nt + h * Nt + j;
    const float4 w0 = *reinterpret_cast<const float4*>(uc + fidx(crow, 0, N, r0));
    const float4 w1 = *reinterpret_cast<const float4*>(uc + fidx(crow, 1, N, r0));
    const float wr[4] = {w0.x, w0.y, w0.z, w0.w}, wi[4] = {w1.x, w1.y, w1.z, w1.w};
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) {
      const cx<float> pv = ld<SP, float>(P, s * 12 + 6 * h + cc, Nt, j);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        // fma_(acc, p, w): acc.re += p.re w.re - p.im w.im, acc.im += p.re w.im + p.im w.re
        are[cc][e] = fmaf(-pv.im, wi[e], fmaf(pv.re, wr[e], are[cc][e]));
        aim[cc][e] = fmaf(pv.im, wr[e], fmaf(pv.re, wi[e], aim[cc][e]));
      }
    }
  }
#pragma unroll
  for (int cc = 0; cc < 6; ++cc) {
    const size_t row = s * 12 + 6 * h + cc;
    *reinterpret_cast<float4*>(u + fidx(row, 0, N, r0)) = make_float4(are[cc][0], are[cc][1], are[cc][2], are[cc][3]);
    *reinterpret_cast<float4*>(u + fidx(row, 1, N, r0)) = make_float4(aim[cc][0], aim[cc][1], aim[cc][2], aim[cc][3]);
  }
}

template <class S>
__global__ void k_sub_from(const S* b, S* w, size_t n) {  // w = b - w
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t < n) w[t] = from_r<S>(to_r(b[t]) - to_r(w[t]));
}

template <class S>
__global__ void k_scale_rhs(const S* x, S* y, size_t rows, int N, const double* s) {
  using R = typename Real<S>::type;
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= rows * N) return;
  int r = (int)(t % N);
  size_t row = t / N;
  R f = (R)s[r];
  y[fidx(row, 0, N, r)] = from_r<S>(to_r(x[fidx(row, 0, N, r)]) * f);
  y[fidx(row, 1, N, r)] = from_r<S>(to_r(x[fidx(row, 1, N, r)]) * f);
}

// ------------------------------------------------------- GMRES state ------
struct GmState {
  cx<double>* H;    // [N][m+1][m]
  cx<double>* cs;   // [N][m]
  cx<double>* sn;   // [N][m]
  cx<double>* g;    // [N][m+1]
  double* y;        // [m][N][2]  (coefficients for the solution update)
  double* h1;       // [m+1][N][2]
  double* h2;       // [m+1][N][2]
  double* hn2;      // [N][2]
  double* beta2;    // [N][2]
  double* bnorm2;   // [N][2]
  double* inv;      // [N]
  int* conv;        // [N]
  int* active;      // [N]
  int* its;         // [N]
  int* kend;        // [N]
  int* counter;     // [1]
};

__global__ void k_gm_init(GmState st, int N) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  st.conv[r] = st.bnorm2[2 * r] == 0.0;
  st.its[r] = 0;
  st.active[r] = 0;
  st.kend[r] = 0;
}

// start of a cycle: r = b - A x is in w with |w|^2 in beta2
__global__ void k_gm_start(GmState st, int N, int m, double tol, int maxit) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  st.kend[r] = 0;
  st.active[r] = 0;
  st.inv[r] = 0;
  if (st.conv[r] || st.its[r] >= maxit) return;
  double beta = sqrt(st.beta2[2 * r]);
  if (beta <= tol * sqrt(st.bnorm2[2 * r])) {
    st.conv[r] = 1;
    return;
  }
  st.active[r] = 1;
  st.inv[r] = 1.0 / beta;
  for (int i = 0; i <= m; ++i) st.g[(size_t)r * (m + 1) + i] = mk(0.0, 0.0);
  st.g[(size_t)r * (m + 1)] = mk(beta, 0.0);
  atomicAdd(st.counter, 1);
}

// Arnoldi column k: h = h1 + h2 (two classical Gram-Schmidt passes), then
// the Givens rotations and the residual estimate |g_{k+1}|
__global__ void k_gm_step(GmState st, int N, int m, int k, double tol, int maxit) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  st.inv[r] = 0;
  if (!st.active[r]) return;
  cx<double>* H = st.H + (size_t)r * (m + 1) * m;
  cx<double>* cs = st.cs + (size_t)r * m;
  cx<double>* sn = st.sn + (size_t)r * m;
  cx<double>* g = st.g + (size_t)r * (m + 1);
  for (int i = 0; i <= k; ++i)
    H[i * m + k] = mk(st.h1[((size_t)i * N + r) * 2] + st.h2[((size_t)i * N + r) * 2],
                      st.h1[((size_t)i * N + r) * 2 + 1] + st.h2[((size_t)i * N + r) * 2 + 1]);
  double hk1 = sqrt(st.hn2[2 * r]);
  H[(k + 1) * m + k] = mk(hk1, 0.0);
  for (int i = 0; i < k; ++i) {
    cx<double> a = H[i * m + k], b = H[(i + 1) * m + k];
    H[i * m + k] = cnj(cs[i]) * a + cnj(sn[i]) * b;
    H[(i + 1) * m + k] = mk(0.0, 0.0) - sn[i] * a + cs[i] * b;
  }
  cx<double> a = H[k * m + k], b = H[(k + 1) * m + k];
  double nu = sqrt(a.re * a.re + a.im * a.im + b.re * b.re + b.im * b.im);
  if (nu == 0) {
    cs[k] = mk(1.0, 0.0);
    sn[k] = mk(0.0, 0.0);
  } else {
    cs[k] = scale(a, 1.0 / nu);
    sn[k] = scale(b, 1.0 / nu);
  }
  H[k * m + k] = mk(nu, 0.0);
  H[(k + 1) * m + k] = mk(0.0, 0.0);
  cx<double> g0 = g[k];
  g[k] = cnj(cs[k]) * g0;
  g[k + 1] = mk(0.0, 0.0) - sn[k] * g0;
  st.its[r] += 1;
  st.kend[r] = k + 1;
  double res = sqrt(g[k + 1].re * g[k + 1].re + g[k + 1].im * g[k + 1].im);
  bool conv = res <= tol * sqrt(st.bnorm2[2 * r]) || hk1 == 0;
  if (conv) st.conv[r] = 1;
  if (conv || st.its[r] >= maxit || k + 1 == m) {
    st.active[r] = 0;
  } else {
    st.inv[r] = 1.0 / hk1;
    atomicAdd(st.counter, 1);
  }
}

// back substitution of the leading kend x kend triangle, y = coefficients
__global__ void k_gm_solve(GmState st, int N, int m) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  const cx<double>* H = st.H + (size_t)r * (m + 1) * m;
  const cx<double>* g = st.g + (size_t)r * (m + 1);
  int ke = st.kend[r];
  cx<double> yv[64];
  for (int i = ke - 1; i >= 0; --i) {
    cx<double> c = g[i];
    for (int l = i + 1; l < ke; ++l) c = c - H[i * m + l] * yv[l];
    double d = H[i * m + i].re;  // real and positive after the rotation
    yv[i] = scale(c, 1.0 / d);
  }
  for (int i = 0; i < m; ++i) {
    cx<double> v = i < ke ? yv[i] : mk(0.0, 0.0);
    st.y[((size_t)i * N + r) * 2] = v.re;
    st.y[((size_t)i * N + r) * 2 + 1] = v.im;
  }
}

template <class T>
T* carve(char*& p, size_t n) {
  T* r = (T*)p;
  p += ((n * sizeof(T) + 255) / 256) * 256;
  return r;
}

}  // namespace

// ------------------------------------------------------------------ host ---
void build_Dc(mrhs_ctx c) {
  MRHS_REQUIRE(c->have_P, MRHS_ERR_STATE, "mrhs_build_Dc before mrhs_build_P");
  MRHS_REQUIRE(c->have_clover, MRHS_ERR_STATE, "mrhs_build_Dc before mrhs_build_clover");
  const int Nt = c->ntv, nc = 2 * Nt;
  size_t n = (size_t)c->g.nagg * 9 * nc * nc;
  if (!c->Dc) c->Dc = dalloc(c, n * 2 * dtype_size(c->work_dtype));
  Agg4 ag;
  for (int m = 0; m < 4; ++m) ag.a[m] = c->g.a[m];
  const bool tiled = Nt % 4 == 0 && nc <= 64;
  // tensor-core contraction: chosen explicitly, or by default for the mixed setups
  int fmt = -1;
  bool split = false;
  switch (c->dc_engine) {
    case MRHS_DC_TC_BF16: fmt = tc_fmt_bf16; break;
    case MRHS_DC_TC_F16: fmt = tc_fmt_f16; break;
    case MRHS_DC_TC_TF32: fmt = tc_fmt_tf32; break;
    case MRHS_DC_TC_TF32X3: fmt = tc_fmt_tf32; split = true; break;
    case MRHS_DC_AUTO:
      // FP32: the split-tf32 contraction (FP32 accuracy; 184 ms per build at
      // 48^3x96 against 210 ms for the CUDA-core form); mixed setups: one
      // rounding to bf16 or tf32
      if (c->prec == MRHS_PREC_FP32) fmt = tc_fmt_tf32, split = true;
      if (c->prec == MRHS_PREC_MIX_BF16) fmt = tc_fmt_bf16;
      if (c->prec == MRHS_PREC_MIX_FP16) fmt = tc_fmt_tf32;
      break;
    default: break;
  }
  if (fmt >= 0 && build_Dc_tc(c, fmt, split)) {
    size_t tot = (size_t)c->g.nagg * 4 * nc * nc;
    k_coarse_backward<float><<<grid_for(tot, 256), 256, 0, c->stream>>>((cx<float>*)c->Dc, c->aggnbr, c->g.nagg, Nt);
    MRHS_LAUNCH_CHECK("coarse_backward");
    c->have_Dc = true;
    ++c->dc_version;
    dc_images_build(c);
    return;
  }
  MRHS_REQUIRE(c->dc_engine == MRHS_DC_AUTO || c->dc_engine == MRHS_DC_ALU, MRHS_ERR_SHAPE,
               "tensor-core D_c contraction needs FP32 work fields and 2*ntv <= 64");
  Prof pr(c, "coarse_op");
  MRHS_DISPATCH(c->tv_dtype, SP, {
    using R = typename Real<SP>::type;
    const cx<R>* U = (const cx<R>*)(sizeof(R) == 8 ? (const void*)c->U64 : (const void*)c->U32);
    const R* Acl = (const R*)(sizeof(R) == 8 ? (const void*)c->A64 : (const void*)c->A32);
    if (tiled) {
      size_t smem = sizeof(cx<R>) * kTileSites * 12 * (size_t)(nc + Nt);
      auto kern = k_coarse_op_tiled<SP, R>;
      MRHS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      kern<<<c->g.nagg * 5, 256, smem, c->stream>>>((const SP*)c->P, U, Acl, c->nbr, Nt, ag, c->g.Va, (cx<R>*)c->Dc);
      MRHS_LAUNCH_CHECK("coarse_op_tiled");
      size_t tot = (size_t)c->g.nagg * 4 * nc * nc;
      k_coarse_backward<R><<<grid_for(tot, 256), 256, 0, c->stream>>>((cx<R>*)c->Dc, c->aggnbr, c->g.nagg, Nt);
      MRHS_LAUNCH_CHECK("coarse_backward");
    } else {
      int threads = std::max(128, ((nc * nc + 15) / 16 + 31) / 32 * 32);
      MRHS_REQUIRE(threads <= 1024, MRHS_ERR_SHAPE, "ntv too large for the coarse-operator kernel");
      size_t smem = sizeof(cx<R>) * kSites * 12 * (size_t)(nc + Nt);
      auto kern = k_coarse_op<SP, R, 16>;
      MRHS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      kern<<<c->g.nagg * 9, threads, smem, c->stream>>>((const SP*)c->P, U, Acl, c->nbr, Nt, ag, c->g.Va,
                                                        (cx<R>*)c->Dc);
      MRHS_LAUNCH_CHECK("coarse_op");
    }
  });
  c->have_Dc = true;
  ++c->dc_version;
  dc_images_build(c);
}

// restriction from a fine field of type dv into a coarse field of type dc
void restrict_typed(mrhs_ctx c, const void* v, int dv, void* vc, int dc, int N) {
  MRHS_REQUIRE(c->have_P, MRHS_ERR_STATE, "restriction before mrhs_build_P");
  MRHS_REQUIRE(N >= 1 && N <= 64, MRHS_ERR_ARG, "restriction: 1 <= nrhs <= 64");
  const int Nt = c->ntv, nc = 2 * Nt;
  int threads = std::max(64, ((nc * N + 7) / 8 + 31) / 32 * 32);
  MRHS_REQUIRE(threads <= 1024, MRHS_ERR_SHAPE, "restriction: ntv*nrhs too large");
  MRHS_REQUIRE(dc == MRHS_F64 || dc == MRHS_F32, MRHS_ERR_ARG, "coarse fields are F64 or F32");
  Prof pr(c, "restrict");
  static const bool stream_off = [] {
    const char* e = std::getenv("MRHS_RESTRICT");
    return e && std::string(e) == "tiled";
  }();
  if (!stream_off && c->tv_dtype == MRHS_F32 && dv == MRHS_F32 && dc == MRHS_F32 && Nt % 4 == 0 && N % 4 == 0 &&
      2 * (Nt / 4) * (N / 4) <= 128) {
    k_restrict_stream<<<c->g.nagg, 128, 0, c->stream>>>((const float*)c->P, (const float*)v, (float*)vc, Nt, N,
                                                        c->g.Va);
    MRHS_LAUNCH_CHECK("restrict_stream");
    return;
  }
  const bool tiled = Nt % 4 == 0 && N % 2 == 0 && (nc / 4) * (N / 2) <= 256;
  MRHS_DISPATCH(c->tv_dtype, SP, MRHS_DISPATCH(dv, SV, {
    if (tiled) {
      if (dc == MRHS_F64) {
        size_t smem = sizeof(cx<double>) * kSites * 12 * (size_t)(Nt + N);
        auto kern = k_restrict_tiled<SP, SV, double>;
        MRHS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<c->g.nagg, 256, smem, c->stream>>>((const SP*)c->P, (const SV*)v, (double*)vc, Nt, N, c->g.Va);
      } else {
        size_t smem = sizeof(cx<float>) * kSites * 12 * (size_t)(Nt + N);
        auto kern = k_restrict_tiled<SP, SV, float>;
        MRHS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<c->g.nagg, 256, smem, c->stream>>>((const SP*)c->P, (const SV*)v, (float*)vc, Nt, N, c->g.Va);
      }
    } else if (dc == MRHS_F64) {
      size_t smem = sizeof(cx<double>) * kSites * 12 * (size_t)(Nt + N);
      auto kern = k_restrict<SP, SV, double, 8>;
      MRHS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      kern<<<c->g.nagg, threads, smem, c->stream>>>((const SP*)c->P, (const SV*)v, (double*)vc, Nt, N, c->g.Va);
    } else {
      size_t smem = sizeof(cx<float>) * kSites * 12 * (size_t)(Nt + N);
      auto kern = k_restrict<SP, SV, float, 8>;
      MRHS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      kern<<<c->g.nagg, threads, smem, c->stream>>>((const SP*)c->P, (const SV*)v, (float*)vc, Nt, N, c->g.Va);
    }
  }));
  MRHS_LAUNCH_CHECK("restrict");
}

void prolong_typed(mrhs_ctx c, const void* uc, int dc, void* u, int du, int N) {
  MRHS_REQUIRE(c->have_P, MRHS_ERR_STATE, "prolongation before mrhs_build_P");
  MRHS_REQUIRE(dc == MRHS_F64 || dc == MRHS_F32, MRHS_ERR_ARG, "coarse fields are F64 or F32");
  size_t work = (size_t)c->g.V * 2 * N;
  Prof pr(c, "prolong");
  if (dc == MRHS_F32 && du == MRHS_F32 && N % 4 == 0 && ((uintptr_t)uc & 15) == 0 && ((uintptr_t)u & 15) == 0) {
    const size_t w4 = (size_t)c->g.V * 2 * (N / 4);
    MRHS_DISPATCH(c->tv_dtype, SP, (k_prolong6x4<SP><<<grid_for(w4, 256), 256, 0, c->stream>>>((const SP*)c->P, (const float*)uc, (float*)u, c->ntv, N, c->g.Va, w4)));
    MRHS_LAUNCH_CHECK("prolong");
    return;
  }
  MRHS_DISPATCH(c->tv_dtype, SP, MRHS_DISPATCH(du, SU, {
    if (dc == MRHS_F64)
      k_prolong6<SP, double, SU><<<grid_for(work, 256), 256, 0, c->stream>>>((const SP*)c->P, (const double*)uc, (SU*)u, c->ntv, N, c->g.Va, work);
    else
      k_prolong6<SP, float, SU><<<grid_for(work, 256), 256, 0, c->stream>>>((const SP*)c->P, (const float*)uc, (SU*)u, c->ntv, N, c->g.Va, work);
  }));
  MRHS_LAUNCH_CHECK("prolong");
}

void restrict_(mrhs_ctx c, const void* v, void* vc, int nrhs, int dtype) {
  MRHS_REQUIRE(dtype == c->work_dtype, MRHS_ERR_ARG, "restriction: dtype must be the context's work type");
  restrict_typed(c, v, dtype, vc, dtype, nrhs);
}

void prolong(mrhs_ctx c, const void* uc, void* u, int nrhs, int dtype) {
  MRHS_REQUIRE(dtype == c->work_dtype, MRHS_ERR_ARG, "prolongation: dtype must be the context's work type");
  prolong_typed(c, uc, dtype, u, dtype, nrhs);
}

void apply_Dc(mrhs_ctx c, const void* xc, void* yc, int nrhs, int dtype) {
  apply_Dc_part(c, DcPart{nullptr, c->g.nagg, nullptr, 0, 9, xc, xc, nullptr}, yc, nrhs, dtype);
}

void apply_Dc_part(mrhs_ctx c, const DcPart& pt, void* yc, int nrhs, int dtype) {
  MRHS_REQUIRE(c->have_Dc, MRHS_ERR_STATE, "D_c used before mrhs_build_Dc");
  MRHS_REQUIRE(dtype == c->work_dtype, MRHS_ERR_ARG, "D_c apply: dtype must be the context's work type");
  const int nc = 2 * c->ntv;
  // tensor cores unless the CUDA-core engine is chosen: split tf32 (FP32
  // accuracy) for the FP32 setup, single tf32 for the mixed ones
  static const bool apply_alu = [] {
    const char* e = std::getenv("MRHS_DC_APPLY");
    return e && std::string(e) == "alu";
  }();
  if (c->dc_engine != MRHS_DC_ALU && dtype == MRHS_F32 && !apply_alu) {
    const bool split = c->prec == MRHS_PREC_FP32;
    if (apply_Dc_tc(c, pt, yc, nrhs, split)) return;
  }
  Prof pr(c, "apply_dc");
  auto launch = [&](auto* tag) {
    using SC = std::remove_pointer_t<decltype(tag)>;
    using R = typename Real<SC>::type;
    const DcPartArgs<SC> pa{pt.alist, pt.pos, pt.kb, pt.ke, (const SC*)pt.x0, (const SC*)pt.xh, (const SC*)pt.add};
    if (nc % 8 == 0) {
      const size_t work = (size_t)pt.na * (nc / 8) * nrhs;
      k_apply_dc_tiled<SC><<<grid_for(work, 128), 128, 0, c->stream>>>((const cx<R>*)c->Dc, pa, (SC*)yc, c->aggnbr,
                                                                        nc, nrhs, work);
    } else {
      const size_t work = (size_t)pt.na * nc * nrhs;
      k_apply_dc<SC><<<grid_for(work, 256), 256, 0, c->stream>>>((const cx<R>*)c->Dc, pa, (SC*)yc, c->aggnbr, nc,
                                                                  nrhs, work);
    }
  };
  if (dtype == MRHS_F64)
    launch((double*)nullptr);
  else
    launch((float*)nullptr);
  MRHS_LAUNCH_CHECK("apply_dc");
}

// ------------------------------------------------------------------------
// Even-odd preconditioned coarse solve. The aggregates carry the red-black
// colour of the SAP domains and every hop block of D_c joins aggregates of
// different colour, so D_c = [[D_ee, D_eo], [D_oe, D_oo]] with block-diagonal
// D_ee, D_oo (the self blocks). GMRES runs on S = D_ee - D_eo D_oo^-1 D_oe
// over the even aggregates only, then x_o = D_oo^-1 (b_o - D_oe x_e). Every
// vector of the solve is compact: the row blocks of one colour in the order
// of that colour's aggregate list (blocks_col), so the Krylov basis and its
// dots and updates are half the size of the plain solve's.
namespace {
// the inverse self block of every odd aggregate (CTA b: aggregate
// blist[b], stored at Dinv[b]): Gauss-Jordan in place with partial pivoting
// (row interchanges, undone as column interchanges in reverse order at the
// end) on the block in shared memory; *bad set for a singular block
template <class R>
__global__ void k_self_inverse(const cx<R>* __restrict__ Dc, cx<R>* __restrict__ Dinv, const int* __restrict__ blist,
                               int nc, int* bad) {
  extern __shared__ double smem_d[];
  cx<R>* m = (cx<R>*)smem_d;  // [nc][nc]
  __shared__ cx<R> s_f[128];
  __shared__ int s_piv[128];
  __shared__ int s_p;
  const int A = blist[blockIdx.x];
  const cx<R>* S = Dc + (size_t)A * 9 * nc * nc;
  for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) m[e] = S[e];
  __syncthreads();
  for (int k = 0; k < nc; ++k) {
    if (threadIdx.x < 32) {
      // pivot: the largest |m[i][k]|^2, i >= k (the first on ties), by warp 0
      const int lane = threadIdx.x;
      R best = -1;
      int p = -1;
      for (int i = k + lane; i < nc; i += 32) {
        const cx<R> v = m[i * nc + k];
        const R a = v.re * v.re + v.im * v.im;
        if (a > best) best = a, p = i;
      }
      for (int off = 16; off > 0; off >>= 1) {
        const R ob = __shfl_down_sync(0xffffffffu, best, off);
        const int op = __shfl_down_sync(0xffffffffu, p, off);
        if (op >= 0 && (ob > best || (ob == best && op < p))) best = ob, p = op;
      }
      if (lane == 0) {
        s_p = best > 0 ? p : -1;
        s_piv[k] = p;
      }
    }
    __syncthreads();
    const int p = s_p;
    if (p < 0) {
      if (threadIdx.x == 0) atomicExch(bad, 1);
      return;
    }
    if (p != k)
      for (int j = threadIdx.x; j < nc; j += blockDim.x) {
        const cx<R> t = m[p * nc + j];
        m[p * nc + j] = m[k * nc + j];
        m[k * nc + j] = t;
      }
    __syncthreads();
    const cx<R> piv = m[k * nc + k];
    const R pn = piv.re * piv.re + piv.im * piv.im;
    const cx<R> d = mk<R>(piv.re / pn, -piv.im / pn);
    for (int i = threadIdx.x; i < nc; i += blockDim.x) s_f[i] = i == k ? mk<R>(0, 0) : m[i * nc + k];
    __syncthreads();
    // row k scaled by d, with d itself in column k
    for (int j = threadIdx.x; j < nc; j += blockDim.x) m[k * nc + j] = j == k ? d : m[k * nc + j] * d;
    __syncthreads();
    // every other row: minus f_i times row k; column k becomes -f_i d
    for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) {
      const int i = e / nc, j = e % nc;
      if (i == k) continue;
      m[e] = j == k ? mk<R>(0, 0) - s_f[i] * d : m[e] - s_f[i] * m[k * nc + j];
    }
    __syncthreads();
  }
  for (int k = nc - 1; k >= 0; --k) {
    const int p = s_piv[k];
    if (p != k)
      for (int i = threadIdx.x; i < nc; i += blockDim.x) {
        const cx<R> t = m[i * nc + p];
        m[i * nc + p] = m[i * nc + k];
        m[i * nc + k] = t;
      }
    __syncthreads();
  }
  cx<R>* out = Dinv + (size_t)blockIdx.x * nc * nc;
  for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) out[e] = m[e];
}

// y[b] = s Dinv[b] (a[b] - c[b]) for the compact odd row blocks b (c may be
// null); 8 rows x 1 right-hand side per thread (nc % 8 = 0), so that every
// load of a serves eight rows
template <class S, class R>
__global__ void k_inverse_apply8(const cx<R>* __restrict__ Dinv, const S* __restrict__ a, const S* __restrict__ c,
                                 S* __restrict__ y, R s, int nc, int N, size_t nwork) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= nwork) return;
  const int r = (int)(t % N);
  const size_t q = t / N;
  const int nrt = nc / 8;
  const size_t b = q / nrt;
  const size_t row0 = b * nc + 8 * (q % nrt);
  cx<R> acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = mk<R>(0, 0);
  for (int j = 0; j < nc; ++j) {
    cx<R> v = ld<S, R>(a, b * nc + j, N, r);
    if (c) v = v - ld<S, R>(c, b * nc + j, N, r);
#pragma unroll
    for (int k = 0; k < 8; ++k) fma_(acc[k], Dinv[(row0 + k) * nc + j], v);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) st<S, R>(y, row0 + k, N, r, scale(acc[k], s));
}

// the same with one CTA per compact odd block: its inverse (nc x nc) staged
// in shared memory once, read there by every (8-row group, rhs) item of the
// block; the same sums in the same order as k_inverse_apply8
template <class S, class R>
__global__ void __launch_bounds__(256) k_inverse_apply_blk(const cx<R>* __restrict__ Dinv, const S* __restrict__ a,
                                                           const S* __restrict__ c, S* __restrict__ y, R s, int nc,
                                                           int N) {
  extern __shared__ double smem_iv[];
  cx<R>* M = reinterpret_cast<cx<R>*>(smem_iv);  // [nc][nc]
  const size_t b = blockIdx.x;
  for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) M[e] = Dinv[b * nc * nc + e];
  __syncthreads();
  const int nrt = nc / 8;
  for (int w = threadIdx.x; w < nrt * N; w += blockDim.x) {
    const int r = w % N, g = w / N;
    const size_t row0 = b * nc + 8 * g;
    cx<R> acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = mk<R>(0, 0);
    for (int j = 0; j < nc; ++j) {
      cx<R> v = ld<S, R>(a, b * nc + j, N, r);
      if (c) v = v - ld<S, R>(c, b * nc + j, N, r);
#pragma unroll
      for (int k = 0; k < 8; ++k) fma_(acc[k], M[(8 * g + k) * nc + j], v);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) st<S, R>(y, row0 + k, N, r, scale(acc[k], s));
  }
}

// the same with one row per thread (any nc)
template <class S, class R>
__global__ void k_inverse_apply(const cx<R>* __restrict__ Dinv, const S* __restrict__ a, const S* __restrict__ c,
                                S* __restrict__ y, R s, int nc, int N, size_t nwork) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= nwork) return;
  const int r = (int)(t % N);
  const size_t row = t / N;  // b * nc + i
  const size_t b = row / nc;
  const cx<R>* M = Dinv + row * nc;
  cx<R> acc = mk<R>(0, 0);
  for (int j = 0; j < nc; ++j) {
    cx<R> v = ld<S, R>(a, b * nc + j, N, r);
    if (c) v = v - ld<S, R>(c, b * nc + j, N, r);
    fma_(acc, M[j], v);
  }
  st<S, R>(y, row, N, r, scale(acc, s));
}

// compact row blocks <-> the full coarse field: part b of the colour list
// blist is the row block blist[b] of the full field
template <class S>
__global__ void k_colour_gather(const S* __restrict__ full, S* __restrict__ part, const int* __restrict__ blist,
                                size_t blk, size_t nwork) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= nwork) return;
  part[t] = full[(size_t)blist[t / blk] * blk + t % blk];
}
template <class S>
__global__ void k_colour_scatter(const S* __restrict__ part, S* __restrict__ full, const int* __restrict__ blist,
                                 size_t blk, size_t nwork) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= nwork) return;
  full[(size_t)blist[t / blk] * blk + t % blk] = part[t];
}
}  // namespace

// the inverse self blocks of the odd aggregates for the current D_c
static void ensure_self_inverses(mrhs_ctx c) {
  const int nc = 2 * c->ntv;
  MRHS_REQUIRE(nc <= 128, MRHS_ERR_SHAPE, "even-odd coarse solve: 2 ntv must be at most 128");
  if (c->dc_inv && c->dc_inv_version == c->dc_version) return;
  const size_t es = c->work_dtype == MRHS_F64 ? sizeof(cx<double>) : sizeof(cx<float>);
  const size_t smem = (size_t)nc * nc * es;
  int optin = 0;
  MRHS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
  MRHS_REQUIRE(smem <= (size_t)optin, MRHS_ERR_SHAPE,
               "even-odd coarse solve: a self block of this size does not fit in shared memory");
  if (!c->dc_inv) c->dc_inv = dalloc(c, (size_t)c->ncol[1] * nc * nc * es);
  MRHS_CUDA(cudaMemsetAsync(c->dflag + 5, 0, sizeof(int), c->stream));
  const int* odd = c->blocks_col + c->ncol[0];
  Prof pr(c, "self_inverse");
  if (c->work_dtype == MRHS_F64) {
    MRHS_CUDA(cudaFuncSetAttribute(k_self_inverse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_self_inverse<double><<<c->ncol[1], 256, smem, c->stream>>>((const cx<double>*)c->Dc, (cx<double>*)c->dc_inv,
                                                                 odd, nc, c->dflag + 5);
  } else {
    MRHS_CUDA(cudaFuncSetAttribute(k_self_inverse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_self_inverse<float><<<c->ncol[1], 256, smem, c->stream>>>((const cx<float>*)c->Dc, (cx<float>*)c->dc_inv, odd,
                                                                nc, c->dflag + 5);
  }
  MRHS_LAUNCH_CHECK("self_inverse");
  MRHS_CUDA(cudaMemcpyAsync(c->hflag + 5, c->dflag + 5, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MRHS_CUDA(cudaStreamSynchronize(c->stream));
  MRHS_REQUIRE(c->hflag[5] == 0, MRHS_ERR_NONFINITE, "even-odd coarse solve: a self block of D_c is singular");
  c->dc_inv_version = c->dc_version;
}

namespace {
// y = s D_oo^-1 (a - b) on compact odd blocks (b may be null)
void inverse_apply(mrhs_ctx c, const void* a, const void* b, void* y, double s, int N, int dtype) {
  const int nc = 2 * c->ntv;
  Prof pr(c, "inverse_apply");
  const size_t es = dtype == MRHS_F64 ? sizeof(cx<double>) : sizeof(cx<float>);
  const size_t smem = (size_t)nc * nc * es;
  if (nc % 8 == 0 && smem <= 48 * 1024) {
    if (dtype == MRHS_F64)
      k_inverse_apply_blk<double, double><<<c->ncol[1], 256, smem, c->stream>>>(
          (const cx<double>*)c->dc_inv, (const double*)a, (const double*)b, (double*)y, s, nc, N);
    else
      k_inverse_apply_blk<float, float><<<c->ncol[1], 256, smem, c->stream>>>(
          (const cx<float>*)c->dc_inv, (const float*)a, (const float*)b, (float*)y, (float)s, nc, N);
    MRHS_LAUNCH_CHECK("inverse_apply");
    return;
  }
  if (nc % 8 == 0) {
    const size_t work = (size_t)c->ncol[1] * (nc / 8) * N;
    if (dtype == MRHS_F64)
      k_inverse_apply8<double, double><<<grid_for(work, 128), 128, 0, c->stream>>>(
          (const cx<double>*)c->dc_inv, (const double*)a, (const double*)b, (double*)y, s, nc, N, work);
    else
      k_inverse_apply8<float, float><<<grid_for(work, 128), 128, 0, c->stream>>>(
          (const cx<float>*)c->dc_inv, (const float*)a, (const float*)b, (float*)y, (float)s, nc, N, work);
    MRHS_LAUNCH_CHECK("inverse_apply");
    return;
  }
  const size_t work = (size_t)c->ncol[1] * nc * N;
  if (dtype == MRHS_F64)
    k_inverse_apply<double, double><<<grid_for(work, 256), 256, 0, c->stream>>>(
        (const cx<double>*)c->dc_inv, (const double*)a, (const double*)b, (double*)y, s, nc, N, work);
  else
    k_inverse_apply<float, float><<<grid_for(work, 256), 256, 0, c->stream>>>(
        (const cx<float>*)c->dc_inv, (const float*)a, (const float*)b, (float*)y, (float)s, nc, N, work);
  MRHS_LAUNCH_CHECK("inverse_apply");
}
void colour_copy(mrhs_ctx c, const void* src, void* dst, int colour, bool gather, int N, int dtype) {
  const size_t blk = (size_t)2 * c->ntv * 2 * N;
  const size_t work = (size_t)c->ncol[colour] * blk;
  const int* bl = c->blocks_col + (colour ? c->ncol[0] : 0);
  MRHS_DISPATCH(dtype, S, (gather ? k_colour_gather<S><<<grid_for(work, 256), 256, 0, c->stream>>>((const S*)src, (S*)dst, bl, blk, work)
                                  : k_colour_scatter<S><<<grid_for(work, 256), 256, 0, c->stream>>>((const S*)src, (S*)dst, bl, blk, work)));
  MRHS_LAUNCH_CHECK("colour_copy");
}
// the part of the stencil over the aggregates of one colour, on compact fields
DcPart colour_part(mrhs_ctx c, int colour, int kb, const void* x0, const void* xh, const void* add) {
  return DcPart{c->blocks_col + (colour ? c->ncol[0] : 0), c->ncol[colour], c->colpos, kb, 9, x0, xh, add};
}
}  // namespace

// y = S x on compact even fields: t_o = D_oe x, u_o = -D_oo^-1 t_o,
// y = D_ee x + D_eo u_o (t and u: compact odd work fields)
static void apply_schur(mrhs_ctx c, const void* x, void* y, void* t, void* u, int N, int dtype) {
  apply_Dc_part(c, colour_part(c, 1, 1, nullptr, x, nullptr), t, N, dtype);
  inverse_apply(c, t, nullptr, u, -1.0, N, dtype);
  apply_Dc_part(c, colour_part(c, 0, 0, x, u, nullptr), y, N, dtype);
}

// restarted GMRES on `rows` coarse rows: op(x, y) is D_c, or S on compact
// even fields
template <class Op>
static void coarse_gmres(mrhs_ctx c, const void* bc, void* xc, int N, int dtype, double tol, int m, int maxit,
                         int* iters, size_t rows, Op op) {
  const size_t fe = rows * 2 * N;  // elements of one coarse field
  const size_t es = dtype_size(dtype);
  char* basis = (char*)scratch(c, SC_KRYLOV, (size_t)(m + 2) * fe * es);
  char* w = basis + (size_t)(m + 1) * fe * es;
  auto Vk = [&](int k) { return (void*)(basis + (size_t)k * fe * es); };
  size_t sbytes = 0;
  sbytes += 3 * sizeof(cx<double>) * N * (size_t)(m + 1) * m + 256 * 16;
  char* sp = (char*)scratch(c, SC_HESS, sbytes + sizeof(double) * 16 * N * (size_t)(m + 2) + 4096);
  GmState st;
  st.H = carve<cx<double>>(sp, (size_t)N * (m + 1) * m);
  st.cs = carve<cx<double>>(sp, (size_t)N * m);
  st.sn = carve<cx<double>>(sp, (size_t)N * m);
  st.g = carve<cx<double>>(sp, (size_t)N * (m + 1));
  st.y = carve<double>(sp, (size_t)m * N * 2);
  st.h1 = carve<double>(sp, (size_t)(m + 1) * N * 2);
  st.h2 = carve<double>(sp, (size_t)(m + 1) * N * 2);
  st.hn2 = carve<double>(sp, (size_t)N * 2);
  st.beta2 = carve<double>(sp, (size_t)N * 2);
  st.bnorm2 = carve<double>(sp, (size_t)N * 2);
  st.inv = carve<double>(sp, (size_t)N);
  st.conv = carve<int>(sp, N);
  st.active = carve<int>(sp, N);
  st.its = carve<int>(sp, N);
  st.kend = carve<int>(sp, N);
  st.counter = carve<int>(sp, 1);
  int* hcount = c->hflag + 1;
  auto read_counter = [&]() {
    MRHS_CUDA(cudaMemcpyAsync(hcount, st.counter, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    MRHS_CUDA(cudaStreamSynchronize(c->stream));
    return *hcount;
  };
  auto scale_into = [&](const void* x, void* y) {
    MRHS_DISPATCH(dtype, S, (k_scale_rhs<S><<<grid_for(rows * N, 256), 256, 0, c->stream>>>((const S*)x, (S*)y, rows, N, st.inv)));
    MRHS_LAUNCH_CHECK("scale_rhs");
  };
  MRHS_CUDA(cudaMemsetAsync(xc, 0, fe * es, c->stream));
  norms(c, bc, rows, N, dtype, st.bnorm2);
  k_gm_init<<<grid_for(N, 64), 64, 0, c->stream>>>(st, N);
  MRHS_LAUNCH_CHECK("gm_init");
  for (;;) {
    op(xc, w);
    MRHS_DISPATCH(dtype, S, (k_sub_from<S><<<grid_for(fe, 256), 256, 0, c->stream>>>((const S*)bc, (S*)w, fe)));
    MRHS_LAUNCH_CHECK("sub_from");
    norms(c, w, rows, N, dtype, st.beta2);
    MRHS_CUDA(cudaMemsetAsync(st.counter, 0, sizeof(int), c->stream));
    k_gm_start<<<grid_for(N, 64), 64, 0, c->stream>>>(st, N, m, tol, maxit);
    MRHS_LAUNCH_CHECK("gm_start");
    if (read_counter() == 0) break;
    scale_into(w, Vk(0));
    int kmax = 0;
    for (int k = 0; k < m; ++k) {
      op(Vk(k), w);
      multi_dot(c, Vk(0), fe, k + 1, w, rows, N, dtype, st.h1);
      multi_axpy(c, Vk(0), fe, k + 1, w, rows, N, dtype, st.h1, -1.0);
      multi_dot(c, Vk(0), fe, k + 1, w, rows, N, dtype, st.h2);
      multi_axpy(c, Vk(0), fe, k + 1, w, rows, N, dtype, st.h2, -1.0);
      norms(c, w, rows, N, dtype, st.hn2);
      MRHS_CUDA(cudaMemsetAsync(st.counter, 0, sizeof(int), c->stream));
      k_gm_step<<<grid_for(N, 64), 64, 0, c->stream>>>(st, N, m, k, tol, maxit);
      MRHS_LAUNCH_CHECK("gm_step");
      kmax = k + 1;
      int more = read_counter();
      if (more == 0) break;
      scale_into(w, Vk(k + 1));
    }
    k_gm_solve<<<grid_for(N, 64), 64, 0, c->stream>>>(st, N, m);
    MRHS_LAUNCH_CHECK("gm_solve");
    multi_axpy(c, Vk(0), fe, kmax, xc, rows, N, dtype, st.y, 1.0);
  }
  if (iters) {
    MRHS_CUDA(cudaMemcpyAsync(iters, st.its, sizeof(int) * N, cudaMemcpyDeviceToHost, c->stream));
    MRHS_CUDA(cudaStreamSynchronize(c->stream));
  }
  check_tc_timeout(c);
}

void coarse_solve(mrhs_ctx c, const void* bc, void* xc, int N, int dtype, double tol, int m, int maxit, int* iters) {
  MRHS_REQUIRE(c->have_Dc, MRHS_ERR_STATE, "coarse solve before mrhs_build_Dc");
  MRHS_REQUIRE(dtype == c->work_dtype, MRHS_ERR_ARG, "coarse solve: dtype must be the context's work type");
  MRHS_REQUIRE(N >= 1 && N <= 256 && m >= 1 && m <= 64 && maxit >= 0 && tol >= 0, MRHS_ERR_ARG,
               "coarse solve: need 1 <= nrhs <= 256, 1 <= restart <= 64, maxit >= 0, tol >= 0");
  const int nc = 2 * c->ntv;
  if (!c->coarse_eo) {
    coarse_gmres(c, bc, xc, N, dtype, tol, m, maxit, iters, (size_t)c->g.nagg * nc,
                 [&](const void* x, void* y) { apply_Dc(c, x, y, N, dtype); });
    return;
  }
  ensure_self_inverses(c);
  // compact fields: b_e, b_o, bhat_e, x_e, and two odd work fields
  const size_t hb = (size_t)c->ncol[0] * nc * 2 * N * dtype_size(dtype);
  char* wk = (char*)scratch(c, SC_COARSE_EO, 6 * hb);
  void* be = wk;
  void* bo = wk + hb;
  void* bh = wk + 2 * hb;
  void* xe = wk + 3 * hb;
  void* t = wk + 4 * hb;
  void* u = wk + 5 * hb;
  colour_copy(c, bc, be, 0, true, N, dtype);
  colour_copy(c, bc, bo, 1, true, N, dtype);
  // bhat_e = b_e - D_eo D_oo^-1 b_o
  inverse_apply(c, bo, nullptr, u, -1.0, N, dtype);
  apply_Dc_part(c, colour_part(c, 0, 1, nullptr, u, be), bh, N, dtype);
  // GMRES on S from x_e = 0
  coarse_gmres(c, bh, xe, N, dtype, tol, m, maxit, iters, (size_t)c->ncol[0] * nc,
               [&](const void* x, void* y) { apply_schur(c, x, y, t, u, N, dtype); });
  // x_o = D_oo^-1 (b_o - D_oe x_e)
  apply_Dc_part(c, colour_part(c, 1, 1, nullptr, xe, nullptr), t, N, dtype);
  inverse_apply(c, bo, t, u, 1.0, N, dtype);
  colour_copy(c, xe, xc, 0, false, N, dtype);
  colour_copy(c, u, xc, 1, false, N, dtype);
}

// ------------------------------------------------------------------------
// The same coarse GMRES on one caller-supplied workspace: basis, GMRES state
// and reduction partials are carved from ws; nothing is allocated.
namespace {
struct WsLayout {
  size_t basis, state, part, total;
};
WsLayout ws_layout(mrhs_ctx c, int N, int dtype, int m) {
  const size_t rows = (size_t)c->g.nagg * 2 * c->ntv;
  const size_t fe = rows * 2 * N;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  WsLayout L;
  L.basis = up((size_t)(m + 2) * fe * dtype_size(dtype));
  size_t st = 0;
  st += up(sizeof(cx<double>) * (size_t)N * (m + 1) * m);      // H
  st += 2 * up(sizeof(cx<double>) * (size_t)N * m);            // cs, sn
  st += up(sizeof(cx<double>) * (size_t)N * (m + 1));          // g
  st += up(sizeof(double) * (size_t)m * N * 2);                 // y
  st += 2 * up(sizeof(double) * (size_t)(m + 1) * N * 2);      // h1, h2
  st += 3 * up(sizeof(double) * (size_t)N * 2);                // hn2, beta2, bnorm2
  st += up(sizeof(double) * (size_t)N);                        // inv
  st += 4 * up(sizeof(int) * (size_t)N) + up(sizeof(int));     // conv, active, its, kend, counter
  L.state = st;
  L.part = up(multi_dot_partials_bytes(rows, N, m + 1));
  L.total = L.basis + L.state + L.part;
  return L;
}
}  // namespace

size_t coarse_solve_ws_bytes(mrhs_ctx c, int nrhs, int dtype, int restart) {
  return ws_layout(c, nrhs, dtype, restart).total;
}

void coarse_solve_ws(mrhs_ctx c, const void* bc, void* xc, int N, int dtype, double tol, int m, int maxit, int* iters,
                     void* ws, size_t ws_bytes) {
  MRHS_REQUIRE(c->have_Dc, MRHS_ERR_STATE, "coarse solve before mrhs_build_Dc");
  MRHS_REQUIRE(dtype == c->work_dtype, MRHS_ERR_ARG, "coarse solve: dtype must be the context's work type");
  MRHS_REQUIRE(N >= 1 && N <= 256 && m >= 1 && m <= 64 && maxit >= 0 && tol >= 0, MRHS_ERR_ARG,
               "coarse solve: need 1 <= nrhs <= 256, 1 <= restart <= 64, maxit >= 0, tol >= 0");
  const WsLayout L = ws_layout(c, N, dtype, m);
  MRHS_REQUIRE(L.total <= ws_bytes, MRHS_ERR_SHAPE, "coarse solve workspace too small");
  const size_t rows = (size_t)c->g.nagg * 2 * c->ntv;
  const size_t fe = rows * 2 * N;
  const size_t es = dtype_size(dtype);
  char* basis = (char*)ws;
  char* w = basis + (size_t)(m + 1) * fe * es;
  auto Vk = [&](int k) { return (void*)(basis + (size_t)k * fe * es); };
  char* sp = basis + L.basis;
  GmState st;
  st.H = carve<cx<double>>(sp, (size_t)N * (m + 1) * m);
  st.cs = carve<cx<double>>(sp, (size_t)N * m);
  st.sn = carve<cx<double>>(sp, (size_t)N * m);
  st.g = carve<cx<double>>(sp, (size_t)N * (m + 1));
  st.y = carve<double>(sp, (size_t)m * N * 2);
  st.h1 = carve<double>(sp, (size_t)(m + 1) * N * 2);
  st.h2 = carve<double>(sp, (size_t)(m + 1) * N * 2);
  st.hn2 = carve<double>(sp, (size_t)N * 2);
  st.beta2 = carve<double>(sp, (size_t)N * 2);
  st.bnorm2 = carve<double>(sp, (size_t)N * 2);
  st.inv = carve<double>(sp, (size_t)N);
  st.conv = carve<int>(sp, N);
  st.active = carve<int>(sp, N);
  st.its = carve<int>(sp, N);
  st.kend = carve<int>(sp, N);
  st.counter = carve<int>(sp, 1);
  double* part = (double*)(basis + L.basis + L.state);
  int* hcount = c->hflag + 1;
  auto read_counter = [&]() {
    MRHS_CUDA(cudaMemcpyAsync(hcount, st.counter, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    MRHS_CUDA(cudaStreamSynchronize(c->stream));
    return *hcount;
  };
  auto scale_into = [&](const void* x, void* y) {
    MRHS_DISPATCH(dtype, S, (k_scale_rhs<S><<<grid_for(rows * N, 256), 256, 0, c->stream>>>((const S*)x, (S*)y, rows, N, st.inv)));
    MRHS_LAUNCH_CHECK("scale_rhs");
  };
  MRHS_CUDA(cudaMemsetAsync(xc, 0, fe * es, c->stream));
  multi_dot_ws(c, bc, 0, 1, bc, rows, N, dtype, st.bnorm2, part);
  k_gm_init<<<grid_for(N, 64), 64, 0, c->stream>>>(st, N);
  MRHS_LAUNCH_CHECK("gm_init");
  for (;;) {
    apply_Dc(c, xc, w, N, dtype);
    MRHS_DISPATCH(dtype, S, (k_sub_from<S><<<grid_for(fe, 256), 256, 0, c->stream>>>((const S*)bc, (S*)w, fe)));
    MRHS_LAUNCH_CHECK("sub_from");
    multi_dot_ws(c, w, 0, 1, w, rows, N, dtype, st.beta2, part);
    MRHS_CUDA(cudaMemsetAsync(st.counter, 0, sizeof(int), c->stream));
    k_gm_start<<<grid_for(N, 64), 64, 0, c->stream>>>(st, N, m, tol, maxit);
    MRHS_LAUNCH_CHECK("gm_start");
    if (read_counter() == 0) break;
    scale_into(w, Vk(0));
    int kmax = 0;
    for (int k = 0; k < m; ++k) {
      apply_Dc(c, Vk(k), w, N, dtype);
      multi_dot_ws(c, Vk(0), fe, k + 1, w, rows, N, dtype, st.h1, part);
      multi_axpy(c, Vk(0), fe, k + 1, w, rows, N, dtype, st.h1, -1.0);
      multi_dot_ws(c, Vk(0), fe, k + 1, w, rows, N, dtype, st.h2, part);
      multi_axpy(c, Vk(0), fe, k + 1, w, rows, N, dtype, st.h2, -1.0);
      multi_dot_ws(c, w, 0, 1, w, rows, N, dtype, st.hn2, part);
      MRHS_CUDA(cudaMemsetAsync(st.counter, 0, sizeof(int), c->stream));
      k_gm_step<<<grid_for(N, 64), 64, 0, c->stream>>>(st, N, m, k, tol, maxit);
      MRHS_LAUNCH_CHECK("gm_step");
      kmax = k + 1;
      if (read_counter() == 0) break;
      scale_into(w, Vk(k + 1));
    }
    k_gm_solve<<<grid_for(N, 64), 64, 0, c->stream>>>(st, N, m);
    MRHS_LAUNCH_CHECK("gm_solve");
    multi_axpy(c, Vk(0), fe, kmax, xc, rows, N, dtype, st.y, 1.0);
  }
  if (iters) {
    MRHS_CUDA(cudaMemcpyAsync(iters, st.its, sizeof(int) * N, cudaMemcpyDeviceToHost, c->stream));
    MRHS_CUDA(cudaStreamSynchronize(c->stream));
  }
  check_tc_timeout(c);
}

}  // namespace mrhs

using namespace mrhs;

extern "C" {

int mrhs_build_Dc(mrhs_ctx c) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c, MRHS_ERR_ARG, "null context");
    build_Dc(c);
  });
}

int mrhs_set_dc_engine(mrhs_ctx c, int engine) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c, MRHS_ERR_ARG, "null context");
    MRHS_REQUIRE(engine >= MRHS_DC_AUTO && engine <= MRHS_DC_TC_TF32X3, MRHS_ERR_ARG, "unknown D_c engine");
    c->dc_engine = engine;
  });
}

int mrhs_restrict(mrhs_ctx c, const void* v, void* vc, int nrhs, int dtype) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && v && vc, MRHS_ERR_ARG, "null argument");
    require_dev(c, v, "mrhs_restrict v");
    require_dev(c, vc, "mrhs_restrict vc");
    restrict_(c, v, vc, nrhs, dtype);
  });
}

int mrhs_prolong(mrhs_ctx c, const void* uc, void* u, int nrhs, int dtype) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && uc && u, MRHS_ERR_ARG, "null argument");
    require_dev(c, uc, "mrhs_prolong uc");
    require_dev(c, u, "mrhs_prolong u");
    prolong(c, uc, u, nrhs, dtype);
  });
}

int mrhs_apply_Dc(mrhs_ctx c, const void* xc, void* yc, int nrhs, int dtype) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && xc && yc, MRHS_ERR_ARG, "null argument");
    require_dev(c, xc, "mrhs_apply_Dc xc");
    require_dev(c, yc, "mrhs_apply_Dc yc");
    MRHS_REQUIRE(nrhs >= 1, MRHS_ERR_ARG, "nrhs must be >= 1");
    apply_Dc(c, xc, yc, nrhs, dtype);
  });
}

int mrhs_set_coarse_solver(mrhs_ctx c, int even_odd) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c, MRHS_ERR_ARG, "null context");
    MRHS_REQUIRE(even_odd == 0 || even_odd == 1, MRHS_ERR_ARG, "even_odd must be 0 or 1");
    c->coarse_eo = even_odd;
  });
}

int mrhs_coarse_solve(mrhs_ctx c, const void* bc, void* xc, int nrhs, int dtype, double tol, int restart, int maxit,
                      int* iters) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && bc && xc, MRHS_ERR_ARG, "null argument");
    require_dev(c, bc, "mrhs_coarse_solve bc");
    require_dev(c, xc, "mrhs_coarse_solve xc");
    coarse_solve(c, bc, xc, nrhs, dtype, tol, restart, maxit, iters);
  });
}

}  // extern "C"
