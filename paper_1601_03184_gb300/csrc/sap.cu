// SAP colour phase (the smoother of Sec. 2 of the paper) with the Schwarz
// domain held on chip (FP32 work fields).
//
// One CTA per domain of the colour being updated. The domain's links and
// clover blocks are staged once in shared memory (structure-of-arrays over the
// domain's sites, padded against bank conflicts); the right-hand sides are
// processed in chunks of G. Per chunk:
//   1. x of the chunk is staged in shared memory and kept in registers,
//   2. r = b - D x on the domain (neighbours in other domains read from
//      global memory: they belong to the other colour and do not change),
//   3. n_mr minimal-residual steps on D_B e = r entirely on chip:
//      q = D_B rho, alpha = <q,rho>/<q,q> (block reduction in double),
//      x += alpha rho, rho -= alpha q,
//   4. x is written back.
// Only b and x of the colour's sites (and the face neighbours of x) touch HBM.
#include <cstdlib>

#include "stencil.cuh"

namespace mrhs {
namespace {

constexpr int kMaxVa = 256;

struct SapSmem {
  float* U;   // [4*9*2][LS]
  float* A;   // [72][LS]
  float* R;   // [12*2][Va][G]
  double* red;
  int LS;
};

template <int G>
__device__ __forceinline__ void load_rho(cx<float> psi[G][12], const float* sR, int Va, int n) {
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    if (G == 2) {
      float2 re = *reinterpret_cast<const float2*>(sR + ((size_t)(c * 2 + 0) * Va + n) * 2);
      float2 im = *reinterpret_cast<const float2*>(sR + ((size_t)(c * 2 + 1) * Va + n) * 2);
      psi[0][c] = mk(re.x, im.x);
      psi[G - 1][c] = mk(re.y, im.y);
    } else {
#pragma unroll
      for (int g = 0; g < G; ++g)
        psi[g][c] = mk(sR[((size_t)(c * 2 + 0) * Va + n) * G + g], sR[((size_t)(c * 2 + 1) * Va + n) * G + g]);
    }
  }
}

template <int G>
__device__ __forceinline__ void store_rho(const cx<float> v[G][12], float* sR, int Va, int n) {
#pragma unroll
  for (int c = 0; c < 12; ++c)
#pragma unroll
    for (int g = 0; g < G; ++g) {
      sR[((size_t)(c * 2 + 0) * Va + n) * G + g] = v[g][c].re;
      sR[((size_t)(c * 2 + 1) * Va + n) * G + g] = v[g][c].im;
    }
}

__device__ __forceinline__ void link_smem(cx<float> u[3][3], const float* sU, int LS, int l, int mu) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      int e = (mu * 9 + a * 3 + b) * 2;
      u[a][b] = mk(sU[e * LS + l], sU[(e + 1) * LS + l]);
    }
}

__device__ __forceinline__ void link_global(cx<float> u[3][3], const float* U, size_t n, int mu) {
  const float2* p = reinterpret_cast<const float2*>(U + (n * 4 + mu) * 18);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      float2 v = p[a * 3 + b];
      u[a][b] = mk(v.x, v.y);
    }
}

// out = A(l) psi for G right-hand sides, clover from shared memory
template <int G>
__device__ __forceinline__ void clover_smem(cx<float> out[G][12], const cx<float> psi[G][12], const float* sA, int LS,
                                            int l) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float q[36];
#pragma unroll
    for (int k = 0; k < 36; ++k) q[k] = sA[(h * 36 + k) * LS + l];
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        cx<float> acc = scale(psi[g][6 * h + a], q[a]);
#pragma unroll
        for (int b = 0; b < 6; ++b) {
          if (b == a) continue;
          cx<float> m = b > a ? mk(q[herm_idx(a, b)], q[herm_idx(a, b) + 1]) : mk(q[herm_idx(b, a)], -q[herm_idx(b, a) + 1]);
          fma_(acc, m, psi[g][6 * h + b]);
        }
        out[g][6 * h + a] = acc;
      }
  }
}

// one hop direction for G right-hand sides; neighbour spinor and link supplied
template <int MU, int DIR, int G>
__device__ __forceinline__ void hop_g(cx<float> out[G][12], const cx<float> psi[G][12], const cx<float> u[3][3], float sg) {
#pragma unroll
  for (int g = 0; g < G; ++g) hop_reg_u<MU, DIR, float>(out[g], psi[g], u, sg);
}

// D (or D_B) applied at local site l for the staged chunk. RESID: neighbours
// outside the domain are read from global x (columns r0..r0+G-1) and their
// links from global U; otherwise (MR) they are skipped (Dirichlet).
template <int G, bool RESID>
__device__ __forceinline__ void apply_local(cx<float> out[G][12], const SapSmem& sm, int Va, int l, int s, int blk,
                                            const int* nbr, const float* x, const float* U, int N, int r0) {
  cx<float> psi[G][12];
  load_rho<G>(psi, sm.R, Va, l);
  clover_smem<G>(out, psi, sm.A, sm.LS, l);
#define MRHS_SAP_HOP(MU)                                                                                   \
  {                                                                                                        \
    _Pragma("unroll") for (int d = 0; d < 2; ++d) {                                                        \
      int e = nbr[(size_t)s * 8 + d * 4 + MU];                                                             \
      int n = e & 0x3fffffff;                                                                              \
      float sg = (e & 0x40000000) ? -1.f : 1.f;                                                            \
      bool inside = n / Va == blk;                                                                         \
      if (inside || RESID) {                                                                               \
        cx<float> u[3][3];                                                                                 \
        if (inside) {                                                                                      \
          load_rho<G>(psi, sm.R, Va, n - blk * Va);                                                        \
          link_smem(u, sm.U, sm.LS, d == 0 ? l : n - blk * Va, MU);                                        \
        } else {                                                                                           \
          _Pragma("unroll") for (int c = 0; c < 12; ++c)                                                   \
          _Pragma("unroll") for (int g = 0; g < G; ++g)                                                    \
            psi[g][c] = mk(x[(((size_t)n * 12 + c) * 2 + 0) * N + r0 + g],                                 \
                           x[(((size_t)n * 12 + c) * 2 + 1) * N + r0 + g]);                                \
          if (d == 0) link_smem(u, sm.U, sm.LS, l, MU);                                                    \
          else link_global(u, U, (size_t)n, MU);                                                           \
        }                                                                                                  \
        if (d == 0) hop_g<MU, +1, G>(out, psi, u, sg);                                                     \
        else hop_g<MU, -1, G>(out, psi, u, sg);                                                            \
      }                                                                                                    \
    }                                                                                                      \
  }
  MRHS_SAP_HOP(0)
  MRHS_SAP_HOP(1)
  MRHS_SAP_HOP(2)
  MRHS_SAP_HOP(3)
#undef MRHS_SAP_HOP
}

// Block-wide sums of NV per-thread partials, fixed order: warp sums in FP32
// (each thread's partial already covers 12 components), the cross-warp sum in
// double by one thread per value. FP64 is slow on this GPU, so no thread does
// more than a handful of double operations. Result in red[0..NV).
template <int NV>
__device__ __forceinline__ void block_sum(float v[NV], double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[NV + w * NV + k] = (double)v[k];
  __syncthreads();
  if (threadIdx.x < NV) {
    double a = 0;
    for (int i = 0; i < nw; ++i) a += red[NV + i * NV + threadIdx.x];
    red[threadIdx.x] = a;
  }
  __syncthreads();
}

template <class SB, int G>
__global__ void k_sap_fused(const SB* __restrict__ b, float* x, const float* __restrict__ U,
                            const float* __restrict__ Acl, const int* __restrict__ nbr, int N, int Va,
                            const int* __restrict__ blist, int n_mr) {
  extern __shared__ double smem_d[];
  SapSmem sm;
  sm.LS = Va + 1;
  sm.U = (float*)smem_d;
  sm.A = sm.U + 72 * sm.LS;
  sm.R = sm.A + 72 * sm.LS;
  sm.red = (double*)(sm.R + ((24 * Va * G + 1) & ~1));
  const int blk = blist[blockIdx.x];
  const int l = threadIdx.x;
  const bool act = l < Va;
  const int s = blk * Va + l;
  // links and clover of the domain: coalesced global reads, SoA in shared memory
  for (int i = threadIdx.x; i < Va * 72; i += blockDim.x) {
    int ls = i / 72, e = i % 72;
    sm.U[e * sm.LS + ls] = U[(size_t)blk * Va * 72 + i];
    sm.A[e * sm.LS + ls] = Acl[(size_t)blk * Va * 72 + i];
  }
  __syncthreads();
  for (int r0 = 0; r0 < N; r0 += G) {
    cx<float> xr[G][12];
    if (act) {
#pragma unroll
      for (int c = 0; c < 12; ++c)
#pragma unroll
        for (int g = 0; g < G; ++g)
          xr[g][c] = mk(x[(((size_t)s * 12 + c) * 2 + 0) * N + r0 + g], x[(((size_t)s * 12 + c) * 2 + 1) * N + r0 + g]);
      store_rho<G>(xr, sm.R, Va, l);
    }
    __syncthreads();
    // r = b - D x on the domain
    cx<float> q[G][12];
    if (act) {
      apply_local<G, true>(q, sm, Va, l, s, blk, nbr, x, U, N, r0);
#pragma unroll
      for (int c = 0; c < 12; ++c)
#pragma unroll
        for (int g = 0; g < G; ++g) {
          cx<float> bv = mk((float)to_r(b[(((size_t)s * 12 + c) * 2 + 0) * N + r0 + g]),
                            (float)to_r(b[(((size_t)s * 12 + c) * 2 + 1) * N + r0 + g]));
          q[g][c] = bv - q[g][c];
        }
    }
    __syncthreads();
    if (act) store_rho<G>(q, sm.R, Va, l);
    __syncthreads();
    float* salpha = (float*)(sm.red + 3 * G + (blockDim.x >> 5) * 3 * G);  // [G][2]
    for (int it = 0; it < n_mr; ++it) {
      float v[3 * G];
#pragma unroll
      for (int k = 0; k < 3 * G; ++k) v[k] = 0;
      if (act) {
        apply_local<G, false>(q, sm, Va, l, s, blk, nbr, x, U, N, r0);
        cx<float> rho[G][12];
        load_rho<G>(rho, sm.R, Va, l);
#pragma unroll
        for (int g = 0; g < G; ++g) {
          float pr = 0, pi = 0, pq = 0;
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            pr = fmaf(q[g][c].re, rho[g][c].re, fmaf(q[g][c].im, rho[g][c].im, pr));
            pi = fmaf(q[g][c].re, rho[g][c].im, fmaf(-q[g][c].im, rho[g][c].re, pi));
            pq = fmaf(q[g][c].re, q[g][c].re, fmaf(q[g][c].im, q[g][c].im, pq));
          }
          v[3 * g] = pr;
          v[3 * g + 1] = pi;
          v[3 * g + 2] = pq;
        }
      }
      block_sum<3 * G>(v, sm.red);  // contains the barrier after all reads of rho
      if (threadIdx.x < G) {
        const int g = threadIdx.x;
        double qq = sm.red[3 * g + 2];
        salpha[2 * g] = qq > 0 ? (float)(sm.red[3 * g] / qq) : 0.f;
        salpha[2 * g + 1] = qq > 0 ? (float)(sm.red[3 * g + 1] / qq) : 0.f;
      }
      __syncthreads();
      if (act) {
        cx<float> rho[G][12];
        load_rho<G>(rho, sm.R, Va, l);
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const cx<float> al = mk(salpha[2 * g], salpha[2 * g + 1]);
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            fma_(xr[g][c], al, rho[g][c]);
            cx<float> t = mk(-q[g][c].re, -q[g][c].im);
            fma_(rho[g][c], al, t);
          }
        }
        store_rho<G>(rho, sm.R, Va, l);
      }
      __syncthreads();
    }
    if (act) {
#pragma unroll
      for (int c = 0; c < 12; ++c)
#pragma unroll
        for (int g = 0; g < G; ++g) {
          x[(((size_t)s * 12 + c) * 2 + 0) * N + r0 + g] = xr[g][c].re;
          x[(((size_t)s * 12 + c) * 2 + 1) * N + r0 + g] = xr[g][c].im;
        }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// 8-RHS form (N % 8 == 0): one chunk of 8 right-hand sides is exactly one
// 32-byte sector of every spin-colour row, so every global access of x, b and
// q moves whole sectors. rho of the chunk lives in shared memory (all Va sites);
// q and x are updated in place in global memory (the chunk of one domain stays
// in L2 while its CTA runs); links and clover come through L1, shared by the 8
// threads of a site. Items (site l, rhs g) = 8*l + g; a thread keeps one g.
constexpr int kG8 = 8;
constexpr int kThreads8 = 512;

__device__ __forceinline__ void load_rho8(cx<float> psi[12], const float* sR, int Va, int n, int g) {
#pragma unroll
  for (int c = 0; c < 12; ++c)
    psi[c] = mk(sR[((size_t)(c * 2 + 0) * Va + n) * kG8 + g], sR[((size_t)(c * 2 + 1) * Va + n) * kG8 + g]);
}

__device__ __forceinline__ size_t gidx(size_t s, int c, int reim, int N, int r) {
  return ((s * 12 + c) * 2 + reim) * (size_t)N + r;
}

// D (RESID: all hops; neighbours outside the domain from global x) or D_B at
// site l of the domain for right-hand side g of the chunk starting at r0
template <bool RESID>
__device__ __forceinline__ void apply8(cx<float> out[12], const float* sR, int Va, int l, int s, int blk, int g,
                                       const int* __restrict__ nbr, const float* x, const float* __restrict__ U,
                                       const float* __restrict__ Acl, int N, int r0) {
  cx<float> psi[12];
  load_rho8(psi, sR, Va, l, g);
  clover_apply_reg<float>(out, psi, Acl + (size_t)s * 72);
  const cx<float>* Uc = reinterpret_cast<const cx<float>*>(U);
#pragma unroll 1
  for (int d = 0; d < 2; ++d) {
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int e = nbr[(size_t)s * 8 + d * 4 + mu];
      const int n = e & 0x3fffffff;
      const float sg = (e & 0x40000000) ? -1.f : 1.f;
      const bool inside = n / Va == blk;
      if (!inside && !RESID) continue;
      if (inside) {
        load_rho8(psi, sR, Va, n - blk * Va, g);
      } else {
#pragma unroll
        for (int c = 0; c < 12; ++c) psi[c] = mk(x[gidx(n, c, 0, N, r0 + g)], x[gidx(n, c, 1, N, r0 + g)]);
      }
      const cx<float>* Ul = d == 0 ? Uc + (size_t)s * 36 + mu * 9 : Uc + (size_t)n * 36 + mu * 9;
      if (d == 0) {
        switch (mu) {
          case 0: hop_reg<0, +1, float>(out, psi, Ul, sg); break;
          case 1: hop_reg<1, +1, float>(out, psi, Ul, sg); break;
          case 2: hop_reg<2, +1, float>(out, psi, Ul, sg); break;
          default: hop_reg<3, +1, float>(out, psi, Ul, sg); break;
        }
      } else {
        switch (mu) {
          case 0: hop_reg<0, -1, float>(out, psi, Ul, sg); break;
          case 1: hop_reg<1, -1, float>(out, psi, Ul, sg); break;
          case 2: hop_reg<2, -1, float>(out, psi, Ul, sg); break;
          default: hop_reg<3, -1, float>(out, psi, Ul, sg); break;
        }
      }
    }
  }
}

template <class SB>
__global__ void __launch_bounds__(kThreads8) k_sap_fused8(const SB* __restrict__ b, float* x, float* qbuf,
                                                          const float* __restrict__ U, const float* __restrict__ Acl,
                                                          const int* __restrict__ nbr, int N, int Va,
                                                          const int* __restrict__ blist, int n_mr) {
  extern __shared__ double smem_d[];
  float* sR = (float*)smem_d;                                  // [12][2][Va][8]
  float* sred = sR + (size_t)24 * Va * kG8;                    // [warps][8][3]
  double* salpha_d = (double*)(sred + (kThreads8 / 32) * kG8 * 3 + 8);
  float* salpha = (float*)(salpha_d + 0);                      // [8][2]
  const int blk = blist[blockIdx.x];
  const int g = threadIdx.x % kG8;
  const int items = Va * kG8;
  float* q = qbuf + (size_t)blockIdx.x * Va * 24 * kG8;        // this CTA's q: [Va][12][2][8]
  for (int r0 = 0; r0 < N; r0 += kG8) {
    // stage x of the chunk
    for (int it = threadIdx.x; it < items; it += kThreads8) {
      const int l = it / kG8;
      const size_t s = (size_t)blk * Va + l;
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        sR[((size_t)(c * 2 + 0) * Va + l) * kG8 + g] = x[gidx(s, c, 0, N, r0 + g)];
        sR[((size_t)(c * 2 + 1) * Va + l) * kG8 + g] = x[gidx(s, c, 1, N, r0 + g)];
      }
    }
    __syncthreads();
    // r = b - D x into q (global), then into shared memory
    for (int it = threadIdx.x; it < items; it += kThreads8) {
      const int l = it / kG8;
      const int s = blk * Va + l;
      cx<float> out[12];
      apply8<true>(out, sR, Va, l, s, blk, g, nbr, x, U, Acl, N, r0);
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        q[((size_t)l * 24 + c * 2 + 0) * kG8 + g] = (float)to_r(b[gidx(s, c, 0, N, r0 + g)]) - out[c].re;
        q[((size_t)l * 24 + c * 2 + 1) * kG8 + g] = (float)to_r(b[gidx(s, c, 1, N, r0 + g)]) - out[c].im;
      }
    }
    __syncthreads();
    for (int it = threadIdx.x; it < items; it += kThreads8) {
      const int l = it / kG8;
#pragma unroll
      for (int k = 0; k < 24; ++k) sR[((size_t)k * Va + l) * kG8 + g] = q[((size_t)l * 24 + k) * kG8 + g];
    }
    __syncthreads();
    for (int step = 0; step < n_mr; ++step) {
      float pr = 0, pi = 0, pq = 0;
      for (int it = threadIdx.x; it < items; it += kThreads8) {
        const int l = it / kG8;
        const int s = blk * Va + l;
        cx<float> out[12], rho[12];
        apply8<false>(out, sR, Va, l, s, blk, g, nbr, x, U, Acl, N, r0);
        load_rho8(rho, sR, Va, l, g);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          q[((size_t)l * 24 + c * 2 + 0) * kG8 + g] = out[c].re;
          q[((size_t)l * 24 + c * 2 + 1) * kG8 + g] = out[c].im;
          pr = fmaf(out[c].re, rho[c].re, fmaf(out[c].im, rho[c].im, pr));
          pi = fmaf(out[c].re, rho[c].im, fmaf(-out[c].im, rho[c].re, pi));
          pq = fmaf(out[c].re, out[c].re, fmaf(out[c].im, out[c].im, pq));
        }
      }
      // sums over the lanes that share g (lane % 8 == g), then over warps
#pragma unroll
      for (int o = 8; o < 32; o <<= 1) {
        pr += __shfl_xor_sync(0xffffffffu, pr, o);
        pi += __shfl_xor_sync(0xffffffffu, pi, o);
        pq += __shfl_xor_sync(0xffffffffu, pq, o);
      }
      const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
      if (lane < kG8) {
        sred[(w * kG8 + lane) * 3 + 0] = pr;
        sred[(w * kG8 + lane) * 3 + 1] = pi;
        sred[(w * kG8 + lane) * 3 + 2] = pq;
      }
      __syncthreads();
      if (threadIdx.x < kG8) {
        double a = 0, bb = 0, cc = 0;
        for (int i = 0; i < kThreads8 / 32; ++i) {
          a += sred[(i * kG8 + threadIdx.x) * 3 + 0];
          bb += sred[(i * kG8 + threadIdx.x) * 3 + 1];
          cc += sred[(i * kG8 + threadIdx.x) * 3 + 2];
        }
        salpha[2 * threadIdx.x] = cc > 0 ? (float)(a / cc) : 0.f;
        salpha[2 * threadIdx.x + 1] = cc > 0 ? (float)(bb / cc) : 0.f;
      }
      __syncthreads();
      const cx<float> al = mk(salpha[2 * g], salpha[2 * g + 1]);
      for (int it = threadIdx.x; it < items; it += kThreads8) {
        const int l = it / kG8;
        const size_t s = (size_t)blk * Va + l;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          const size_t i0 = ((size_t)(c * 2 + 0) * Va + l) * kG8 + g, i1 = ((size_t)(c * 2 + 1) * Va + l) * kG8 + g;
          cx<float> rv = mk(sR[i0], sR[i1]);
          cx<float> qv = mk(q[((size_t)l * 24 + c * 2 + 0) * kG8 + g], q[((size_t)l * 24 + c * 2 + 1) * kG8 + g]);
          const size_t x0 = gidx(s, c, 0, N, r0 + g), x1 = gidx(s, c, 1, N, r0 + g);
          cx<float> xv = mk(x[x0], x[x1]);
          fma_(xv, al, rv);
          x[x0] = xv.re;
          x[x1] = xv.im;
          cx<float> t = mk(-qv.re, -qv.im);
          fma_(rv, al, t);
          sR[i0] = rv.re;
          sR[i1] = rv.im;
        }
      }
      __syncthreads();
    }
  }
}

template <class SB>
void launch_fused8(mrhs_ctx c, const SB* b, float* x, int N, int colour, int n_mr) {
  const int Va = c->g.Va;
  size_t smem = sizeof(float) * ((size_t)24 * Va * kG8 + (kThreads8 / 32) * kG8 * 3 + 8) + sizeof(float) * 2 * kG8 + 16;
  auto kern = k_sap_fused8<SB>;
  MRHS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int nblk = c->ncol[colour];
  float* qbuf = (float*)scratch(c, SC_Q, sizeof(float) * (size_t)nblk * Va * 24 * kG8);
  const int* blist = c->blocks_col + (colour ? c->ncol[0] : 0);
  Prof pr(c, "sap_fused8");
  kern<<<nblk, kThreads8, smem, c->stream>>>(b, x, qbuf, c->U32, c->A32, c->nbr, N, Va, blist, n_mr);
  MRHS_LAUNCH_CHECK("sap_fused8");
}

template <class SB, int G>
void launch_fused(mrhs_ctx c, const SB* b, float* x, int N, int colour, int n_mr) {
  const int Va = c->g.Va;
  const int threads = (Va + 31) / 32 * 32;
  const int LS = Va + 1;
  size_t smem = sizeof(float) * (144 * (size_t)LS + ((24 * (size_t)Va * G + 1) & ~(size_t)1)) +
                sizeof(double) * (3 * G + (threads / 32) * 3 * G) + sizeof(float) * 2 * G;
  auto kern = k_sap_fused<SB, G>;
  MRHS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int* blist = c->blocks_col + (colour ? c->ncol[0] : 0);
  Prof pr(c, "sap_fused");
  kern<<<c->ncol[colour], threads, smem, c->stream>>>(b, x, c->U32, c->A32, c->nbr, N, Va, blist, n_mr);
  MRHS_LAUNCH_CHECK("sap_fused");
}

}  // namespace

// The on-chip SAP needs FP32 work fields and a domain of at most 256 sites
// whose links, clover and a 2-RHS chunk fit in shared memory.
bool sap_fused_ok(mrhs_ctx c, int dtype) {
  if (dtype != MRHS_F32 || c->g.Va > kMaxVa) return false;
  int maxsm = 0;
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  size_t need = sizeof(float) * (144 * (size_t)(c->g.Va + 1) + 48 * (size_t)c->g.Va + 2) + sizeof(double) * 64;
  return need <= (size_t)maxsm;
}

void sap_fused(mrhs_ctx c, const void* b, int bdtype, void* x, int nrhs, int n_sweeps, int n_mr, bool x0_zero) {
  // the on-chip forms (tensor memory for the running solution): packed pairs
  // of right-hand sides per thread when nrhs % 4 == 0, else one (site, rhs)
  // item per thread; MRHS_SAP_KERNEL=tm asks for the item form always,
  // MRHS_SAP_KERNEL=smem for the shared-memory/global forms below
  static const int mode = [] {
    const char* e = std::getenv("MRHS_SAP_KERNEL");
    if (!e) return 0;
    return std::string(e) == "smem" ? 2 : std::string(e) == "tm" ? 1 : 0;
  }();
  const bool tm_off = mode == 2;
  if (mode == 0 && sap_pk_ok(c, nrhs)) {
    sap_pk(c, b, bdtype, x, nrhs, n_sweeps, n_mr, x0_zero);
    return;
  }
  if (!tm_off && sap_tm_ok(c, nrhs)) {
    sap_tm(c, b, bdtype, x, nrhs, n_sweeps, n_mr);
    return;
  }
  const bool g8 = nrhs % kG8 == 0 &&
                  sizeof(float) * ((size_t)24 * c->g.Va * kG8 + 1024) <= (size_t)[&] {
                    int m = 0;
                    cudaDeviceGetAttribute(&m, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
                    return m;
                  }();
  for (int sw = 0; sw < n_sweeps; ++sw)
    for (int col = 0; col < 2; ++col) {
      if (g8) {
        MRHS_DISPATCH(bdtype, SB, (launch_fused8<SB>(c, (const SB*)b, (float*)x, nrhs, col, n_mr)));
      } else if (nrhs % 2 == 0) {
        MRHS_DISPATCH(bdtype, SB, (launch_fused<SB, 2>(c, (const SB*)b, (float*)x, nrhs, col, n_mr)));
      } else {
        MRHS_DISPATCH(bdtype, SB, (launch_fused<SB, 1>(c, (const SB*)b, (float*)x, nrhs, col, n_mr)));
      }
    }
}

}  // namespace mrhs
