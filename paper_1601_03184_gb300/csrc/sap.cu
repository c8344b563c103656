// SAP colour phase with the Schwarz domain held on chip (FP32 work fields).
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

// block-wide sum of NV doubles per thread, fixed order; result in red[0..NV)
template <int NV>
__device__ __forceinline__ void block_sum(double v[NV], double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[NV + w * NV + k] = v[k];
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
    for (int it = 0; it < n_mr; ++it) {
      double v[3 * G];
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
      if (act) {
        cx<float> rho[G][12];
        load_rho<G>(rho, sm.R, Va, l);
#pragma unroll
        for (int g = 0; g < G; ++g) {
          double qq = sm.red[3 * g + 2];
          cx<float> al = qq > 0 ? mk((float)(sm.red[3 * g] / qq), (float)(sm.red[3 * g + 1] / qq)) : mk(0.f, 0.f);
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

template <class SB, int G>
void launch_fused(mrhs_ctx c, const SB* b, float* x, int N, int colour, int n_mr) {
  const int Va = c->g.Va;
  const int threads = (Va + 31) / 32 * 32;
  const int LS = Va + 1;
  size_t smem = sizeof(float) * (144 * (size_t)LS + ((24 * (size_t)Va * G + 1) & ~(size_t)1)) +
                sizeof(double) * (3 * G + (threads / 32) * 3 * G);
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

void sap_fused(mrhs_ctx c, const void* b, int bdtype, void* x, int nrhs, int n_sweeps, int n_mr) {
  for (int sw = 0; sw < n_sweeps; ++sw)
    for (int col = 0; col < 2; ++col) {
      if (nrhs % 2 == 0) {
        MRHS_DISPATCH(bdtype, SB, (launch_fused<SB, 2>(c, (const SB*)b, (float*)x, nrhs, col, n_mr)));
      } else {
        MRHS_DISPATCH(bdtype, SB, (launch_fused<SB, 1>(c, (const SB*)b, (float*)x, nrhs, col, n_mr)));
      }
    }
}

}  // namespace mrhs
