// SAP sweep (Sec. 2 of the paper; red-black multiplicative Schwarz with
// minimal-residual block solves) with the whole state of a domain on chip.
//
// Per colour, one CTA per (domain, chunk of G right-hand sides): the CTAs of a
// domain run side by side, so each 32-byte sector of x and b that they share
// comes from HBM once. Per chunk:
//   shared memory  rho [24][Va][G] (the block residual of the MR iteration)
//                  and the domain's links (1/2) sgn U [4][5][Va+1] float4
//                  (G = 2 also the clover [18][Va+1] float4 and the
//                  domain-local neighbour table);
//   tensor memory  the running solution x_B = x0 + sum_k alpha_k rho_k of the
//                  thread's own items (tcgen05.st / tcgen05.ld, 24 columns per
//                  item), so x is read once and written once per chunk;
//   registers      q = D_B rho of the thread's items between the reduction
//                  for alpha and the update.
// Items (site l, rhs g) = G*l + g. Per colour: r = b - D x on the domain
// (neighbours outside it from x in global memory, which the other colour owns
// and nobody writes during the launch), then n_mr MR steps e += alpha rho,
// rho -= alpha q with alpha = <q, rho> / <q, q>, then x_B += e.
#include <algorithm>
#include <cstdlib>

#include "stencil.cuh"
#include "tc.cuh"

namespace mrhs {
namespace {

constexpr int kG = 4;            // right-hand sides per chunk
constexpr int kMaxT = 512;       // threads for a 256-site domain
constexpr int kColsItem = 24;    // tensor-memory columns per item

// one hop for one right-hand side: pr/pi the neighbour spinor, u the halved
// link (9 complex, row-major, sign of the time boundary folded in)
template <int MU, int DIR>
__device__ __forceinline__ void hop1(float ore[12], float oim[12], const float pr[12], const float pi[12],
                                     const float u[18]) {
  float hre[2][3], him[2][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cx<float> p2 = mk(pr[6 + c], pi[6 + c]), p3 = mk(pr[9 + c], pi[9 + c]);
    cx<float> b0, b1;
    b_low<MU>(p2, p3, b0, b1);
    cx<float> h0 = DIR > 0 ? mk(pr[c], pi[c]) - b0 : mk(pr[c], pi[c]) + b0;
    cx<float> h1 = DIR > 0 ? mk(pr[3 + c], pi[3 + c]) - b1 : mk(pr[3 + c], pi[3 + c]) + b1;
    hre[0][c] = h0.re;
    him[0][c] = h0.im;
    hre[1][c] = h1.re;
    him[1][c] = h1.im;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cx<float> ch[2];
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      cx<float> acc = mk(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        cx<float> hv = mk(hre[sp][b], him[sp][b]);
        if (DIR > 0) fma_(acc, mk(u[2 * (a * 3 + b)], u[2 * (a * 3 + b) + 1]), hv);
        else fmac_(acc, mk(u[2 * (b * 3 + a)], u[2 * (b * 3 + a) + 1]), hv);
      }
      ch[sp] = acc;
    }
    cx<float> l0, l1;
    bdag<MU>(ch[0], ch[1], l0, l1);
    ore[a] -= ch[0].re;
    oim[a] -= ch[0].im;
    ore[3 + a] -= ch[1].re;
    oim[3 + a] -= ch[1].im;
    if (DIR > 0) {
      ore[6 + a] += l0.re;
      oim[6 + a] += l0.im;
      ore[9 + a] += l1.re;
      oim[9 + a] += l1.im;
    } else {
      ore[6 + a] -= l0.re;
      oim[6 + a] -= l0.im;
      ore[9 + a] -= l1.re;
      oim[9 + a] -= l1.im;
    }
  }
}

struct Dom {
  const float2* sR;  // [12][Va][4] (re, im)
  const float4* sU;  // [20][Va+1]
  const int* sN;     // [8][Va]: neighbour inside the domain (local index) or ~(device site) outside
  int Va, l, g;
  size_t s0;         // first device site of the domain
};

__device__ __forceinline__ void load_rho(const Dom& d, int n, float pr[12], float pi[12]) {
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const float2 v = d.sR[(c * d.Va + n) * kG + d.g];
    pr[c] = v.x;
    pi[c] = v.y;
  }
}

__device__ __forceinline__ void load_u_smem(const Dom& d, int site, int mu, float u[18]) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const float4 t = d.sU[(mu * 5 + k) * (d.Va + 1) + site];
    u[4 * k] = t.x;
    u[4 * k + 1] = t.y;
    if (4 * k + 2 < 18) u[4 * k + 2] = t.z;
    if (4 * k + 3 < 18) u[4 * k + 3] = t.w;
  }
}

__device__ __forceinline__ void load_u_glob(const float* __restrict__ U20, size_t site, int mu, float u[18]) {
  const float4* p = reinterpret_cast<const float4*>(U20 + (site * 4 + mu) * 20);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const float4 t = __ldg(p + k);
    u[4 * k] = t.x;
    u[4 * k + 1] = t.y;
    if (4 * k + 2 < 18) u[4 * k + 2] = t.z;
    if (4 * k + 3 < 18) u[4 * k + 3] = t.w;
  }
}

// hop (MU, DIR) at the item's site: inside the domain from shared memory;
// outside (RESID only) from x and the links in global memory
template <int MU, int DIR, bool RESID>
__device__ __forceinline__ void hop_dom(const Dom& d, float ore[12], float oim[12], const float* __restrict__ x,
                                        const float* __restrict__ U20, int N, int r0) {
  const int e = d.sN[((DIR > 0 ? 0 : 4) + MU) * d.Va + d.l];
  float pr[12], pi[12], u[18];
  if (e >= 0) {
    load_rho(d, e, pr, pi);
    load_u_smem(d, DIR > 0 ? d.l : e, MU, u);
  } else {
    if (!RESID) return;
    const size_t n = (size_t)(~e);
    const float* xn = x + n * 24 * N + r0 + d.g;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      pr[c] = xn[(2 * c) * N];
      pi[c] = xn[(2 * c + 1) * N];
    }
    if (DIR > 0) load_u_smem(d, d.l, MU, u);
    else load_u_glob(U20, n, MU, u);
  }
  hop1<MU, DIR>(ore, oim, pr, pi, u);
}

// out = D x (RESID) or D_B rho at the item's site
template <bool RESID>
__device__ __forceinline__ void apply_dom(const Dom& d, float ore[12], float oim[12], const float* __restrict__ Acl,
                                          const float* __restrict__ x, const float* __restrict__ U20, int N, int r0) {
  {
    float pr[12], pi[12];
    load_rho(d, d.l, pr, pi);
    const float4* A4 = reinterpret_cast<const float4*>(Acl + (d.s0 + d.l) * 72);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float q[36];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const float4 v = __ldg(A4 + 9 * h + k);
        q[4 * k] = v.x;
        q[4 * k + 1] = v.y;
        q[4 * k + 2] = v.z;
        q[4 * k + 3] = v.w;
      }
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        cx<float> acc = scale(mk(pr[6 * h + a], pi[6 * h + a]), q[a]);
#pragma unroll
        for (int b2 = 0; b2 < 6; ++b2) {
          if (b2 == a) continue;
          cx<float> m = b2 > a ? mk(q[herm_idx(a, b2)], q[herm_idx(a, b2) + 1])
                               : mk(q[herm_idx(b2, a)], -q[herm_idx(b2, a) + 1]);
          fma_(acc, m, mk(pr[6 * h + b2], pi[6 * h + b2]));
        }
        ore[6 * h + a] = acc.re;
        oim[6 * h + a] = acc.im;
      }
    }
  }
  hop_dom<0, +1, RESID>(d, ore, oim, x, U20, N, r0);
  hop_dom<1, +1, RESID>(d, ore, oim, x, U20, N, r0);
  hop_dom<2, +1, RESID>(d, ore, oim, x, U20, N, r0);
  hop_dom<3, +1, RESID>(d, ore, oim, x, U20, N, r0);
  hop_dom<0, -1, RESID>(d, ore, oim, x, U20, N, r0);
  hop_dom<1, -1, RESID>(d, ore, oim, x, U20, N, r0);
  hop_dom<2, -1, RESID>(d, ore, oim, x, U20, N, r0);
  hop_dom<3, -1, RESID>(d, ore, oim, x, U20, N, r0);
}

// four consecutive right-hand sides of one row of b (16-byte / 8-byte load)
__device__ __forceinline__ void ld4(const float* p, float v[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, float v[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = (float)p[i];
}
template <class H>
__device__ __forceinline__ void ld4(const H* p, float v[4]) {
  const uint2 t = *reinterpret_cast<const uint2*>(p);
  H h[4];
  *reinterpret_cast<uint2*>(h) = t;
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = (float)to_r(h[i]);
}

__device__ __forceinline__ void tm_put(uint32_t ta, const float v[24]) {
  tc::tmem_st8(ta, v);
  tc::tmem_st8(ta + 8, v + 8);
  tc::tmem_st8(ta + 16, v + 16);
}
__device__ __forceinline__ void tm_get(uint32_t ta, float v[24]) {
  tc::tmem_ld8(ta, v);
  tc::tmem_ld8(ta + 8, v + 8);
  tc::tmem_ld8(ta + 16, v + 16);
}

template <class SB>
__global__ void __launch_bounds__(kMaxT, 1) k_sap_tm(const SB* __restrict__ b, float* __restrict__ x,
                                                     const float* __restrict__ U20, const float* __restrict__ Acl,
                                                     const int* __restrict__ nbr, int N, int Va,
                                                     const int* __restrict__ blist, int n_mr, uint32_t tm_cols,
                                                     int cpb) {
  extern __shared__ float4 smem4[];
  const int T = blockDim.x;
  float4* sU = smem4;                                          // [20][Va+1]
  float* sR = reinterpret_cast<float*>(sU + 20 * (Va + 1));   // [12][Va][4] x (re, im)
  float2* sR2 = reinterpret_cast<float2*>(sR);
  float4* sred4 = reinterpret_cast<float4*>(sR + 24 * Va * kG);  // [T/32][4] (pr, pi, pq, -)
  int* sN = reinterpret_cast<int*>(sred4 + (T / 32) * kG);     // [8][Va]
  __shared__ uint32_t s_tmem;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nit = kG * Va;
  Dom d;
  d.Va = Va;
  d.g = tid & (kG - 1);
  d.s0 = (size_t)blist[blockIdx.x / cpb] * Va;
  d.sR = sR2;
  d.sU = sU;
  d.sN = sN;

  if (warp == 0) {
    tc::tmem_alloc(&s_tmem, tm_cols);
    tc::tmem_relinquish();
  }
  {
    const float4* U4 = reinterpret_cast<const float4*>(U20) + d.s0 * 20;
    for (int i = tid; i < 20 * Va; i += T) sU[(i % 20) * (Va + 1) + i / 20] = __ldg(U4 + i);
    for (int i = tid; i < 8 * Va; i += T) {
      const int l = i >> 3, k = i & 7;
      const int n = __ldg(nbr + (d.s0 + l) * 8 + k) & 0x3fffffff;
      const int nl = n - (int)d.s0;
      sN[k * Va + l] = (nl >= 0 && nl < Va) ? nl : ~n;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  // lane quarter of the warp; warps w, w+4, w+8, w+12 share it and take
  // disjoint column ranges: x_B of item 0, x_B of item 1, q of item 0
  const uint32_t tm = s_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * 3 * kColsItem);
  const uint32_t tmq = tm + 2 * kColsItem;

  for (int r0 = (blockIdx.x % cpb) * kG; r0 < N; r0 += cpb * kG) {
    // stage x0 into shared memory, one (component pair c, site l) per unit:
    // the real and the imaginary row of the chunk's four right-hand sides
    // (two 16-byte loads) become the four (re, im) pairs of [c][l][g]
    for (int u = tid; u < 12 * Va; u += T) {
      const int c = u / Va, l = u % Va;
      const float* xs = x + ((d.s0 + l) * 24 + 2 * c) * N + r0;
      const float4 re = *reinterpret_cast<const float4*>(xs);
      const float4 im = *reinterpret_cast<const float4*>(xs + N);
      float4* dst = reinterpret_cast<float4*>(sR2 + (c * Va + l) * kG);
      dst[0] = make_float4(re.x, im.x, re.y, im.y);
      dst[1] = make_float4(re.z, im.z, re.w, im.w);
    }
    __syncthreads();
    // the thread's items of x0 -> tensor memory (running solution)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int i = tid + j * T;
      float v[24];
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        const float2 t = i < nit ? sR2[(c * Va + (i >> 2)) * kG + d.g] : make_float2(0.f, 0.f);
        v[2 * c] = t.x;
        v[2 * c + 1] = t.y;
      }
      tm_put(tm + j * kColsItem, v);
    }
    tc::tmem_wait_st();
    // D x0 item by item; q of item 0 waits in tensor memory, q of item 1 in registers
    float qr[12], qi[12];
#pragma unroll 1
    for (int j = 0; j < 2; ++j) {
      const int i = tid + j * T;
      if (i < nit) {
        d.l = i >> 2;
        apply_dom<true>(d, qr, qi, Acl, x, U20, N, r0);
      }
      if (j == 0) {
        float v[24];
#pragma unroll
        for (int c = 0; c < 12; ++c) v[2 * c] = qr[c], v[2 * c + 1] = qi[c];
        tm_put(tmq, v);
      }
    }
    tc::tmem_wait_st();
    __syncthreads();
    // stage b the same way as x0, then rho = b - D x0 item by item
    for (int u = tid; u < 12 * Va; u += T) {
      const int c = u / Va, l = u % Va;
      const SB* bs = b + ((d.s0 + l) * 24 + 2 * c) * N + r0;
      float re[4], im[4];
      ld4(bs, re);
      ld4(bs + N, im);
      float4* dst = reinterpret_cast<float4*>(sR2 + (c * Va + l) * kG);
      dst[0] = make_float4(re[0], im[0], re[1], im[1]);
      dst[1] = make_float4(re[2], im[2], re[3], im[3]);
    }
    __syncthreads();
    {
      float q0[24];
      tm_get(tmq, q0);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int i = tid + j * T;
        if (i < nit) {
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            const int ix = (c * Va + (i >> 2)) * kG + d.g;
            const float2 bv = sR2[ix];
            sR2[ix] = j == 0 ? make_float2(bv.x - q0[2 * c], bv.y - q0[2 * c + 1])
                             : make_float2(bv.x - qr[c], bv.y - qi[c]);
          }
        }
      }
    }
    __syncthreads();
    for (int step = 0; step < n_mr; ++step) {
      float pr = 0.f, pi = 0.f, pq = 0.f;
#pragma unroll 1
      for (int j = 0; j < 2; ++j) {
        const int i = tid + j * T;
        if (i < nit) {
          d.l = i >> 2;
          apply_dom<false>(d, qr, qi, Acl, x, U20, N, r0);
          float rr[12], ri[12];
          load_rho(d, d.l, rr, ri);
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            pr = fmaf(qr[c], rr[c], fmaf(qi[c], ri[c], pr));
            pi = fmaf(qr[c], ri[c], fmaf(-qi[c], rr[c], pi));
            pq = fmaf(qr[c], qr[c], fmaf(qi[c], qi[c], pq));
          }
        }
        if (j == 0) {
          float v[24];
#pragma unroll
          for (int c = 0; c < 12; ++c) v[2 * c] = qr[c], v[2 * c + 1] = qi[c];
          tm_put(tmq, v);
        }
      }
      // sums over the lanes of the same rhs (lane % 4), then over warps:
      // every thread adds the per-warp partials of its rhs in the same order,
      // so all threads of one rhs hold the same alpha
#pragma unroll
      for (int o = kG; o < 32; o <<= 1) {
        pr += __shfl_xor_sync(0xffffffffu, pr, o);
        pi += __shfl_xor_sync(0xffffffffu, pi, o);
        pq += __shfl_xor_sync(0xffffffffu, pq, o);
      }
      if (lane < kG) sred4[warp * kG + lane] = make_float4(pr, pi, pq, 0.f);
      tc::tmem_wait_st();
      __syncthreads();
      float a = 0.f, bb = 0.f, cc = 0.f;
      for (int w = 0; w < T / 32; ++w) {
        const float4 t = sred4[w * kG + d.g];
        a += t.x;
        bb += t.y;
        cc += t.z;
      }
      const cx<float> al = cc > 0.f ? mk(a / cc, bb / cc) : mk(0.f, 0.f);
      // x_B += alpha rho (tensor memory), rho -= alpha q (shared memory)
      float q0[24];
      tm_get(tmq, q0);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        float xv[24];
        tm_get(tm + j * kColsItem, xv);
        const int i = tid + j * T;
        if (i < nit) {
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            const int i0 = (c * Va + (i >> 2)) * kG + d.g;
            const float2 r2 = sR2[i0];
            cx<float> rv = mk(r2.x, r2.y);
            cx<float> xc = mk(xv[2 * c], xv[2 * c + 1]);
            fma_(xc, al, rv);
            xv[2 * c] = xc.re;
            xv[2 * c + 1] = xc.im;
            const cx<float> qv = j == 0 ? mk(-q0[2 * c], -q0[2 * c + 1]) : mk(-qr[c], -qi[c]);
            fma_(rv, al, qv);
            sR2[i0] = make_float2(rv.re, rv.im);
          }
        }
        tm_put(tm + j * kColsItem, xv);
      }
      tc::tmem_wait_st();
      __syncthreads();
    }
    // x = x_B: items -> shared memory, then 16-byte rows back to x
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      float xv[24];
      tm_get(tm + j * kColsItem, xv);
      const int i = tid + j * T;
      if (i < nit) {
#pragma unroll
        for (int c = 0; c < 12; ++c) sR2[(c * Va + (i >> 2)) * kG + d.g] = make_float2(xv[2 * c], xv[2 * c + 1]);
      }
    }
    __syncthreads();
    for (int u = tid; u < 12 * Va; u += T) {
      const int c = u / Va, l = u % Va;
      float* xs = x + ((d.s0 + l) * 24 + 2 * c) * N + r0;
      const float4* src = reinterpret_cast<const float4*>(sR2 + (c * Va + l) * kG);
      const float4 p0 = src[0], p1 = src[1];
      *reinterpret_cast<float4*>(xs) = make_float4(p0.x, p0.z, p1.x, p1.z);
      *reinterpret_cast<float4*>(xs + N) = make_float4(p0.y, p0.w, p1.y, p1.w);
    }
    __syncthreads();
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(s_tmem, tm_cols);
}

// ---------------------------------------------------------------------------
// Two right-hand sides per chunk, every operand of the MR steps on chip:
// shared memory holds rho [24][Va][2], the halved links [20][Va+1] float4,
// the clover [18][Va+1] float4 and the domain-local neighbour table [8][Va]
// (-1 outside the domain); tensor memory the running solution (24 columns
// per thread); one item (site l = t/2, rhs g = t%2) per thread, q in
// registers. Only the residual reads global memory inside the chunk (b and
// the neighbours outside the domain).
constexpr int kG2 = 2;

struct Dom2 {
  const float* sR;   // [24][Va][2]
  const float4* sU;  // [20][Va+1]
  const float4* sA;  // [18][Va+1]
  const int* sN;     // [8][Va]
  int Va, l, g;
  size_t s0;
};

__device__ __forceinline__ void load_rho2(const Dom2& d, int n, float pr[12], float pi[12]) {
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    pr[c] = d.sR[((2 * c) * d.Va + n) * kG2 + d.g];
    pi[c] = d.sR[((2 * c + 1) * d.Va + n) * kG2 + d.g];
  }
}

__device__ __forceinline__ void load_u2(const Dom2& d, int site, int mu, float u[18]) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const float4 t = d.sU[(mu * 5 + k) * (d.Va + 1) + site];
    u[4 * k] = t.x;
    u[4 * k + 1] = t.y;
    if (4 * k + 2 < 18) u[4 * k + 2] = t.z;
    if (4 * k + 3 < 18) u[4 * k + 3] = t.w;
  }
}

template <int MU, int DIR, bool RESID>
__device__ __forceinline__ void hop_dom2(const Dom2& d, float ore[12], float oim[12], const int* __restrict__ nbr,
                                         const float* __restrict__ x, const float* __restrict__ U20, int N, int r0) {
  const int nl = d.sN[((DIR > 0 ? 0 : 4) + MU) * d.Va + d.l];
  float pr[12], pi[12], u[18];
  if (nl >= 0) {
    load_rho2(d, nl, pr, pi);
    load_u2(d, DIR > 0 ? d.l : nl, MU, u);
  } else {
    if (!RESID) return;
    const int n = __ldg(nbr + (d.s0 + d.l) * 8 + (DIR > 0 ? 0 : 4) + MU) & 0x3fffffff;
    const float* xn = x + (size_t)n * 24 * N + r0 + d.g;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      pr[c] = xn[(2 * c) * N];
      pi[c] = xn[(2 * c + 1) * N];
    }
    if (DIR > 0) load_u2(d, d.l, MU, u);
    else load_u_glob(U20, (size_t)n, MU, u);
  }
  hop1<MU, DIR>(ore, oim, pr, pi, u);
}

template <bool RESID>
__device__ __forceinline__ void apply_dom2(const Dom2& d, float ore[12], float oim[12], const int* __restrict__ nbr,
                                           const float* __restrict__ x, const float* __restrict__ U20, int N, int r0) {
  {
    float pr[12], pi[12];
    load_rho2(d, d.l, pr, pi);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float q[36];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const float4 v = d.sA[(9 * h + k) * (d.Va + 1) + d.l];
        q[4 * k] = v.x;
        q[4 * k + 1] = v.y;
        q[4 * k + 2] = v.z;
        q[4 * k + 3] = v.w;
      }
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        cx<float> acc = scale(mk(pr[6 * h + a], pi[6 * h + a]), q[a]);
#pragma unroll
        for (int b2 = 0; b2 < 6; ++b2) {
          if (b2 == a) continue;
          cx<float> m = b2 > a ? mk(q[herm_idx(a, b2)], q[herm_idx(a, b2) + 1])
                               : mk(q[herm_idx(b2, a)], -q[herm_idx(b2, a) + 1]);
          fma_(acc, m, mk(pr[6 * h + b2], pi[6 * h + b2]));
        }
        ore[6 * h + a] = acc.re;
        oim[6 * h + a] = acc.im;
      }
    }
  }
  hop_dom2<0, +1, RESID>(d, ore, oim, nbr, x, U20, N, r0);
  hop_dom2<1, +1, RESID>(d, ore, oim, nbr, x, U20, N, r0);
  hop_dom2<2, +1, RESID>(d, ore, oim, nbr, x, U20, N, r0);
  hop_dom2<3, +1, RESID>(d, ore, oim, nbr, x, U20, N, r0);
  hop_dom2<0, -1, RESID>(d, ore, oim, nbr, x, U20, N, r0);
  hop_dom2<1, -1, RESID>(d, ore, oim, nbr, x, U20, N, r0);
  hop_dom2<2, -1, RESID>(d, ore, oim, nbr, x, U20, N, r0);
  hop_dom2<3, -1, RESID>(d, ore, oim, nbr, x, U20, N, r0);
}

template <class SB>
__global__ void __launch_bounds__(kMaxT, 1) k_sap_tm2(const SB* __restrict__ b, float* __restrict__ x,
                                                      const float* __restrict__ U20, const float* __restrict__ Acl,
                                                      const int* __restrict__ nbr, int N, int Va,
                                                      const int* __restrict__ blist, int n_mr, uint32_t tm_cols,
                                                      int cpb) {
  extern __shared__ float4 smem4[];
  const int T = blockDim.x;
  float4* sU = smem4;                                      // [20][Va+1]
  float4* sA = sU + 20 * (Va + 1);                         // [18][Va+1]
  int* sN = reinterpret_cast<int*>(sA + 18 * (Va + 1));    // [8][Va]
  float* sR = reinterpret_cast<float*>(sN + 8 * Va);       // [24][Va][2]
  float* sred = sR + 24 * Va * kG2;                        // [T/32][2][3]
  float* salpha = sred + (T / 32) * kG2 * 3;               // [2][2]
  __shared__ uint32_t s_tmem;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool valid = tid < kG2 * Va;
  Dom2 d;
  d.Va = Va;
  d.g = tid & 1;
  d.l = valid ? tid >> 1 : 0;
  d.s0 = (size_t)blist[blockIdx.x / cpb] * Va;
  d.sR = sR;
  d.sU = sU;
  d.sA = sA;
  d.sN = sN;

  if (warp == 0) {
    tc::tmem_alloc(&s_tmem, tm_cols);
    tc::tmem_relinquish();
  }
  {
    const float4* U4 = reinterpret_cast<const float4*>(U20) + d.s0 * 20;
    for (int i = tid; i < 20 * Va; i += T) sU[(i % 20) * (Va + 1) + i / 20] = __ldg(U4 + i);
    const float4* A4 = reinterpret_cast<const float4*>(Acl) + d.s0 * 18;
    for (int i = tid; i < 18 * Va; i += T) sA[(i % 18) * (Va + 1) + i / 18] = __ldg(A4 + i);
    for (int i = tid; i < 8 * Va; i += T) {
      const int l = i >> 3, k = i & 7;
      const int n = (__ldg(nbr + (d.s0 + l) * 8 + k) & 0x3fffffff) - (int)d.s0;
      sN[k * Va + l] = (n >= 0 && n < Va) ? n : -1;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = s_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * kColsItem);

  for (int r0 = (blockIdx.x % cpb) * kG2; r0 < N; r0 += cpb * kG2) {
    {
      float v[24];
      if (valid) {
        const float* xs = x + (d.s0 + d.l) * 24 * N + r0 + d.g;
#pragma unroll
        for (int k = 0; k < 24; ++k) {
          v[k] = xs[k * N];
          sR[(k * Va + d.l) * kG2 + d.g] = v[k];
        }
      } else {
#pragma unroll
        for (int k = 0; k < 24; ++k) v[k] = 0.f;
      }
      tm_put(tm, v);
    }
    tc::tmem_wait_st();
    __syncthreads();
    float qr[12], qi[12];
    if (valid) {
      apply_dom2<true>(d, qr, qi, nbr, x, U20, N, r0);
      const SB* bs = b + (d.s0 + d.l) * 24 * N + r0 + d.g;
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        qr[c] = (float)to_r(bs[(2 * c) * N]) - qr[c];
        qi[c] = (float)to_r(bs[(2 * c + 1) * N]) - qi[c];
      }
    }
    __syncthreads();
    if (valid) {
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        sR[((2 * c) * Va + d.l) * kG2 + d.g] = qr[c];
        sR[((2 * c + 1) * Va + d.l) * kG2 + d.g] = qi[c];
      }
    }
    __syncthreads();
    for (int step = 0; step < n_mr; ++step) {
      float pr = 0.f, pi = 0.f, pq = 0.f;
      if (valid) {
        apply_dom2<false>(d, qr, qi, nbr, x, U20, N, r0);
        float rr[12], ri[12];
        load_rho2(d, d.l, rr, ri);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          pr = fmaf(qr[c], rr[c], fmaf(qi[c], ri[c], pr));
          pi = fmaf(qr[c], ri[c], fmaf(-qi[c], rr[c], pi));
          pq = fmaf(qr[c], qr[c], fmaf(qi[c], qi[c], pq));
        }
      }
#pragma unroll
      for (int o = kG2; o < 32; o <<= 1) {
        pr += __shfl_xor_sync(0xffffffffu, pr, o);
        pi += __shfl_xor_sync(0xffffffffu, pi, o);
        pq += __shfl_xor_sync(0xffffffffu, pq, o);
      }
      if (lane < kG2) {
        sred[(warp * kG2 + lane) * 3 + 0] = pr;
        sred[(warp * kG2 + lane) * 3 + 1] = pi;
        sred[(warp * kG2 + lane) * 3 + 2] = pq;
      }
      __syncthreads();
      if (tid < kG2) {
        double a = 0, bb = 0, cc = 0;
        for (int w = 0; w < T / 32; ++w) {
          a += sred[(w * kG2 + tid) * 3 + 0];
          bb += sred[(w * kG2 + tid) * 3 + 1];
          cc += sred[(w * kG2 + tid) * 3 + 2];
        }
        salpha[2 * tid] = cc > 0 ? (float)(a / cc) : 0.f;
        salpha[2 * tid + 1] = cc > 0 ? (float)(bb / cc) : 0.f;
      }
      __syncthreads();
      const cx<float> al = mk(salpha[2 * d.g], salpha[2 * d.g + 1]);
      {
        float xv[24];
        tm_get(tm, xv);
        if (valid) {
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            const int i0 = ((2 * c) * Va + d.l) * kG2 + d.g, i1 = ((2 * c + 1) * Va + d.l) * kG2 + d.g;
            cx<float> rv = mk(sR[i0], sR[i1]);
            cx<float> xc = mk(xv[2 * c], xv[2 * c + 1]);
            fma_(xc, al, rv);
            xv[2 * c] = xc.re;
            xv[2 * c + 1] = xc.im;
            fma_(rv, al, mk(-qr[c], -qi[c]));
            sR[i0] = rv.re;
            sR[i1] = rv.im;
          }
        }
        tm_put(tm, xv);
      }
      tc::tmem_wait_st();
      __syncthreads();
    }
    {
      float xv[24];
      tm_get(tm, xv);
      if (valid) {
        float* xs = x + (d.s0 + d.l) * 24 * N + r0 + d.g;
#pragma unroll
        for (int k = 0; k < 24; ++k) xs[k * N] = xv[k];
      }
    }
    __syncthreads();
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(s_tmem, tm_cols);
}

}  // namespace

// threads for a domain of Va sites: G items per site, at most two items per
// thread (G = 4) or one (G = 2), whole warpgroups
static int sap_tm_threads(int Va, int G) { return G == 4 ? 128 * ((kG * Va + 255) / 256) : 128 * ((2 * Va + 127) / 128); }

static size_t sap_tm_smem(int Va, int T, int G) {
  if (G == 4)
    return sizeof(float4) * 20 * (size_t)(Va + 1) + sizeof(float) * ((size_t)24 * Va * kG + (T / 32) * kG * 4) +
           sizeof(int) * 8 * (size_t)Va;
  return sizeof(float4) * 38 * (size_t)(Va + 1) + sizeof(int) * 8 * (size_t)Va +
         sizeof(float) * ((size_t)24 * Va * kG2 + (T / 32) * kG2 * 3 + 2 * kG2);
}

static int max_smem(mrhs_ctx c) {
  int maxsm = 0;
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  return maxsm;
}

// chunk width: 4 (clover through L1; measured faster) unless MRHS_SAP_CHUNK=2
// asks for the two-RHS form (everything on chip) or nrhs is not a multiple of 4
static int sap_tm_width(mrhs_ctx c, int nrhs) {
  static const int forced = [] {
    const char* e = std::getenv("MRHS_SAP_CHUNK");
    return e ? std::atoi(e) : 0;
  }();
  const int Va = c->g.Va;
  if (Va > 256 || !c->U20) return 0;
  const bool ok2 = nrhs % 2 == 0 && sap_tm_smem(Va, sap_tm_threads(Va, 2), 2) <= (size_t)max_smem(c);
  const bool ok4 = nrhs % 4 == 0 && sap_tm_smem(Va, sap_tm_threads(Va, 4), 4) <= (size_t)max_smem(c);
  if (forced == 2 && ok2) return 2;
  if (ok4) return 4;
  return ok2 ? 2 : 0;
}

bool sap_tm_ok(mrhs_ctx c, int nrhs) { return sap_tm_width(c, nrhs) > 0; }

void sap_tm(mrhs_ctx c, const void* b, int bdtype, void* x, int nrhs, int n_sweeps, int n_mr) {
  const int Va = c->g.Va;
  const int G = sap_tm_width(c, nrhs);
  const int T = sap_tm_threads(Va, G);
  const size_t smem = sap_tm_smem(Va, T, G);
  // columns: (T/128) warpgroups x 24 per item (G = 4: two items and the
  // stashed q of the first), rounded up to a power of two >= 32
  uint32_t cols = 32;
  while (cols < (uint32_t)(T / 128) * (G == 4 ? 3 : 1) * kColsItem) cols <<= 1;
  // CTAs per domain: by default one chunk of G right-hand sides each, so that
  // the CTAs of a domain run side by side and share every 32-byte sector of
  // x and b in L2 (MRHS_SAP_CPB overrides, 1 = one CTA loops over the chunks)
  static const int cpb_env = [] {
    const char* e = std::getenv("MRHS_SAP_CPB");
    return e ? std::atoi(e) : 0;
  }();
  const int nch = nrhs / G;
  const int cpb = cpb_env > 0 ? std::min(cpb_env, nch) : nch;
  for (int sw = 0; sw < n_sweeps; ++sw)
    for (int col = 0; col < 2; ++col) {
      const int* blist = c->blocks_col + (col ? c->ncol[0] : 0);
      Prof pr(c, G == 4 ? "sap_tm" : "sap_tm2");
      MRHS_DISPATCH(bdtype, SB, {
        auto kern = G == 4 ? k_sap_tm<SB> : k_sap_tm2<SB>;
        MRHS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<c->ncol[col] * cpb, T, smem, c->stream>>>((const SB*)b, (float*)x, c->U20, c->A32, c->nbr, nrhs, Va,
                                                         blist, n_mr, cols, cpb);
      });
      MRHS_LAUNCH_CHECK("sap_tm");
    }
}

}  // namespace mrhs
