// SAP sweep (Sec. 2 of the paper; red-black multiplicative Schwarz with
// minimal-residual block solves) with the domain on chip and the arithmetic
// on packed pairs of right-hand sides.
//
// Per colour, one CTA per (domain, chunk of 4 right-hand sides), as in
// sap_tm.cu, but a thread owns one SITE and a PAIR of right-hand sides
// (thread t: site t/2, pair t%2 of the chunk) instead of two (site, rhs)
// items: every complex operation is one .f32x2 instruction on the pair, and
// the links and the clover term of the site are loaded once for both
// right-hand sides of the pair.
//   shared memory  rho [12][Va][2] float4 = (re_a, re_b, im_a, im_b) of the
//                  pair and the domain-local neighbour table [8][Va] (the
//                  domain's halved links [20][Va+1] float4 too in the "2s"
//                  form; by default the links are read through L1);
//   tensor memory  the running solution x_B of the thread's pair
//                  (48 columns: 12 components x (re_a, re_b, im_a, im_b)) and
//                  a copy of the clover term of the thread's site (72
//                  columns), staged once per CTA: the five applications of D
//                  per chunk read it there instead of from global memory;
//   registers      q = D_B rho between the reduction for alpha and the
//                  update.
// Per colour and chunk: r = b - D x on the domain (neighbours outside it from
// x in global memory, owned by the other colour and not written during the
// launch), then n_mr MR steps e += alpha rho, rho -= alpha q with
// alpha = <q, rho> / <q, q> per right-hand side, then x_B += e.
#include <algorithm>
#include <cstdlib>
#include <string>

#include "stencil.cuh"
#include "tc.cuh"

namespace mrhs {
namespace {

// PP pairs of right-hand sides per chunk: PP = 2 (512 threads for a 256-site
// domain, one CTA per SM) or PP = 1 (256 threads, two CTAs per SM); LG: the
// links read from global memory (through L1) instead of staged in shared
// memory, which leaves room for the second CTA
constexpr int kPCols = 48;    // tensor-memory columns of one thread's x_B
constexpr int kPClov = 72;    // tensor-memory columns of its site's clover term
constexpr int kPWarpCols = kPCols + kPClov;

struct DomP {
  const float4* sR;  // [12][Va][PP]
  const float4* sU;  // [20][Va+1]: float4 k of link mu at row mu*5 + k
  const int* sN;     // [8][Va]: neighbour inside the domain (local) or ~(device site)
  uint32_t tclov;    // tensor-memory address of the thread's copy of its site's clover term
  int Va, l, p;
  size_t s0;
};

template <int PP>
__device__ __forceinline__ c2 ldR(const DomP& d, int c, int n) {
  const float4 v = d.sR[(c * d.Va + n) * PP + d.p];
  return mk2(make_float2(v.x, v.y), make_float2(v.z, v.w));
}

__device__ __forceinline__ void ld_link(const float4* src, int stride, float u[20]) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const float4 t = src[k * stride];
    u[4 * k] = t.x, u[4 * k + 1] = t.y, u[4 * k + 2] = t.z, u[4 * k + 3] = t.w;
  }
}
// link mu of device site n from global memory (read-only path)
__device__ __forceinline__ void ld_link_g(const float* __restrict__ U20, size_t n, int mu, float u[20]) {
  const float4* src = reinterpret_cast<const float4*>(U20 + (n * 4 + mu) * 20);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const float4 t = __ldg(src + k);
    u[4 * k] = t.x, u[4 * k + 1] = t.y, u[4 * k + 2] = t.z, u[4 * k + 3] = t.w;
  }
}

// o += hop (MU, DIR) at the thread's site for its pair: the neighbour spinor
// from shared memory inside the domain; outside it (RESID only) from x, with
// the link of a backward hop from global memory. The two halves of the
// projected spinor (h_0 from spins 0 and SB0, h_1 from spins 1 and SB1) are
// done one after the other, so that only one half is live in registers; each
// half feeds one upper and one lower spin of o.
template <int MU, int DIR, int SP>
__device__ __forceinline__ void half_pk(c2 o[12], const c2 h[3], const float u[20]) {
  using Tb = BTab<MU>;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    c2 ch;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      // U[a][b] forward, conj(U[b][a]) backward (the sign of the time
      // boundary and the factor 1/2 are folded into the stored links)
      const int q = DIR > 0 ? a * 3 + b : b * 3 + a;
      const float2 ure = bc2(u[2 * q]);
      const float2 uim = bc2(DIR > 0 ? u[2 * q + 1] : -u[2 * q + 1]);
      const float2 nuim = bc2(DIR > 0 ? -u[2 * q + 1] : u[2 * q + 1]);
      const c2 hv = h[b];
      if (b == 0) {
        ch.re = mul2(ure, hv.re);
        ch.im = mul2(ure, hv.im);
      } else {
        ch.re = fma2(ure, hv.re, ch.re);
        ch.im = fma2(ure, hv.im, ch.im);
      }
      ch.re = fma2(nuim, hv.im, ch.re);
      ch.im = fma2(uim, hv.re, ch.im);
    }
    // upper spin SP -= chi_SP; the lower spin that B^dag takes chi_SP to
    o[3 * SP + a] = o[3 * SP + a] - ch;
    if (Tb::SD0 == SP) o[6 + a] = axpy_ph<Tb::KD0, DIR>(o[6 + a], ch);
    if (Tb::SD1 == SP) o[9 + a] = axpy_ph<Tb::KD1, DIR>(o[9 + a], ch);
  }
}

template <int MU, int DIR, bool RESID, int PP, bool LG>
__device__ __forceinline__ void hop_pk(const DomP& d, c2 o[12], const float* __restrict__ x,
                                       const float* __restrict__ U20, int N, int r0) {
  using Tb = BTab<MU>;
  const int e = d.sN[((DIR > 0 ? 0 : 4) + MU) * d.Va + d.l];
  if (!RESID && e < 0) return;
  float u[20];
  const float* xn = nullptr;
  if (e >= 0) {
    if (LG) ld_link_g(U20, d.s0 + (DIR > 0 ? d.l : e), MU, u);
    else ld_link(d.sU + MU * 5 * (d.Va + 1) + (DIR > 0 ? d.l : e), d.Va + 1, u);
  } else {
    const size_t n = (size_t)(~e);
    xn = x + n * 24 * N + r0 + 2 * d.p;
    if (DIR > 0) {
      if (LG) ld_link_g(U20, d.s0 + d.l, MU, u);
      else ld_link(d.sU + MU * 5 * (d.Va + 1) + d.l, d.Va + 1, u);
    } else {
      ld_link(reinterpret_cast<const float4*>(U20 + (n * 4 + MU) * 20), 1, u);
    }
  }
  auto ld = [&](int comp) -> c2 {
    if (e >= 0) return ldR<PP>(d, comp, e);
    return mk2(*reinterpret_cast<const float2*>(xn + (2 * comp) * N),
               *reinterpret_cast<const float2*>(xn + (2 * comp + 1) * N));
  };
  {
    c2 h[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) h[c] = axpy_ph<Tb::KB0, -DIR>(ld(c), ld(3 * Tb::SB0 + c));
    half_pk<MU, DIR, 0>(o, h, u);
  }
  {
    c2 h[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) h[c] = axpy_ph<Tb::KB1, -DIR>(ld(3 + c), ld(3 * Tb::SB1 + c));
    half_pk<MU, DIR, 1>(o, h, u);
  }
}

// o = D x (RESID: x inside the domain from shared memory, outside from global
// memory) or o = D_B rho (couplings leaving the domain dropped)
template <bool RESID, int PP, bool LG>
__device__ __forceinline__ void apply_pk(const DomP& d, c2 o[12], const float* __restrict__ Acl,
                                         const float* __restrict__ x, const float* __restrict__ U20, int N,
                                         int r0) {
  {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float q[36];
      tc::tmem_ld36(d.tclov + 36 * h, q);
      c2 ps[6];
#pragma unroll
      for (int a = 0; a < 6; ++a) ps[a] = ldR<PP>(d, 6 * h + a, d.l);
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        const float2 qa = bc2(q[a]);
        c2 acc = mk2(mul2(ps[a].re, qa), mul2(ps[a].im, qa));
#pragma unroll
        for (int b2 = 0; b2 < 6; ++b2) {
          if (b2 == a) continue;
          const int ei = b2 > a ? herm_idx(a, b2) : herm_idx(b2, a);
          const float mim = b2 > a ? q[ei + 1] : -q[ei + 1];
          const float2 mre2 = bc2(q[ei]), mim2 = bc2(mim), nmim2 = bc2(-mim);
          acc.re = fma2(mre2, ps[b2].re, acc.re);
          acc.re = fma2(nmim2, ps[b2].im, acc.re);
          acc.im = fma2(mre2, ps[b2].im, acc.im);
          acc.im = fma2(mim2, ps[b2].re, acc.im);
        }
        o[6 * h + a] = acc;
      }
    }
  }
  // one hop per iteration of a loop the compiler keeps rolled, so that it does
  // not start the loads of later hops early (they would not fit in the
  // registers next to o)
#pragma unroll 1
  for (int k = 0; k < 8; ++k) {
    switch (k) {
      case 0: hop_pk<0, +1, RESID, PP, LG>(d, o, x, U20, N, r0); break;
      case 1: hop_pk<1, +1, RESID, PP, LG>(d, o, x, U20, N, r0); break;
      case 2: hop_pk<2, +1, RESID, PP, LG>(d, o, x, U20, N, r0); break;
      case 3: hop_pk<3, +1, RESID, PP, LG>(d, o, x, U20, N, r0); break;
      case 4: hop_pk<0, -1, RESID, PP, LG>(d, o, x, U20, N, r0); break;
      case 5: hop_pk<1, -1, RESID, PP, LG>(d, o, x, U20, N, r0); break;
      case 6: hop_pk<2, -1, RESID, PP, LG>(d, o, x, U20, N, r0); break;
      default: hop_pk<3, -1, RESID, PP, LG>(d, o, x, U20, N, r0); break;
    }
  }
}

// a pair of right-hand sides of b (two consecutive values) in FP32
__device__ __forceinline__ float2 ld_pair(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ float2 ld_pair(const double* p) { return make_float2((float)p[0], (float)p[1]); }
__device__ __forceinline__ float2 ld_pair(const __nv_bfloat16* p) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
}
__device__ __forceinline__ float2 ld_pair(const __half* p) {
  return __half22float2(*reinterpret_cast<const __half2*>(p));
}

__device__ __forceinline__ void xb_put(uint32_t ta, const c2 v[12]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float f[16];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const c2 t = v[4 * k + i];
      f[4 * i] = t.re.x, f[4 * i + 1] = t.re.y, f[4 * i + 2] = t.im.x, f[4 * i + 3] = t.im.y;
    }
    tc::tmem_st16(ta + 16 * k, f);
  }
}

template <class SB, int PP, bool LG>
__global__ void __launch_bounds__(256 * PP, 3 - PP) k_sap_pk(const SB* __restrict__ b, float* __restrict__ x,
                                                      const float* __restrict__ U20, const float* __restrict__ Acl,
                                                      const int* __restrict__ nbr, int N, int Va,
                                                      const int* __restrict__ blist, int n_mr, uint32_t tm_cols,
                                                      int cpb, int x0z) {
  extern __shared__ float4 smem4[];
  const int T = blockDim.x;
  constexpr int kG = 2 * PP;                                          // right-hand sides per chunk
  float4* sU = smem4;                                                 // [20][Va+1] (not LG)
  float4* sR = LG ? smem4 : sU + 20 * (Va + 1);                       // [12][Va][PP]
  float2* sred = reinterpret_cast<float2*>(sR + 12 * PP * Va);        // [T/32][PP][3]
  int* sN = reinterpret_cast<int*>(sred + (T / 32) * PP * 3);        // [8][Va]
  __shared__ uint32_t s_tmem;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  DomP d;
  d.Va = Va;
  d.l = tid / PP;
  d.p = tid % PP;
  const bool valid = d.l < Va;
  if (!valid) d.l = 0;  // idle threads read site 0 and write nothing
  d.s0 = (size_t)blist[blockIdx.x / cpb] * Va;
  d.sR = sR;
  d.sU = sU;
  d.sN = sN;

  if (warp == 0) {
    tc::tmem_alloc(&s_tmem, tm_cols);
    tc::tmem_relinquish();
  }
  {
    const float4* U4 = reinterpret_cast<const float4*>(U20) + d.s0 * 20;
    if (!LG)
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
  // disjoint column ranges of kPCols
  const uint32_t tm = s_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * kPWarpCols);
  d.tclov = tm + kPCols;
  {
    // the clover term of the thread's site -> tensor memory (72 columns)
    const float4* A4 = reinterpret_cast<const float4*>(Acl + (d.s0 + d.l) * 72);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float f[16];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float4 v = __ldg(A4 + 4 * k + i);
        f[4 * i] = v.x, f[4 * i + 1] = v.y, f[4 * i + 2] = v.z, f[4 * i + 3] = v.w;
      }
      tc::tmem_st16(d.tclov + 16 * k, f);
    }
    float f[8];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float4 v = __ldg(A4 + 16 + i);
      f[4 * i] = v.x, f[4 * i + 1] = v.y, f[4 * i + 2] = v.z, f[4 * i + 3] = v.w;
    }
    tc::tmem_st8(d.tclov + 64, f);
    tc::tmem_wait_st();
  }

  for (int r0 = (blockIdx.x % cpb) * kG; r0 < N; r0 += cpb * kG) {
    // stage x0: one (component c, site l) per unit, the real and imaginary
    // rows of the chunk's right-hand sides become the pairs' float4
    // (re_a, re_b, im_a, im_b)
    // (x0z: x = 0 everywhere, the stage and D x0 are skipped)
    for (int u = x0z ? 12 * Va : tid; u < 12 * Va; u += T) {
      const int c = u / Va, l = u % Va;
      const float* xs = x + ((d.s0 + l) * 24 + 2 * c) * N + r0;
      if (PP == 2) {
        const float4 re = *reinterpret_cast<const float4*>(xs);
        const float4 im = *reinterpret_cast<const float4*>(xs + N);
        sR[(c * Va + l) * 2] = make_float4(re.x, re.y, im.x, im.y);
        sR[(c * Va + l) * 2 + 1] = make_float4(re.z, re.w, im.z, im.w);
      } else {
        const float2 re = *reinterpret_cast<const float2*>(xs);
        const float2 im = *reinterpret_cast<const float2*>(xs + N);
        sR[c * Va + l] = make_float4(re.x, re.y, im.x, im.y);
      }
    }
    __syncthreads();
    c2 o[12];
    // x_B = x0 of the thread's pair -> tensor memory; then q0 = D x0
#pragma unroll
    for (int c = 0; c < 12; ++c) o[c] = x0z ? mk2(make_float2(0.f, 0.f), make_float2(0.f, 0.f)) : ldR<PP>(d, c, d.l);
    xb_put(tm, o);
    if (!x0z) apply_pk<true, PP, LG>(d, o, Acl, x, U20, N, r0);
    tc::tmem_wait_st();
    __syncthreads();  // every read of x0 in shared memory is done
    // rho = b - D x0 at the thread's site
    if (valid) {
      const SB* bs = b + (d.s0 + d.l) * 24 * N + r0 + 2 * d.p;
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        const float2 bre = ld_pair(bs + (2 * c) * N), bim = ld_pair(bs + (2 * c + 1) * N);
        const c2 r = mk2(sub2(bre, o[c].re), sub2(bim, o[c].im));
        sR[(c * Va + d.l) * PP + d.p] = make_float4(r.re.x, r.re.y, r.im.x, r.im.y);
      }
    }
    __syncthreads();
    for (int step = 0; step < n_mr; ++step) {
      float2 pr = make_float2(0.f, 0.f), pi = pr, pq = pr;
      apply_pk<false, PP, LG>(d, o, Acl, x, U20, N, r0);  // o = q = D_B rho
      if (valid) {
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          const c2 r = ldR<PP>(d, c, d.l);
          pr = fma2(o[c].re, r.re, fma2(o[c].im, r.im, pr));
          pi = fma2(o[c].re, r.im, fma2(make_float2(-o[c].im.x, -o[c].im.y), r.re, pi));
          pq = fma2(o[c].re, o[c].re, fma2(o[c].im, o[c].im, pq));
        }
      }
      // sums over the sites of the warp (lanes of the same pair parity),
      // then over the warps in order: every thread of a pair gets the same
      // alpha for both of its right-hand sides
#pragma unroll
      for (int s = PP; s < 32; s <<= 1) {
        pr.x += __shfl_xor_sync(0xffffffffu, pr.x, s);
        pr.y += __shfl_xor_sync(0xffffffffu, pr.y, s);
        pi.x += __shfl_xor_sync(0xffffffffu, pi.x, s);
        pi.y += __shfl_xor_sync(0xffffffffu, pi.y, s);
        pq.x += __shfl_xor_sync(0xffffffffu, pq.x, s);
        pq.y += __shfl_xor_sync(0xffffffffu, pq.y, s);
      }
      if (lane < PP) {
        sred[(warp * PP + lane) * 3] = pr;
        sred[(warp * PP + lane) * 3 + 1] = pi;
        sred[(warp * PP + lane) * 3 + 2] = pq;
      }
      __syncthreads();
      float2 a = make_float2(0.f, 0.f), bb = a, cc = a;
      for (int w = 0; w < T / 32; ++w) {
        const float2 t0 = sred[(w * PP + d.p) * 3], t1 = sred[(w * PP + d.p) * 3 + 1],
                     t2 = sred[(w * PP + d.p) * 3 + 2];
        a.x += t0.x, a.y += t0.y;
        bb.x += t1.x, bb.y += t1.y;
        cc.x += t2.x, cc.y += t2.y;
      }
      const float2 alr = make_float2(cc.x > 0.f ? a.x / cc.x : 0.f, cc.y > 0.f ? a.y / cc.y : 0.f);
      const float2 ali = make_float2(cc.x > 0.f ? bb.x / cc.x : 0.f, cc.y > 0.f ? bb.y / cc.y : 0.f);
      const float2 nali = make_float2(-ali.x, -ali.y);
      // x_B += alpha rho (tensor memory), rho -= alpha q (shared memory)
      // four components (16 tensor-memory columns) at a time
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float f[16];
        tc::tmem_ld16(tm + 16 * k, f);
        if (valid) {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int c = 4 * k + i;
            c2 xv = mk2(make_float2(f[4 * i], f[4 * i + 1]), make_float2(f[4 * i + 2], f[4 * i + 3]));
            c2 r = ldR<PP>(d, c, d.l);
            xv.re = fma2(alr, r.re, xv.re);
            xv.re = fma2(nali, r.im, xv.re);
            xv.im = fma2(alr, r.im, xv.im);
            xv.im = fma2(ali, r.re, xv.im);
            // rho += alpha (-q)
            const c2 nq = mk2(make_float2(-o[c].re.x, -o[c].re.y), make_float2(-o[c].im.x, -o[c].im.y));
            r.re = fma2(alr, nq.re, r.re);
            r.re = fma2(nali, nq.im, r.re);
            r.im = fma2(alr, nq.im, r.im);
            r.im = fma2(ali, nq.re, r.im);
            sR[(c * Va + d.l) * PP + d.p] = make_float4(r.re.x, r.re.y, r.im.x, r.im.y);
            f[4 * i] = xv.re.x, f[4 * i + 1] = xv.re.y, f[4 * i + 2] = xv.im.x, f[4 * i + 3] = xv.im.y;
          }
        }
        tc::tmem_st16(tm + 16 * k, f);
      }
      tc::tmem_wait_st();
      __syncthreads();
    }
    // x = x_B for the thread's site and pair
    {
      float* xs = x + (d.s0 + d.l) * 24 * N + r0 + 2 * d.p;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float f[16];
        tc::tmem_ld16(tm + 16 * k, f);
        if (valid) {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int c = 4 * k + i;
            *reinterpret_cast<float2*>(xs + (2 * c) * N) = make_float2(f[4 * i], f[4 * i + 1]);
            *reinterpret_cast<float2*>(xs + (2 * c + 1) * N) = make_float2(f[4 * i + 2], f[4 * i + 3]);
          }
        }
      }
    }
    __syncthreads();
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(s_tmem, tm_cols);
}

}  // namespace

// the form of the kernel: MRHS_SAP_PK = "2g" (default: two pairs per CTA,
// links read through L1), "2s" (links staged in shared memory) or "1g" (one
// pair per CTA, two CTAs per SM). Measured at 48^3x96 with 32 right-hand
// sides: 83.2 ms per colour launch (2g), 88.8 (2s), 108.7 (1g): the links of
// a domain stay in L1 across the hops, and staging them cost more than it
// saved; two CTAs per SM each restage the clover term and re-read the links
// for half the right-hand sides.
struct PkForm {
  int pp;
  bool lg;
};
static PkForm pk_form() {
  static const PkForm f = [] {
    const char* e = std::getenv("MRHS_SAP_PK");
    const std::string v = e ? e : "";
    if (v == "1g") return PkForm{1, true};
    if (v == "2s") return PkForm{2, false};
    return PkForm{2, true};
  }();
  return f;
}

static int sap_pk_threads(int Va, int pp) { return 128 * ((pp * Va + 127) / 128); }

static size_t sap_pk_smem(int Va, int T, PkForm f) {
  return sizeof(float4) * ((f.lg ? 0 : 20 * (size_t)(Va + 1)) + 12 * (size_t)f.pp * Va) +
         sizeof(float2) * (T / 32) * f.pp * 3 + sizeof(int) * 8 * (size_t)Va;
}

bool sap_pk_ok(mrhs_ctx c, int nrhs) {
  const int Va = c->g.Va;
  const PkForm f = pk_form();
  if (Va > 256 || !c->U20 || nrhs % (2 * f.pp) != 0) return false;
  int maxsm = 0;
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  return sap_pk_smem(Va, sap_pk_threads(Va, f.pp), f) <= (size_t)maxsm;
}

void sap_pk(mrhs_ctx c, const void* b, int bdtype, void* x, int nrhs, int n_sweeps, int n_mr, bool x0_zero) {
  const int Va = c->g.Va;
  const PkForm f = pk_form();
  const int T = sap_pk_threads(Va, f.pp);
  const size_t smem = sap_pk_smem(Va, T, f);
  const int kG = 2 * f.pp;
  // x_B and the clover copy: kPWarpCols columns per thread, (T / 128) warps
  // per lane quarter (at most 4 x 120 = 480 of the 512 columns)
  uint32_t cols = 32;
  while (cols < (uint32_t)(T / 128) * kPWarpCols) cols <<= 1;
  // CTAs per domain: by default one chunk each, so that a domain's CTAs run
  // side by side and share the 32-byte sectors of x and b in L2;
  // MRHS_SAP_CPB = c: c CTAs per domain, each looping over nrhs / (4 c) chunks
  // (the links and clover term staged once per CTA serve all its chunks)
  static const int cpb_env = [] {
    const char* e = std::getenv("MRHS_SAP_CPB");
    return e ? std::atoi(e) : 0;
  }();
  const int cpb = cpb_env > 0 ? std::min(cpb_env, nrhs / kG) : nrhs / kG;
  for (int sw = 0; sw < n_sweeps; ++sw)
    for (int col = 0; col < 2; ++col) {
      const int* blist = c->blocks_col + (col ? c->ncol[0] : 0);
      Prof pr(c, "sap_pk");
      MRHS_DISPATCH(bdtype, SB, {
        auto kern = f.pp == 1 ? k_sap_pk<SB, 1, true> : f.lg ? k_sap_pk<SB, 2, true> : k_sap_pk<SB, 2, false>;
        MRHS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<c->ncol[col] * cpb, T, smem, c->stream>>>((const SB*)b, (float*)x, c->U20, c->A32, c->nbr, nrhs, Va,
                                                         blist, n_mr, cols, cpb, x0_zero && sw == 0 && col == 0);
      });
      MRHS_LAUNCH_CHECK("sap_pk");
    }
}

}  // namespace mrhs
