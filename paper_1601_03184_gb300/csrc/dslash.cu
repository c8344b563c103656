// Multi-right-hand-side Wilson-clover stencil (full, block-restricted and
// residual forms) and the SAP smoother built on it: the operator of Sec. 1-2
// of the paper, with the right-hand sides as the innermost index like the
// SIMD vectors of Sec. 5, and the smoother of Sec. 2.
#include <cstdlib>

#include "stencil.cuh"

// tuning switches of the FP32 stencil (compile time): MRHS_DS_PRELOAD = 1
// loads a site's eight neighbour records before its first hop;
// MRHS_DS_MINB = CTAs of 128 threads per SM the register budget is sized for
#ifndef MRHS_DS_PRELOAD
#define MRHS_DS_PRELOAD 1
#endif
#ifndef MRHS_DS_MINB
#define MRHS_DS_MINB 4
#endif

namespace mrhs {
namespace {

// y = D x, y = D_B x, or y = b - D x; over all sites, or over the sites of
// the aggregates listed in blist (nblk of them)
template <int MODE, class S, class SB, class R>
__global__ void k_dslash(const S* __restrict__ x, S* __restrict__ y, const SB* __restrict__ b,
                         const cx<R>* __restrict__ U, const R* __restrict__ A, const int* __restrict__ nbr, int N,
                         int Va, const int* __restrict__ blist, size_t nwork) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= nwork) return;
  int r = (int)(t % N);
  size_t sl = t / N;
  int s = blist ? blist[sl / Va] * Va + (int)(sl % Va) : (int)sl;
  cx<R> out[12];
  dslash_site<MODE == DS_BLOCK, S, R>(out, x, s, N, r, U, A, nbr, Va);
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    cx<R> v = out[c];
    if (MODE == DS_RESID) v = ld<SB, R>(b, (size_t)s * 12 + c, N, r) - v;
    st<S, R>(y, (size_t)s * 12 + c, N, r, v);
  }
}

// n_mr minimal-residual steps on D_B e = rho for every aggregate in blist,
// one CTA per aggregate, all right-hand sides; x += alpha rho and
// rho -= alpha q are applied directly (e starts at 0, so x_B += e).
// rho, q, x are read and written by the CTA only (no read-only cache path).
template <class S, class R>
__global__ void k_block_mr(S* x, S* rho, S* q, const cx<R>* __restrict__ U, const R* __restrict__ A,
                           const int* __restrict__ nbr, int N, int Va, const int* __restrict__ blist, int n_mr) {
  extern __shared__ double smem[];
  const int lanes = blockDim.x / N;  // site lanes; thread -> (lane, rhs)
  const int tid = threadIdx.x;
  const int r = tid % N;
  const int lane = tid / N;
  const bool active = lane < lanes;
  double* sqr_re = smem;                 // [lanes][N]
  double* sqr_im = sqr_re + lanes * N;
  double* sqq = sqr_im + lanes * N;
  double* salpha = sqq + lanes * N;      // [N][2]
  const int blk = blist[blockIdx.x];
  const int s0 = blk * Va;
  for (int it = 0; it < n_mr; ++it) {
    double qr_re = 0, qr_im = 0, qq = 0;
    if (active) {
      for (int l = lane; l < Va; l += lanes) {
        int s = s0 + l;
        cx<R> out[12];
        dslash_site<true, S, R>(out, rho, s, N, r, U, A, nbr, Va);
        R pr = 0, pi = 0, pq = 0;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          cx<R> rv = ld<S, R>(rho, (size_t)s * 12 + c, N, r);
          cx<R> qv = out[c];
          st<S, R>(q, (size_t)s * 12 + c, N, r, qv);
          qv = ld<S, R>(q, (size_t)s * 12 + c, N, r);  // the stored (rounded) value
          pr += qv.re * rv.re + qv.im * rv.im;
          pi += qv.re * rv.im - qv.im * rv.re;
          pq += qv.re * qv.re + qv.im * qv.im;
        }
        qr_re += (double)pr;
        qr_im += (double)pi;
        qq += (double)pq;
      }
      sqr_re[lane * N + r] = qr_re;
      sqr_im[lane * N + r] = qr_im;
      sqq[lane * N + r] = qq;
    }
    __syncthreads();
    if (tid < N) {
      double a = 0, bb = 0, c = 0;
      for (int l = 0; l < lanes; ++l) {
        a += sqr_re[l * N + tid];
        bb += sqr_im[l * N + tid];
        c += sqq[l * N + tid];
      }
      salpha[2 * tid] = c > 0 ? a / c : 0.0;
      salpha[2 * tid + 1] = c > 0 ? bb / c : 0.0;
    }
    __syncthreads();
    if (active) {
      cx<R> al = mk<R>((R)salpha[2 * r], (R)salpha[2 * r + 1]);
      for (int l = lane; l < Va; l += lanes) {
        size_t row = (size_t)(s0 + l) * 12;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          cx<R> rv = ld<S, R>(rho, row + c, N, r);
          cx<R> qv = ld<S, R>(q, row + c, N, r);
          cx<R> xv = ld<S, R>(x, row + c, N, r);
          fma_(xv, al, rv);
          cx<R> t = mk<R>(-qv.re, -qv.im);
          fma_(rv, al, t);
          st<S, R>(x, row + c, N, r, xv);
          st<S, R>(rho, row + c, N, r, rv);
        }
      }
    }
    __syncthreads();
  }
}

// Even-odd preconditioned domain solves: n_mr minimal-residual steps on the
// Schur complement of the even sites, S = A_EE - H_EO A_OO^-1 H_OE, for
// every aggregate in blist (one CTA per aggregate, all right-hand sides),
// from the residual r of the colour:
//   u_O = A_OO^-1 r_O,  rho_E = r_E - H_EO u_O,  e_E = 0;
//   n_mr times: u_O = A_OO^-1 H_OE rho_E, q_E = A_EE rho_E - H_EO u_O,
//               alpha = <q, rho>_E / <q, q>_E, e_E += alpha rho, rho -= alpha q;
//   e_O = A_OO^-1 (r_O - H_OE e_E);  x_B += e.
// H = the hopping terms inside the domain (they change the site parity, so
// every hop reads only sites of the other parity). ru holds rho on even and
// u on odd sites; q and e are separate fields.
struct EoGeom {
  int a[4], nb[4];
};

template <class S, class R>
__device__ __forceinline__ void site_apply_packed(cx<R> out[12], const S* x, size_t row, int N, int r, const R* M) {
  cx<R> psi[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) psi[c] = ld<S, R>(x, row + c, N, r);
  clover_apply_reg<R>(out, psi, M);
}

template <class S, class R>
__global__ void k_block_mr_eo(S* x, const S* rres, S* ru, S* q, S* e, const cx<R>* __restrict__ U,
                              const R* __restrict__ A, const R* __restrict__ Ainv, const int* __restrict__ nbr, int N,
                              int Va, const int* __restrict__ blist, int n_mr, EoGeom g) {
  extern __shared__ double smem[];
  const int lanes = blockDim.x / N;
  const int tid = threadIdx.x;
  const int r = tid % N;
  const int lane = tid / N;
  const bool active = lane < lanes;
  double* sqr_re = smem;
  double* sqr_im = sqr_re + lanes * N;
  double* sqq = sqr_im + lanes * N;
  double* salpha = sqq + lanes * N;
  const int blk = blist[blockIdx.x];
  const int s0 = blk * Va;
  // parity of the aggregate's first site, then of site l inside it
  int pb = 0;
  {
    int i = blk;
    for (int m = 0; m < 4; ++m) {
      pb += (i % g.nb[m]) * g.a[m];
      i /= g.nb[m];
    }
  }
  auto parity = [&](int l) {
    int p = pb;
    for (int m = 0; m < 4; ++m) {
      p += l % g.a[m];
      l /= g.a[m];
    }
    return p & 1;
  };
  // u_O = A_OO^-1 r_O
  if (active)
    for (int l = lane; l < Va; l += lanes)
      if (parity(l) == 1) {
        const int s = s0 + l;
        cx<R> o[12];
        site_apply_packed<S, R>(o, rres, (size_t)s * 12, N, r, Ainv + (size_t)s * 72);
#pragma unroll
        for (int c = 0; c < 12; ++c) st<S, R>(ru, (size_t)s * 12 + c, N, r, o[c]);
      }
  __syncthreads();
  // rho_E = r_E - H_EO u_O, e_E = 0
  if (active)
    for (int l = lane; l < Va; l += lanes)
      if (parity(l) == 0) {
        const int s = s0 + l;
        cx<R> h[12];
        dslash_site<true, S, R, false>(h, ru, s, N, r, U, A, nbr, Va);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
          st<S, R>(ru, (size_t)s * 12 + c, N, r, ld<S, R>(rres, (size_t)s * 12 + c, N, r) - h[c]);
          st<S, R>(e, (size_t)s * 12 + c, N, r, mk<R>(0, 0));
        }
      }
  __syncthreads();
  for (int it = 0; it < n_mr; ++it) {
    // u_O = A_OO^-1 H_OE rho_E
    if (active)
      for (int l = lane; l < Va; l += lanes)
        if (parity(l) == 1) {
          const int s = s0 + l;
          cx<R> h[12], u[12];
          dslash_site<true, S, R, false>(h, ru, s, N, r, U, A, nbr, Va);
          clover_apply_reg<R>(u, h, Ainv + (size_t)s * 72);
#pragma unroll
          for (int c = 0; c < 12; ++c) st<S, R>(ru, (size_t)s * 12 + c, N, r, u[c]);
        }
    __syncthreads();
    // q_E = A_EE rho_E - H_EO u_O and the two inner products over the even sites
    double qr_re = 0, qr_im = 0, qq = 0;
    if (active) {
      for (int l = lane; l < Va; l += lanes)
        if (parity(l) == 0) {
          const int s = s0 + l;
          cx<R> a[12], h[12];
          site_apply_packed<S, R>(a, ru, (size_t)s * 12, N, r, A + (size_t)s * 72);
          dslash_site<true, S, R, false>(h, ru, s, N, r, U, A, nbr, Va);
          R pr = 0, pi = 0, pq = 0;
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            st<S, R>(q, (size_t)s * 12 + c, N, r, a[c] - h[c]);
            const cx<R> qv = ld<S, R>(q, (size_t)s * 12 + c, N, r);  // the stored (rounded) value
            const cx<R> rv = ld<S, R>(ru, (size_t)s * 12 + c, N, r);
            pr += qv.re * rv.re + qv.im * rv.im;
            pi += qv.re * rv.im - qv.im * rv.re;
            pq += qv.re * qv.re + qv.im * qv.im;
          }
          qr_re += (double)pr;
          qr_im += (double)pi;
          qq += (double)pq;
        }
      sqr_re[lane * N + r] = qr_re;
      sqr_im[lane * N + r] = qr_im;
      sqq[lane * N + r] = qq;
    }
    __syncthreads();
    if (tid < N) {
      double a = 0, bb = 0, c = 0;
      for (int l = 0; l < lanes; ++l) {
        a += sqr_re[l * N + tid];
        bb += sqr_im[l * N + tid];
        c += sqq[l * N + tid];
      }
      salpha[2 * tid] = c > 0 ? a / c : 0.0;
      salpha[2 * tid + 1] = c > 0 ? bb / c : 0.0;
    }
    __syncthreads();
    // e_E += alpha rho_E, rho_E -= alpha q_E
    if (active) {
      const cx<R> al = mk<R>((R)salpha[2 * r], (R)salpha[2 * r + 1]);
      for (int l = lane; l < Va; l += lanes)
        if (parity(l) == 0) {
          const size_t row = (size_t)(s0 + l) * 12;
#pragma unroll
          for (int c = 0; c < 12; ++c) {
            cx<R> rv = ld<S, R>(ru, row + c, N, r);
            const cx<R> qv = ld<S, R>(q, row + c, N, r);
            cx<R> ev = ld<S, R>(e, row + c, N, r);
            fma_(ev, al, rv);
            fma_(rv, al, mk<R>(-qv.re, -qv.im));
            st<S, R>(e, row + c, N, r, ev);
            st<S, R>(ru, row + c, N, r, rv);
          }
        }
    }
    __syncthreads();
  }
  // e_O = A_OO^-1 (r_O - H_OE e_E)
  if (active)
    for (int l = lane; l < Va; l += lanes)
      if (parity(l) == 1) {
        const int s = s0 + l;
        cx<R> h[12], o[12];
        dslash_site<true, S, R, false>(h, e, s, N, r, U, A, nbr, Va);
#pragma unroll
        for (int c = 0; c < 12; ++c) h[c] = ld<S, R>(rres, (size_t)s * 12 + c, N, r) - h[c];
        clover_apply_reg<R>(o, h, Ainv + (size_t)s * 72);
#pragma unroll
        for (int c = 0; c < 12; ++c) st<S, R>(e, (size_t)s * 12 + c, N, r, o[c]);
      }
  __syncthreads();
  // x_B += e
  if (active)
    for (int l = lane; l < Va; l += lanes) {
      const size_t row = (size_t)(s0 + l) * 12;
#pragma unroll
      for (int c = 0; c < 12; ++c) st<S, R>(x, row + c, N, r, ld<S, R>(x, row + c, N, r) + ld<S, R>(e, row + c, N, r));
    }
}

// ---------------------------------------------------------------------------
// FP32 full operator, y = D x, on packed pairs of right-hand sides: P pairs
// per thread (2P interleaved right-hand sides, 8- or 16-byte loads), links
// padded to 20 floats (one float4-aligned record per link, loaded once per
// thread and applied to all its right-hand sides), the clover term read as
// float4; threads in site order so that the CTAs running at one time cover a
// compact range of aggregates; output stores are streaming (evict-first) so
// that L2 keeps the input field.
template <int P>
__device__ __forceinline__ void ldp(const float* p, float2 v[P]) {
  if constexpr (P == 1) {
    v[0] = *reinterpret_cast<const float2*>(p);
  } else {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = make_float2(t.x, t.y);
    v[1] = make_float2(t.z, t.w);
  }
}
// bf16 / fp16 storage: one pair of right-hand sides (4 bytes) widened to FP32
template <int P>
__device__ __forceinline__ void ldp(const __nv_bfloat16* p, float2 v[P]) {
  static_assert(P == 1, "reduced storage: one pair per thread");
  v[0] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
}
template <int P>
__device__ __forceinline__ void ldp(const __half* p, float2 v[P]) {
  static_assert(P == 1, "reduced storage: one pair per thread");
  v[0] = __half22float2(*reinterpret_cast<const __half2*>(p));
}
// store one pair (streaming: the output is not read again by this kernel)
__device__ __forceinline__ void stp(float* p, float2 v) { __stcs(reinterpret_cast<float2*>(p), v); }
__device__ __forceinline__ void stp(__nv_bfloat16* p, float2 v) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
  __stcs(reinterpret_cast<unsigned int*>(p), *reinterpret_cast<const unsigned int*>(&h));
}
__device__ __forceinline__ void stp(__half* p, float2 v) {
  const __half2 h = __floats2half2_rn(v.x, v.y);
  __stcs(reinterpret_cast<unsigned int*>(p), *reinterpret_cast<const unsigned int*>(&h));
}

template <int MU, int DIR, int P, int NC, class S>
__device__ __forceinline__ void hop_f2(c2 o[12][P], const S* __restrict__ xn, int Nrt,
                                       const float* __restrict__ Ul) {
  const int N = NC > 0 ? NC : Nrt;
  c2 h[2][3][P];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float2 pr[4][P], pi[4][P];
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
      ldp<P>(xn + ((3 * sp + c) * 2 + 0) * N, pr[sp]);
      ldp<P>(xn + ((3 * sp + c) * 2 + 1) * N, pi[sp]);
    }
#pragma unroll
    for (int g = 0; g < P; ++g) {
      using T = BTab<MU>;
      // h_s = psi_s -/+ (B psi_low)_s
      h[0][c][g] = axpy_ph<T::KB0, -DIR>(mk2(pr[0][g], pi[0][g]), mk2(pr[T::SB0][g], pi[T::SB0][g]));
      h[1][c][g] = axpy_ph<T::KB1, -DIR>(mk2(pr[1][g], pi[1][g]), mk2(pr[T::SB1][g], pi[T::SB1][g]));
    }
  }
  float u[20];
  const float4* U4 = reinterpret_cast<const float4*>(Ul);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    float4 t = __ldg(U4 + k);
    u[4 * k] = t.x;
    u[4 * k + 1] = t.y;
    u[4 * k + 2] = t.z;
    u[4 * k + 3] = t.w;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    c2 ch[2][P];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      // U[a][b] forward, conj(U[b][a]) backward
      const int e = DIR > 0 ? a * 3 + b : b * 3 + a;
      const float2 ure = bc2(u[2 * e]);
      const float2 uim = bc2(DIR > 0 ? u[2 * e + 1] : -u[2 * e + 1]);
      const float2 nuim = bc2(DIR > 0 ? -u[2 * e + 1] : u[2 * e + 1]);
#pragma unroll
      for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int g = 0; g < P; ++g) {
          const c2 hv = h[sp][b][g];
          if (b == 0) {
            ch[sp][g].re = mul2(ure, hv.re);
            ch[sp][g].im = mul2(ure, hv.im);
          } else {
            ch[sp][g].re = fma2(ure, hv.re, ch[sp][g].re);
            ch[sp][g].im = fma2(ure, hv.im, ch[sp][g].im);
          }
          ch[sp][g].re = fma2(nuim, hv.im, ch[sp][g].re);
          ch[sp][g].im = fma2(uim, hv.re, ch[sp][g].im);
        }
    }
#pragma unroll
    for (int g = 0; g < P; ++g) {
      using T = BTab<MU>;
      // upper spins -= chi, lower spins +/-= B^dag chi
      o[a][g] = o[a][g] - ch[0][g];
      o[3 + a][g] = o[3 + a][g] - ch[1][g];
      o[6 + a][g] = axpy_ph<T::KD0, DIR>(o[6 + a][g], ch[T::SD0][g]);
      o[9 + a][g] = axpy_ph<T::KD1, DIR>(o[9 + a][g], ch[T::SD1][g]);
    }
  }
}

template <class S, int P, int NC, int MINB>
__global__ void __launch_bounds__(128, MINB) k_dslash_f2(const S* __restrict__ x, S* __restrict__ y,
                                                         const float* __restrict__ U20,
                                                         const float* __restrict__ Acl,
                                                         const int* __restrict__ nbr, int Nrt, int q0, int nq,
                                                         size_t nwork) {
  constexpr int G = 2 * P;
  const int N = NC > 0 ? NC : Nrt;
  const int ng = nq / G;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= nwork) return;
  const int r0 = q0 + (int)(t % ng) * G;
  const size_t s = t / ng;
  // the eight neighbour records of the site, loaded first (their latency
  // overlaps the clover term) so that every hop waits for one round trip
  // (its spinor), not two (index, then spinor)
  int nb[8];
#if MRHS_DS_PRELOAD
  {
    const int4 n0 = __ldg(reinterpret_cast<const int4*>(nbr + s * 8));
    const int4 n1 = __ldg(reinterpret_cast<const int4*>(nbr + s * 8) + 1);
    nb[0] = n0.x, nb[1] = n0.y, nb[2] = n0.z, nb[3] = n0.w;
    nb[4] = n1.x, nb[5] = n1.y, nb[6] = n1.z, nb[7] = n1.w;
  }
#endif
  c2 o[12][P];
  {
    const float4* A4 = reinterpret_cast<const float4*>(Acl + s * 72);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float q[36];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        float4 v = __ldg(A4 + 9 * h + k);
        q[4 * k] = v.x;
        q[4 * k + 1] = v.y;
        q[4 * k + 2] = v.z;
        q[4 * k + 3] = v.w;
      }
      float2 pr[6][P], pi[6][P];
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        ldp<P>(x + ((s * 12 + 6 * h + a) * 2 + 0) * N + r0, pr[a]);
        ldp<P>(x + ((s * 12 + 6 * h + a) * 2 + 1) * N + r0, pi[a]);
      }
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        const float2 qa = bc2(q[a]);
#pragma unroll
        for (int g = 0; g < P; ++g) o[6 * h + a][g] = mk2(mul2(pr[a][g], qa), mul2(pi[a][g], qa));
#pragma unroll
        for (int b2 = 0; b2 < 6; ++b2) {
          if (b2 == a) continue;
          const int e = b2 > a ? herm_idx(a, b2) : herm_idx(b2, a);
          const float mim = b2 > a ? q[e + 1] : -q[e + 1];
          const float2 mre2 = bc2(q[e]), mim2 = bc2(mim), nmim2 = bc2(-mim);
#pragma unroll
          for (int g = 0; g < P; ++g) {
            c2& acc = o[6 * h + a][g];
            acc.re = fma2(mre2, pr[b2][g], acc.re);
            acc.re = fma2(nmim2, pi[b2][g], acc.re);
            acc.im = fma2(mre2, pi[b2][g], acc.im);
            acc.im = fma2(mim2, pr[b2][g], acc.im);
          }
        }
      }
    }
  }
#pragma unroll
  for (int d = 0; d < 2; ++d) {
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
#if !MRHS_DS_PRELOAD
      nb[d * 4 + mu] = __ldg(nbr + s * 8 + d * 4 + mu);
#endif
      const size_t n = (size_t)(nb[d * 4 + mu] & 0x3fffffff);
      const S* xn = x + n * 24 * N + r0;
      const float* Ul = U20 + ((d == 0 ? s : n) * 4 + mu) * 20;
      if (d == 0) {
        if (mu == 0) hop_f2<0, +1, P, NC, S>(o, xn, Nrt, Ul);
        if (mu == 1) hop_f2<1, +1, P, NC, S>(o, xn, Nrt, Ul);
        if (mu == 2) hop_f2<2, +1, P, NC, S>(o, xn, Nrt, Ul);
        if (mu == 3) hop_f2<3, +1, P, NC, S>(o, xn, Nrt, Ul);
      } else {
        if (mu == 0) hop_f2<0, -1, P, NC, S>(o, xn, Nrt, Ul);
        if (mu == 1) hop_f2<1, -1, P, NC, S>(o, xn, Nrt, Ul);
        if (mu == 2) hop_f2<2, -1, P, NC, S>(o, xn, Nrt, Ul);
        if (mu == 3) hop_f2<3, -1, P, NC, S>(o, xn, Nrt, Ul);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    S* yr = y + ((s * 12 + c) * 2 + 0) * N + r0;
    S* yi = y + ((s * 12 + c) * 2 + 1) * N + r0;
    if constexpr (P == 1) {
      stp(yr, o[c][0].re);
      stp(yi, o[c][0].im);
    } else {
      __stcs(reinterpret_cast<float4*>(yr), make_float4(o[c][0].re.x, o[c][0].re.y, o[c][1].re.x, o[c][1].re.y));
      __stcs(reinterpret_cast<float4*>(yi), make_float4(o[c][0].im.x, o[c][0].im.y, o[c][1].im.x, o[c][1].im.y));
    }
  }
}

// The right-hand sides are processed in `passes` sweeps over the lattice (a
// sweep over fewer right-hand sides keeps a larger part of the lattice in L2,
// at the price of reading links and clover once per sweep).
static int stencil_passes(int N, int G) {
  static int forced = [] {
    const char* e = getenv("MRHS_STENCIL_PASSES");
    return e ? atoi(e) : 0;
  }();
  int p = forced > 0 ? forced : 1;
  while (p > 1 && (N % p != 0 || (N / p) % G != 0)) --p;
  return p;
}

template <class S, int NC>
void launch_dslash_f2(mrhs_ctx c, const S* x, S* y, int N) {
  const int passes = stencil_passes(N, 2);
  const int nq = N / passes;
  const size_t work = (size_t)c->g.V * (nq / 2);
  for (int p = 0; p < passes; ++p)
    k_dslash_f2<S, 1, NC, MRHS_DS_MINB><<<grid_for(work, 128), 128, 0, c->stream>>>(x, y, c->U20, c->A32, c->nbr, N,
                                                                                  p * nq, nq, work);
}

template <class S>
void dslash_f2(mrhs_ctx c, const S* x, S* y, int N) {
  switch (N) {
    case 8: launch_dslash_f2<S, 8>(c, x, y, N); break;
    case 16: launch_dslash_f2<S, 16>(c, x, y, N); break;
    case 20: launch_dslash_f2<S, 20>(c, x, y, N); break;
    case 24: launch_dslash_f2<S, 24>(c, x, y, N); break;
    case 32: launch_dslash_f2<S, 32>(c, x, y, N); break;
    default: launch_dslash_f2<S, 0>(c, x, y, N); break;
  }
}

template <class S, class SB>
void dslash_t(mrhs_ctx c, const S* x, S* y, const SB* b, int N, int mode, const int* blist, int nblk) {
  using R = typename Real<S>::type;
  const cx<R>* U;
  const R* A;
  if constexpr (sizeof(R) == 8) {
    U = (const cx<R>*)c->U64;
    A = (const R*)c->A64;
  } else {
    U = (const cx<R>*)c->U32;
    A = (const R*)c->A32;
  }
  size_t nsites = blist ? (size_t)nblk * c->g.Va : (size_t)c->g.V;
  size_t work = nsites * N;
  const int bs = 128;
  Prof pr(c, mode == DS_FULL ? "dslash_full" : mode == DS_BLOCK ? "dslash_block" : "dslash_resid");
  switch (mode) {
    case DS_FULL:
      k_dslash<DS_FULL, S, SB, R><<<grid_for(work, bs), bs, 0, c->stream>>>(x, y, b, U, A, c->nbr, N, c->g.Va, blist, work);
      break;
    case DS_BLOCK:
      k_dslash<DS_BLOCK, S, SB, R><<<grid_for(work, bs), bs, 0, c->stream>>>(x, y, b, U, A, c->nbr, N, c->g.Va, blist, work);
      break;
    case DS_RESID:
      k_dslash<DS_RESID, S, SB, R><<<grid_for(work, bs), bs, 0, c->stream>>>(x, y, b, U, A, c->nbr, N, c->g.Va, blist, work);
      break;
  }
  MRHS_LAUNCH_CHECK("dslash");
}

template <class S>
void block_mr_t(mrhs_ctx c, S* x, S* rho, S* q, int N, const int* blist, int nblk, int n_mr) {
  using R = typename Real<S>::type;
  const cx<R>* U;
  const R* A;
  if constexpr (sizeof(R) == 8) {
    U = (const cx<R>*)c->U64;
    A = (const R*)c->A64;
  } else {
    U = (const cx<R>*)c->U32;
    A = (const R*)c->A32;
  }
  int bs = 256;
  if (N > bs) bs = ((N + 31) / 32) * 32;
  int lanes = bs / N;
  size_t smem = sizeof(double) * (3 * (size_t)lanes * N + 2 * N);
  Prof pr(c, "sap_block_mr");
  k_block_mr<S, R><<<nblk, bs, smem, c->stream>>>(x, rho, q, U, A, c->nbr, N, c->g.Va, blist, n_mr);
  MRHS_LAUNCH_CHECK("block_mr");
}

// the even-odd domain solves of one colour: r the colour's residual, work
// fields ru, q, e of the same size
template <class S>
void block_mr_eo_t(mrhs_ctx c, S* x, const S* r, S* ru, S* q, S* e, int N, const int* blist, int nblk, int n_mr) {
  using R = typename Real<S>::type;
  const cx<R>* U;
  const R *A, *Ainv;
  if constexpr (sizeof(R) == 8) {
    U = (const cx<R>*)c->U64;
    A = (const R*)c->A64;
    Ainv = (const R*)c->Ainv64;
  } else {
    U = (const cx<R>*)c->U32;
    A = (const R*)c->A32;
    Ainv = (const R*)c->Ainv32;
  }
  int bs = 256;
  if (N > bs) bs = ((N + 31) / 32) * 32;
  int lanes = bs / N;
  size_t smem = sizeof(double) * (3 * (size_t)lanes * N + 2 * N);
  EoGeom g;
  for (int m = 0; m < 4; ++m) g.a[m] = c->g.a[m], g.nb[m] = c->g.nb[m];
  Prof pr(c, "sap_block_mr_eo");
  k_block_mr_eo<S, R><<<nblk, bs, smem, c->stream>>>(x, r, ru, q, e, U, A, Ainv, c->nbr, N, c->g.Va, blist, n_mr, g);
  MRHS_LAUNCH_CHECK("block_mr_eo");
}

}  // namespace

void dslash(mrhs_ctx c, const void* x, void* y, const void* b, int nrhs, int dtype, int mode, int colour) {
  MRHS_REQUIRE(c->have_clover, MRHS_ERR_STATE, "operator used before mrhs_build_clover");
  MRHS_REQUIRE(nrhs >= 1, MRHS_ERR_ARG, "nrhs must be >= 1");
  // FP32 arithmetic, even nrhs: the packed-pair kernel for FP32, bf16 and
  // fp16 storage (an odd count and FP64 take the generic one)
  if (dtype != MRHS_F64 && mode == DS_FULL && colour < 0 && c->U20 && nrhs % 2 == 0) {
    Prof pr(c, "dslash_full");
    if (dtype == MRHS_F32) dslash_f2(c, (const float*)x, (float*)y, nrhs);
    else if (dtype == MRHS_BF16) dslash_f2(c, (const __nv_bfloat16*)x, (__nv_bfloat16*)y, nrhs);
    else dslash_f2(c, (const __half*)x, (__half*)y, nrhs);
    MRHS_LAUNCH_CHECK("dslash_f2");
    return;
  }
  const int* blist = nullptr;
  int nblk = 0;
  if (colour >= 0) {
    blist = c->blocks_col + (colour ? c->ncol[0] : 0);
    nblk = c->ncol[colour];
  }
  MRHS_DISPATCH(dtype, S, (dslash_t<S, S>(c, (const S*)x, (S*)y, (const S*)b, nrhs, mode, blist, nblk)));
}

// residual with a right-hand side b stored in a different type than x
static void resid_mixed(mrhs_ctx c, const void* x, void* y, const void* b, int bdtype, int N, int dtype, int colour) {
  const int* blist = c->blocks_col + (colour ? c->ncol[0] : 0);
  int nblk = c->ncol[colour];
  if (dtype == MRHS_F64) {
    MRHS_REQUIRE(bdtype == MRHS_F64, MRHS_ERR_ARG, "F64 smoother needs an F64 right-hand side");
    dslash_t<double, double>(c, (const double*)x, (double*)y, (const double*)b, N, DS_RESID, blist, nblk);
  } else {
    MRHS_REQUIRE(dtype == MRHS_F32, MRHS_ERR_ARG, "smoother work fields must be F64 or F32");
    MRHS_DISPATCH(bdtype, SB, (dslash_t<float, SB>(c, (const float*)x, (float*)y, (const SB*)b, N, DS_RESID, blist, nblk)));
  }
}

// SAP with b stored in bdtype (possibly reduced precision) and x in dtype
void sap_mixed(mrhs_ctx c, const void* b, int bdtype, void* x, int nrhs, int dtype, int n_sweeps, int n_mr, bool x0_zero) {
  MRHS_REQUIRE(c->have_clover, MRHS_ERR_STATE, "smoother used before mrhs_build_clover");
  MRHS_REQUIRE(n_sweeps >= 0 && n_mr >= 0 && nrhs >= 1, MRHS_ERR_ARG, "bad smoother parameters");
  if (c->even_odd) {
    // domain solves on the Schur complement of the even sites: residual
    // kernel + one CTA per domain (no on-chip form)
    ensure_clover_inverse(c);
    const size_t bytes = fine_elems(c, nrhs) * dtype_size(dtype);
    void* r = scratch(c, SC_R, bytes);
    void* ru = scratch(c, SC_EO1, bytes);
    char* qe = (char*)scratch(c, SC_EO2, 2 * bytes);
    for (int sw = 0; sw < n_sweeps; ++sw)
      for (int col = 0; col < 2; ++col) {
        resid_mixed(c, x, r, b, bdtype, nrhs, dtype, col);
        const int* blist = c->blocks_col + (col ? c->ncol[0] : 0);
        if (dtype == MRHS_F64)
          block_mr_eo_t<double>(c, (double*)x, (const double*)r, (double*)ru, (double*)qe, (double*)(qe + bytes),
                                nrhs, blist, c->ncol[col], n_mr);
        else
          block_mr_eo_t<float>(c, (float*)x, (const float*)r, (float*)ru, (float*)qe, (float*)(qe + bytes), nrhs,
                               blist, c->ncol[col], n_mr);
      }
    return;
  }
  if (sap_fused_ok(c, dtype)) {
    sap_fused(c, b, bdtype, x, nrhs, n_sweeps, n_mr, x0_zero);
    return;
  }
  size_t bytes = fine_elems(c, nrhs) * dtype_size(dtype);
  void* r = scratch(c, SC_R, bytes);
  void* q = scratch(c, SC_Q, bytes);
  for (int sw = 0; sw < n_sweeps; ++sw)
    for (int col = 0; col < 2; ++col) {
      resid_mixed(c, x, r, b, bdtype, nrhs, dtype, col);
      const int* blist = c->blocks_col + (col ? c->ncol[0] : 0);
      if (dtype == MRHS_F64) block_mr_t<double>(c, (double*)x, (double*)r, (double*)q, nrhs, blist, c->ncol[col], n_mr);
      else block_mr_t<float>(c, (float*)x, (float*)r, (float*)q, nrhs, blist, c->ncol[col], n_mr);
    }
}

void sap(mrhs_ctx c, const void* b, void* x, int nrhs, int dtype, int n_sweeps, int n_mr) {
  sap_mixed(c, b, dtype, x, nrhs, dtype, n_sweeps, n_mr);
}

}  // namespace mrhs

using namespace mrhs;

extern "C" {

int mrhs_apply_D(mrhs_ctx c, const void* x, void* y, int nrhs, int dtype) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && x && y, MRHS_ERR_ARG, "null argument");
    require_dev(c, x, "mrhs_apply_D x");
    require_dev(c, y, "mrhs_apply_D y");
    dslash(c, x, y, nullptr, nrhs, dtype, DS_FULL, -1);
  });
}

int mrhs_apply_D_block(mrhs_ctx c, const void* x, void* y, int nrhs, int dtype) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && x && y, MRHS_ERR_ARG, "null argument");
    require_dev(c, x, "mrhs_apply_D_block x");
    require_dev(c, y, "mrhs_apply_D_block y");
    dslash(c, x, y, nullptr, nrhs, dtype, DS_BLOCK, -1);
  });
}

int mrhs_set_smoother(mrhs_ctx c, int even_odd) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c, MRHS_ERR_ARG, "null context");
    MRHS_REQUIRE(even_odd == 0 || even_odd == 1, MRHS_ERR_ARG, "even_odd must be 0 or 1");
    c->even_odd = even_odd;
  });
}

int mrhs_sap(mrhs_ctx c, const void* b, void* x, int nrhs, int dtype, int n_sweeps, int n_mr) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && b && x, MRHS_ERR_ARG, "null argument");
    require_dev(c, b, "mrhs_sap b");
    require_dev(c, x, "mrhs_sap x");
    MRHS_REQUIRE(dtype == MRHS_F64 || dtype == MRHS_F32, MRHS_ERR_ARG, "smoother fields must be F64 or F32");
    sap(c, b, x, nrhs, dtype, n_sweeps, n_mr);
  });
}

}  // extern "C"
