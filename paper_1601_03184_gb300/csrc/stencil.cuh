// Device-side Wilson-clover building blocks shared by the stencil, the
// smoother and the coarse-operator assembly.
//
// D psi(x) = A(x) psi(x) - 1/2 sum_mu [(1-gamma_mu) U_mu(x) psi(x+mu)
//                                    + (1+gamma_mu) U_mu(x-mu)^dag psi(x-mu)]
// In the chiral basis gamma_mu = [[0, B_mu], [B_mu^dag, 0]] with
// B_{0,1,2} = -i sigma_{1,2,3}, B_3 = 1, so (1 -/+ gamma_mu) psi is fixed by
// the two-spin "half spinor" h = psi_up -/+ B psi_low:
//   (1 - gamma) psi = (h, -B^dag h),   (1 + gamma) psi = (h, +B^dag h).
// Only the half spinor is multiplied by the link (6 instead of 12 complex
// colour products per hop).
#pragma once

#include "common.cuh"

namespace mrhs {

template <class S, class R>
__device__ __forceinline__ cx<R> ld(const S* f, size_t row, int N, int r) {
  return mk<R>(to_r(f[fidx(row, 0, N, r)]), to_r(f[fidx(row, 1, N, r)]));
}
template <class S, class R>
__device__ __forceinline__ void st(S* f, size_t row, int N, int r, cx<R> v) {
  f[fidx(row, 0, N, r)] = from_r<S>(v.re);
  f[fidx(row, 1, N, r)] = from_r<S>(v.im);
}

// (B_mu psi_low)_s for s = 0, 1 ; psi_low = (p2, p3)
template <int MU, class R>
__device__ __forceinline__ void b_low(const cx<R>& p2, const cx<R>& p3, cx<R>& o0, cx<R>& o1) {
  if (MU == 0) { o0 = tmi(p3); o1 = tmi(p2); }
  if (MU == 1) { o0 = mk<R>(-p3.re, -p3.im); o1 = p2; }
  if (MU == 2) { o0 = tmi(p2); o1 = ti(p3); }
  if (MU == 3) { o0 = p2; o1 = p3; }
}
// (B_mu^dag chi)_s for s = 0, 1
template <int MU, class R>
__device__ __forceinline__ void bdag(const cx<R>& c0, const cx<R>& c1, cx<R>& o0, cx<R>& o1) {
  if (MU == 0) { o0 = ti(c1); o1 = ti(c0); }
  if (MU == 1) { o0 = c1; o1 = mk<R>(-c0.re, -c0.im); }
  if (MU == 2) { o0 = ti(c0); o1 = tmi(c1); }
  if (MU == 3) { o0 = c0; o1 = c1; }
}

// out += hop term of direction MU, DIR (+1 forward, -1 backward) for the
// neighbour spinor psi with link Ul (U_mu(x) forward, U_mu(x-mu) backward,
// applied as dagger), sign sg (-1 across the t boundary)
template <int MU, int DIR, class R>
__device__ __forceinline__ void hop_reg_u(cx<R> out[12], const cx<R> psi[12], const cx<R> u[3][3], R sg) {
  cx<R> h[2][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cx<R> p0 = psi[c];
    cx<R> p1 = psi[3 + c];
    cx<R> p2 = psi[6 + c];
    cx<R> p3 = psi[9 + c];
    cx<R> b0, b1;
    b_low<MU>(p2, p3, b0, b1);
    if (DIR > 0) { h[0][c] = p0 - b0; h[1][c] = p1 - b1; }
    else { h[0][c] = p0 + b0; h[1][c] = p1 + b1; }
  }
  cx<R> ch[2][3];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cx<R> acc = mk<R>(0, 0);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (DIR > 0) fma_(acc, u[a][b], h[s][b]);
        else fmac_(acc, u[b][a], h[s][b]);
      }
      ch[s][a] = scale(acc, sg * (R)0.5);
    }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cx<R> l0, l1;
    bdag<MU>(ch[0][a], ch[1][a], l0, l1);
    out[a] = out[a] - ch[0][a];
    out[3 + a] = out[3 + a] - ch[1][a];
    if (DIR > 0) { out[6 + a] = out[6 + a] + l0; out[9 + a] = out[9 + a] + l1; }
    else { out[6 + a] = out[6 + a] - l0; out[9 + a] = out[9 + a] - l1; }
  }
}

template <int MU, int DIR, class R>
__device__ __forceinline__ void hop_reg(cx<R> out[12], const cx<R> psi[12], const cx<R>* Ul, R sg) {
  cx<R> u[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) u[a][b] = Ul[a * 3 + b];
  hop_reg_u<MU, DIR, R>(out, psi, u, sg);
}

// the same, loading the neighbour spinor at row base nrow (= n*12)
template <int MU, int DIR, class S, class R>
__device__ __forceinline__ void hop(cx<R> out[12], const S* x, size_t nrow, int N, int r, const cx<R>* Ul, R sg) {
  cx<R> psi[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) psi[c] = ld<S, R>(x, nrow + c, N, r);
  hop_reg<MU, DIR, R>(out, psi, Ul, sg);
}

__device__ __forceinline__ int herm_idx(int a, int b) { return 6 + 2 * (5 * a - a * (a - 1) / 2 + (b - a - 1)); }

// out = A(x) psi(x), A packed per chirality (6 diagonals, 15 upper entries)
template <class R>
__device__ __forceinline__ void clover_apply_reg(cx<R> out[12], const cx<R> psi[12], const R* Ap) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const cx<R>* p = psi + 6 * h;
    const R* q = Ap + 36 * h;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      cx<R> acc = scale(p[a], q[a]);
#pragma unroll
      for (int b = 0; b < 6; ++b) {
        if (b == a) continue;
        cx<R> m = b > a ? mk<R>(q[herm_idx(a, b)], q[herm_idx(a, b) + 1])
                        : mk<R>(q[herm_idx(b, a)], -q[herm_idx(b, a) + 1]);
        fma_(acc, m, p[b]);
      }
      out[6 * h + a] = acc;
    }
  }
}

template <class S, class R>
__device__ __forceinline__ void clover_apply(cx<R> out[12], const S* x, size_t row, int N, int r, const R* Ap) {
  cx<R> psi[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) psi[c] = ld<S, R>(x, row + c, N, r);
  clover_apply_reg<R>(out, psi, Ap);
}

// D (BLOCK = false) or D_B (BLOCK = true) at device site s, right-hand side r
// CLOVER = false: the hopping terms alone (out starts at zero; A unused)
template <bool BLOCK, class S, class R, bool CLOVER = true>
__device__ __forceinline__ void dslash_site(cx<R> out[12], const S* x, int s, int N, int r, const cx<R>* U,
                                            const R* A, const int* nbr, int Va) {
  if constexpr (CLOVER) {
    clover_apply<S, R>(out, x, (size_t)s * 12, N, r, A + (size_t)s * 72);
  } else {
#pragma unroll
    for (int c = 0; c < 12; ++c) out[c] = mk<R>(0, 0);
  }
  const int blk = s / Va;
  const cx<R>* Us = U + (size_t)s * 36;
#define MRHS_HOP(MU)                                                                                   \
  {                                                                                                    \
    int e = nbr[s * 8 + MU];                                                                           \
    int n = e & 0x3fffffff;                                                                            \
    if (!BLOCK || n / Va == blk)                                                                       \
      hop<MU, +1, S, R>(out, x, (size_t)n * 12, N, r, Us + MU * 9, (e & 0x40000000) ? (R)-1 : (R)1);  \
    e = nbr[s * 8 + 4 + MU];                                                                           \
    n = e & 0x3fffffff;                                                                                \
    if (!BLOCK || n / Va == blk)                                                                       \
      hop<MU, -1, S, R>(out, x, (size_t)n * 12, N, r, U + (size_t)n * 36 + MU * 9,                     \
                        (e & 0x40000000) ? (R)-1 : (R)1);                                              \
  }
  MRHS_HOP(0)
  MRHS_HOP(1)
  MRHS_HOP(2)
  MRHS_HOP(3)
#undef MRHS_HOP
}

// Packed pairs of right-hand sides (FP32): a float2 holds one real component
// of two neighbouring right-hand sides and every arithmetic step is one
// fma/add/mul .rn.f32x2 instruction doing the work of two. The rounding is
// per lane, so a packed kernel that performs the scalar operations in the
// same order gives the same bits. Link and clover entries are broadcast
// into both lanes.
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b, exactly rounded like the scalar subtraction (one fused step)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

struct c2 {
  float2 re, im;
};
__device__ __forceinline__ c2 mk2(float2 re, float2 im) {
  c2 r;
  r.re = re;
  r.im = im;
  return r;
}
__device__ __forceinline__ c2 operator+(c2 a, c2 b) { return mk2(add2(a.re, b.re), add2(a.im, b.im)); }
__device__ __forceinline__ c2 operator-(c2 a, c2 b) { return mk2(sub2(a.re, b.re), sub2(a.im, b.im)); }
template <int SG>
__device__ __forceinline__ float2 pm2(float2 a, float2 b) {
  return SG > 0 ? add2(a, b) : sub2(a, b);
}
// a + SG i^K x (K = 0..3): the phase only selects components and signs
template <int K, int SG>
__device__ __forceinline__ c2 axpy_ph(c2 a, c2 x) {
  constexpr int sre = (K == 0 || K == 3) ? SG : -SG;
  constexpr int sim = (K == 0 || K == 1) ? SG : -SG;
  return mk2(pm2<sre>(a.re, (K & 1) ? x.im : x.re), pm2<sim>(a.im, (K & 1) ? x.re : x.im));
}

// The chiral-basis B_mu (B psi_low) and B_mu^dag as (phase i^K, source spin):
// (B psi_low)_s = i^KB0 psi_{SB0}, ... with psi_low = (psi_2, psi_3), and
// (B^dag chi)_s = i^KD0 chi_{SD0}, ... with chi = (chi_0, chi_1).
template <int MU>
struct BTab {
  static constexpr int KB0 = MU == 0 ? 3 : MU == 1 ? 2 : MU == 2 ? 3 : 0;
  static constexpr int SB0 = MU == 0 ? 3 : MU == 1 ? 3 : 2;
  static constexpr int KB1 = MU == 0 ? 3 : MU == 1 ? 0 : MU == 2 ? 1 : 0;
  static constexpr int SB1 = MU == 0 ? 2 : MU == 1 ? 2 : 3;
  static constexpr int KD0 = MU == 0 ? 1 : MU == 1 ? 0 : MU == 2 ? 1 : 0;
  static constexpr int SD0 = MU == 0 ? 1 : MU == 1 ? 1 : 0;
  static constexpr int KD1 = MU == 0 ? 1 : MU == 1 ? 2 : MU == 2 ? 3 : 0;
  static constexpr int SD1 = MU == 0 ? 0 : MU == 1 ? 0 : 1;
};

}  // namespace mrhs
