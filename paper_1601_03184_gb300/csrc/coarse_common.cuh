// Helpers shared by the coarse-operator kernels (ALU and tensor-core forms):
// aggregate face enumeration and the hop of one column of P.
#pragma once
#include "stencil.cuh"

namespace mrhs {

struct Agg4 {
  int a[4];
};

// local site index of face site f of an aggregate: l_mu fixed to lmu, the
// other three coordinates enumerated lexicographically
static __device__ __forceinline__ int face_site(const Agg4& g, int mu, int lmu, int f) {
  int l[4];
  for (int m = 0; m < 4; ++m) {
    if (m == mu) {
      l[m] = lmu;
    } else {
      l[m] = f % g.a[m];
      f /= g.a[m];
    }
  }
  return l[0] + g.a[0] * (l[1] + g.a[1] * (l[2] + g.a[2] * l[3]));
}

// column col = (h', j) of P: P_j restricted to chirality h', at site n
template <class SP, class R>
static __device__ __forceinline__ void load_pcol(cx<R> psi[12], const SP* P, int n, int Nt, int col) {
  const int hp = col / Nt, j = col % Nt;
#pragma unroll
  for (int c = 0; c < 12; ++c)
    psi[c] = (c / 6 == hp) ? ld<SP, R>(P, (size_t)n * 12 + c, Nt, j) : mk<R>(0, 0);
}

template <int MU, class SP, class R>
static __device__ __forceinline__ void hop_pcol(cx<R> out[12], const SP* P, const cx<R>* U, const int* nbr, int s, int dir,
                                         int Nt, int col, bool only_same_block, int Va) {
  int e = nbr[s * 8 + (dir > 0 ? 0 : 4) + MU];
  int n = e & 0x3fffffff;
  if (only_same_block && n / Va != s / Va) return;
  R sg = (e & 0x40000000) ? (R)-1 : (R)1;
  cx<R> psi[12];
  load_pcol<SP, R>(psi, P, n, Nt, col);
  if (dir > 0) hop_reg<MU, +1, R>(out, psi, U + (size_t)s * 36 + MU * 9, sg);
  else hop_reg<MU, -1, R>(out, psi, U + (size_t)n * 36 + MU * 9, sg);
}


// the same with the column's chirality HP known at compile time: the other
// chirality's components are constant zeros, so the clover term touches one
// 6x6 block and the spin projection of the hops folds away
template <int HP, class SP, class R>
static __device__ __forceinline__ void load_pcol_t(cx<R> psi[12], const SP* P, int n, int Nt, int j) {
#pragma unroll
  for (int c = 0; c < 12; ++c) psi[c] = (c / 6 == HP) ? ld<SP, R>(P, (size_t)n * 12 + c, Nt, j) : mk<R>(0, 0);
}

template <int MU, int HP, class SP, class R>
static __device__ __forceinline__ void hop_pcol_t(cx<R> out[12], const SP* P, const cx<R>* U, const int* nbr, int s,
                                                  int dir, int Nt, int j, int blk0, int Va, bool only_same_block) {
  const int e = nbr[s * 8 + (dir > 0 ? 0 : 4) + MU];
  const int n = e & 0x3fffffff;
  if (only_same_block && (unsigned)(n - blk0) >= (unsigned)Va) return;
  const R sg = (e & 0x40000000) ? (R)-1 : (R)1;
  cx<R> psi[12];
  load_pcol_t<HP, SP, R>(psi, P, n, Nt, j);
  if (dir > 0) hop_reg<MU, +1, R>(out, psi, U + (size_t)s * 36 + MU * 9, sg);
  else hop_reg<MU, -1, R>(out, psi, U + (size_t)n * 36 + MU * 9, sg);
}

// Y(x) = (D_k P_col)(x) for column col = (HP, j): k = 0 the aggregate-local
// operator (clover + hops inside the aggregate), k = 1+mu the hop from x+mu
template <int HP, class SP, class R>
static __device__ __forceinline__ void dk_pcol(cx<R> out[12], const SP* P, const cx<R>* U, const R* Acl,
                                               const int* nbr, int s, int k, int Nt, int j, int blk0, int Va) {
#pragma unroll
  for (int c = 0; c < 12; ++c) out[c] = mk<R>(0, 0);
  if (k == 0) {
    cx<R> psi[12];
    load_pcol_t<HP, SP, R>(psi, P, s, Nt, j);
    // A is block diagonal in chirality: only block HP meets a nonzero psi
    cx<R> blk[12];
    clover_apply_reg<R>(blk, psi, Acl + (size_t)s * 72);
#pragma unroll
    for (int c = 0; c < 6; ++c) out[6 * HP + c] = blk[6 * HP + c];
#pragma unroll
    for (int d = -1; d <= 1; d += 2) {
      hop_pcol_t<0, HP, SP, R>(out, P, U, nbr, s, d, Nt, j, blk0, Va, true);
      hop_pcol_t<1, HP, SP, R>(out, P, U, nbr, s, d, Nt, j, blk0, Va, true);
      hop_pcol_t<2, HP, SP, R>(out, P, U, nbr, s, d, Nt, j, blk0, Va, true);
      hop_pcol_t<3, HP, SP, R>(out, P, U, nbr, s, d, Nt, j, blk0, Va, true);
    }
  } else {
    switch (k - 1) {
      case 0: hop_pcol_t<0, HP, SP, R>(out, P, U, nbr, s, +1, Nt, j, blk0, Va, false); break;
      case 1: hop_pcol_t<1, HP, SP, R>(out, P, U, nbr, s, +1, Nt, j, blk0, Va, false); break;
      case 2: hop_pcol_t<2, HP, SP, R>(out, P, U, nbr, s, +1, Nt, j, blk0, Va, false); break;
      default: hop_pcol_t<3, HP, SP, R>(out, P, U, nbr, s, +1, Nt, j, blk0, Va, false); break;
    }
  }
}
}  // namespace mrhs
