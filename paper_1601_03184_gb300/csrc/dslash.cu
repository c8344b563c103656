// Multi-right-hand-side Wilson-clover stencil (full, block-restricted and
// residual forms) and the SAP smoother built on it.
#include "stencil.cuh"

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

}  // namespace

void dslash(mrhs_ctx c, const void* x, void* y, const void* b, int nrhs, int dtype, int mode, int colour) {
  MRHS_REQUIRE(c->have_clover, MRHS_ERR_STATE, "operator used before mrhs_build_clover");
  MRHS_REQUIRE(nrhs >= 1, MRHS_ERR_ARG, "nrhs must be >= 1");
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
void sap_mixed(mrhs_ctx c, const void* b, int bdtype, void* x, int nrhs, int dtype, int n_sweeps, int n_mr) {
  MRHS_REQUIRE(c->have_clover, MRHS_ERR_STATE, "smoother used before mrhs_build_clover");
  MRHS_REQUIRE(n_sweeps >= 0 && n_mr >= 0 && nrhs >= 1, MRHS_ERR_ARG, "bad smoother parameters");
  if (sap_fused_ok(c, dtype)) {
    sap_fused(c, b, bdtype, x, nrhs, n_sweeps, n_mr);
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
    dslash(c, x, y, nullptr, nrhs, dtype, DS_FULL, -1);
  });
}

int mrhs_apply_D_block(mrhs_ctx c, const void* x, void* y, int nrhs, int dtype) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && x && y, MRHS_ERR_ARG, "null argument");
    dslash(c, x, y, nullptr, nrhs, dtype, DS_BLOCK, -1);
  });
}

int mrhs_sap(mrhs_ctx c, const void* b, void* x, int nrhs, int dtype, int n_sweeps, int n_mr) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && b && x, MRHS_ERR_ARG, "null argument");
    MRHS_REQUIRE(dtype == MRHS_F64 || dtype == MRHS_F32, MRHS_ERR_ARG, "smoother fields must be F64 or F32");
    sap(c, b, x, nrhs, dtype, n_sweeps, n_mr);
  });
}

}  // extern "C"
