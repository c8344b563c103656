// Coarse-operator contraction D_c[A,k] = P_A^dag (D_k P) on the fifth-
// generation tensor cores (tcgen05), for the mixed-precision setup: the
// link products are dense 2N_tv x 2N_tv blocks (Sec. 2 of the paper builds
// D_c from P = R^dag; D_c = P^dag D P with the aggregate-local structure of P).
//
// One CTA per (aggregate A, k in 0..4): k = 0 the self block, k = 1+mu the
// forward block towards A+mu. Sites of the block (all of A for k = 0, the +mu
// face for k > 0) are taken in chunks of Q. For each chunk
//   B[n][kk]: Y = D_k P evaluated by the CUDA cores (one (site, column) per
//             thread, FP32), n = (re/im part, column), kk = (site, component);
//   A[m][kk]: P, m = (re/im part, row (h, i)), zero where the component's
//             chirality is not h;
// and one elected thread issues the MMAs D += A B^T (M = 128, N = 2*2N_tv
// rounded up to 16, FP32 accumulation in tensor memory). With
// D[(p,i)][(p',j)] = sum Re/Im(P) Re/Im(Y), the coarse entry is
//   Re C[i][j] = D[(0,i)][(0,j)] + D[(1,i)][(1,j)],
//   Im C[i][j] = D[(0,i)][(1,j)] - D[(1,i)][(0,j)]    (C = P^dag Y).
// The operand buffers are double-buffered: the CUDA cores fill chunk t+1
// while the tensor core multiplies chunk t. Operands are bf16 or fp16
// (kind::f16) or tf32 (kind::tf32); P is exact in each of them when it is
// stored in that precision or in fp16.
#include "coarse_common.cuh"
#include "tc.cuh"

#include <algorithm>
#include <cstdlib>
#include <string>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace mrhs {
namespace {

constexpr int kThreads = 256;
constexpr int kRows = 128;          // M of the MMA, and rows of both operand tiles
constexpr int kKG = 12;             // 16-byte K groups per chunk (both element widths)
constexpr int kTileBytes = kRows / 8 * kKG * 128;  // 24 KB
constexpr uint32_t kWaitLimit = 1u << 20;

// operand element formats
template <int FMT>
struct Elem;
template <>
struct Elem<tc::kFmtBF16> {
  static constexpr int size = 2;
  static __device__ __forceinline__ uint32_t pack(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
  }
};
template <>
struct Elem<tc::kFmtF16> {
  static constexpr int size = 2;
  static __device__ __forceinline__ uint32_t pack(float a, float b) {
    __half2 v = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
  }
};
template <>
struct Elem<tc::kFmtTF32> {
  static constexpr int size = 4;
  static __device__ __forceinline__ uint32_t one(float a) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(a));
    return r;
  }
};

using tc::tf32_split;

// store the pair of elements (row, k), (row, k+1), k even, of a K-major tile
template <int FMT>
__device__ __forceinline__ void put2(unsigned char* tile, int row, int k, float a, float b, int kg = kKG) {
  using E = Elem<FMT>;
  const uint32_t off = tc::kmajor_offset(row, k, E::size, kg);
  if constexpr (E::size == 2) {
    *reinterpret_cast<uint32_t*>(tile + off) = E::pack(a, b);
  } else {
    *reinterpret_cast<uint2*>(tile + off) = make_uint2(E::one(a), E::one(b));
  }
}

// the same for split tf32: v = hi + lo, hi into one tile and lo into the other
__device__ __forceinline__ void put2_split(unsigned char* thi, unsigned char* tlo, int row, int k, float a, float b,
                                           int kg) {
  const uint32_t off = tc::kmajor_offset(row, k, 4, kg);
  uint32_t ha, la, hb, lb;
  tf32_split(a, ha, la);
  tf32_split(b, hb, lb);
  *reinterpret_cast<uint2*>(thi + off) = make_uint2(ha, hb);
  *reinterpret_cast<uint2*>(tlo + off) = make_uint2(la, lb);
}

template <int FMT, class SP, bool SPLIT>
__global__ void __launch_bounds__(kThreads) k_coarse_op_tc(const SP* __restrict__ P, const cx<float>* __restrict__ U,
                                                           const float* __restrict__ Acl, const int* __restrict__ nbr,
                                                           int Nt, Agg4 ag, int Va, cx<float>* __restrict__ Dc,
                                                           int* __restrict__ err) {
  constexpr int ES = Elem<FMT>::size;
  // 16-byte K groups per chunk: 12. Split tf32 keeps one stage of four tiles
  // (96 KB, two CTAs per SM): its chunk waits for the previous chunk's MMAs
  // before it overwrites the operands, which cost less than the chunks of
  // half the size that two stages would leave room for
  constexpr int KGT = kKG;
  constexpr bool ONE = SPLIT;                  // a single stage
  constexpr int TB = kRows / 8 * KGT * 128;    // bytes of one tile
  constexpr int Q = KGT * 16 / ES / 12;        // sites per chunk: 8 (2-byte), 4 (tf32), 2 (split tf32)
  constexpr int KSTEP_BYTES = 256;            // two core matrices along K per MMA
  extern __shared__ __align__(1024) unsigned char smem[];
  // stage st: A tile at smem + 2*st*kTileBytes, B tile right after it
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_bad;

  const int A = blockIdx.x / 5, k = blockIdx.x % 5;
  const int nc = 2 * Nt;
  const int NN = (2 * nc + 15) / 16 * 16;     // MMA N
  const int mu = k - 1;
  const int nsite = k == 0 ? Va : Va / ag.a[mu];
  const int lmu = k == 0 ? 0 : ag.a[mu] - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // zero both stages once: padding rows and off-chirality entries of A stay zero
  constexpr int NT = SPLIT ? 4 : 2;  // tiles per stage: A, B (and their low parts)
  for (int i = threadIdx.x; i < (ONE ? 1 : 2) * NT * TB / 16; i += kThreads)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::fence_mbar_init();
    s_bad = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(&s_tmem, 256);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  // R (columns 0..127): the MMAs of one chunk; S (128..255): the sum of the
  // chunks, kept by the CUDA cores (warp w: lanes 32 (w % 4).., columns
  // 64 (w / 4)..)
  const uint32_t tbase = s_tmem;
  const uint32_t t_own = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * (warp >> 2));
  const int own_cols = max(0, min(64, NN - 64 * (warp >> 2)));
  {
    float z[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) z[i] = 0.f;
    for (int c0 = 0; c0 < own_cols; c0 += 16) tc::tmem_st16(t_own + 128 + c0, z);
    tc::tmem_wait_st();
  }
  const uint32_t idesc = tc::instr_desc(FMT, FMT, kRows, NN);

  const int nchunk = (nsite + Q - 1) / Q;
  int issued = 0;
  for (int t = 0; t < nchunk; ++t) {
    const int st = ONE ? 0 : t & 1;
    // stage st was last read by the MMAs of chunk t-2 (two stages), complete
    // since the previous iteration waited for chunk t-1; with one stage, wait
    // for chunk t-1 here and fold its partial sum before the operands change
    if (ONE && t >= 1) {
      if (!tc::mbar_wait(&mbar[0], (t - 1) & 1, kWaitLimit)) s_bad = 1;
      tc::fence_after_sync();
      tc::tmem_promote(t_own + 128, t_own, own_cols);
      tc::tmem_wait_st();
      tc::fence_before_sync();
      __syncthreads();
    }
    if (s_bad) break;
    const int q0 = t * Q;
    const int nq = min(Q, nsite - q0);
    unsigned char* tA = smem + NT * st * TB;
    unsigned char* tB = tA + TB;
    unsigned char* tAl = tA + 2 * TB;  // low parts (SPLIT)
    unsigned char* tBl = tA + 3 * TB;
    // B: Y = D_k P for (site q, column col); absent sites of a ragged chunk give zeros
    for (int w = threadIdx.x; w < Q * nc; w += kThreads) {
      const int q = w / nc, col = w % nc;
      cx<float> out[12];
#pragma unroll
      for (int c = 0; c < 12; ++c) out[c] = mk<float>(0, 0);
      if (q < nq) {
        const int l = k == 0 ? q0 + q : face_site(ag, mu, lmu, q0 + q);
        const int s = A * Va + l;
        if (col < Nt) dk_pcol<0, SP, float>(out, P, U, Acl, nbr, s, k, Nt, col, A * Va, Va);
        else dk_pcol<1, SP, float>(out, P, U, Acl, nbr, s, k, Nt, col - Nt, A * Va, Va);
      }
#pragma unroll
      for (int c = 0; c < 12; c += 2) {
        if constexpr (SPLIT) {
          put2_split(tB, tBl, col, q * 12 + c, out[c].re, out[c + 1].re, KGT);
          put2_split(tB, tBl, nc + col, q * 12 + c, out[c].im, out[c + 1].im, KGT);
        } else {
          put2<FMT>(tB, col, q * 12 + c, out[c].re, out[c + 1].re);
          put2<FMT>(tB, nc + col, q * 12 + c, out[c].im, out[c + 1].im);
        }
      }
    }
    // A: P rows (part p, h, j) for the components of chirality h
    for (int w = threadIdx.x; w < nq * 12 * Nt; w += kThreads) {
      const int j = w % Nt;
      int rest = w / Nt;
      const int p = rest % 2;
      rest /= 2;
      const int cp = rest % 3;
      rest /= 3;
      const int h = rest % 2;
      const int q = rest / 2;
      const int c = 6 * h + 2 * cp;
      const int l = k == 0 ? q0 + q : face_site(ag, mu, lmu, q0 + q);
      const size_t s = (size_t)A * Va + l;
      const float a = to_r(P[((s * 12 + c) * 2 + p) * Nt + j]);
      const float b = to_r(P[((s * 12 + c + 1) * 2 + p) * Nt + j]);
      if constexpr (SPLIT) put2_split(tA, tAl, p * nc + h * Nt + j, q * 12 + c, a, b, KGT);
      else put2<FMT>(tA, p * nc + h * Nt + j, q * 12 + c, a, b);
    }
    tc::fence_async_smem();
    // chunk t-1 done: fold its partial sum R into S before R is reused
    if (!ONE && t >= 1) {
      if (!tc::mbar_wait(&mbar[0], (t - 1) & 1, kWaitLimit)) s_bad = 1;
      tc::fence_after_sync();
      tc::tmem_promote(t_own + 128, t_own, own_cols);
      tc::tmem_wait_st();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (s_bad) break;
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(tA), b0 = tc::smem_u32(tB);
      const uint32_t a1 = tc::smem_u32(tAl), b1 = tc::smem_u32(tBl);
#pragma unroll
      for (int ks = 0; ks < KGT / 2; ++ks) {
        const uint64_t ad = tc::smem_desc(a0 + ks * KSTEP_BYTES, 128, KGT * 128);
        const uint64_t bd = tc::smem_desc(b0 + ks * KSTEP_BYTES, 128, KGT * 128);
        if constexpr (FMT == tc::kFmtTF32) {
          tc::mma_tf32(tbase, ad, bd, idesc, ks > 0 ? 1u : 0u);
          if constexpr (SPLIT) {
            tc::mma_tf32(tbase, ad, tc::smem_desc(b1 + ks * KSTEP_BYTES, 128, KGT * 128), idesc, 1u);
            tc::mma_tf32(tbase, tc::smem_desc(a1 + ks * KSTEP_BYTES, 128, KGT * 128), bd, idesc, 1u);
          }
        } else {
          tc::mma_f16(tbase, ad, bd, idesc, ks > 0 ? 1u : 0u);
        }
      }
      tc::mma_commit(&mbar[0]);
    }
    issued = t + 1;
  }
  // the last chunk: wait, fold into S
  if (issued > 0) {
    if (!tc::mbar_wait(&mbar[0], (issued - 1) & 1, kWaitLimit)) s_bad = 1;
    tc::fence_after_sync();
    tc::tmem_promote(t_own + 128, t_own, own_cols);
    tc::tmem_wait_st();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const bool ok = !s_bad && issued == nchunk;
  if (ok) {
    // the sum S -> shared memory (stage buffers are free now)
    float* E = reinterpret_cast<float*>(smem);  // [128][NN + 1]
    const int quarter = warp & 3, half = warp >> 2;
    for (int col0 = half * 64; col0 < min(NN, half * 64 + 64); col0 += 16) {
      float v[16];
      tc::tmem_ld16(tbase + ((uint32_t)(quarter * 32) << 16) + 128u + (uint32_t)col0, v);
      const int row = quarter * 32 + lane;
#pragma unroll
      for (int i = 0; i < 16; ++i) E[row * (NN + 1) + col0 + i] = v[i];
    }
    __syncthreads();
    cx<float>* out = Dc + ((size_t)A * 9 + k) * nc * nc;
    for (int e = threadIdx.x; e < nc * nc; e += kThreads) {
      const int i = e / nc, j = e % nc;
      const float re = E[i * (NN + 1) + j] + E[(nc + i) * (NN + 1) + nc + j];
      const float im = E[i * (NN + 1) + nc + j] - E[(nc + i) * (NN + 1) + j];
      out[e] = mk<float>(re, im);
    }
  } else if (threadIdx.x == 0) {
    atomicExch(err, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 256);
}

// ---------------------------------------------------------------------------
// Coarse stencil y_c(A) = sum_k D_c[A,k] x_c(nbr_k(A)) on the tensor cores.
// One CTA per aggregate A. With nc = 2 N_tv coarse rows and n right-hand
// sides, per block k:
//   A operand (M = 128): rows m < nc the real parts Dr[m][kk] of D_c[A,k],
//             rows nc <= m < 2nc the imaginary parts Di, K = kk the columns;
//   B operand (N = 2n): rows (p, r) = Re/Im of x_c(B_k)[kk][r], K = kk;
//   D[m][(p,r)] accumulates over the nine blocks in tensor memory, and
//   Re y = D[i][(0,r)] - D[nc+i][(1,r)],  Im y = D[i][(1,r)] + D[nc+i][(0,r)].
// SPLIT: every FP32 operand v is split into tf32 parts v = hi + lo and the
// product is hi*hi + hi*lo + lo*hi (the three-pass TF32 scheme; the dropped
// lo*lo term is below 2^-21 of the product), which keeps the result at FP32
// accuracy; without SPLIT the operands are rounded to tf32 once.
// The global loads of block k+1 are issued before the MMAs of block k are
// waited for; two CTAs share an SM.
constexpr int kDcThreads = 512;  // 16 warps: the operand conversion is the CUDA cores' share

// A part of the stencil (the even-odd coarse solve): CTA b takes aggregate
// alist[b] (b without a list) and the blocks kb <= k < ke; block 0 reads x0,
// the hop blocks xh, the row block of aggregate B at pos[B] (B without pos);
// y (plus add, when given) is written at row block b.
template <bool SPLIT, bool PRE>
__global__ void __launch_bounds__(kDcThreads, 1) k_apply_dc_tc(const float* __restrict__ Dc,
                                                               const float* __restrict__ x0,
                                                               const float* __restrict__ xh, float* __restrict__ y,
                                                               const int* __restrict__ aggnbr, int nc, int nrhs,
                                                               uint32_t tm_cols, int* __restrict__ err,
                                                               const int* __restrict__ alist,
                                                               const int* __restrict__ pos, int kb, int ke,
                                                               const float* __restrict__ add) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t full[2], mma_done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_bad;
  const int A = alist ? alist[blockIdx.x] : (int)blockIdx.x;
  const int nk = ke - kb;                    // blocks of this launch (at least 1)
  const int NM = 2 * nrhs;                   // MMA N
  const int KG = nc / 4;                     // 16-byte K groups (tf32)
  const int a_bytes = kRows / 8 * KG * 128;  // A tile
  const int b_bytes = NM / 8 * KG * 128;     // B tile
  const uint32_t d_bytes = (uint32_t)nc * nc * 8, x_bytes = (uint32_t)nc * 2 * nrhs * 4;
  // PRE: the stage holds the block's ready operand images (hi, then lo) in
  // place of the FP32 block, and the MMAs read A from the stage itself
  const uint32_t img_bytes = (SPLIT ? 2 : 1) * (uint32_t)a_bytes;
  const uint32_t x_off = PRE ? img_bytes : d_bytes;  // the x block inside a stage
  const uint32_t raw_bytes = (x_off + x_bytes + 1023) & ~1023u;
  unsigned char* raw0 = smem;                      // stage s: D block (or its images), then the x block
  unsigned char* Ahi = smem + 2 * raw_bytes;       // (not PRE)
  unsigned char* Bhi = PRE ? Ahi : Ahi + a_bytes;
  unsigned char* Alo = Bhi + b_bytes;              // (not PRE)
  unsigned char* Blo = PRE ? Bhi + b_bytes : Alo + a_bytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (!PRE && 2 * nc < kRows) {  // rows of A beyond 2nc stay zero
    const int nz = (SPLIT ? 2 : 1) * (a_bytes + b_bytes) / 16;
    for (int i = tid; i < nz; i += kDcThreads) reinterpret_cast<uint4*>(Ahi)[i] = make_uint4(0, 0, 0, 0);
  }
  if (tid == 0) {
    tc::mbar_init(&full[0], 1);
    tc::mbar_init(&full[1], 1);
    tc::mbar_init(&mma_done, 1);
    tc::fence_mbar_init();
    s_bad = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(&s_tmem, tm_cols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  // R (columns 0..NM-1): the MMAs of one block k; S (NM..2NM-1): the sum over
  // the blocks, kept by the CUDA cores (warp w: lanes 32 (w % 4).., columns
  // (NM/2) (w / 4)..)
  const uint32_t tbase = s_tmem;
  // column slices of 16 (or more) per warp group: warp w takes lanes
  // 32 (w % 4).. and slice w / 4 (warp groups beyond the slices idle here)
  const int nslice = min(kDcThreads / 128, NM / 16);
  const int sw = NM / nslice;                              // columns per slice
  const int slice = warp >> 2;
  const int own = slice < nslice ? sw : 0;
  const uint32_t t_own = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(sw * min(slice, nslice - 1));
  {
    float z[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) z[i] = 0.f;
    for (int c0 = 0; c0 < own; c0 += 16) tc::tmem_st16(t_own + NM + c0, z);
    tc::tmem_wait_st();
  }
  const uint32_t idesc = tc::instr_desc(tc::kFmtTF32, tc::kFmtTF32, kRows, NM);

  // step j: block k = kb + j of the stencil, D_c[A][k] and x_c of its
  // aggregate, one bulk copy each
  auto fetch = [&](int j) {
    const int k = kb + j;
    unsigned char* raw = raw0 + (j & 1) * raw_bytes;
    const int B = k == 0 ? A : aggnbr[A * 8 + k - 1];
    const float* xs = k == 0 ? x0 : xh;
    const int rb = pos ? pos[B] : B;
    tc::mbar_expect_tx(&full[j & 1], x_off + x_bytes);
    if (PRE)
      tc::bulk_g2s(raw, reinterpret_cast<const unsigned char*>(Dc) + ((size_t)A * 9 + k) * img_bytes, img_bytes,
                   &full[j & 1]);
    else
      tc::bulk_g2s(raw, Dc + ((size_t)A * 9 + k) * nc * nc * 2, d_bytes, &full[j & 1]);
    tc::bulk_g2s(raw + x_off, xs + (size_t)rb * nc * 2 * nrhs, x_bytes, &full[j & 1]);
  };
  if (tid == 0) {
    fetch(0);
    if (nk > 1) fetch(1);
  }
  int issued = 0;
  for (int j = 0; j < nk; ++j) {
    const unsigned char* raw = raw0 + (j & 1) * raw_bytes;
    bool ok = tc::mbar_wait(&full[j & 1], (j >> 1) & 1, kWaitLimit);
    if (j >= 1) {
      // step j-1 done: fold its partial sum R into S before R is reused
      ok = ok && tc::mbar_wait(&mma_done, (j - 1) & 1, kWaitLimit);
      tc::fence_after_sync();
      tc::tmem_promote(t_own + NM, t_own, own);  // warp-wide; a failed wait discards the result
      tc::tmem_wait_st();
      // PRE: the MMAs of step j-1 are done with its stage, which takes step j+1
      if (PRE && tid == 0 && ok && j + 1 < nk) fetch(j + 1);
    }
    if (!ok) s_bad = 1;
    tc::fence_before_sync();
    __syncthreads();
    if (s_bad) break;
    // A: 16-byte chunks q (two complex columns) of 8 rows per warp pass; lane
    // (r, qq) takes chunk 8 qq + ((r + t) & 7) of row r, so that the eight
    // lanes of a row group hit eight different bank groups
    if (!PRE) {
      const float4* D4 = reinterpret_cast<const float4*>(raw);
      const int r = lane & 7, qq = lane >> 3;
      for (int pass = warp; pass < (nc / 8) * 8; pass += kDcThreads / 32) {
        const int g8 = pass >> 3, t = pass & 7;
        const int q = qq * 8 + ((r + t) & 7);
        if (q < nc / 2) {
          const int row = 8 * g8 + r, col = 2 * q;
          const float4 v = D4[(row * nc + col) / 2];
          const uint32_t offr = tc::kmajor_offset(row, col, 4, KG), offi = tc::kmajor_offset(nc + row, col, 4, KG);
          uint32_t h0, l0, h1, l1, h2, l2, h3, l3;
          tf32_split(v.x, h0, l0);  // Re D[row][col]
          tf32_split(v.y, h1, l1);  // Im D[row][col]
          tf32_split(v.z, h2, l2);  // Re D[row][col+1]
          tf32_split(v.w, h3, l3);  // Im D[row][col+1]
          *reinterpret_cast<uint2*>(Ahi + offr) = make_uint2(h0, h2);
          *reinterpret_cast<uint2*>(Ahi + offi) = make_uint2(h1, h3);
          if (SPLIT) {
            *reinterpret_cast<uint2*>(Alo + offr) = make_uint2(l0, l2);
            *reinterpret_cast<uint2*>(Alo + offi) = make_uint2(l1, l3);
          }
        }
      }
    }
    // B: one 16-byte core row (row n = (p, r), K group kq) per unit, from four
    // rows (kk, p) of the x block
    {
      const float* X = reinterpret_cast<const float*>(raw + x_off);
      for (int u = tid; u < NM * KG; u += kDcThreads) {
        const int n = u % NM, kq = u / NM;
        const int p = n / nrhs, r = n % nrhs;
        uint32_t h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) tf32_split(X[((4 * kq + j) * 2 + p) * nrhs + r], h[j], l[j]);
        const uint32_t off = tc::kmajor_offset(n, 4 * kq, 4, KG);
        *reinterpret_cast<uint4*>(Bhi + off) = make_uint4(h[0], h[1], h[2], h[3]);
        if (SPLIT) *reinterpret_cast<uint4*>(Blo + off) = make_uint4(l[0], l[1], l[2], l[3]);
      }
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      if (!PRE && j + 2 < nk) fetch(j + 2);  // the raw stage is free: every thread has converted it
      tc::fence_after_sync();
      const uint32_t ah = PRE ? tc::smem_u32(raw) : tc::smem_u32(Ahi), bh = tc::smem_u32(Bhi),
                     al = PRE ? ah + a_bytes : tc::smem_u32(Alo), bl = tc::smem_u32(Blo);
      const uint32_t sbo = KG * 128;
      for (int ks = 0; ks < KG / 2; ++ks) {
        const uint32_t o = ks * 256;
        tc::mma_tf32(tbase, tc::smem_desc(ah + o, 128, sbo), tc::smem_desc(bh + o, 128, sbo), idesc,
                     ks > 0 ? 1u : 0u);
        if (SPLIT) {
          tc::mma_tf32(tbase, tc::smem_desc(ah + o, 128, sbo), tc::smem_desc(bl + o, 128, sbo), idesc, 1u);
          tc::mma_tf32(tbase, tc::smem_desc(al + o, 128, sbo), tc::smem_desc(bh + o, 128, sbo), idesc, 1u);
        }
      }
      tc::mma_commit(&mma_done);
    }
    issued = j + 1;
  }
  if (issued > 0) {
    if (!tc::mbar_wait(&mma_done, (issued - 1) & 1, kWaitLimit)) s_bad = 1;
    tc::fence_after_sync();
    tc::tmem_promote(t_own + NM, t_own, own);
    tc::tmem_wait_st();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (!s_bad && issued == nk) {
    float* E = reinterpret_cast<float*>(smem);  // [128][NM + 1], over the (now idle) raw stages
    const int quarter = warp & 3;
    for (int col0 = slice * sw; col0 < slice * sw + own; col0 += 16) {
      float v[16];
      tc::tmem_ld16(tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(NM + col0), v);
      const int row = quarter * 32 + lane;
#pragma unroll
      for (int i = 0; i < 16; ++i) E[row * (NM + 1) + col0 + i] = v[i];
    }
    __syncthreads();
    float* yA = y + (size_t)blockIdx.x * nc * 2 * nrhs;
    const float* addA = add ? add + (size_t)blockIdx.x * nc * 2 * nrhs : nullptr;
    for (int e = tid; e < nc * 2 * nrhs; e += kDcThreads) {
      const int r = e % nrhs, p = (e / nrhs) % 2, i = e / (2 * nrhs);
      float v = p == 0 ? E[i * (NM + 1) + r] - E[(nc + i) * (NM + 1) + nrhs + r]
                       : E[i * (NM + 1) + nrhs + r] + E[(nc + i) * (NM + 1) + r];
      if (addA) v += addA[e];
      yA[e] = v;
    }
  } else {
    // a wait ran out: let the copies still in flight land before the CTA's
    // shared memory is released
    if (tid == 0) {
      atomicExch(err, 1);
      for (int j = issued; j < nk && j < issued + 2; ++j) tc::mbar_wait(&full[j & 1], (j >> 1) & 1, kWaitLimit);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, tm_cols);
}

// D_c blocks as the byte images of k_apply_dc_tc's A operand tiles (tf32 hi,
// then lo with SPLIT), written once per build of D_c so that the coarse
// stencil copies them into shared memory as they are. One thread per 16-byte
// core row (row r, K group kq); the eight rows of a core matrix are adjacent
// threads, so each warp writes whole 128-byte core matrices. Rows beyond 2 nc
// are zero.
template <bool SPLIT>
__global__ void k_format_dc(const float* __restrict__ Dc, unsigned char* __restrict__ img, int nc, size_t nblk) {
  const int KG = nc / 4;
  const uint32_t a_bytes = kRows / 8 * KG * 128;
  const size_t per_blk = (size_t)kRows * KG;  // core rows of one image
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= nblk * per_blk) return;
  const size_t blk = t / per_blk;
  const int u = (int)(t % per_blk);
  const int r8 = u & 7, kq = (u >> 3) % KG, g8 = (u >> 3) / KG;
  const int m = 8 * g8 + r8;  // A row: Re rows 0..nc-1, Im rows nc..2nc-1
  unsigned char* hi = img + blk * (SPLIT ? 2 : 1) * a_bytes;
  uint32_t h[4] = {0, 0, 0, 0}, l[4] = {0, 0, 0, 0};
  if (m < 2 * nc) {
    const int row = m < nc ? m : m - nc, p = m < nc ? 0 : 1;
    const float* D = Dc + (blk * nc + row) * nc * 2;  // complex row of the block
#pragma unroll
    for (int j = 0; j < 4; ++j) tf32_split(D[2 * (4 * kq + j) + p], h[j], l[j]);
  }
  const uint32_t off = tc::kmajor_offset(m, 4 * kq, 4, KG);
  *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
  if (SPLIT) *reinterpret_cast<uint4*>(hi + a_bytes + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

}  // namespace

// tensor-core contraction for the self and forward blocks (split: tf32
// operands as hi + lo parts, FP32 accuracy); false when the shape is outside
// what the kernel handles
bool build_Dc_tc(mrhs_ctx c, int fmt, bool split) {
  const int Nt = c->ntv, nc = 2 * Nt;
  if (c->work_dtype != MRHS_F32 || 2 * nc > kRows) return false;
  for (int m = 0; m < 4; ++m)
    if ((c->g.Va / c->g.a[m]) < 1) return false;
  Agg4 ag;
  for (int m = 0; m < 4; ++m) ag.a[m] = c->g.a[m];
  split = split && fmt == tc::kFmtTF32;
  // two stages of 2 tiles, or one stage of 4 tiles (split; chunks of eight
  // sites in one stage of 196 KB per CTA measured slower: 270 against 184 ms
  // per build at 48^3x96)
  const size_t smem = 4 * (size_t)kTileBytes;
  const cx<float>* U = (const cx<float>*)c->U32;
  const float* Acl = (const float*)c->A32;
  int* err = c->dflag + 2;
  MRHS_CUDA(cudaMemsetAsync(err, 0, sizeof(int), c->stream));
  Prof pr(c, "coarse_op_tc");
  MRHS_DISPATCH(c->tv_dtype, SP, {
    auto kern = fmt == tc::kFmtBF16 ? k_coarse_op_tc<tc::kFmtBF16, SP, false>
                : fmt == tc::kFmtF16 ? k_coarse_op_tc<tc::kFmtF16, SP, false>
                : split              ? k_coarse_op_tc<tc::kFmtTF32, SP, true>
                                     : k_coarse_op_tc<tc::kFmtTF32, SP, false>;
    MRHS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<c->g.nagg * 5, kThreads, smem, c->stream>>>((const SP*)c->P, U, Acl, c->nbr, Nt, ag, c->g.Va,
                                                        (cx<float>*)c->Dc, err);
  });
  MRHS_LAUNCH_CHECK("coarse_op_tc");
  int* h = c->hflag + 2;
  MRHS_CUDA(cudaMemcpyAsync(h, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MRHS_CUDA(cudaStreamSynchronize(c->stream));
  MRHS_REQUIRE(*h == 0, MRHS_ERR_TIMEOUT, "coarse_op_tc: tensor-core pipeline wait ran out");
  return true;
}

// the operand images of D_c for the tensor-core coarse stencil, made by every
// build of D_c (so that the coarse solves, including the allocation-free one,
// only read them): tf32 hi + lo for the FP32 setup, tf32 for the mixed ones.
// Skipped (the stencil then converts each block itself) when the stencil
// would not use them, when MRHS_DC_IMAGES=0, or when they do not fit in
// device memory.
void dc_images_build(mrhs_ctx c) {
  static const bool off = [] {
    const char* e = std::getenv("MRHS_DC_IMAGES");
    const char* a = std::getenv("MRHS_DC_APPLY");
    return (e && std::atoi(e) == 0) || (a && std::string(a) == "alu");
  }();
  const int nc = 2 * c->ntv, KG = nc / 4;
  if (off || c->dc_engine == MRHS_DC_ALU || c->work_dtype != MRHS_F32 || nc % 8 != 0 || nc > 64) return;
  const bool split = c->prec == MRHS_PREC_FP32;
  const size_t a_bytes = (size_t)kRows / 8 * KG * 128;
  const size_t nblk = (size_t)c->g.nagg * 9;
  if (!c->dc_img) {
    const size_t bytes = nblk * 2 * a_bytes;  // room for either form
    size_t free_b = 0, total_b = 0;
    MRHS_CUDA(cudaMemGetInfo(&free_b, &total_b));
    if (bytes + ((size_t)1 << 30) > free_b) return;
    c->dc_img = dalloc(c, bytes);
  }
  const size_t n = nblk * (size_t)kRows * KG;
  Prof pr(c, "format_dc");
  if (split)
    k_format_dc<true><<<grid_for(n, 256), 256, 0, c->stream>>>((const float*)c->Dc, (unsigned char*)c->dc_img, nc, nblk);
  else
    k_format_dc<false><<<grid_for(n, 256), 256, 0, c->stream>>>((const float*)c->Dc, (unsigned char*)c->dc_img, nc, nblk);
  MRHS_LAUNCH_CHECK("format_dc");
  c->dc_img_version = c->dc_version;
  c->dc_img_split = (int)split;
}

// coarse stencil on the tensor cores (FP32 coarse fields): split-tf32 (FP32
// accuracy) or single tf32; false when the shape is outside the kernel's
bool apply_Dc_tc(mrhs_ctx c, const DcPart& pt, void* yc, int nrhs, bool split) {
  const int nc = 2 * c->ntv;
  if (c->work_dtype != MRHS_F32 || nc % 8 != 0 || nc > 64 || nrhs % 16 != 0 || nrhs > 64) return false;
  const int KG = nc / 4;
  const size_t tiles = (size_t)(kRows / 8 * KG * 128 + 2 * nrhs / 8 * KG * 128);
  const size_t raw = ((size_t)nc * nc * 8 + (size_t)nc * 2 * nrhs * 4 + 1023) & ~(size_t)1023;
  size_t smem = std::max(2 * raw, sizeof(float) * kRows * (2 * nrhs + 1)) + (split ? 2 : 1) * tiles;
  uint32_t cols = 32;
  while (cols < (uint32_t)(4 * nrhs)) cols <<= 1;  // R and S regions of 2 nrhs columns each
  int* err = c->dflag + 3;
  const void* src = c->Dc;
  const bool pre = c->dc_img && c->dc_img_version == c->dc_version && c->dc_img_split == (int)split;
  if (pre) {
    src = c->dc_img;
    // stages hold the operand images instead of the FP32 blocks; no A tiles
    const size_t img = (size_t)(split ? 2 : 1) * (kRows / 8 * KG * 128);
    const size_t stage = (img + (size_t)nc * 2 * nrhs * 4 + 1023) & ~(size_t)1023;
    const size_t btiles = (size_t)(split ? 2 : 1) * (2 * nrhs / 8 * KG * 128);
    smem = std::max(2 * stage, sizeof(float) * kRows * (2 * nrhs + 1)) + btiles;
  }
  // a shape whose pipeline stages do not fit in shared memory (e.g. 64
  // right-hand sides in split form at 2 ntv = 64) takes the CUDA-core stencil
  int maxsm = 0;
  MRHS_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
  if (smem > (size_t)maxsm) return false;
  Prof pr(c, "apply_dc_tc");
  auto kern = pre ? (split ? k_apply_dc_tc<true, true> : k_apply_dc_tc<false, true>)
                  : (split ? k_apply_dc_tc<true, false> : k_apply_dc_tc<false, false>);
  MRHS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<pt.na, kDcThreads, smem, c->stream>>>((const float*)src, (const float*)pt.x0, (const float*)pt.xh,
                                               (float*)yc, c->aggnbr, nc, nrhs, cols, err, pt.alist, pt.pos, pt.kb,
                                               pt.ke, (const float*)pt.add);
  MRHS_LAUNCH_CHECK("apply_dc_tc");
  return true;
}

// report (and clear) a bounded wait of the tensor-core coarse stencil that
// ran out since the last check; synchronises the context's stream
void check_tc_timeout(mrhs_ctx c) {
  MRHS_CUDA(cudaMemcpyAsync(c->hflag + 3, c->dflag + 3, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MRHS_CUDA(cudaStreamSynchronize(c->stream));
  if (c->hflag[3] != 0) {
    MRHS_CUDA(cudaMemsetAsync(c->dflag + 3, 0, sizeof(int), c->stream));
    MRHS_REQUIRE(false, MRHS_ERR_TIMEOUT, "apply_dc_tc: tensor-core pipeline wait ran out");
  }
}

}  // namespace mrhs
