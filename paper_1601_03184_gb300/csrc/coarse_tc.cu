// Coarse-operator contraction D_c[A,k] = P_A^dag (D_k P) on the fifth-
// generation tensor cores (tcgen05), for the mixed-precision setup: the
// link products are dense 2N_tv x 2N_tv blocks (Sec. 3.2 / Eq. 6 of the
// paper: D_c = P^dag D P with the aggregate-local structure of P).
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

// store the pair of elements (row, k), (row, k+1), k even, of a K-major tile
template <int FMT>
__device__ __forceinline__ void put2(unsigned char* tile, int row, int k, float a, float b) {
  using E = Elem<FMT>;
  const uint32_t off = tc::kmajor_offset(row, k, E::size, kKG);
  if constexpr (E::size == 2) {
    *reinterpret_cast<uint32_t*>(tile + off) = E::pack(a, b);
  } else {
    *reinterpret_cast<uint2*>(tile + off) = make_uint2(E::one(a), E::one(b));
  }
}

template <int FMT, class SP>
__global__ void __launch_bounds__(kThreads) k_coarse_op_tc(const SP* __restrict__ P, const cx<float>* __restrict__ U,
                                                           const float* __restrict__ Acl, const int* __restrict__ nbr,
                                                           int Nt, Agg4 ag, int Va, cx<float>* __restrict__ Dc,
                                                           int* __restrict__ err) {
  constexpr int ES = Elem<FMT>::size;
  constexpr int Q = kKG * 16 / ES / 12;       // sites per chunk: 8 (2-byte) or 4 (tf32)
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
  for (int i = threadIdx.x; i < 4 * kTileBytes / 16; i += kThreads)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::fence_mbar_init();
    s_bad = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(&s_tmem, 128);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = s_tmem;
  const uint32_t idesc = tc::instr_desc(FMT, FMT, kRows, NN);

  const int nchunk = (nsite + Q - 1) / Q;
  int issued = 0;
  for (int t = 0; t < nchunk; ++t) {
    const int st = t & 1;
    if (t >= 2 && !tc::mbar_wait(&mbar[st], ((t >> 1) - 1) & 1, kWaitLimit)) s_bad = 1;
    __syncthreads();
    if (s_bad) break;
    const int q0 = t * Q;
    const int nq = min(Q, nsite - q0);
    unsigned char* tA = smem + 2 * st * kTileBytes;
    unsigned char* tB = tA + kTileBytes;
    // B: Y = D_k P for (site q, column col); absent sites of a ragged chunk give zeros
    for (int w = threadIdx.x; w < Q * nc; w += kThreads) {
      const int q = w / nc, col = w % nc;
      cx<float> out[12];
#pragma unroll
      for (int c = 0; c < 12; ++c) out[c] = mk<float>(0, 0);
      if (q < nq) {
        const int l = k == 0 ? q0 + q : face_site(ag, mu, lmu, q0 + q);
        const int s = A * Va + l;
        if (k == 0) {
          cx<float> psi[12];
          load_pcol<SP, float>(psi, P, s, Nt, col);
          clover_apply_reg<float>(out, psi, Acl + (size_t)s * 72);
          for (int d = -1; d <= 1; d += 2) {
            hop_pcol<0, SP, float>(out, P, U, nbr, s, d, Nt, col, true, Va);
            hop_pcol<1, SP, float>(out, P, U, nbr, s, d, Nt, col, true, Va);
            hop_pcol<2, SP, float>(out, P, U, nbr, s, d, Nt, col, true, Va);
            hop_pcol<3, SP, float>(out, P, U, nbr, s, d, Nt, col, true, Va);
          }
        } else {
          switch (mu) {
            case 0: hop_pcol<0, SP, float>(out, P, U, nbr, s, +1, Nt, col, false, Va); break;
            case 1: hop_pcol<1, SP, float>(out, P, U, nbr, s, +1, Nt, col, false, Va); break;
            case 2: hop_pcol<2, SP, float>(out, P, U, nbr, s, +1, Nt, col, false, Va); break;
            default: hop_pcol<3, SP, float>(out, P, U, nbr, s, +1, Nt, col, false, Va); break;
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 12; c += 2) {
        put2<FMT>(tB, col, q * 12 + c, out[c].re, out[c + 1].re);
        put2<FMT>(tB, nc + col, q * 12 + c, out[c].im, out[c + 1].im);
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
      put2<FMT>(tA, p * nc + h * Nt + j, q * 12 + c, a, b);
    }
    tc::fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(tA), b0 = tc::smem_u32(tB);
#pragma unroll
      for (int ks = 0; ks < kKG / 2; ++ks) {
        const uint64_t ad = tc::smem_desc(a0 + ks * KSTEP_BYTES, 128, kKG * 128);
        const uint64_t bd = tc::smem_desc(b0 + ks * KSTEP_BYTES, 128, kKG * 128);
        if constexpr (FMT == tc::kFmtTF32)
          tc::mma_tf32(tbase, ad, bd, idesc, (t > 0 || ks > 0) ? 1u : 0u);
        else
          tc::mma_f16(tbase, ad, bd, idesc, (t > 0 || ks > 0) ? 1u : 0u);
      }
      tc::mma_commit(&mbar[st]);
    }
    issued = t + 1;
  }
  // the last commit covers every MMA issued before it
  if (issued > 0) {
    const int tl = issued - 1;
    if (!tc::mbar_wait(&mbar[tl & 1], (tl >> 1) & 1, kWaitLimit)) s_bad = 1;
  }
  tc::fence_after_sync();
  __syncthreads();
  const bool ok = !s_bad && issued == nchunk;
  if (ok) {
    // accumulator rows -> shared memory (stage buffers are free now)
    float* E = reinterpret_cast<float*>(smem);  // [128][NN + 1]
    const int quarter = warp & 3, half = warp >> 2;
    for (int col0 = half * 64; col0 < min(NN, half * 64 + 64); col0 += 16) {
      float v[16];
      tc::tmem_ld16(tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col0, v);
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
  if (warp == 0) tc::tmem_dealloc(tbase, 128);
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
constexpr int kDcThreads = 256;

__device__ __forceinline__ void tf32_split(float v, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(v));
  const float r = v - __uint_as_float(hi);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}

template <bool SPLIT>
__global__ void __launch_bounds__(kDcThreads) k_apply_dc_tc(const float* __restrict__ Dc, const float* __restrict__ x,
                                                            float* __restrict__ y, const int* __restrict__ aggnbr,
                                                            int nc, int nrhs, uint32_t tm_cols, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_bad;
  const int A = blockIdx.x;
  const int NM = 2 * nrhs;                   // MMA N
  const int KG = nc / 4;                     // 16-byte K groups (tf32)
  const int a_bytes = kRows / 8 * KG * 128;  // A tile
  const int b_bytes = NM / 8 * KG * 128;     // B tile
  unsigned char* Ahi = smem;
  unsigned char* Bhi = Ahi + a_bytes;
  unsigned char* Alo = Bhi + b_bytes;
  unsigned char* Blo = Alo + a_bytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // rows of A beyond 2nc stay zero
  if (2 * nc < kRows) {
    const int nz = (SPLIT ? 2 : 1) * (a_bytes + b_bytes) / 16;
    for (int i = threadIdx.x; i < nz; i += kDcThreads) reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  }
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar, 1);
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
  const uint32_t tbase = s_tmem;
  const uint32_t idesc = tc::instr_desc(tc::kFmtTF32, tc::kFmtTF32, kRows, NM);

  // per thread and block: A units (two K-adjacent core matrices of Dr and Di
  // per warp pass) and B units (4 kk x 4 rhs of one part p)
  const int a_units = (nc / 8) * (nc / 8);          // warp passes
  const int b_units = (nc / 4) * 2 * (nrhs / 4);    // thread units
  constexpr int kMaxA = 8, kMaxB = 2;               // nc <= 64, nrhs <= 64
  float4 ra[kMaxA];
  float4 rb[kMaxB][4];
  auto load = [&](int k) {
    const float4* D4 = reinterpret_cast<const float4*>(Dc + ((size_t)A * 9 + k) * nc * nc * 2);
#pragma unroll
    for (int j = 0; j < kMaxA; ++j) {
      const int u = warp + 8 * j;
      if (u < a_units) {
        const int g8 = u / (nc / 8), kgp = u % (nc / 8);
        const int row = 8 * g8 + ((lane >> 1) & 7);
        const int col = (2 * kgp + (lane >> 4)) * 4 + 2 * (lane & 1);
        ra[j] = __ldg(D4 + (row * nc + col) / 2);
      }
    }
    const int B = k == 0 ? A : aggnbr[A * 8 + k - 1];
#pragma unroll
    for (int j = 0; j < kMaxB; ++j) {
      const int u = threadIdx.x + kDcThreads * j;
      if (u < b_units) {
        const int rq = u % (nrhs / 4), p = (u / (nrhs / 4)) % 2, kq = u / (nrhs / 4) / 2;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          rb[j][q] = __ldg(reinterpret_cast<const float4*>(x + (((size_t)B * nc + 4 * kq + q) * 2 + p) * nrhs + 4 * rq));
      }
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int j = 0; j < kMaxA; ++j) {
      const int u = warp + 8 * j;
      if (u < a_units) {
        const int g8 = u / (nc / 8), kgp = u % (nc / 8);
        const int row = 8 * g8 + ((lane >> 1) & 7);
        const int col = (2 * kgp + (lane >> 4)) * 4 + 2 * (lane & 1);
        const uint32_t offr = tc::kmajor_offset(row, col, 4, KG), offi = tc::kmajor_offset(nc + row, col, 4, KG);
        uint32_t h0, l0, h1, l1, h2, l2, h3, l3;
        tf32_split(ra[j].x, h0, l0);  // Re D[row][col]
        tf32_split(ra[j].y, h1, l1);  // Im D[row][col]
        tf32_split(ra[j].z, h2, l2);  // Re D[row][col+1]
        tf32_split(ra[j].w, h3, l3);  // Im D[row][col+1]
        *reinterpret_cast<uint2*>(Ahi + offr) = make_uint2(h0, h2);
        *reinterpret_cast<uint2*>(Ahi + offi) = make_uint2(h1, h3);
        if (SPLIT) {
          *reinterpret_cast<uint2*>(Alo + offr) = make_uint2(l0, l2);
          *reinterpret_cast<uint2*>(Alo + offi) = make_uint2(l1, l3);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kMaxB; ++j) {
      const int u = threadIdx.x + kDcThreads * j;
      if (u < b_units) {
        const int rq = u % (nrhs / 4), p = (u / (nrhs / 4)) % 2, kq = u / (nrhs / 4) / 2;
        // transpose 4 (kk) x 4 (rhs): row n = p*nrhs + 4rq + c holds kk = 4kq .. 4kq+3
        const float v[4][4] = {{rb[j][0].x, rb[j][0].y, rb[j][0].z, rb[j][0].w},
                               {rb[j][1].x, rb[j][1].y, rb[j][1].z, rb[j][1].w},
                               {rb[j][2].x, rb[j][2].y, rb[j][2].z, rb[j][2].w},
                               {rb[j][3].x, rb[j][3].y, rb[j][3].z, rb[j][3].w}};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const uint32_t off = tc::kmajor_offset(p * nrhs + 4 * rq + c, 4 * kq, 4, KG);
          uint32_t h[4], l[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) tf32_split(v[q][c], h[q], l[q]);
          *reinterpret_cast<uint4*>(Bhi + off) = make_uint4(h[0], h[1], h[2], h[3]);
          if (SPLIT) *reinterpret_cast<uint4*>(Blo + off) = make_uint4(l[0], l[1], l[2], l[3]);
        }
      }
    }
  };

  load(0);
  int issued = 0;
  for (int k = 0; k < 9; ++k) {
    if (k >= 1 && !tc::mbar_wait(&mbar, (k - 1) & 1, kWaitLimit)) s_bad = 1;
    __syncthreads();
    if (s_bad) break;
    store();
    if (k + 1 < 9) load(k + 1);
    tc::fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
      const uint32_t ah = tc::smem_u32(Ahi), bh = tc::smem_u32(Bhi), al = tc::smem_u32(Alo), bl = tc::smem_u32(Blo);
      const uint32_t sbo = KG * 128;
      for (int ks = 0; ks < KG / 2; ++ks) {
        const uint32_t o = ks * 256;
        tc::mma_tf32(tbase, tc::smem_desc(ah + o, 128, sbo), tc::smem_desc(bh + o, 128, sbo), idesc,
                     (k > 0 || ks > 0) ? 1u : 0u);
        if (SPLIT) {
          tc::mma_tf32(tbase, tc::smem_desc(ah + o, 128, sbo), tc::smem_desc(bl + o, 128, sbo), idesc, 1u);
          tc::mma_tf32(tbase, tc::smem_desc(al + o, 128, sbo), tc::smem_desc(bh + o, 128, sbo), idesc, 1u);
        }
      }
      tc::mma_commit(&mbar);
    }
    issued = k + 1;
  }
  if (issued > 0 && !tc::mbar_wait(&mbar, (issued - 1) & 1, kWaitLimit)) s_bad = 1;
  tc::fence_after_sync();
  __syncthreads();
  if (!s_bad && issued == 9) {
    float* E = reinterpret_cast<float*>(smem);  // [128][NM + 1]
    const int quarter = warp & 3, half = warp >> 2;
    const int ch = NM / 2;
    for (int col0 = half * ch; col0 < half * ch + ch; col0 += 16) {
      float v[16];
      tc::tmem_ld16(tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col0, v);
      const int row = quarter * 32 + lane;
#pragma unroll
      for (int i = 0; i < 16; ++i) E[row * (NM + 1) + col0 + i] = v[i];
    }
    __syncthreads();
    float* yA = y + (size_t)A * nc * 2 * nrhs;
    for (int e = threadIdx.x; e < nc * 2 * nrhs; e += kDcThreads) {
      const int r = e % nrhs, p = (e / nrhs) % 2, i = e / (2 * nrhs);
      const float v = p == 0 ? E[i * (NM + 1) + r] - E[(nc + i) * (NM + 1) + nrhs + r]
                             : E[i * (NM + 1) + nrhs + r] + E[(nc + i) * (NM + 1) + r];
      yA[e] = v;
    }
  } else if (threadIdx.x == 0) {
    atomicExch(err, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, tm_cols);
}

}  // namespace

// tensor-core contraction for the self and forward blocks of the mixed
// setups; false when the shape is outside what the kernel handles
bool build_Dc_tc(mrhs_ctx c, int fmt) {
  const int Nt = c->ntv, nc = 2 * Nt;
  if (c->work_dtype != MRHS_F32 || 2 * nc > kRows) return false;
  for (int m = 0; m < 4; ++m)
    if ((c->g.Va / c->g.a[m]) < 1) return false;
  Agg4 ag;
  for (int m = 0; m < 4; ++m) ag.a[m] = c->g.a[m];
  const size_t smem = 4 * (size_t)kTileBytes;
  const cx<float>* U = (const cx<float>*)c->U32;
  const float* Acl = (const float*)c->A32;
  int* err = c->dflag + 2;
  MRHS_CUDA(cudaMemsetAsync(err, 0, sizeof(int), c->stream));
  Prof pr(c, "coarse_op_tc");
  MRHS_DISPATCH(c->tv_dtype, SP, {
    if (fmt == tc::kFmtBF16) {
      auto kern = k_coarse_op_tc<tc::kFmtBF16, SP>;
      MRHS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      kern<<<c->g.nagg * 5, kThreads, smem, c->stream>>>((const SP*)c->P, U, Acl, c->nbr, Nt, ag, c->g.Va,
                                                          (cx<float>*)c->Dc, err);
    } else if (fmt == tc::kFmtF16) {
      auto kern = k_coarse_op_tc<tc::kFmtF16, SP>;
      MRHS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      kern<<<c->g.nagg * 5, kThreads, smem, c->stream>>>((const SP*)c->P, U, Acl, c->nbr, Nt, ag, c->g.Va,
                                                          (cx<float>*)c->Dc, err);
    } else {
      auto kern = k_coarse_op_tc<tc::kFmtTF32, SP>;
      MRHS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      kern<<<c->g.nagg * 5, kThreads, smem, c->stream>>>((const SP*)c->P, U, Acl, c->nbr, Nt, ag, c->g.Va,
                                                          (cx<float>*)c->Dc, err);
    }
  });
  MRHS_LAUNCH_CHECK("coarse_op_tc");
  int* h = c->hflag + 2;
  MRHS_CUDA(cudaMemcpyAsync(h, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MRHS_CUDA(cudaStreamSynchronize(c->stream));
  MRHS_REQUIRE(*h == 0, MRHS_ERR_TIMEOUT, "coarse_op_tc: tensor-core pipeline wait ran out");
  return true;
}

// coarse stencil on the tensor cores (FP32 coarse fields): split-tf32 (FP32
// accuracy) or single tf32; false when the shape is outside the kernel's
bool apply_Dc_tc(mrhs_ctx c, const void* xc, void* yc, int nrhs, bool split) {
  const int nc = 2 * c->ntv;
  if (c->work_dtype != MRHS_F32 || nc % 8 != 0 || nc > 64 || nrhs % 16 != 0 || nrhs > 64) return false;
  const int KG = nc / 4;
  const size_t tiles = (size_t)(kRows / 8 * KG * 128 + 2 * nrhs / 8 * KG * 128);
  const size_t smem = std::max((split ? 2 : 1) * tiles, sizeof(float) * kRows * (2 * nrhs + 1));
  uint32_t cols = 32;
  while (cols < (uint32_t)(2 * nrhs)) cols <<= 1;
  int* err = c->dflag + 3;
  Prof pr(c, "apply_dc_tc");
  auto kern = split ? k_apply_dc_tc<true> : k_apply_dc_tc<false>;
  MRHS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<c->g.nagg, kDcThreads, smem, c->stream>>>((const float*)c->Dc, (const float*)xc, (float*)yc, c->aggnbr, nc,
                                                   nrhs, cols, err);
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
