// One layer of the learned test-vector generator (the gauge-covariant
// convolution on colour triplets, nn.cu) for inference, with the channel
// mixing on the tensor cores (tcgen05, bf16 operands, FP32 accumulation):
//   z(x)[o] = sum_{k=0..8} sum_c W[k][o][c] s_k T_k(x) h(n_k(x))[c].
// W acts on channels only, so per step k the layer is a dense product of the
// weight block W[k] (C_out x C_in complex) and the transported inputs of a
// tile of sites. Real form: with A_k = [[Re W, -Im W], [Im W, Re W]] (rows:
// Re z then Im z of the C_out channels; columns: (c, Re/Im) of the inputs)
// and B_k = the transported inputs, one column per (site, colour, rhs) and
// one K row per (c, Re/Im),
//   [Re z; Im z] = sum_k A_k B_k,
// an MMA of M = 128 (2 C_out rows used), N = the tile's columns, K = 2 C_in
// (padded to 16) per k; the nine k accumulate in tensor memory.
//
// Persistent CTAs of 16 warps: the nine A_k sit in shared memory for the
// whole launch; the CUDA cores build B_{k+1} (colour transport, sign, bf16
// rounding) into the other buffer while the tensor core multiplies B_k; the
// transports of the tile's sites for all nine steps are staged in shared
// memory at the start of the tile, and the inputs of step k+1 are loaded into
// registers while step k is computed. The
// operands are bf16: the weights are the bf16-rounded compute copy (exact),
// the activations are rounded once to bf16 when they enter B; products and
// sums are FP32.
#include <algorithm>

#include "common.cuh"
#include "tc.cuh"

namespace mrhs {
namespace {

constexpr int kNnThreads = 512;
constexpr int kNnRows = 128;        // MMA M
constexpr int kNnCols = 192;        // MMA N: 3 colours x (sites x rhs) of a tile, padded
constexpr uint32_t kNnWait = 1u << 20;
constexpr int kNnMaxS = 32;         // sites per tile: min(32, 64 / rhs)
constexpr int kNnItems = 4;         // operand items per thread and step (S x C_in x rhs <= 2048)

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}

// (row, k), (row, k+1) of a K-major no-swizzle bf16 tile with kg 16-byte K groups
__device__ __forceinline__ void put_bf16(unsigned char* tile, int row, int k, float a, float b, int kg) {
  *reinterpret_cast<uint32_t*>(tile + tc::kmajor_offset(row, k, 2, kg)) = pack_bf16(a, b);
}

template <int KC>
__global__ void __launch_bounds__(kNnThreads, 1) k_covconv_tc(const float* __restrict__ h, float* __restrict__ z,
                                                              const float* __restrict__ W,
                                                              const float* __restrict__ U32,
                                                              const int* __restrict__ nbr, int cin, int cout, int N,
                                                              int S, int V, int ntiles, int* __restrict__ err) {
  constexpr int KG = KC / 8;                        // 16-byte K groups per step
  constexpr int ABYTES = kNnRows * KC * 2;          // one A_k
  constexpr int BBYTES = kNnCols * KC * 2;          // one B buffer
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                         // [9] A_k
  unsigned char* sB = smem + 9 * ABYTES;            // [2] B buffers
  // the transports of the tile's sites for all nine steps: s_k T_k(x) (sign
  // folded in) as 18 floats (padded to 20) and the neighbour n_k(x)
  float* sT = reinterpret_cast<float*>(sB + 2 * BBYTES);   // [9][kNnMaxS][20]
  int* sNb = reinterpret_cast<int*>(sT + 9 * kNnMaxS * 20); // [9][kNnMaxS]
  __shared__ uint64_t bar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // zero everything once: padding rows of A, padding K entries and padding
  // columns of B stay zero for the whole launch
  for (int i = tid; i < (9 * ABYTES + 2 * BBYTES + 9 * kNnMaxS * 21 * 4) / 16; i += kNnThreads)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  for (int e = tid; e < 9 * cout * cin; e += kNnThreads) {
    const int c = e % cin, o = (e / cin) % cout, k = e / (cin * cout);
    const float wr = W[2 * e], wi = W[2 * e + 1];
    unsigned char* Ak = sA + k * ABYTES;
    put_bf16(Ak, o, 2 * c, wr, -wi, KG);
    put_bf16(Ak, cout + o, 2 * c, wi, wr, KG);
  }
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::fence_mbar_init();
    s_bad = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(&s_tmem, 256);
    tc::tmem_relinquish();
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = s_tmem;
  const uint32_t idesc = tc::instr_desc(tc::kFmtBF16, tc::kFmtBF16, kNnRows, kNnCols);
  const int items = S * cin * N;                    // (site, input channel, rhs) of one step
  uint32_t st = 0;                                  // steps issued by this CTA

  // the operand items of thread tid, the same at every step and tile:
  // item i = tid + j * threads is (site s, input channel c, rhs r); its
  // input rows sit at n * 6 C_in N + it_h (+ (2 bb + part) N) for the
  // neighbour n, its three colours go to B rows (s*3 + a) N + r, K = 2c
  int it_s[kNnItems], it_h[kNnItems];
  uint32_t it_b[kNnItems][3];
#pragma unroll
  for (int j = 0; j < kNnItems; ++j) {
    const int i = tid + j * kNnThreads;
    const int r = i % N, c = (i / N) % cin;
    it_s[j] = i < items ? i / (N * cin) : kNnMaxS;  // kNnMaxS: no item
    it_h[j] = c * 6 * N + r;
#pragma unroll
    for (int a = 0; a < 3; ++a) it_b[j][a] = tc::kmajor_offset(((i / (N * cin)) * 3 + a) * N + r, 2 * c, 2, KG);
  }
  const size_t nstride = (size_t)6 * cin * N;       // floats per site of h
  auto load_items = [&](int k, int ns, float (&hb)[kNnItems][6]) {
#pragma unroll
    for (int j = 0; j < kNnItems; ++j) {
      const bool on = it_s[j] < ns;
      const float* hp = h + (on ? (size_t)sNb[k * kNnMaxS + it_s[j]] * nstride + it_h[j] : 0);
#pragma unroll
      for (int q = 0; q < 6; ++q) hb[j][q] = on ? __ldg(hp + q * N) : 0.f;
    }
  };
  // epilogue: column n of the accumulator is (site, colour, rhs); its offset
  // in z from the tile's first site, without the row's channel and part
  int* s_col = sNb + 9 * kNnMaxS;                   // [kNnCols]
  for (int n = tid; n < kNnCols; n += kNnThreads) {
    const int r = n % N, a = (n / N) % 3, ss = n / (3 * N);
    s_col[n] = (ss * cout * 3 + a) * 2 * N + r;
  }
  __syncthreads();

  for (int tile = blockIdx.x; tile < ntiles && !s_bad; tile += gridDim.x) {
    const int s0 = tile * S;
    const int ns = min(S, V - s0);
    // the transports of all nine steps, one (step, site) per thread
    for (int u = tid; u < 9 * S; u += kNnThreads) {
      const int k = u / S, s = u % S;
      float* T = sT + (k * kNnMaxS + s) * 20;
      int n = 0;
      if (s < ns) {
        const size_t x = (size_t)s0 + s;
        if (k == 0) {
          n = (int)x;
#pragma unroll
          for (int q = 0; q < 18; ++q) T[q] = (q == 0 || q == 8 || q == 16) ? 1.f : 0.f;
        } else {
          const int mu = (k - 1) & 3;
          const int e = __ldg(nbr + x * 8 + (k <= 4 ? 0 : 4) + mu);
          n = e & 0x3fffffff;
          const float sg = (e & 0x40000000) ? -1.f : 1.f;
          const float* uu = U32 + ((k <= 4 ? x : (size_t)n) * 4 + mu) * 18;
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int bb = 0; bb < 3; ++bb) {
              // T = U forward, U^dag backward: T[a][bb] at 2 (3a + bb)
              const int q = k <= 4 ? a * 3 + bb : bb * 3 + a;
              T[2 * (a * 3 + bb)] = sg * __ldg(uu + 2 * q);
              T[2 * (a * 3 + bb) + 1] = sg * (k <= 4 ? __ldg(uu + 2 * q + 1) : -__ldg(uu + 2 * q + 1));
            }
        }
      }
      sNb[k * kNnMaxS + s] = n;
    }
    __syncthreads();
    // the inputs of step k+1 are loaded while step k is computed
    float hc[kNnItems][6], hn[kNnItems][6];
    load_items(0, ns, hc);
    for (int k = 0; k < 9; ++k, ++st) {
      const int b = st & 1;
      unsigned char* Bb = sB + b * BBYTES;
      if (k < 8) load_items(k + 1, ns, hn);
      // the MMAs of step st-2 read this buffer
      if (st >= 2 && !tc::mbar_wait(&bar[b], ((st - 2) >> 1) & 1, kNnWait)) s_bad = 1;
#pragma unroll
      for (int j = 0; j < kNnItems; ++j) {
        if (it_s[j] < kNnMaxS) {
          // rows of absent sites get zeros (their inputs were loaded as 0)
          const float* T = sT + (k * kNnMaxS + it_s[j]) * 20;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            float sr = 0.f, si = 0.f;
#pragma unroll
            for (int bb = 0; bb < 3; ++bb) {
              const float ur = T[2 * (a * 3 + bb)], ui = T[2 * (a * 3 + bb) + 1];
              sr = fmaf(ur, hc[j][2 * bb], fmaf(-ui, hc[j][2 * bb + 1], sr));
              si = fmaf(ur, hc[j][2 * bb + 1], fmaf(ui, hc[j][2 * bb], si));
            }
            *reinterpret_cast<uint32_t*>(Bb + it_b[j][a]) = pack_bf16(sr, si);
          }
        }
      }
      tc::fence_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      if (s_bad) break;
      if (tid == 0) {
        tc::fence_after_sync();
        const uint32_t a0 = tc::smem_u32(sA + k * ABYTES), b0 = tc::smem_u32(Bb);
#pragma unroll
        for (int ks = 0; ks < KC / 16; ++ks)
          tc::mma_f16(tbase, tc::smem_desc(a0 + ks * 256, 128, KG * 128), tc::smem_desc(b0 + ks * 256, 128, KG * 128),
                      idesc, (k > 0 || ks > 0) ? 1u : 0u);
        tc::mma_commit(&bar[b]);
      }
#pragma unroll
      for (int j = 0; j < kNnItems; ++j)
#pragma unroll
        for (int q = 0; q < 6; ++q) hc[j][q] = hn[j][q];
    }
    if (s_bad) break;
    // the tile's last step done: every MMA of the tile is
    if (!tc::mbar_wait(&bar[(st - 1) & 1], ((st - 1) >> 1) & 1, kNnWait)) s_bad = 1;
    tc::fence_after_sync();
    if (!s_bad) {
      // warp w: lanes 32 (w % 4) .. (rows), columns 48 (w / 4) .. +47
      const int row = 32 * (warp & 3) + lane;
      const int col0 = 48 * (warp >> 2);
      const bool live = row < 2 * cout;
      const int part = live ? row / cout : 0, o = live ? row % cout : 0;
      const int ncols = 3 * ns * N;
      float* zt = z + (size_t)s0 * cout * 6 * N + (size_t)o * 6 * N + (size_t)part * N;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        float v[16];
        tc::tmem_ld16(tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(col0 + 16 * j), v);
        if (live) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int n = col0 + 16 * j + q;
            if (n < ncols) zt[s_col[n]] = v[q];
          }
        }
      }
    }
    // every read of the accumulator is done before the next tile's first MMA
    tc::fence_before_sync();
    __syncthreads();
  }
  if (s_bad && tid == 0) {
    atomicExch(err, 1);
    // let MMAs still in flight finish before the CTA's shared memory goes
    if (st >= 1) tc::mbar_wait(&bar[(st - 1) & 1], ((st - 1) >> 1) & 1, kNnWait);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 256);
}

template <int KC>
void launch_tc(mrhs_ctx c, const float* h, float* z, const float* W, int cin, int cout, int N) {
  const int S = std::min(kNnMaxS, std::max(1, 64 / N));
  const int V = c->g.V;
  const int ntiles = (V + S - 1) / S;
  const size_t smem = 9 * (size_t)kNnRows * KC * 2 + 2 * (size_t)kNnCols * KC * 2 +
                      9 * kNnMaxS * 20 * sizeof(float) + 9 * kNnMaxS * sizeof(int) + kNnCols * sizeof(int);
  const int grid = std::min(ntiles, c->num_sms);
  MRHS_CUDA(cudaFuncSetAttribute(k_covconv_tc<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_covconv_tc<KC><<<grid, kNnThreads, smem, c->stream>>>(h, z, W, c->U32, c->nbr, cin, cout, N, S, V, ntiles,
                                                          c->dflag + 6);
  MRHS_LAUNCH_CHECK("covconv_tc");
}

}  // namespace

// z = covconv(h) with the channel mixing on the tensor cores (bf16 operands);
// false when the shape is outside the kernel's (more than 32 channels or 8
// right-hand sides)
bool covconv_tc(mrhs_ctx c, const float* h, float* z, const float* W, int cin, int cout, int N) {
  if (cin < 1 || cin > 32 || cout < 1 || cout > 32 || N < 1 || N > 8) return false;
  const int kc = (2 * cin + 15) / 16 * 16;
  Prof pr(c, "nn_covconv_tc");
  switch (kc) {
    case 16: launch_tc<16>(c, h, z, W, cin, cout, N); break;
    case 32: launch_tc<32>(c, h, z, W, cin, cout, N); break;
    case 48: launch_tc<48>(c, h, z, W, cin, cout, N); break;
    default: launch_tc<64>(c, h, z, W, cin, cout, N); break;
  }
  return true;
}

// report (and clear) a bounded wait of the tensor-core layer that ran out;
// synchronises the context's stream
void check_nn_tc_timeout(mrhs_ctx c) {
  MRHS_CUDA(cudaMemcpyAsync(c->hflag + 6, c->dflag + 6, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MRHS_CUDA(cudaStreamSynchronize(c->stream));
  if (c->hflag[6] != 0) {
    MRHS_CUDA(cudaMemsetAsync(c->dflag + 6, 0, sizeof(int), c->stream));
    MRHS_REQUIRE(false, MRHS_ERR_TIMEOUT, "covconv_tc: tensor-core pipeline wait ran out");
  }
}

}  // namespace mrhs
