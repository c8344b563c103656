// Learned test-vector generator: a gauge-covariant nearest-neighbour
// convolution network on colour triplets, trained on the GPU with its own
// forward and backward kernels.
//
// Layer (C_in -> C_out channels, every channel a colour triplet):
//   z(x)[c] = sum_{k=0..8} sum_c' W[k][c][c'] s_k(x) T_k(x) h(n_k(x))[c']
// k = 0: n = x, T = 1; k = 1+mu: n = x+mu, T = U_mu(x); k = 5+mu: n = x-mu,
// T = U_mu(x-mu)^dag; s_k = -1 on hops across the t boundary.
// modReLU between layers: h[c] = z[c] max(0, |z[c]| + b[c]) / |z[c]|.
// Network 4 -> C1 -> C2 -> 4 channels (a spinor is 4 spin channels x 3
// colours, so the first and last layers read and write fine fields).
// Activations use the interleaved field layout with rows (site, channel,
// colour). Gradients: dL/dRe(p) + i dL/dIm(p) for complex parameters.
//
// The backward data pass is the forward kernel with W'[k'] = W[mirror(k')]^dag
// (mirror exchanges +mu and -mu): the adjoint of hopping from x+mu with
// U_mu(x) is hopping from y-mu with U_mu(y-mu)^dag.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace mrhs {

struct NNState {
  int C[4] = {4, 0, 0, 4};
  size_t nw = 0, nb = 0;        // complex weights, real biases
  float* W = nullptr;           // master weights (float2 complex), then biases
  float* Wc = nullptr;          // compute copy: bf16-rounded when bf16 weights are on
  float* Wm = nullptr;          // mirrored conjugate-transposed copy of Wc (backward data)
  float* G = nullptr;           // gradients, same packing as W
  float* m1 = nullptr;          // Adam first moment
  float* m2 = nullptr;          // Adam second moment
  bool bf16 = true;
  int nrhs = 0;                 // activations held for this many right-hand sides
  float* z1 = nullptr;
  float* h1 = nullptr;
  float* z2 = nullptr;
  float* h2 = nullptr;
  float* in = nullptr;          // copy of the forward input
  double* part = nullptr;       // reduction partials
  size_t part_elems = 0;
};

}  // namespace mrhs

namespace {
using namespace mrhs;

constexpr int kMaxC = 32;
constexpr int kCB = 12;         // output channels per thread (one block for the 11-triplet hidden layers)

size_t layer_w(const NNState& s, int l) { return (size_t)9 * s.C[l + 1] * s.C[l]; }
size_t layer_off(const NNState& s, int l) {
  size_t o = 0;
  for (int i = 0; i < l; ++i) o += layer_w(s, i);
  return o;
}

// colour transport of the triplet at neighbour row base, by T_k(x) with sign
__device__ __forceinline__ void link_k(cx<float> T[3][3], const float* U32, const int* nbr, size_t x, int k, size_t& n,
                                       float& sg) {
  if (k == 0) {
    n = x;
    sg = 1.f;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) T[a][b] = mk(a == b ? 1.f : 0.f, 0.f);
    return;
  }
  const int mu = (k - 1) % 4;
  const int e = nbr[x * 8 + (k <= 4 ? 0 : 4) + mu];
  n = (size_t)(e & 0x3fffffff);
  sg = (e & 0x40000000) ? -1.f : 1.f;
  const float* u = U32 + ((k <= 4 ? x : n) * 4 + mu) * 18;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (k <= 4) T[a][b] = mk(u[(a * 3 + b) * 2], u[(a * 3 + b) * 2 + 1]);
      else T[a][b] = mk(u[(b * 3 + a) * 2], -u[(b * 3 + a) * 2 + 1]);
    }
}

// z = covconv(h): thread per (site, rhs, block of kCB output channels)
__global__ void k_covconv(const float* __restrict__ h, float* __restrict__ z, const float* __restrict__ W,
                          const float* __restrict__ U32, const int* __restrict__ nbr, int cin, int cout, int N,
                          size_t nwork) {
  extern __shared__ float sW[];  // [9][cout][cin] complex
  const int nwc = 9 * cout * cin * 2;
  for (int i = threadIdx.x; i < nwc; i += blockDim.x) sW[i] = W[i];
  __syncthreads();
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= nwork) return;
  const int nblk = (cout + kCB - 1) / kCB;
  const int r = (int)(t % N);
  const int cb = (int)((t / N) % nblk);
  const size_t x = t / N / nblk;
  const int c0 = cb * kCB;
  cx<float> acc[kCB][3];
#pragma unroll
  for (int i = 0; i < kCB; ++i)
#pragma unroll
    for (int a = 0; a < 3; ++a) acc[i][a] = mk(0.f, 0.f);
  for (int k = 0; k < 9; ++k) {
    cx<float> T[3][3];
    size_t n;
    float sg;
    link_k(T, U32, nbr, x, k, n, sg);
    for (int cp = 0; cp < cin; ++cp) {
      cx<float> hv[3], tv[3];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const size_t row = (n * cin + cp) * 3 + b;
        hv[b] = mk(h[fidx(row, 0, N, r)], h[fidx(row, 1, N, r)]);
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        cx<float> s = mk(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < 3; ++b) fma_(s, T[a][b], hv[b]);
        tv[a] = scale(s, sg);
      }
#pragma unroll
      for (int i = 0; i < kCB; ++i) {
        if (c0 + i >= cout) break;
        const float* w = sW + (((size_t)k * cout + c0 + i) * cin + cp) * 2;
        cx<float> wv = mk(w[0], w[1]);
#pragma unroll
        for (int a = 0; a < 3; ++a) fma_(acc[i][a], wv, tv[a]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < kCB; ++i) {
    if (c0 + i >= cout) break;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const size_t row = (x * cout + c0 + i) * 3 + a;
      z[fidx(row, 0, N, r)] = acc[i][a].re;
      z[fidx(row, 1, N, r)] = acc[i][a].im;
    }
  }
}

// Wm[k'][c'][c] = conj(W[mirror(k')][c][c']) for one layer
__global__ void k_mirror(const float* W, float* Wm, int cin, int cout) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 9 * cout * cin) return;
  const int kp = t / (cin * cout), cp = (t / cout) % cin, c = t % cout;
  const int k = kp == 0 ? 0 : (kp <= 4 ? kp + 4 : kp - 4);
  const float* w = W + (((size_t)k * cout + c) * cin + cp) * 2;
  Wm[t * 2] = w[0];
  Wm[t * 2 + 1] = -w[1];
}

__global__ void k_modrelu(const float* z, float* h, const float* bias, int C, int N, size_t nwork) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= nwork) return;
  const int r = (int)(t % N);
  const size_t q = t / N;  // site*C + c
  const int c = (int)(q % C);
  float n2 = 0;
  cx<float> v[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    v[a] = mk(z[fidx(q * 3 + a, 0, N, r)], z[fidx(q * 3 + a, 1, N, r)]);
    n2 += v[a].re * v[a].re + v[a].im * v[a].im;
  }
  const float n = sqrtf(n2);
  const float f = (n > 0.f && n + bias[c] > 0.f) ? (n + bias[c]) / n : 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    h[fidx(q * 3 + a, 0, N, r)] = v[a].re * f;
    h[fidx(q * 3 + a, 1, N, r)] = v[a].im * f;
  }
}

// dz = modReLU'(z)^T dh (in place allowed), and per-CTA partials of the bias
// gradient: thread (channel c = tid % C, lane = tid / C) walks the CTA's
// sites and the right-hand sides r = lane, lane + lanes, ...; the lanes of a
// channel are summed in a fixed order
__global__ void k_modrelu_back(const float* z, const float* dh, float* dz, const float* bias, int C, int N,
                               size_t nsites, double* dbpart) {
  __shared__ float sdb[256];
  const int lanes = blockDim.x / C;
  const int c = threadIdx.x % C, lane = threadIdx.x / C;
  const bool act = lane < lanes;
  const size_t per = (nsites + gridDim.x - 1) / gridDim.x;
  const size_t s0 = blockIdx.x * per, s1 = min(nsites, s0 + per);
  float db = 0.f;
  if (act) {
    const float bc = bias[c];
    for (size_t x = s0; x < s1; ++x)
      for (int r = lane; r < N; r += lanes) {
        const size_t q = x * C + c;
        cx<float> v[3], d[3];
        float n2 = 0, zd = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          v[a] = mk(z[fidx(q * 3 + a, 0, N, r)], z[fidx(q * 3 + a, 1, N, r)]);
          d[a] = mk(dh[fidx(q * 3 + a, 0, N, r)], dh[fidx(q * 3 + a, 1, N, r)]);
          n2 += v[a].re * v[a].re + v[a].im * v[a].im;
          zd += v[a].re * d[a].re + v[a].im * d[a].im;
        }
        const float n = sqrtf(n2);
        const bool on = n > 0.f && n + bc > 0.f;
        const float f = on ? 1.f + bc / n : 0.f;
        const float g = on ? bc / (n * n * n) * zd : 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          dz[fidx(q * 3 + a, 0, N, r)] = f * d[a].re - g * v[a].re;
          dz[fidx(q * 3 + a, 1, N, r)] = f * d[a].im - g * v[a].im;
        }
        if (on) db += zd / n;
      }
  }
  sdb[threadIdx.x] = act ? db : 0.f;
  __syncthreads();
  if (threadIdx.x < C) {
    double a = 0;
    for (int l = 0; l < lanes; ++l) a += sdb[l * C + threadIdx.x];
    dbpart[(size_t)blockIdx.x * C + threadIdx.x] = a;
  }
}

// weight gradient partials: CTA (k, site range); thread (c, c') pairs over
// the CTA's sites and all right-hand sides; one right-hand side and 8 sites
// staged at a time
constexpr int kWgSites = 8;
__global__ void k_wgrad(const float* __restrict__ dz, const float* __restrict__ h, const float* __restrict__ U32,
                        const int* __restrict__ nbr, int cin, int cout, int N, size_t V, size_t sites_per_cta,
                        double* part) {
  __shared__ cx<float> sdz[kWgSites][kMaxC][3];
  __shared__ cx<float> stv[kWgSites][kMaxC][3];
  const int k = blockIdx.y;
  const size_t s0 = blockIdx.x * sites_per_cta;
  const size_t s1 = min(V, s0 + sites_per_cta);
  const int npair = cout * cin;
  double accr[4] = {0, 0, 0, 0}, acci[4] = {0, 0, 0, 0};
  for (size_t sb = s0; sb < s1; sb += kWgSites) {
    const int ns = (int)min((size_t)kWgSites, s1 - sb);
    for (int r = 0; r < N; ++r) {
      for (int w = threadIdx.x; w < ns * cout * 3; w += blockDim.x) {
        const int q = w / (cout * 3), c = (w / 3) % cout, a = w % 3;
        const size_t row = ((sb + q) * cout + c) * 3 + a;
        sdz[q][c][a] = mk(dz[fidx(row, 0, N, r)], dz[fidx(row, 1, N, r)]);
      }
      for (int w = threadIdx.x; w < ns * cin; w += blockDim.x) {
        const int q = w / cin, cp = w % cin;
        cx<float> T[3][3];
        size_t n;
        float sg;
        link_k(T, U32, nbr, sb + q, k, n, sg);
        cx<float> hv[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const size_t row = (n * cin + cp) * 3 + b;
          hv[b] = mk(h[fidx(row, 0, N, r)], h[fidx(row, 1, N, r)]);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          cx<float> s = mk(0.f, 0.f);
#pragma unroll
          for (int b = 0; b < 3; ++b) fma_(s, T[a][b], hv[b]);
          stv[q][cp][a] = scale(s, sg);
        }
      }
      __syncthreads();
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int p = threadIdx.x + e * blockDim.x;
        if (p >= npair) break;
        const int c = p / cin, cp = p % cin;
        cx<float> s = mk(0.f, 0.f);
        for (int q = 0; q < ns; ++q)
#pragma unroll
          for (int a = 0; a < 3; ++a) fmac_(s, stv[q][cp][a], sdz[q][c][a]);  // dz conj(t)
        accr[e] += s.re;
        acci[e] += s.im;
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int p = threadIdx.x + e * blockDim.x;
    if (p >= npair) break;
    double* o = part + (((size_t)k * gridDim.x + blockIdx.x) * npair + p) * 2;
    o[0] = accr[e];
    o[1] = acci[e];
  }
}

// G[k][p] += factor * sum of the per-CTA partials (fixed order)
__global__ void k_wgrad_sum(const double* part, int nchunk, int npair, float* G, float factor) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 9 * npair) return;
  const int k = t / npair, p = t % npair;
  double a = 0, b = 0;
  for (int ch = 0; ch < nchunk; ++ch) {
    a += part[(((size_t)k * nchunk + ch) * npair + p) * 2];
    b += part[(((size_t)k * nchunk + ch) * npair + p) * 2 + 1];
  }
  G[2 * t] += (float)(factor * a);
  G[2 * t + 1] += (float)(factor * b);
}

__global__ void k_bias_sum(const double* part, int nchunk, int C, float* G) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double a = 0;
  for (int ch = 0; ch < nchunk; ++ch) a += part[(size_t)ch * C + c];
  G[c] += (float)a;
}

__global__ void k_round_bf16(const float* W, float* Wc, size_t n, int on) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t < n) Wc[t] = on ? __bfloat162float(__float2bfloat16(W[t])) : W[t];
}

__global__ void k_adam(float* W, const float* G, float* m1, float* m2, size_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float g = G[t];
  const float a = b1 * m1[t] + (1.f - b1) * g;
  const float v = b2 * m2[t] + (1.f - b2) * g * g;
  m1[t] = a;
  m2[t] = v;
  W[t] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

// loss pieces: dv = 2 (DDv/vv - dd v/vv^2) + 2 lam (q/vv - qq v/vv^2), q = v - P P^dag v
__global__ void k_loss_grad(const float* v, const float* DDv, const float* q, const double* vv, const double* dd,
                            const double* qq, float* dv, float lam, int N, size_t nwork) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= nwork) return;
  const int r = (int)(t % N);
  const float a = (float)(1.0 / vv[2 * r]);
  const float b = (float)(dd[2 * r] / (vv[2 * r] * vv[2 * r]));
  const float c = (float)(qq[2 * r] / (vv[2 * r] * vv[2 * r]));
  dv[t] = 2.f * (DDv[t] * a - b * v[t]) + 2.f * lam * (q[t] * a - c * v[t]);
}

__global__ void k_gamma5(const float* x, float* y, int N, size_t nwork) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= nwork) return;
  const size_t row = t / (2 * (size_t)N);
  y[t] = ((row % 12) < 6) ? x[t] : -x[t];
}

// y (N_y = nr right-hand sides) <- x (right-hand sides r0 .. r0+nr-1 of N_x)
__global__ void k_gather_rhs(const float* x, int Nx, int r0, float* y, int nr, size_t rows) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= rows * 2 * nr) return;
  const int r = (int)(t % nr);
  const size_t q = t / nr;  // row*2 + reim
  y[t] = x[q * Nx + r0 + r];
}
__global__ void k_scatter_rhs(const float* y, int nr, float* x, int Nx, int r0, size_t rows) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= rows * 2 * nr) return;
  const int r = (int)(t % nr);
  const size_t q = t / nr;
  x[q * Nx + r0 + r] = y[t];
}

__global__ void k_sub(const float* a, const float* b, float* c, size_t n) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t < n) c[t] = a[t] - b[t];
}

}  // namespace

namespace mrhs {
void nn_destroy(mrhs_ctx c) {
  delete c->nn;
  c->nn = nullptr;
}
}  // namespace mrhs

namespace {

NNState& nn_of(mrhs_ctx c) {
  MRHS_REQUIRE(c, MRHS_ERR_ARG, "null context");
  MRHS_REQUIRE(c->nn, MRHS_ERR_STATE, "mrhs_nn_create has not been called");
  return *c->nn;
}

void ensure_acts(mrhs_ctx c, NNState& s, int N) {
  if (s.nrhs >= N) return;
  const size_t V = c->g.V;
  s.z1 = (float*)dalloc(c, sizeof(float) * V * s.C[1] * 6 * N);
  s.h1 = (float*)dalloc(c, sizeof(float) * V * s.C[1] * 6 * N);
  s.z2 = (float*)dalloc(c, sizeof(float) * V * s.C[2] * 6 * N);
  s.h2 = (float*)dalloc(c, sizeof(float) * V * s.C[2] * 6 * N);
  s.in = (float*)dalloc(c, sizeof(float) * V * s.C[0] * 6 * N);
  s.nrhs = N;
}

void covconv(mrhs_ctx c, const float* h, float* z, const float* W, int cin, int cout, int N) {
  const int nblk = (cout + kCB - 1) / kCB;
  const size_t work = (size_t)c->g.V * nblk * N;
  const size_t smem = sizeof(float) * 2 * 9 * cin * cout;
  MRHS_CUDA(cudaFuncSetAttribute(k_covconv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  Prof pr(c, "nn_covconv");
  k_covconv<<<grid_for(work, 128), 128, smem, c->stream>>>(h, z, W, c->U32, c->nbr, cin, cout, N, work);
  MRHS_LAUNCH_CHECK("covconv");
}

void nn_forward_impl(mrhs_ctx c, const float* in, float* out, int N) {
  NNState& s = nn_of(c);
  ensure_acts(c, s, N);
  const size_t V = c->g.V;
  MRHS_CUDA(cudaMemcpyAsync(s.in, in, sizeof(float) * V * 24 * N, cudaMemcpyDeviceToDevice, c->stream));
  const float* bias = s.Wc + 2 * s.nw;
  covconv(c, in, s.z1, s.Wc + 2 * layer_off(s, 0), s.C[0], s.C[1], N);
  k_modrelu<<<grid_for(V * s.C[1] * N, 256), 256, 0, c->stream>>>(s.z1, s.h1, bias, s.C[1], N, V * s.C[1] * N);
  MRHS_LAUNCH_CHECK("modrelu");
  covconv(c, s.h1, s.z2, s.Wc + 2 * layer_off(s, 1), s.C[1], s.C[2], N);
  k_modrelu<<<grid_for(V * s.C[2] * N, 256), 256, 0, c->stream>>>(s.z2, s.h2, bias + s.C[1], s.C[2], N,
                                                                   V * s.C[2] * N);
  MRHS_LAUNCH_CHECK("modrelu");
  covconv(c, s.h2, out, s.Wc + 2 * layer_off(s, 2), s.C[2], s.C[3], N);
}

void wgrad(mrhs_ctx c, NNState& s, const float* dz, const float* h, int l, int N) {
  const int cin = s.C[l], cout = s.C[l + 1];
  const size_t V = c->g.V;
  const int nchunk = (int)std::min<size_t>(256, (V + 511) / 512);
  const size_t per = (V + nchunk - 1) / nchunk;
  const size_t need = (size_t)9 * nchunk * cout * cin * 2;
  MRHS_REQUIRE(need <= s.part_elems, MRHS_ERR_ARG, "nn: partial buffer too small");
  dim3 grid(nchunk, 9);
  Prof pr(c, "nn_wgrad");
  k_wgrad<<<grid, 256, 0, c->stream>>>(dz, h, c->U32, c->nbr, cin, cout, N, V, per, s.part);
  MRHS_LAUNCH_CHECK("wgrad");
  k_wgrad_sum<<<grid_for((size_t)9 * cout * cin, 256), 256, 0, c->stream>>>(s.part, nchunk, cout * cin,
                                                                            s.G + 2 * layer_off(s, l), 1.f);
  MRHS_LAUNCH_CHECK("wgrad_sum");
}

void modrelu_back(mrhs_ctx c, NNState& s, const float* z, const float* dh, float* dz, int l, int N) {
  const int C = s.C[l];
  const size_t V = c->g.V;
  const int nb = 512;
  const float* bias = s.Wc + 2 * s.nw + (l == 1 ? 0 : s.C[1]);
  k_modrelu_back<<<nb, 256, 0, c->stream>>>(z, dh, dz, bias, C, N, V, s.part);
  MRHS_LAUNCH_CHECK("modrelu_back");
  k_bias_sum<<<1, 64, 0, c->stream>>>(s.part, nb, C, s.G + 2 * s.nw + (l == 1 ? 0 : s.C[1]));
  MRHS_LAUNCH_CHECK("bias_sum");
}

// gradient of a real loss through the network. dout = dL/dRe(out) + i dL/dIm(out).
// Weight gradients accumulate into G; din (may be null) receives dL/dRe(in) + i dL/dIm(in).
void nn_backward(mrhs_ctx c, const float* dout, float* din, int N) {
  NNState& s = nn_of(c);
  MRHS_REQUIRE(s.nrhs >= N, MRHS_ERR_STATE, "nn backward before a forward pass of that many right-hand sides");
  const size_t V = c->g.V;
  float* d2 = (float*)scratch(c, SC_FINE1, sizeof(float) * V * std::max(s.C[1], s.C[2]) * 6 * N);
  float* d1 = (float*)scratch(c, SC_FINE2, sizeof(float) * V * std::max(s.C[1], s.C[2]) * 6 * N);
  // mirrored conjugate-transposed weights for the backward data passes
  for (int l = 0; l < 3; ++l) {
    const int n = 9 * s.C[l] * s.C[l + 1];
    k_mirror<<<grid_for(n, 256), 256, 0, c->stream>>>(s.Wc + 2 * layer_off(s, l), s.Wm + 2 * layer_off(s, l), s.C[l],
                                                      s.C[l + 1]);
    MRHS_LAUNCH_CHECK("mirror");
  }
  // layer 2: out = covconv(h2)
  wgrad(c, s, dout, s.h2, 2, N);
  covconv(c, dout, d2, s.Wm + 2 * layer_off(s, 2), s.C[3], s.C[2], N);  // dL/dh2
  modrelu_back(c, s, s.z2, d2, d2, 2, N);                                // dL/dz2
  wgrad(c, s, d2, s.h1, 1, N);
  covconv(c, d2, d1, s.Wm + 2 * layer_off(s, 1), s.C[2], s.C[1], N);    // dL/dh1
  modrelu_back(c, s, s.z1, d1, d1, 1, N);                                // dL/dz1
  wgrad(c, s, d1, s.in, 0, N);
  if (din) covconv(c, d1, din, s.Wm + 2 * layer_off(s, 0), s.C[1], s.C[0], N);
}

// loss and dL/dv of the test vectors v (FP32 field, N right-hand sides) using
// the context's current P as the plain vectors' prolongation
double nn_loss(mrhs_ctx c, const float* v, float* dv, int N, double lam, double* per_rhs) {
  MRHS_REQUIRE(c->have_P, MRHS_ERR_STATE, "nn loss needs the plain setup's P (run the setup first)");
  MRHS_REQUIRE(c->work_dtype == MRHS_F32, MRHS_ERR_ARG, "nn loss runs on FP32 contexts");
  const size_t V = c->g.V;
  const size_t n = V * 24 * (size_t)N;
  float* Dv = (float*)scratch(c, SC_FINE1, sizeof(float) * n * 3);
  float* DDv = Dv + n;
  float* q = DDv + n;
  float* cbuf = (float*)scratch(c, SC_COARSE, coarse_elems(c, N) * sizeof(float));
  double* nr = (double*)scratch(c, SC_MISC, sizeof(double) * 6 * N);
  dslash(c, v, Dv, nullptr, N, MRHS_F32, DS_FULL, -1);
  k_gamma5<<<grid_for(n, 256), 256, 0, c->stream>>>(Dv, q, N, n);
  dslash(c, q, DDv, nullptr, N, MRHS_F32, DS_FULL, -1);
  k_gamma5<<<grid_for(n, 256), 256, 0, c->stream>>>(DDv, DDv, N, n);
  MRHS_LAUNCH_CHECK("gamma5");
  restrict_(c, v, cbuf, N, MRHS_F32);
  prolong(c, cbuf, q, N, MRHS_F32);
  k_sub<<<grid_for(n, 256), 256, 0, c->stream>>>(v, q, q, n);
  MRHS_LAUNCH_CHECK("sub");
  norms(c, v, V * 12, N, MRHS_F32, nr);
  norms(c, Dv, V * 12, N, MRHS_F32, nr + 2 * N);
  norms(c, q, V * 12, N, MRHS_F32, nr + 4 * N);
  if (dv) {
    k_loss_grad<<<grid_for(n, 256), 256, 0, c->stream>>>(v, DDv, q, nr, nr + 2 * N, nr + 4 * N, dv, (float)lam, N, n);
    MRHS_LAUNCH_CHECK("loss_grad");
  }
  std::vector<double> h(6 * N);
  MRHS_CUDA(cudaMemcpyAsync(h.data(), nr, sizeof(double) * 6 * N, cudaMemcpyDeviceToHost, c->stream));
  MRHS_CUDA(cudaStreamSynchronize(c->stream));
  double tot = 0;
  for (int r = 0; r < N; ++r) {
    double l = h[2 * N + 2 * r] / h[2 * r] + lam * h[4 * N + 2 * r] / h[2 * r];
    if (per_rhs) per_rhs[r] = l;
    tot += l;
  }
  return tot;
}

void refresh_compute_weights(mrhs_ctx c, NNState& s) {
  const size_t n = 2 * s.nw + s.nb;
  k_round_bf16<<<grid_for(n, 256), 256, 0, c->stream>>>(s.W, s.Wc, 2 * s.nw, s.bf16 ? 1 : 0);
  MRHS_LAUNCH_CHECK("round_bf16");
  MRHS_CUDA(cudaMemcpyAsync(s.Wc + 2 * s.nw, s.W + 2 * s.nw, sizeof(float) * s.nb, cudaMemcpyDeviceToDevice,
                            c->stream));
  (void)n;
}

}  // namespace

// one layer for inference: the channel mixing on the tensor cores (bf16
// operands) when the weights are bf16 and the layer has 16 or more channels
// on one side, else on the CUDA cores. Measured at 48^3x96 with 32 vectors:
// the 4-11-11-4 network takes 1545 ms on the tensor-core layer against 829 ms
// on the CUDA cores (the tensor-core layer's per-tile cost of staging, steps
// and epilogue dominates at few channels), the 4-32-32-4 network 2254 ms
// against 6008 ms.
void infer_layer(mrhs_ctx c, const NNState& s, const float* h, float* z, int l, int N) {
  const float* W = s.Wc + 2 * layer_off(s, l);
  if (s.bf16 && std::max(s.C[l], s.C[l + 1]) >= 16 && covconv_tc(c, h, z, W, s.C[l], s.C[l + 1], N)) return;
  covconv(c, h, z, W, s.C[l], s.C[l + 1], N);
}

// inference only (no activations kept): right-hand sides in chunks, two
// ping-pong buffers for the hidden layers
void nn_infer_chunked(mrhs_ctx c, const float* in, float* out, int N, int chunk) {
  NNState& s = nn_of(c);
  const size_t V = c->g.V;
  const int hid = std::max(s.C[1], s.C[2]);
  const int cs = std::min(N, chunk);
  float* a = (float*)scratch(c, SC_FINE1, sizeof(float) * V * hid * 6 * cs);
  float* b = (float*)scratch(c, SC_FINE2, sizeof(float) * V * hid * 6 * cs);
  float* io = (float*)scratch(c, SC_FINE3, sizeof(float) * V * 24 * cs * 2);
  float* xin = io;
  float* xout = io + V * 24 * cs;
  const float* bias = s.Wc + 2 * s.nw;
  for (int r0 = 0; r0 < N; r0 += cs) {
    const int nr = std::min(cs, N - r0);
    k_gather_rhs<<<grid_for(V * 12 * 2 * nr, 256), 256, 0, c->stream>>>(in, N, r0, xin, nr, V * 12);
    MRHS_LAUNCH_CHECK("gather_rhs");
    infer_layer(c, s, xin, a, 0, nr);
    k_modrelu<<<grid_for(V * s.C[1] * nr, 256), 256, 0, c->stream>>>(a, a, bias, s.C[1], nr, V * s.C[1] * nr);
    MRHS_LAUNCH_CHECK("modrelu");
    infer_layer(c, s, a, b, 1, nr);
    k_modrelu<<<grid_for(V * s.C[2] * nr, 256), 256, 0, c->stream>>>(b, b, bias + s.C[1], s.C[2], nr,
                                                                     V * s.C[2] * nr);
    MRHS_LAUNCH_CHECK("modrelu");
    infer_layer(c, s, b, xout, 2, nr);
    k_scatter_rhs<<<grid_for(V * 12 * 2 * nr, 256), 256, 0, c->stream>>>(xout, nr, out, N, r0, V * 12);
    MRHS_LAUNCH_CHECK("scatter_rhs");
  }
}

namespace mrhs {
void nn_forward(mrhs_ctx c, const float* in, float* out, int N) { nn_forward_impl(c, in, out, N); }
// inference in chunks of right-hand sides: up to 8 at a time, fewer when the
// activations of 8 (two hidden fields and the chunk's input and output) would
// take more than half of the device memory still available
void nn_infer(mrhs_ctx c, const float* in, float* out, int N) {
  NNState& s = nn_of(c);
  const int hid = std::max(s.C[1], s.C[2]);
  const size_t per_rhs = sizeof(float) * (size_t)c->g.V * (2 * (size_t)hid * 6 + 2 * 24);
  size_t free_b = 0, total_b = 0;
  MRHS_CUDA(cudaMemGetInfo(&free_b, &total_b));
  size_t avail = free_b;
  for (int k : {SC_FINE1, SC_FINE2, SC_FINE3}) avail += c->scratch[k].bytes;  // reusable
  int chunk = 8;
  while (chunk > 1 && (size_t)chunk * per_rhs > avail / 2) --chunk;
  nn_infer_chunked(c, in, out, N, chunk);
  check_nn_tc_timeout(c);
}
}  // namespace mrhs

using namespace mrhs;

extern "C" {

int mrhs_nn_create(mrhs_ctx c, const int widths[4], int bf16_weights) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && widths, MRHS_ERR_ARG, "null argument");
    MRHS_REQUIRE(widths[0] == 4 && widths[3] == 4, MRHS_ERR_SHAPE, "the network maps spinors: widths[0] = widths[3] = 4");
    MRHS_REQUIRE(widths[1] >= 1 && widths[1] <= kMaxC && widths[2] >= 1 && widths[2] <= kMaxC, MRHS_ERR_SHAPE,
                 "hidden widths must be in 1..32");
    MRHS_REQUIRE(!c->nn, MRHS_ERR_STATE, "the network already exists");
    NNState* s = new NNState();
    for (int i = 0; i < 4; ++i) s->C[i] = widths[i];
    s->nw = layer_off(*s, 3);
    s->nb = (size_t)widths[1] + widths[2];
    s->bf16 = bf16_weights != 0;
    const size_t n = 2 * s->nw + s->nb;
    s->W = (float*)dalloc(c, sizeof(float) * n);
    s->Wc = (float*)dalloc(c, sizeof(float) * n);
    s->Wm = (float*)dalloc(c, sizeof(float) * 2 * s->nw);
    s->G = (float*)dalloc(c, sizeof(float) * n);
    s->m1 = (float*)dalloc(c, sizeof(float) * n);
    s->m2 = (float*)dalloc(c, sizeof(float) * n);
    s->part_elems = (size_t)9 * 256 * kMaxC * kMaxC * 2;
    s->part = (double*)dalloc(c, sizeof(double) * s->part_elems);
    MRHS_CUDA(cudaMemsetAsync(s->W, 0, sizeof(float) * n, c->stream));
    MRHS_CUDA(cudaMemsetAsync(s->G, 0, sizeof(float) * n, c->stream));
    MRHS_CUDA(cudaMemsetAsync(s->m1, 0, sizeof(float) * n, c->stream));
    MRHS_CUDA(cudaMemsetAsync(s->m2, 0, sizeof(float) * n, c->stream));
    c->nn = s;
    refresh_compute_weights(c, *s);
  });
}

int mrhs_nn_num_params(mrhs_ctx c, long long* n_complex, long long* n_real) {
  return guarded(c, [&] {
    NNState& s = nn_of(c);
    if (n_complex) *n_complex = (long long)s.nw;
    if (n_real) *n_real = (long long)s.nb;
  });
}

int mrhs_nn_set_weights(mrhs_ctx c, const float* host) {
  return guarded(c, [&] {
    MRHS_REQUIRE(host, MRHS_ERR_ARG, "null argument");
    NNState& s = nn_of(c);
    require_host(c, host, "mrhs_nn_set_weights host");
    MRHS_CUDA(cudaMemcpyAsync(s.W, host, sizeof(float) * (2 * s.nw + s.nb), cudaMemcpyHostToDevice, c->stream));
    refresh_compute_weights(c, s);
    MRHS_CUDA(cudaStreamSynchronize(c->stream));
  });
}

int mrhs_nn_get_weights(mrhs_ctx c, float* host, int compute_copy) {
  return guarded(c, [&] {
    MRHS_REQUIRE(host, MRHS_ERR_ARG, "null argument");
    NNState& s = nn_of(c);
    require_host(c, host, "mrhs_nn_get_weights host");
    MRHS_CUDA(cudaMemcpyAsync(host, compute_copy ? s.Wc : s.W, sizeof(float) * (2 * s.nw + s.nb),
                              cudaMemcpyDeviceToHost, c->stream));
    MRHS_CUDA(cudaStreamSynchronize(c->stream));
  });
}

int mrhs_nn_get_grads(mrhs_ctx c, float* host) {
  return guarded(c, [&] {
    MRHS_REQUIRE(host, MRHS_ERR_ARG, "null argument");
    NNState& s = nn_of(c);
    require_host(c, host, "mrhs_nn_get_grads host");
    MRHS_CUDA(cudaMemcpyAsync(host, s.G, sizeof(float) * (2 * s.nw + s.nb), cudaMemcpyDeviceToHost, c->stream));
    MRHS_CUDA(cudaStreamSynchronize(c->stream));
  });
}

int mrhs_nn_zero_grads(mrhs_ctx c) {
  return guarded(c, [&] {
    NNState& s = nn_of(c);
    MRHS_CUDA(cudaMemsetAsync(s.G, 0, sizeof(float) * (2 * s.nw + s.nb), c->stream));
  });
}

int mrhs_nn_forward(mrhs_ctx c, const void* in, void* out, int nrhs) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && in && out && nrhs >= 1, MRHS_ERR_ARG, "bad argument");
    require_dev(c, in, "mrhs_nn_forward in");
    require_dev(c, out, "mrhs_nn_forward out");
    MRHS_REQUIRE(c->have_gauge, MRHS_ERR_STATE, "nn forward before mrhs_set_gauge");
    nn_forward_impl(c, (const float*)in, (float*)out, nrhs);
  });
}

int mrhs_nn_infer(mrhs_ctx c, const void* in, void* out, int nrhs) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && in && out && nrhs >= 1, MRHS_ERR_ARG, "bad argument");
    require_dev(c, in, "mrhs_nn_infer in");
    require_dev(c, out, "mrhs_nn_infer out");
    MRHS_REQUIRE(c->have_gauge, MRHS_ERR_STATE, "nn inference before mrhs_set_gauge");
    nn_infer(c, (const float*)in, (float*)out, nrhs);
  });
}

int mrhs_nn_backward(mrhs_ctx c, const void* grad_out, void* grad_in, int nrhs) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && grad_out && nrhs >= 1, MRHS_ERR_ARG, "bad argument");
    require_dev(c, grad_out, "mrhs_nn_backward grad_out");
    require_dev(c, grad_in, "mrhs_nn_backward grad_in");
    nn_backward(c, (const float*)grad_out, (float*)grad_in, nrhs);
  });
}

int mrhs_nn_loss(mrhs_ctx c, const void* v, void* grad_v, int nrhs, double lambda, double* loss, double* per_rhs) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && v && loss && nrhs >= 1, MRHS_ERR_ARG, "bad argument");
    require_dev(c, v, "mrhs_nn_loss v");
    require_dev(c, grad_v, "mrhs_nn_loss grad_v");
    require_host(c, per_rhs, "mrhs_nn_loss per_rhs");
    *loss = nn_loss(c, (const float*)v, (float*)grad_v, nrhs, lambda, per_rhs);
  });
}

int mrhs_nn_adam(mrhs_ctx c, float lr, float beta1, float beta2, float eps, int step) {
  return guarded(c, [&] {
    NNState& s = nn_of(c);
    MRHS_REQUIRE(step >= 1, MRHS_ERR_ARG, "Adam step counts from 1");
    const size_t n = 2 * s.nw + s.nb;
    const float c1 = 1.f - std::pow(beta1, (float)step), c2 = 1.f - std::pow(beta2, (float)step);
    k_adam<<<grid_for(n, 256), 256, 0, c->stream>>>(s.W, s.G, s.m1, s.m2, n, lr, beta1, beta2, eps, c1, c2);
    MRHS_LAUNCH_CHECK("adam");
    refresh_compute_weights(c, s);
  });
}

int mrhs_nn_train_step(mrhs_ctx c, const void* v_in, int nrhs, double lambda, float lr, int step, double* loss) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && v_in && loss && nrhs >= 1, MRHS_ERR_ARG, "bad argument");
    require_dev(c, v_in, "mrhs_nn_train_step v_in");
    NNState& s = nn_of(c);
    const size_t n = (size_t)c->g.V * 24 * nrhs;
    float* out = (float*)scratch(c, SC_FINE3, sizeof(float) * n * 2);
    float* dv = out + n;
    nn_forward_impl(c, (const float*)v_in, out, nrhs);
    *loss = nn_loss(c, out, dv, nrhs, lambda, nullptr);
    MRHS_CUDA(cudaMemsetAsync(s.G, 0, sizeof(float) * (2 * s.nw + s.nb), c->stream));
    nn_backward(c, dv, nullptr, nrhs);
    const size_t np = 2 * s.nw + s.nb;
    const float c1 = 1.f - std::pow(0.9f, (float)step), c2 = 1.f - std::pow(0.999f, (float)step);
    k_adam<<<grid_for(np, 256), 256, 0, c->stream>>>(s.W, s.G, s.m1, s.m2, np, lr, 0.9f, 0.999f, 1e-8f, c1, c2);
    MRHS_LAUNCH_CHECK("adam");
    refresh_compute_weights(c, s);
  });
}

}  // extern "C"
