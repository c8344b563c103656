// Context, index tables, gauge field and clover term, field transfer and the
// C ABI entry points that do not belong to a specific solver stage.
#include <cstring>
#include <mutex>

#include "common.cuh"

using namespace mrhs;

namespace {
thread_local std::string g_create_error;
}  // namespace

namespace mrhs {
std::string& create_error_slot() { return g_create_error; }

void* dalloc(mrhs_ctx c, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  MRHS_CUDA(cudaMalloc(&p, bytes));
  c->allocs.push_back(p);
  c->held_bytes += bytes;
  return p;
}

void* scratch(mrhs_ctx c, int which, size_t bytes) {
  DevBuf& b = c->scratch[which];
  if (b.bytes < bytes) {
    if (b.p) {
      MRHS_CUDA(cudaStreamSynchronize(c->stream));
      MRHS_CUDA(cudaFree(b.p));
      c->held_bytes -= b.bytes;
      b.p = nullptr;
      b.bytes = 0;
    }
    MRHS_CUDA(cudaMalloc(&b.p, bytes));
    b.bytes = bytes;
    c->held_bytes += bytes;
  }
  return b.p;
}

double* host_scratch(mrhs_ctx c, size_t bytes) {
  if (c->hbuf_bytes < bytes) {
    if (c->hbuf) {
      MRHS_CUDA(cudaStreamSynchronize(c->stream));
      MRHS_CUDA(cudaFreeHost(c->hbuf));
      c->hbuf = nullptr;
    }
    MRHS_CUDA(cudaMallocHost((void**)&c->hbuf, bytes));
    c->hbuf_bytes = bytes;
  }
  return c->hbuf;
}

}  // namespace mrhs

// ------------------------------------------------------------- kernels ----
namespace {

struct GeomArgs {
  int L[4], a[4], nb[4];
  int V, Va, nagg;
};

GeomArgs geom_args(const Geometry& g) {
  GeomArgs r;
  for (int i = 0; i < 4; ++i) {
    r.L[i] = g.L[i];
    r.a[i] = g.a[i];
    r.nb[i] = g.nb[i];
  }
  r.V = g.V;
  r.Va = g.Va;
  r.nagg = g.nagg;
  return r;
}

__device__ __forceinline__ void unlex(const int* ext, int i, int* x) {
  for (int m = 0; m < 4; ++m) {
    x[m] = i % ext[m];
    i /= ext[m];
  }
}
__device__ __forceinline__ int lex(const int* ext, const int* x) {
  return x[0] + ext[0] * (x[1] + ext[1] * (x[2] + ext[2] * x[3]));
}
__device__ __forceinline__ int dev_site(const GeomArgs& g, const int* x) {
  int b[4], l[4];
  for (int m = 0; m < 4; ++m) {
    b[m] = x[m] / g.a[m];
    l[m] = x[m] % g.a[m];
  }
  return lex(g.nb, b) * g.Va + lex(g.a, l);
}

// device-order neighbour table and the canonical <-> device permutation
__global__ void k_tables(GeomArgs g, int* nbr, int* perm, int* iperm) {
  int sd = blockIdx.x * blockDim.x + threadIdx.x;
  if (sd >= g.V) return;
  int b[4], l[4], x[4];
  unlex(g.nb, sd / g.Va, b);
  unlex(g.a, sd % g.Va, l);
  for (int m = 0; m < 4; ++m) x[m] = b[m] * g.a[m] + l[m];
  int s = lex(g.L, x);
  perm[s] = sd;
  iperm[sd] = s;
  for (int mu = 0; mu < 4; ++mu)
    for (int d = 0; d < 2; ++d) {
      int y[4] = {x[0], x[1], x[2], x[3]};
      int v = y[mu] + (d == 0 ? 1 : -1);
      int wrap = 0;
      if (v < 0) { v += g.L[mu]; wrap = 1; }
      if (v >= g.L[mu]) { v -= g.L[mu]; wrap = 1; }
      y[mu] = v;
      int flip = (mu == 3) ? wrap : 0;
      nbr[sd * 8 + d * 4 + mu] = dev_site(g, y) | (flip << 30);
    }
}

__global__ void k_aggnbr(GeomArgs g, int* aggnbr) {
  int A = blockIdx.x * blockDim.x + threadIdx.x;
  if (A >= g.nagg) return;
  int b[4];
  unlex(g.nb, A, b);
  for (int mu = 0; mu < 4; ++mu)
    for (int d = 0; d < 2; ++d) {
      int c[4] = {b[0], b[1], b[2], b[3]};
      c[mu] = (c[mu] + (d == 0 ? 1 : -1) + g.nb[mu]) % g.nb[mu];
      aggnbr[A * 8 + d * 4 + mu] = lex(g.nb, c);
    }
}

// canonical-order export of the tables
__global__ void k_tables_canon(GeomArgs g, const int* nbr, const int* perm, const int* iperm, int* nbr_c,
                               int* aggof_c) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int sd = perm[s];
  for (int k = 0; k < 8; ++k) {
    int e = nbr[sd * 8 + k];
    nbr_c[s * 8 + k] = iperm[e & 0x3fffffff] | (e & 0x40000000);
  }
  aggof_c[2 * s] = sd / g.Va;
  aggof_c[2 * s + 1] = sd % g.Va;
}

// gauge field: canonical sites s0.. of [V][4][9] complex128 (staging) ->
// device order, f64 + f32 copies
// U20[x][mu] = (1/2) sgn(x, mu) U_mu(x) in FP32, padded to 20 floats: the hop
// factor 1/2 and the antiperiodic sign of a hop across the t boundary belong
// to the link (the forward hop from x and the backward hop from x+mu cross the
// boundary together)
__global__ void k_gauge_in(int s0, int ns, const int* perm, const double* Uc, double* U64, float* U32, float* U20,
                           int Lt_last_start) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)ns * 80) return;
  size_t s = t / 80, e = t % 80;
  size_t sd = (size_t)perm[s0 + s];
  size_t mu = e / 20, k = e % 20;
  if (k < 18) {
    double v = Uc[s * 72 + mu * 18 + k];
    U64[sd * 72 + mu * 18 + k] = v;
    U32[sd * 72 + mu * 18 + k] = (float)v;
    const bool flip = mu == 3 && (size_t)(s0 + s) >= (size_t)Lt_last_start;
    U20[sd * 80 + e] = (float)(flip ? -0.5 * v : 0.5 * v);
  } else {
    U20[sd * 80 + e] = 0.f;
  }
}

// ------------------------------------------------------------ clover ------
struct M3 {
  cx<double> m[3][3];
};
__device__ __forceinline__ M3 ld_link(const double* U, int s, int mu) {
  M3 r;
  const double* p = U + ((size_t)s * 4 + mu) * 18;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) r.m[a][b] = mk(p[(a * 3 + b) * 2], p[(a * 3 + b) * 2 + 1]);
  return r;
}
__device__ __forceinline__ M3 mm(const M3& x, const M3& y) {
  M3 r;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      cx<double> c = mk(0.0, 0.0);
      for (int k = 0; k < 3; ++k) fma_(c, x.m[a][k], y.m[k][b]);
      r.m[a][b] = c;
    }
  return r;
}
// x * y^dag
__device__ __forceinline__ M3 mmd(const M3& x, const M3& y) {
  M3 r;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      cx<double> c = mk(0.0, 0.0);
      for (int k = 0; k < 3; ++k) fma_(c, x.m[a][k], cnj(y.m[b][k]));
      r.m[a][b] = c;
    }
  return r;
}
// x^dag * y
__device__ __forceinline__ M3 mdm(const M3& x, const M3& y) {
  M3 r;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      cx<double> c = mk(0.0, 0.0);
      for (int k = 0; k < 3; ++k) fmac_(c, x.m[k][a], y.m[k][b]);
      r.m[a][b] = c;
    }
  return r;
}
__device__ __forceinline__ int hop(const int* nbr, int s, int mu, int d) {
  return nbr[s * 8 + (d > 0 ? 0 : 4) + mu] & 0x3fffffff;
}

// F_{mu nu}(x) = (Q - Q^dag)/8, Q = sum of the four plaquette leaves at x
__device__ void field_strength(const double* U, const int* nbr, int s, int mu, int nu, M3& F) {
  int xpm = hop(nbr, s, mu, +1), xpn = hop(nbr, s, nu, +1);
  int xmm = hop(nbr, s, mu, -1), xmn = hop(nbr, s, nu, -1);
  int xmm_pn = hop(nbr, xmm, nu, +1), xmm_mn = hop(nbr, xmm, nu, -1), xpm_mn = hop(nbr, xpm, nu, -1);
  M3 Q;
  // leaf in the (+mu,+nu) quadrant
  M3 t = mmd(mm(ld_link(U, s, mu), ld_link(U, xpm, nu)), mm(ld_link(U, s, nu), ld_link(U, xpn, mu)));
  Q = t;
  // (-mu,+nu): U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu)
  t = mm(mmd(ld_link(U, s, nu), mm(ld_link(U, xmm, nu), ld_link(U, xmm_pn, mu))), ld_link(U, xmm, mu));
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Q.m[a][b] = Q.m[a][b] + t.m[a][b];
  // (-mu,-nu): U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
  t = mdm(mm(ld_link(U, xmm_mn, nu), ld_link(U, xmm, mu)), mm(ld_link(U, xmm_mn, mu), ld_link(U, xmn, nu)));
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Q.m[a][b] = Q.m[a][b] + t.m[a][b];
  // (+mu,-nu): U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^dag
  t = mmd(mdm(ld_link(U, xmn, nu), mm(ld_link(U, xmn, mu), ld_link(U, xpm_mn, nu))), ld_link(U, s, mu));
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Q.m[a][b] = Q.m[a][b] + t.m[a][b];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) F.m[a][b] = scale(Q.m[a][b] - cnj(Q.m[b][a]), 0.125);
}

__host__ __device__ __forceinline__ int herm_off(int a, int b) {  // a < b
  return 5 * a - a * (a - 1) / 2 + (b - a - 1);
}

// Clover blocks. In the chiral basis sigma_{mu nu} restricted to chirality h
// is: spatial planes (k,l): -eps_klm sigma_m for both h; planes (k,t): +sigma_k
// for h = 0 and -sigma_k for h = 1 (Pauli sigma, k = mu+1). Hence
//   A_h = (4+m0) + (csw/2) i sum_m sigma_m (x) G_m,
//   G_1 = eta F_03 - F_12, G_2 = eta F_13 + F_02, G_3 = eta F_23 - F_01,
// eta = +1 (h=0), -1 (h=1). Packed per h: 6 real diagonals, then the 15
// upper off-diagonal entries (row-major, a<b) as (re, im).
__global__ void k_clover(int V, const double* U, const int* nbr, double m0, double csw, double* A64, float* A32) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  M3 F01, F02, F03, F12, F13, F23;
  field_strength(U, nbr, s, 0, 1, F01);
  field_strength(U, nbr, s, 0, 2, F02);
  field_strength(U, nbr, s, 0, 3, F03);
  field_strength(U, nbr, s, 1, 2, F12);
  field_strength(U, nbr, s, 1, 3, F13);
  field_strength(U, nbr, s, 2, 3, F23);
  const double hc = 0.5 * csw;
  for (int h = 0; h < 2; ++h) {
    double eta = h == 0 ? 1.0 : -1.0;
    cx<double> blk[6][6];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        cx<double> g1 = scale(F03.m[a][b], eta) - F12.m[a][b];
        cx<double> g2 = scale(F13.m[a][b], eta) + F02.m[a][b];
        cx<double> g3 = scale(F23.m[a][b], eta) - F01.m[a][b];
        cx<double> d = a == b ? mk(4.0 + m0, 0.0) : mk(0.0, 0.0);
        blk[a][b] = d + scale(ti(g3), hc);                 // spin (0,0)
        blk[3 + a][3 + b] = d - scale(ti(g3), hc);         // spin (1,1)
        blk[a][3 + b] = scale(ti(g1) + g2, hc);            // spin (0,1)
        blk[3 + a][b] = scale(ti(g1) - g2, hc);            // spin (1,0)
      }
    double* o64 = A64 + ((size_t)s * 2 + h) * 36;
    float* o32 = A32 + ((size_t)s * 2 + h) * 36;
    for (int a = 0; a < 6; ++a) {
      o64[a] = blk[a][a].re;
      o32[a] = (float)blk[a][a].re;
      for (int b = a + 1; b < 6; ++b) {
        int k = 6 + 2 * herm_off(a, b);
        o64[k] = blk[a][b].re;
        o64[k + 1] = blk[a][b].im;
        o32[k] = (float)blk[a][b].re;
        o32[k + 1] = (float)blk[a][b].im;
      }
    }
  }
}

// inverse of the clover term, per site and chirality (Gauss-Jordan with
// partial pivoting on the 6x6 block in FP64), packed like the clover term;
// *bad is set if a block is singular
__global__ void k_clover_inverse(int V, const double* A64, double* I64, float* I32, int* bad) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * V) return;
  const double* q = A64 + (size_t)t * 36;
  cx<double> m[6][12];
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 12; ++b) {
      if (b >= 6) m[a][b] = mk(b - 6 == a ? 1.0 : 0.0, 0.0);
      else if (a == b) m[a][b] = mk(q[a], 0.0);
      else if (b > a) m[a][b] = mk(q[6 + 2 * herm_off(a, b)], q[6 + 2 * herm_off(a, b) + 1]);
      else m[a][b] = mk(q[6 + 2 * herm_off(b, a)], -q[6 + 2 * herm_off(b, a) + 1]);
    }
  for (int c = 0; c < 6; ++c) {
    int p = c;
    double best = m[c][c].re * m[c][c].re + m[c][c].im * m[c][c].im;
    for (int i = c + 1; i < 6; ++i) {
      const double v = m[i][c].re * m[i][c].re + m[i][c].im * m[i][c].im;
      if (v > best) best = v, p = i;
    }
    if (!(best > 0)) {
      atomicExch(bad, 1);
      return;
    }
    if (p != c)
      for (int j = 0; j < 12; ++j) {
        const cx<double> tmp = m[p][j];
        m[p][j] = m[c][j];
        m[c][j] = tmp;
      }
    // row c /= pivot: multiply by conj(pivot) / |pivot|^2
    const cx<double> pc = scale(cnj(m[c][c]), 1.0 / best);
    for (int j = 0; j < 12; ++j) m[c][j] = m[c][j] * pc;
    for (int i = 0; i < 6; ++i) {
      if (i == c) continue;
      const cx<double> f = m[i][c];
      for (int j = 0; j < 12; ++j) m[i][j] = m[i][j] - f * m[c][j];
    }
  }
  double* o64 = I64 + (size_t)t * 36;
  float* o32 = I32 + (size_t)t * 36;
  for (int a = 0; a < 6; ++a) {
    o64[a] = m[a][6 + a].re;
    o32[a] = (float)m[a][6 + a].re;
    for (int b = a + 1; b < 6; ++b) {
      const int k = 6 + 2 * herm_off(a, b);
      o64[k] = m[a][6 + b].re;
      o64[k + 1] = m[a][6 + b].im;
      o32[k] = (float)m[a][6 + b].re;
      o32[k + 1] = (float)m[a][6 + b].im;
    }
  }
}

// packed clover -> dense canonical [V][2][6][6] complex128
__global__ void k_clover_out(int V, const int* perm, const double* A64, double* out) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  int sd = perm[s];
  for (int h = 0; h < 2; ++h) {
    const double* p = A64 + ((size_t)sd * 2 + h) * 36;
    double* o = out + ((size_t)s * 2 + h) * 72;
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 6; ++b) {
        double re, im;
        if (a == b) { re = p[a]; im = 0; }
        else if (a < b) { int k = 6 + 2 * herm_off(a, b); re = p[k]; im = p[k + 1]; }
        else { int k = 6 + 2 * herm_off(b, a); re = p[k]; im = -p[k + 1]; }
        o[(a * 6 + b) * 2] = re;
        o[(a * 6 + b) * 2 + 1] = im;
      }
  }
}

// ------------------------------------------------------- field transfer ---
// staging chunk: [nrhs][ns sites][12] complex (HT = double or float), sites
// s0..s0+ns-1 canonical; the device field has rows (site*12 + c)
template <class HT, class S>
__global__ void k_pack(const HT* st, S* dev, const int* perm, int s0, int ns, int nrhs) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t tot = (size_t)ns * 12 * nrhs;
  if (t >= tot) return;
  int r = t % nrhs;
  size_t q = t / nrhs;
  int c = q % 12;
  int sc = (int)(q / 12);
  const HT* src = st + (((size_t)r * ns + sc) * 12 + c) * 2;
  size_t row = (size_t)perm[s0 + sc] * 12 + c;
  dev[fidx(row, 0, nrhs, r)] = from_r<S>((double)src[0]);
  dev[fidx(row, 1, nrhs, r)] = from_r<S>((double)src[1]);
}

template <class HT, class S>
__global__ void k_unpack(HT* st, const S* dev, const int* perm, int s0, int ns, int nrhs) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t tot = (size_t)ns * 12 * nrhs;
  if (t >= tot) return;
  int r = t % nrhs;
  size_t q = t / nrhs;
  int c = q % 12;
  int sc = (int)(q / 12);
  HT* dst = st + (((size_t)r * ns + sc) * 12 + c) * 2;
  size_t row = (size_t)perm[s0 + sc] * 12 + c;
  dst[0] = (HT)to_r(dev[fidx(row, 0, nrhs, r)]);
  dst[1] = (HT)to_r(dev[fidx(row, 1, nrhs, r)]);
}

// coarse: host [nrhs][rows] complex, device rows (A*2ntv + i)
template <class HT, class S>
__global__ void k_pack_c(const HT* st, S* dev, size_t rows, int nrhs) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= rows * nrhs) return;
  int r = t % nrhs;
  size_t row = t / nrhs;
  dev[fidx(row, 0, nrhs, r)] = from_r<S>((double)st[(r * rows + row) * 2]);
  dev[fidx(row, 1, nrhs, r)] = from_r<S>((double)st[(r * rows + row) * 2 + 1]);
}
template <class HT, class S>
__global__ void k_unpack_c(HT* st, const S* dev, size_t rows, int nrhs) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= rows * nrhs) return;
  int r = t % nrhs;
  size_t row = t / nrhs;
  st[(r * rows + row) * 2] = (HT)to_r(dev[fidx(row, 0, nrhs, r)]);
  st[(r * rows + row) * 2 + 1] = (HT)to_r(dev[fidx(row, 1, nrhs, r)]);
}

template <class SI, class SO>
__global__ void k_convert(const SI* x, SO* y, size_t n) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t < n) y[t] = from_r<SO>(to_r(x[t]));
}

template <class SI, class SO>
__global__ void k_convert_scaled(const SI* x, SO* y, size_t n, float scale) {
  using R = typename Real<SI>::type;  // double data stays double
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t < n) y[t] = from_r<SO>(to_r(x[t]) * (R)scale);
}

void check_host_dtype(int hd) {
  MRHS_REQUIRE(hd == MRHS_F64 || hd == MRHS_F32, MRHS_ERR_ARG, "host dtype must be MRHS_F64 or MRHS_F32");
}

// transfer a fine field between host canonical and device interleaved, in
// chunks of sites through the staging buffer
void transfer_fine(mrhs_ctx c, const void* host_in, void* host_out, int hd, const void* dev_in, void* dev_out,
                   int dd, int nrhs) {
  check_host_dtype(hd);
  MRHS_REQUIRE(nrhs >= 1, MRHS_ERR_ARG, "nrhs must be >= 1");
  const size_t hes = hd == MRHS_F64 ? 16 : 8;  // bytes per complex on the host
  const int V = c->g.V;
  size_t per_site = (size_t)nrhs * 12 * hes;
  size_t chunk = std::max<size_t>(1, std::min<size_t>(V, (size_t(1) << 30) / per_site));
  void* st = scratch(c, SC_STAGE, chunk * per_site);
  for (size_t s0 = 0; s0 < (size_t)V; s0 += chunk) {
    int ns = (int)std::min(chunk, (size_t)V - s0);
    size_t w = (size_t)ns * 12 * hes;
    size_t pitch = (size_t)V * 12 * hes;
    size_t tot = (size_t)ns * 12 * nrhs;
    if (host_in) {
      MRHS_CUDA(cudaMemcpy2DAsync(st, w, (const char*)host_in + s0 * 12 * hes, pitch, w, nrhs,
                                  cudaMemcpyHostToDevice, c->stream));
      if (hd == MRHS_F64) {
        MRHS_DISPATCH(dd, S, (k_pack<double, S><<<grid_for(tot, 256), 256, 0, c->stream>>>(
                                 (const double*)st, (S*)dev_out, c->perm, (int)s0, ns, nrhs)));
      } else {
        MRHS_DISPATCH(dd, S, (k_pack<float, S><<<grid_for(tot, 256), 256, 0, c->stream>>>(
                                 (const float*)st, (S*)dev_out, c->perm, (int)s0, ns, nrhs)));
      }
      MRHS_LAUNCH_CHECK("pack");
    } else {
      if (hd == MRHS_F64) {
        MRHS_DISPATCH(dd, S, (k_unpack<double, S><<<grid_for(tot, 256), 256, 0, c->stream>>>(
                                 (double*)st, (const S*)dev_in, c->perm, (int)s0, ns, nrhs)));
      } else {
        MRHS_DISPATCH(dd, S, (k_unpack<float, S><<<grid_for(tot, 256), 256, 0, c->stream>>>(
                                 (float*)st, (const S*)dev_in, c->perm, (int)s0, ns, nrhs)));
      }
      MRHS_LAUNCH_CHECK("unpack");
      MRHS_CUDA(cudaMemcpy2DAsync((char*)host_out + s0 * 12 * hes, pitch, st, w, w, nrhs,
                                  cudaMemcpyDeviceToHost, c->stream));
    }
  }
  MRHS_CUDA(cudaStreamSynchronize(c->stream));
}

void transfer_coarse(mrhs_ctx c, const void* host_in, void* host_out, int hd, const void* dev_in, void* dev_out,
                     int dd, int nrhs) {
  check_host_dtype(hd);
  MRHS_REQUIRE(nrhs >= 1, MRHS_ERR_ARG, "nrhs must be >= 1");
  const size_t hes = hd == MRHS_F64 ? 16 : 8;
  size_t rows = (size_t)c->g.nagg * 2 * c->ntv;
  size_t bytes = rows * nrhs * hes;
  void* st = scratch(c, SC_STAGE, bytes);
  size_t tot = rows * nrhs;
  if (host_in) {
    MRHS_CUDA(cudaMemcpyAsync(st, host_in, bytes, cudaMemcpyHostToDevice, c->stream));
    if (hd == MRHS_F64) {
      MRHS_DISPATCH(dd, S, (k_pack_c<double, S><<<grid_for(tot, 256), 256, 0, c->stream>>>((const double*)st, (S*)dev_out, rows, nrhs)));
    } else {
      MRHS_DISPATCH(dd, S, (k_pack_c<float, S><<<grid_for(tot, 256), 256, 0, c->stream>>>((const float*)st, (S*)dev_out, rows, nrhs)));
    }
    MRHS_LAUNCH_CHECK("pack_coarse");
  } else {
    if (hd == MRHS_F64) {
      MRHS_DISPATCH(dd, S, (k_unpack_c<double, S><<<grid_for(tot, 256), 256, 0, c->stream>>>((double*)st, (const S*)dev_in, rows, nrhs)));
    } else {
      MRHS_DISPATCH(dd, S, (k_unpack_c<float, S><<<grid_for(tot, 256), 256, 0, c->stream>>>((float*)st, (const S*)dev_in, rows, nrhs)));
    }
    MRHS_LAUNCH_CHECK("unpack_coarse");
    MRHS_CUDA(cudaMemcpyAsync(host_out, st, bytes, cudaMemcpyDeviceToHost, c->stream));
  }
  MRHS_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace

// columns k0 .. k0+nb-1 of a field of ntv right-hand sides <-> a field of nb
// (rows = sites x 12 components x re/im, right-hand sides innermost)
template <class S>
__global__ void k_gather_cols(const S* __restrict__ src, int ntv, S* __restrict__ dst, int nb, int k0, size_t n) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const size_t row = t / nb;
  dst[t] = src[row * ntv + k0 + (int)(t % nb)];
}
template <class SI, class SO>
__global__ void k_scatter_cols(const SI* __restrict__ src, int nb, SO* __restrict__ dst, int ntv, int k0, size_t n,
                               float scale) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const size_t row = t / nb;
  // the product in the source's arithmetic type (double stays double)
  using R = typename Real<SI>::type;
  dst[row * ntv + k0 + (int)(t % nb)] = from_r<SO>(to_r(src[t]) * (R)scale);
}

namespace mrhs {
void convert(mrhs_ctx c, const void* x, int dx, void* y, int dy, size_t n) {
  Prof pr(c, "convert");
  MRHS_DISPATCH(dx, SI, MRHS_DISPATCH(dy, SO, (k_convert<SI, SO><<<grid_for(n, 256), 256, 0, c->stream>>>((const SI*)x, (SO*)y, n))));
  MRHS_LAUNCH_CHECK("convert");
}
void convert_scaled(mrhs_ctx c, const void* x, int dx, void* y, int dy, size_t n, float scale) {
  Prof pr(c, "convert");
  MRHS_DISPATCH(dx, SI, MRHS_DISPATCH(dy, SO, (k_convert_scaled<SI, SO><<<grid_for(n, 256), 256, 0, c->stream>>>((const SI*)x, (SO*)y, n, scale))));
  MRHS_LAUNCH_CHECK("convert_scaled");
}
}  // namespace mrhs

namespace mrhs {
void require_dev(mrhs_ctx c, const void* p, const char* what) {
  if (!p) return;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();  // the failed query is recorded as the last error: clear it
    throw Error(MRHS_ERR_ARG, std::string(what) + ": not a CUDA pointer (" + cudaGetErrorString(e) + ")");
  }
  if (a.type == cudaMemoryTypeManaged) return;
  MRHS_REQUIRE(a.type == cudaMemoryTypeDevice, MRHS_ERR_ARG,
               std::string(what) + ": host memory passed where a device field is required");
  MRHS_REQUIRE(a.device == c->device, MRHS_ERR_ARG,
               std::string(what) + ": device memory of GPU " + std::to_string(a.device) +
                   ", the context lives on GPU " + std::to_string(c->device));
}
void require_host(mrhs_ctx c, const void* p, const char* what) {
  (void)c;
  if (!p) return;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return;  // unknown to CUDA: plain pageable host memory
  }
  MRHS_REQUIRE(a.type != cudaMemoryTypeDevice, MRHS_ERR_ARG,
               std::string(what) + ": device memory passed where a host array is required");
}
void gather_cols(mrhs_ctx c, const void* src, int ntv, void* dst, int nb, int k0, int dtype) {
  const size_t n = (size_t)c->g.V * 24 * nb;
  Prof pr(c, "block_gather");
  MRHS_DISPATCH(dtype, S, (k_gather_cols<S><<<grid_for(n, 256), 256, 0, c->stream>>>((const S*)src, ntv, (S*)dst, nb, k0, n)));
  MRHS_LAUNCH_CHECK("gather_cols");
}
void scatter_cols(mrhs_ctx c, const void* src, int ds, int nb, void* dst, int dd, int ntv, int k0, float scale) {
  const size_t n = (size_t)c->g.V * 24 * nb;
  Prof pr(c, "block_gather");
  MRHS_DISPATCH(ds, SI, MRHS_DISPATCH(dd, SO, (k_scatter_cols<SI, SO><<<grid_for(n, 256), 256, 0, c->stream>>>((const SI*)src, nb, (SO*)dst, ntv, k0, n, scale))));
  MRHS_LAUNCH_CHECK("scatter_cols");
}
// the inverse clover term (for the even-odd domain solves), built once per
// clover term on first use
void ensure_clover_inverse(mrhs_ctx c) {
  MRHS_REQUIRE(c->have_clover, MRHS_ERR_STATE, "even-odd smoother before mrhs_build_clover");
  if (c->have_clover_inv) return;
  const size_t n = (size_t)c->g.V * 72;
  if (!c->Ainv64) {
    c->Ainv64 = (double*)dalloc(c, n * sizeof(double));
    c->Ainv32 = (float*)dalloc(c, n * sizeof(float));
  }
  MRHS_CUDA(cudaMemsetAsync(c->dflag + 4, 0, sizeof(int), c->stream));
  Prof pr(c, "clover_inverse");
  k_clover_inverse<<<grid_for(2 * (size_t)c->g.V, 128), 128, 0, c->stream>>>(c->g.V, c->A64, c->Ainv64, c->Ainv32,
                                                                             c->dflag + 4);
  MRHS_LAUNCH_CHECK("clover_inverse");
  MRHS_CUDA(cudaMemcpyAsync(c->hflag + 4, c->dflag + 4, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MRHS_CUDA(cudaStreamSynchronize(c->stream));
  MRHS_REQUIRE(c->hflag[4] == 0, MRHS_ERR_NONFINITE, "clover term singular on some site (even-odd smoother)");
  c->have_clover_inv = true;
}

}  // namespace mrhs

// ------------------------------------------------------------------ ABI ----
extern "C" {

int mrhs_create(const int dims[4], const int agg[4], int ntv, int prec, void* stream, mrhs_ctx* out) {
  return guarded(nullptr, [&] {
    MRHS_REQUIRE(dims && agg && out, MRHS_ERR_ARG, "null argument");
    MRHS_REQUIRE(prec >= MRHS_PREC_FP64 && prec <= MRHS_PREC_MIX_FP16, MRHS_ERR_ARG, "bad precision");
    Geometry g;
    long long V = 1, Va = 1, na = 1;
    for (int m = 0; m < 4; ++m) {
      MRHS_REQUIRE(dims[m] > 0 && agg[m] > 0 && dims[m] % agg[m] == 0, MRHS_ERR_SHAPE,
                   "lattice extent not divisible by aggregate extent");
      g.L[m] = dims[m];
      g.a[m] = agg[m];
      g.nb[m] = dims[m] / agg[m];
      MRHS_REQUIRE(g.nb[m] % 2 == 0, MRHS_ERR_SHAPE,
                   "the number of aggregates per direction must be even (red-black Schwarz colouring)");
      V *= dims[m];
      Va *= agg[m];
      na *= g.nb[m];
    }
    MRHS_REQUIRE(V < (1LL << 30), MRHS_ERR_SHAPE, "volume must be below 2^30");
    MRHS_REQUIRE(ntv >= 1 && ntv <= 64 && ntv <= 6 * Va, MRHS_ERR_SHAPE, "need 1 <= ntv <= min(64, 6*|aggregate|)");
    g.V = (int)V;
    g.Va = (int)Va;
    g.nagg = (int)na;
    mrhs_ctx c = new mrhs_ctx_s();
    try {
      c->g = g;
      c->ntv = ntv;
      c->prec = prec;
      c->tv_dtype = prec == MRHS_PREC_FP64 ? MRHS_F64
                    : prec == MRHS_PREC_FP32 ? MRHS_F32
                    : prec == MRHS_PREC_MIX_BF16 ? MRHS_BF16 : MRHS_F16;
      c->work_dtype = prec == MRHS_PREC_FP64 ? MRHS_F64 : MRHS_F32;
      c->stream = (cudaStream_t)stream;
      MRHS_CUDA(cudaGetDevice(&c->device));
      MRHS_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
      c->nbr = (int*)dalloc(c, sizeof(int) * 8 * (size_t)V);
      c->perm = (int*)dalloc(c, sizeof(int) * (size_t)V);
      c->iperm = (int*)dalloc(c, sizeof(int) * (size_t)V);
      c->aggnbr = (int*)dalloc(c, sizeof(int) * 8 * (size_t)na);
      c->blocks_col = (int*)dalloc(c, sizeof(int) * (size_t)na);
      c->dflag = (int*)dalloc(c, sizeof(int) * 16);
      c->coef32 = (float*)dalloc(c, sizeof(float) * 65 * 256 * 2);
      MRHS_CUDA(cudaMallocHost((void**)&c->hflag, sizeof(int) * 16));
      GeomArgs ga = geom_args(g);
      k_tables<<<grid_for(V, 256), 256, 0, c->stream>>>(ga, c->nbr, c->perm, c->iperm);
      MRHS_LAUNCH_CHECK("tables");
      k_aggnbr<<<grid_for(na, 256), 256, 0, c->stream>>>(ga, c->aggnbr);
      MRHS_LAUNCH_CHECK("aggnbr");
      // aggregate ids grouped by red-black colour (bookkeeping for launches)
      std::vector<int> col[2];
      for (int A = 0; A < g.nagg; ++A) {
        int i = A, s = 0;
        for (int m = 0; m < 4; ++m) {
          s += i % g.nb[m];
          i /= g.nb[m];
        }
        col[s & 1].push_back(A);
      }
      c->ncol[0] = (int)col[0].size();
      c->ncol[1] = (int)col[1].size();
      std::vector<int> all(col[0]);
      all.insert(all.end(), col[1].begin(), col[1].end());
      MRHS_CUDA(cudaMemcpyAsync(c->blocks_col, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice, c->stream));
      std::vector<int> posv(g.nagg);
      for (int q = 0; q < 2; ++q)
        for (size_t i = 0; i < col[q].size(); ++i) posv[col[q][i]] = (int)i;
      c->colpos = (int*)dalloc(c, sizeof(int) * (size_t)na);
      MRHS_CUDA(cudaMemcpyAsync(c->colpos, posv.data(), sizeof(int) * posv.size(), cudaMemcpyHostToDevice, c->stream));
      MRHS_CUDA(cudaMemsetAsync(c->dflag, 0, sizeof(int) * 16, c->stream));
      MRHS_CUDA(cudaStreamSynchronize(c->stream));
    } catch (...) {
      mrhs_destroy(c);
      throw;
    }
    *out = c;
  });
}

void mrhs_destroy(mrhs_ctx c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (void* p : c->allocs) cudaFree(p);
  for (auto& b : c->scratch)
    if (b.p) cudaFree(b.p);
  if (c->hflag) cudaFreeHost(c->hflag);
  if (c->hbuf) cudaFreeHost(c->hbuf);
  for (cudaEvent_t e : c->prof_events) cudaEventDestroy(e);
  if (c->nn) nn_destroy(c);
  delete c;
}

const char* mrhs_last_error(mrhs_ctx c) { return c ? c->err.c_str() : g_create_error.c_str(); }

int mrhs_sync(mrhs_ctx c) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c, MRHS_ERR_ARG, "null context");
    MRHS_CUDA(cudaStreamSynchronize(c->stream));
    check_tc_timeout(c);
  });
}

int mrhs_trim(mrhs_ctx c) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c, MRHS_ERR_ARG, "null context");
    MRHS_CUDA(cudaStreamSynchronize(c->stream));
    for (auto& b : c->scratch)
      if (b.p) {
        MRHS_CUDA(cudaFree(b.p));
        c->held_bytes -= b.bytes;
        b.p = nullptr;
        b.bytes = 0;
      }
  });
}

int mrhs_info(mrhs_ctx c, long long out[8]) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && out, MRHS_ERR_ARG, "null argument");
    out[0] = c->g.V;
    out[1] = c->g.nagg;
    out[2] = c->g.Va;
    out[3] = c->ntv;
    out[4] = c->prec;
    out[5] = (long long)c->held_bytes;
    out[6] = c->num_sms;
    out[7] = c->device;
  });
}

size_t mrhs_field_bytes(mrhs_ctx c, int nrhs, int dtype, int coarse) {
  if (!c || nrhs < 1 || dtype < 0 || dtype > 3) return 0;
  size_t n = coarse ? coarse_elems(c, nrhs) : fine_elems(c, nrhs);
  return n * dtype_size(dtype);
}

int mrhs_get_tables(mrhs_ctx c, int* nbr, int* aggof, int* aggnbr) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c, MRHS_ERR_ARG, "null context");
    require_host(c, nbr, "mrhs_get_tables nbr");
    require_host(c, aggof, "mrhs_get_tables aggof");
    require_host(c, aggnbr, "mrhs_get_tables aggnbr");
    const Geometry& g = c->g;
    int* d = (int*)scratch(c, SC_STAGE, sizeof(int) * 10 * (size_t)g.V);
    k_tables_canon<<<grid_for(g.V, 256), 256, 0, c->stream>>>(geom_args(g), c->nbr, c->perm, c->iperm, d,
                                                               d + 8 * (size_t)g.V);
    MRHS_LAUNCH_CHECK("tables_canon");
    if (nbr) MRHS_CUDA(cudaMemcpyAsync(nbr, d, sizeof(int) * 8 * (size_t)g.V, cudaMemcpyDeviceToHost, c->stream));
    if (aggof)
      MRHS_CUDA(cudaMemcpyAsync(aggof, d + 8 * (size_t)g.V, sizeof(int) * 2 * (size_t)g.V, cudaMemcpyDeviceToHost, c->stream));
    if (aggnbr)
      MRHS_CUDA(cudaMemcpyAsync(aggnbr, c->aggnbr, sizeof(int) * 8 * (size_t)g.nagg, cudaMemcpyDeviceToHost, c->stream));
    MRHS_CUDA(cudaStreamSynchronize(c->stream));
  });
}

int mrhs_set_gauge(mrhs_ctx c, const double* U) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && U, MRHS_ERR_ARG, "null argument");
    require_host(c, U, "mrhs_set_gauge U");
    size_t n = (size_t)c->g.V * 72;
    if (!c->U64) {
      c->U64 = (double*)dalloc(c, n * sizeof(double));
      c->U32 = (float*)dalloc(c, n * sizeof(float));
      c->U20 = (float*)dalloc(c, (size_t)c->g.V * 80 * sizeof(float));
    }
    // chunks of sites through the staging buffer bound the extra device memory
    const size_t per_site = 72 * sizeof(double);
    const size_t chunk = std::max<size_t>(1, std::min<size_t>(c->g.V, (size_t(1) << 30) / per_site));
    double* st = (double*)scratch(c, SC_STAGE, chunk * per_site);
    for (size_t s0 = 0; s0 < (size_t)c->g.V; s0 += chunk) {
      int ns = (int)std::min(chunk, (size_t)c->g.V - s0);
      MRHS_CUDA(cudaMemcpyAsync(st, U + s0 * 72, ns * per_site, cudaMemcpyHostToDevice, c->stream));
      const int lt_last = c->g.L[0] * c->g.L[1] * c->g.L[2] * (c->g.L[3] - 1);  // first canonical site with t = Lt-1
      k_gauge_in<<<grid_for((size_t)ns * 80, 256), 256, 0, c->stream>>>((int)s0, ns, c->perm, st, c->U64, c->U32, c->U20,
                                                                       lt_last);
      MRHS_LAUNCH_CHECK("gauge_in");
    }
    MRHS_CUDA(cudaStreamSynchronize(c->stream));
    c->have_gauge = true;
    c->have_clover = false;
  });
}

int mrhs_build_clover(mrhs_ctx c, double m0, double csw) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c, MRHS_ERR_ARG, "null context");
    MRHS_REQUIRE(c->have_gauge, MRHS_ERR_STATE, "mrhs_build_clover before mrhs_set_gauge");
    size_t n = (size_t)c->g.V * 72;
    if (!c->A64) {
      c->A64 = (double*)dalloc(c, n * sizeof(double));
      c->A32 = (float*)dalloc(c, n * sizeof(float));
    }
    Prof pr(c, "clover");
    k_clover<<<grid_for(c->g.V, 128), 128, 0, c->stream>>>(c->g.V, c->U64, c->nbr, m0, csw, c->A64, c->A32);
    MRHS_LAUNCH_CHECK("clover");
    c->have_clover = true;
    c->have_clover_inv = false;
  });
}

int mrhs_get_clover(mrhs_ctx c, double* out) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && out, MRHS_ERR_ARG, "null argument");
    require_host(c, out, "mrhs_get_clover out");
    MRHS_REQUIRE(c->have_clover, MRHS_ERR_STATE, "no clover term yet");
    size_t n = (size_t)c->g.V * 144;
    double* st = (double*)scratch(c, SC_STAGE, n * sizeof(double));
    k_clover_out<<<grid_for(c->g.V, 256), 256, 0, c->stream>>>(c->g.V, c->perm, c->A64, st);
    MRHS_LAUNCH_CHECK("clover_out");
    MRHS_CUDA(cudaMemcpyAsync(out, st, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    MRHS_CUDA(cudaStreamSynchronize(c->stream));
  });
}

int mrhs_pack(mrhs_ctx c, const void* host, int hd, void* dev, int dd, int nrhs) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && host && dev, MRHS_ERR_ARG, "null argument");
    require_host(c, host, "mrhs_pack host");
    require_dev(c, dev, "mrhs_pack dev");
    transfer_fine(c, host, nullptr, hd, nullptr, dev, dd, nrhs);
  });
}

int mrhs_unpack(mrhs_ctx c, const void* dev, int dd, void* host, int hd, int nrhs) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && host && dev, MRHS_ERR_ARG, "null argument");
    require_host(c, host, "mrhs_unpack host");
    require_dev(c, dev, "mrhs_unpack dev");
    transfer_fine(c, nullptr, host, hd, dev, nullptr, dd, nrhs);
  });
}

int mrhs_pack_coarse(mrhs_ctx c, const void* host, int hd, void* dev, int dd, int nrhs) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && host && dev, MRHS_ERR_ARG, "null argument");
    require_host(c, host, "mrhs_pack_coarse host");
    require_dev(c, dev, "mrhs_pack_coarse dev");
    transfer_coarse(c, host, nullptr, hd, nullptr, dev, dd, nrhs);
  });
}

int mrhs_unpack_coarse(mrhs_ctx c, const void* dev, int dd, void* host, int hd, int nrhs) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && host && dev, MRHS_ERR_ARG, "null argument");
    require_host(c, host, "mrhs_unpack_coarse host");
    require_dev(c, dev, "mrhs_unpack_coarse dev");
    transfer_coarse(c, nullptr, host, hd, dev, nullptr, dd, nrhs);
  });
}

int mrhs_set_tv(mrhs_ctx c, const void* tv, int dtype) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && tv, MRHS_ERR_ARG, "null argument");
    require_dev(c, tv, "mrhs_set_tv tv");
    size_t n = fine_elems(c, c->ntv);
    if (!c->tv) c->tv = dalloc(c, n * dtype_size(c->tv_dtype));
    convert(c, tv, dtype, c->tv, c->tv_dtype, n);
    c->tv_scale = 1.0;
    c->have_tv = true;
    c->have_P = c->have_Dc = false;
  });
}

int mrhs_get_tv(mrhs_ctx c, void* host, int hd) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && host, MRHS_ERR_ARG, "null argument");
    require_host(c, host, "mrhs_get_tv host");
    MRHS_REQUIRE(c->have_tv, MRHS_ERR_STATE, "no test vectors yet");
    if (c->tv_scale != 1.0) {
      const size_t n = fine_elems(c, c->ntv);
      void* tmp = scratch(c, SC_FINE1, n * sizeof(float));
      convert_scaled(c, c->tv, c->tv_dtype, tmp, MRHS_F32, n, (float)(1.0 / c->tv_scale));
      transfer_fine(c, nullptr, host, hd, tmp, nullptr, MRHS_F32, c->ntv);
    } else {
      transfer_fine(c, nullptr, host, hd, c->tv, nullptr, c->tv_dtype, c->ntv);
    }
  });
}

int mrhs_get_P(mrhs_ctx c, void* host, int hd) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && host, MRHS_ERR_ARG, "null argument");
    require_host(c, host, "mrhs_get_P host");
    MRHS_REQUIRE(c->have_P, MRHS_ERR_STATE, "no P yet");
    transfer_fine(c, nullptr, host, hd, c->P, nullptr, c->tv_dtype, c->ntv);
  });
}

int mrhs_get_Dc(mrhs_ctx c, void* host, int hd) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && host, MRHS_ERR_ARG, "null argument");
    require_host(c, host, "mrhs_get_Dc host");
    MRHS_REQUIRE(c->have_Dc, MRHS_ERR_STATE, "no D_c yet");
    check_host_dtype(hd);
    size_t n = (size_t)c->g.nagg * 9 * 4 * c->ntv * c->ntv * 2;  // reals
    if (hd == c->work_dtype) {
      MRHS_CUDA(cudaMemcpyAsync(host, c->Dc, n * dtype_size(hd), cudaMemcpyDeviceToHost, c->stream));
    } else {
      void* st = scratch(c, SC_STAGE, n * dtype_size(hd));
      convert(c, c->Dc, c->work_dtype, st, hd, n);
      MRHS_CUDA(cudaMemcpyAsync(host, st, n * dtype_size(hd), cudaMemcpyDeviceToHost, c->stream));
    }
    MRHS_CUDA(cudaStreamSynchronize(c->stream));
  });
}

}  // extern "C"


// ------------------------------------------------------------ profiling ----
namespace mrhs {

Prof::Prof(mrhs_ctx ctx, const char* name) : c(ctx) {
  if (!c || !c->prof) return;
  int id = -1;
  for (size_t i = 0; i < c->prof_names.size(); ++i)
    if (c->prof_names[i] == name) id = (int)i;
  if (id < 0) {
    c->prof_names.emplace_back(name);
    c->prof_launches.push_back(0);
    c->prof_ms.push_back(0.0);
    id = (int)c->prof_names.size() - 1;
  }
  while (c->prof_events.size() < c->prof_used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    c->prof_events.push_back(e);
  }
  idx = c->prof_used;
  c->prof_used += 2;
  c->prof_rec_name.push_back(id);
  c->prof_launches[id] += 1;
  cudaEventRecord(c->prof_events[idx], c->stream);
}

Prof::~Prof() {
  if (idx != (size_t)-1) cudaEventRecord(c->prof_events[idx + 1], c->stream);
}

static void prof_fold(mrhs_ctx c) {
  MRHS_CUDA(cudaStreamSynchronize(c->stream));
  for (size_t r = 0; r < c->prof_rec_name.size(); ++r) {
    float ms = 0;
    MRHS_CUDA(cudaEventElapsedTime(&ms, c->prof_events[2 * r], c->prof_events[2 * r + 1]));
    c->prof_ms[c->prof_rec_name[r]] += ms;
  }
  c->prof_rec_name.clear();
  c->prof_used = 0;
}

}  // namespace mrhs

extern "C" {

int mrhs_profile(mrhs_ctx c, int enable) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c, MRHS_ERR_ARG, "null context");
    if (enable) {
      MRHS_CUDA(cudaStreamSynchronize(c->stream));
      c->prof_names.clear();
      c->prof_launches.clear();
      c->prof_ms.clear();
      c->prof_rec_name.clear();
      c->prof_used = 0;
      c->prof = true;
    } else {
      prof_fold(c);
      c->prof = false;
    }
  });
}

int mrhs_profile_read(mrhs_ctx c, int idx, char* name, int name_len, long long* launches, double* ms) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c, MRHS_ERR_ARG, "null context");
    prof_fold(c);
    MRHS_REQUIRE(idx >= 0 && (size_t)idx < c->prof_names.size(), MRHS_ERR_ARG, "no such profile entry");
    if (name && name_len > 0) {
      std::strncpy(name, c->prof_names[idx].c_str(), (size_t)name_len - 1);
      name[name_len - 1] = 0;
    }
    if (launches) *launches = c->prof_launches[idx];
    if (ms) *ms = c->prof_ms[idx];
  });
}

}  // extern "C"
