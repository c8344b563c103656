// The setup phase (Sec. 2 and Algorithm 2 of the paper with block length
// N_b = ntv: the V-cycle is applied to all test vectors at once) and the
// two-level FGMRES solve that measures the quality of a setup.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "common.cuh"

namespace mrhs {

void restrict_typed(mrhs_ctx c, const void* v, int dv, void* vc, int dc, int N);
void prolong_typed(mrhs_ctx c, const void* uc, int dc, void* u, int du, int N);

namespace {

// Block length of the setup phases: N_b of Alg. 2 (0 or >= ntv: all test
// vectors at once, the default).
int block_length(mrhs_ctx c) { return c->block_len > 0 && c->block_len < c->ntv ? c->block_len : c->ntv; }

// The initial phase on the test vectors k0 .. k0+nb-1 (all of them when
// nb = ntv): x = SAP^n_sweeps(b = v, x0 = 0) (init_mode 0) or n_sweeps times
// v <- SAP(b = v, x0 = 0) (init_mode 1); the normalised x replaces v.
// b_src (init_mode 0 with the whole set, may be null): the vectors to smooth
// in the storage type, read in place of the stored test vectors.
void init_block(mrhs_ctx c, int k0, int nb, int init_mode, int n_sweeps, int n_mr, const void* b_src = nullptr) {
  const int N = c->ntv;
  const int wd = c->work_dtype;
  const size_t n = fine_elems(c, nb);
  void* x = scratch(c, SC_X, n * dtype_size(wd));
  void* v = c->tv;  // b: the block's test vectors in their storage type
  if (nb < N) {
    v = scratch(c, SC_BLOCK, n * dtype_size(c->tv_dtype));
    gather_cols(c, c->tv, N, v, nb, k0, c->tv_dtype);
  }
  if (init_mode == 0) {
    MRHS_CUDA(cudaMemsetAsync(x, 0, n * dtype_size(wd), c->stream));
    sap_mixed(c, b_src ? b_src : v, c->tv_dtype, x, nb, wd, n_sweeps, n_mr, true);
  } else {
    for (int it = 0; it < n_sweeps; ++it) {
      MRHS_CUDA(cudaMemsetAsync(x, 0, n * dtype_size(wd), c->stream));
      sap_mixed(c, v, c->tv_dtype, x, nb, wd, 1, n_mr, true);
      if (it + 1 < n_sweeps) convert(c, x, wd, v, c->tv_dtype, n);
    }
  }
  const float scale = (float)(c->tv_dtype == MRHS_F16 ? std::sqrt(12.0 * c->g.V) : 1.0);
  if (nb < N) {
    normalise_rhs(c, x, (size_t)c->g.V * 12, nb, wd);
    scatter_cols(c, x, wd, nb, c->tv, c->tv_dtype, N, k0, scale);
  } else {
    normalise_into(c, x, wd, c->tv, c->tv_dtype, (size_t)c->g.V * 12, N, scale);
  }
}

void setup_init(mrhs_ctx c, const void* tv0, int dtype, int init_mode, int n_sweeps, int n_mr) {
  MRHS_REQUIRE(c->have_clover, MRHS_ERR_STATE, "mrhs_setup_init before mrhs_build_clover");
  MRHS_REQUIRE(init_mode == 0 || init_mode == 1, MRHS_ERR_ARG, "init_mode must be 0 or 1");
  MRHS_REQUIRE(n_sweeps >= 1 && n_mr >= 0, MRHS_ERR_ARG, "need n_sweeps >= 1, n_mr >= 0");
  const int N = c->ntv;
  const size_t n = fine_elems(c, N);
  if (!c->tv) c->tv = dalloc(c, n * dtype_size(c->tv_dtype));
  const int nb = block_length(c);
  // one smoother call on the whole set reads tv0 in place when it has the
  // storage type; otherwise tv0 is converted into the stored vectors first
  const bool direct = init_mode == 0 && nb == N && dtype == c->tv_dtype;
  if (!direct) convert(c, tv0, dtype, c->tv, c->tv_dtype, n);
  c->have_tv = true;
  c->have_P = c->have_Dc = false;
  // blocks of N_b test vectors in order; the last one holds the remainder
  // when N_b does not divide ntv (Alg. 2 and its remainder rule)
  for (int k0 = 0; k0 < N; k0 += nb)
    init_block(c, k0, std::min(nb, N - k0), init_mode, n_sweeps, n_mr, direct ? tv0 : nullptr);
  c->tv_scale = c->tv_dtype == MRHS_F16 ? std::sqrt(12.0 * c->g.V) : 1.0;
  build_P(c);
  build_Dc(c);
}

// learned initial phase: x = SAP^n_sweeps(b = v, x0 = 0), v <- net(x),
// normalised, then P and D_c
void setup_init_learned(mrhs_ctx c, const void* tv0, int dtype, int n_sweeps, int n_mr) {
  MRHS_REQUIRE(c->have_clover, MRHS_ERR_STATE, "mrhs_setup_init_learned before mrhs_build_clover");
  MRHS_REQUIRE(c->nn, MRHS_ERR_STATE, "mrhs_setup_init_learned before mrhs_nn_create");
  MRHS_REQUIRE(c->work_dtype == MRHS_F32, MRHS_ERR_ARG, "the learned initial phase runs on FP32 work fields");
  MRHS_REQUIRE(n_sweeps >= 0 && n_mr >= 0, MRHS_ERR_ARG, "bad smoother parameters");
  const int N = c->ntv;
  const size_t n = fine_elems(c, N);
  if (!c->tv) c->tv = dalloc(c, n * dtype_size(c->tv_dtype));
  void* x = scratch(c, SC_X, n * sizeof(float));
  void* y = scratch(c, SC_R, n * sizeof(float));
  convert(c, tv0, dtype, y, MRHS_F32, n);
  if (n_sweeps > 0) {
    MRHS_CUDA(cudaMemsetAsync(x, 0, n * sizeof(float), c->stream));
    sap_mixed(c, y, MRHS_F32, x, N, MRHS_F32, n_sweeps, n_mr, true);
  } else {
    MRHS_CUDA(cudaMemcpyAsync(x, y, n * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
  }
  nn_infer(c, (const float*)x, (float*)y, N);
  c->tv_scale = c->tv_dtype == MRHS_F16 ? std::sqrt(12.0 * c->g.V) : 1.0;
  normalise_into(c, y, MRHS_F32, c->tv, c->tv_dtype, (size_t)c->g.V * 12, N, (float)c->tv_scale);
  c->have_tv = true;
  build_P(c);
  build_Dc(c);
}

void setup_refine(mrhs_ctx c, int n_iter, int n_sweeps, int n_mr, double ctol, int crestart, int cmaxit,
                  int* coarse_iters) {
  MRHS_REQUIRE(c->have_Dc, MRHS_ERR_STATE, "mrhs_setup_refine before mrhs_setup_init");
  MRHS_REQUIRE(n_iter >= 0 && n_sweeps >= 0 && n_mr >= 0, MRHS_ERR_ARG, "bad refinement parameters");
  const int N = c->ntv;
  const int wd = c->work_dtype;
  const int nb = block_length(c);
  const size_t n = fine_elems(c, nb);
  const size_t nce = coarse_elems(c, nb);
  void* x = scratch(c, SC_X, n * dtype_size(wd));
  char* cbuf = (char*)scratch(c, SC_COARSE, 2 * nce * dtype_size(wd));
  void* vc = cbuf;
  void* uc = cbuf + nce * dtype_size(wd);
  void* vb = nb < N ? scratch(c, SC_BLOCK, n * dtype_size(c->tv_dtype)) : c->tv;
  const float scale = (float)(c->tv_dtype == MRHS_F16 ? std::sqrt(12.0 * c->g.V) : 1.0);
  std::vector<int> its;
  for (int i = 0; i < n_iter; ++i) {
    // the V-cycle on blocks of N_b test vectors in order (Alg. 2; N_b = ntv:
    // all at once; the last block holds the remainder); R, P and D_c stay
    // fixed until every vector has been replaced (Alg. 1 and 2 alike)
    for (int k0 = 0; k0 < N; k0 += nb) {
      const int m = std::min(nb, N - k0);
      if (m < N) gather_cols(c, c->tv, N, vb, m, k0, c->tv_dtype);
      // coarse-grid correction
      restrict_typed(c, vb, c->tv_dtype, vc, wd, m);
      its.assign(m, 0);
      coarse_solve(c, vc, uc, m, wd, ctol, crestart, cmaxit, coarse_iters ? its.data() : nullptr);
      if (coarse_iters)
        for (int j = 0; j < m; ++j) coarse_iters[(size_t)i * N + k0 + j] = its[j];
      prolong_typed(c, uc, wd, x, wd, m);
      // smoother with the coarse-grid result as starting guess
      sap_mixed(c, vb, c->tv_dtype, x, m, wd, n_sweeps, n_mr);
      // replace the block's test vectors by the result
      if (m < N) {
        normalise_rhs(c, x, (size_t)c->g.V * 12, m, wd);
        scatter_cols(c, x, wd, m, c->tv, c->tv_dtype, N, k0, scale);
      } else {
        normalise_into(c, x, wd, c->tv, c->tv_dtype, (size_t)c->g.V * 12, N, scale);
      }
    }
    c->tv_scale = scale;
    // rebuild R = P^dag and D_c from the new test vectors
    build_P(c);
    build_Dc(c);
  }
}

// ---------------------------------------------------------------- FGMRES ---
using zc = std::complex<double>;

struct Fgmres {
  mrhs_ctx c;
  size_t rows;  // V*12 complex rows, one right-hand side
  size_t fe;    // doubles per fine FP64 field
  double* dev_coef;
  double* host_coef;

  void dot_many(const double* X, int K, const double* Y, std::vector<zc>& out) {
    multi_dot(c, X, fe, K, Y, rows, 1, MRHS_F64, dev_coef);
    MRHS_CUDA(cudaMemcpyAsync(host_coef, dev_coef, sizeof(double) * 2 * K, cudaMemcpyDeviceToHost, c->stream));
    MRHS_CUDA(cudaStreamSynchronize(c->stream));
    out.resize(K);
    for (int k = 0; k < K; ++k) out[k] = zc(host_coef[2 * k], host_coef[2 * k + 1]);
  }
  // Y += sum_k a_k X_k
  void axpy_many(const double* X, int K, const std::vector<zc>& a, double* Y) {
    MRHS_CUDA(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < K; ++k) {
      host_coef[2 * k] = a[k].real();
      host_coef[2 * k + 1] = a[k].imag();
    }
    MRHS_CUDA(cudaMemcpyAsync(dev_coef, host_coef, sizeof(double) * 2 * K, cudaMemcpyHostToDevice, c->stream));
    multi_axpy(c, X, fe, K, Y, rows, 1, MRHS_F64, dev_coef, 1.0);
  }
};

int solve_fgmres(mrhs_ctx c, const double* b_host, double* x_host, double tol, int m, int maxit, double ctol,
                 int crestart, int cmaxit, int n_sweeps, int n_mr, int* iters_out, double* relres_out) {
  MRHS_REQUIRE(c->have_Dc, MRHS_ERR_STATE, "mrhs_solve_fgmres before the setup");
  MRHS_REQUIRE(m >= 1 && m <= 256 && maxit >= 1 && tol >= 0, MRHS_ERR_ARG, "bad FGMRES parameters");
  const int wd = c->work_dtype;
  Fgmres F;
  F.c = c;
  F.rows = (size_t)c->g.V * 12;
  F.fe = F.rows * 2;
  const size_t fb = F.fe * sizeof(double);
  // FP64 fields: b, x, w, basis V_0..V_m, Z_0..Z_{m-1}
  double* base = (double*)scratch(c, SC_KRYLOV_F, fb * (size_t)(3 + (m + 1) + m));
  double* b = base;
  double* x = b + F.fe;
  double* w = x + F.fe;
  double* Vb = w + F.fe;
  double* Z = Vb + (size_t)(m + 1) * F.fe;
  auto Vk = [&](int k) { return Vb + (size_t)k * F.fe; };
  auto Zk = [&](int k) { return Z + (size_t)k * F.fe; };
  // preconditioner work in the context precision (one right-hand side)
  const size_t we = F.fe * dtype_size(wd);
  char* pw = (char*)scratch(c, SC_FINE1, 2 * we);
  void* r_w = pw;
  void* z_w = pw + we;
  const size_t nce = coarse_elems(c, 1);
  char* cb = (char*)scratch(c, SC_FINE2, 2 * nce * dtype_size(wd));
  void* rc = cb;
  void* uc = cb + nce * dtype_size(wd);
  F.dev_coef = (double*)scratch(c, SC_FINE3, sizeof(double) * 2 * (m + 2));
  F.host_coef = host_scratch(c, sizeof(double) * 2 * (m + 2));

  int st = mrhs_pack(c, b_host, MRHS_F64, b, MRHS_F64, 1);
  MRHS_REQUIRE(st == MRHS_OK, st, c->err);
  MRHS_CUDA(cudaMemsetAsync(x, 0, fb, c->stream));
  std::vector<zc> tmp;
  F.dot_many(b, 1, b, tmp);
  const double bnorm = std::sqrt(tmp[0].real());
  std::vector<zc> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), h1, h2;
  int it = 0;
  bool conv = false;
  double res = bnorm > 0 ? 1.0 : 0.0;
  if (bnorm == 0) conv = true;
  while (!conv && it < maxit) {
    dslash(c, x, w, b, 1, MRHS_F64, DS_RESID, -1);  // w = b - D x
    F.dot_many(w, 1, w, tmp);
    double beta = std::sqrt(tmp[0].real());
    res = beta / bnorm;
    if (beta <= tol * bnorm) {
      conv = true;
      break;
    }
    MRHS_CUDA(cudaMemsetAsync(Vk(0), 0, fb, c->stream));
    F.axpy_many(w, 1, std::vector<zc>(1, zc(1.0 / beta, 0)), Vk(0));
    std::fill(g.begin(), g.end(), zc(0));
    g[0] = beta;
    int kend = 0;
    for (int k = 0; k < m; ++k) {
      // z_k = M v_k: V-cycle in the context precision
      convert(c, Vk(k), MRHS_F64, r_w, wd, F.fe);
      restrict_typed(c, r_w, wd, rc, wd, 1);
      coarse_solve(c, rc, uc, 1, wd, ctol, crestart, cmaxit, nullptr);
      prolong_typed(c, uc, wd, z_w, wd, 1);
      sap(c, r_w, z_w, 1, wd, n_sweeps, n_mr);
      convert(c, z_w, wd, Zk(k), MRHS_F64, F.fe);
      dslash(c, Zk(k), w, nullptr, 1, MRHS_F64, DS_FULL, -1);
      // two classical Gram-Schmidt passes against V_0..V_k
      F.dot_many(Vb, k + 1, w, h1);
      std::vector<zc> neg(k + 1);
      for (int i = 0; i <= k; ++i) neg[i] = -h1[i];
      F.axpy_many(Vb, k + 1, neg, w);
      F.dot_many(Vb, k + 1, w, h2);
      for (int i = 0; i <= k; ++i) neg[i] = -h2[i];
      F.axpy_many(Vb, k + 1, neg, w);
      F.dot_many(w, 1, w, tmp);
      double hk1 = std::sqrt(tmp[0].real());
      for (int i = 0; i <= k; ++i) H[i * m + k] = h1[i] + h2[i];
      H[(k + 1) * m + k] = hk1;
      for (int i = 0; i < k; ++i) {
        zc a = H[i * m + k], bb = H[(i + 1) * m + k];
        H[i * m + k] = std::conj(cs[i]) * a + std::conj(sn[i]) * bb;
        H[(i + 1) * m + k] = -sn[i] * a + cs[i] * bb;
      }
      zc a = H[k * m + k], bb = H[(k + 1) * m + k];
      double nu = std::sqrt(std::norm(a) + std::norm(bb));
      cs[k] = nu == 0 ? zc(1) : a / nu;
      sn[k] = nu == 0 ? zc(0) : bb / nu;
      H[k * m + k] = nu;
      H[(k + 1) * m + k] = 0;
      zc g0 = g[k];
      g[k] = std::conj(cs[k]) * g0;
      g[k + 1] = -sn[k] * g0;
      ++it;
      kend = k + 1;
      res = std::abs(g[k + 1]) / bnorm;
      if (hk1 > 0) {
        MRHS_CUDA(cudaMemsetAsync(Vk(k + 1), 0, fb, c->stream));
        F.axpy_many(w, 1, std::vector<zc>(1, zc(1.0 / hk1, 0)), Vk(k + 1));
      }
      if (std::abs(g[k + 1]) <= tol * bnorm || hk1 == 0) conv = true;
      if (conv || it >= maxit) break;
    }
    for (int i = kend - 1; i >= 0; --i) {
      zc s = g[i];
      for (int l = i + 1; l < kend; ++l) s -= H[i * m + l] * y[l];
      y[i] = s / H[i * m + i];
    }
    F.axpy_many(Z, kend, std::vector<zc>(y.begin(), y.begin() + kend), x);
  }
  st = mrhs_unpack(c, x, MRHS_F64, x_host, MRHS_F64, 1);
  MRHS_REQUIRE(st == MRHS_OK, st, c->err);
  if (iters_out) *iters_out = it;
  if (relres_out) *relres_out = res;
  return conv ? MRHS_OK : MRHS_ERR_NOCONV;
}

}  // namespace
}  // namespace mrhs

using namespace mrhs;

extern "C" {

int mrhs_setup_init(mrhs_ctx c, const void* tv0, int dtype, int init_mode, int n_sweeps, int n_mr) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && tv0, MRHS_ERR_ARG, "null argument");
    require_dev(c, tv0, "mrhs_setup_init tv0");
    setup_init(c, tv0, dtype, init_mode, n_sweeps, n_mr);
  });
}

int mrhs_setup_init_learned(mrhs_ctx c, const void* tv0, int dtype, int n_sweeps, int n_mr) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c && tv0, MRHS_ERR_ARG, "null argument");
    require_dev(c, tv0, "mrhs_setup_init_learned tv0");
    setup_init_learned(c, tv0, dtype, n_sweeps, n_mr);
  });
}

int mrhs_setup_update(mrhs_ctx c, int n_iter, int n_sweeps, int n_mr, double coarse_tol, int coarse_restart,
                      int coarse_maxit, int* coarse_iters) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c, MRHS_ERR_ARG, "null context");
    MRHS_REQUIRE(c->have_P && c->have_tv, MRHS_ERR_STATE, "mrhs_setup_update before a setup");
    MRHS_REQUIRE(c->have_clover, MRHS_ERR_STATE, "mrhs_setup_update before mrhs_build_clover of the new field");
    // the coarse operator of the kept P with the new links and clover term,
    // then refinement from the kept test vectors
    build_Dc(c);
    setup_refine(c, n_iter, n_sweeps, n_mr, coarse_tol, coarse_restart, coarse_maxit, coarse_iters);
  });
}

int mrhs_set_block_length(mrhs_ctx c, int nb) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c, MRHS_ERR_ARG, "null context");
    MRHS_REQUIRE(nb >= 0, MRHS_ERR_ARG, "block length must be >= 0");
    c->block_len = nb;
  });
}

int mrhs_setup_refine(mrhs_ctx c, int n_iter, int n_sweeps, int n_mr, double coarse_tol, int coarse_restart,
                      int coarse_maxit, int* coarse_iters) {
  return guarded(c, [&] {
    MRHS_REQUIRE(c, MRHS_ERR_ARG, "null context");
    setup_refine(c, n_iter, n_sweeps, n_mr, coarse_tol, coarse_restart, coarse_maxit, coarse_iters);
  });
}

int mrhs_solve_fgmres(mrhs_ctx c, const double* b, double* x, double tol, int restart, int maxit, double coarse_tol,
                      int coarse_restart, int coarse_maxit, int n_sweeps, int n_mr, int* iters, double* relres) {
  int rc = MRHS_OK;
  int st = guarded(c, [&] {
    MRHS_REQUIRE(c && b && x, MRHS_ERR_ARG, "null argument");
    require_host(c, b, "mrhs_solve_fgmres b");
    require_host(c, x, "mrhs_solve_fgmres x");
    rc = solve_fgmres(c, b, x, tol, restart, maxit, coarse_tol, coarse_restart, coarse_maxit, n_sweeps, n_mr, iters,
                      relres);
  });
  if (st != MRHS_OK) return st;
  if (rc == MRHS_ERR_NOCONV) c->err = "FGMRES reached maxit before the tolerance";
  return rc;
}

}  // extern "C"
