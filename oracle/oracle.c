/*
 * FP64 CPU oracle for the multiple-right-hand-side DD-alpha-AMG setup
 * (Richtmann, Heybrock, Wettig, "Multiple right-hand-side setup for the
 * DD-alpha-AMG", arXiv:1601.03184).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this library. The product path (the
 * CUDA library) shares no code with it and never calls it.
 *
 * Everything here is plain double-precision complex arithmetic in the
 * canonical host layout, one right-hand side at a time (the single-RHS loop
 * order of Algorithm 1 of the paper). Nothing is blocked, fused or reordered
 * beyond what the definitions below state.
 *
 * Conventions (the paper defines none of the underlying operators; it defers
 * them to its references, Sec. 2):
 *   site index   s = x + Lx*(y + Ly*(z + Lz*t)), directions mu = 0..3 = x,y,z,t
 *   spinor       psi[s][c], c = 3*spin + colour (12 complex per site)
 *   links        U[s][mu][a][b]  (3x3 complex, row a, column b)
 *   clover       A[s][12][12]    (full matrix; chirality block-diagonal)
 *   boundaries   periodic, except fermion hops across the t boundary (sign -1)
 *   gammas       chiral Euclidean basis: gamma_k = [[0,-i sigma_k],[i sigma_k,0]]
 *                for mu = k-1 = 0,1,2 and gamma_4 = [[0,1],[1,0]] for mu = 3,
 *                so gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1,1,-1,-1)
 *   chirality    h = 0 (spins 0,1, gamma_5 = +1) and h = 1 (spins 2,3)
 *   aggregates   blocks of a[0]x..xa[3] sites, lexicographic block order;
 *                they are also the Schwarz (SAP) domains
 *   test vectors tv[j][s][c], j = 0..ntv-1
 *   coarse index (h*ntv + j) per aggregate; coarse vector xc[A][2*ntv]
 *   coarse op    Dc[A][k][2ntv][2ntv], k = 0 self, 1+mu for the +mu
 *                neighbour aggregate, 5+mu for the -mu neighbour aggregate
 */
#include <complex.h>
#include <stdint.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* geometry                                                            */
/* ------------------------------------------------------------------ */
typedef struct {
  int L[4], V;
  int a[4], nb[4];
  int nagg, Va;
} geom_t;

static int geom_init(geom_t* g, const int* dims, const int* agg) {
  g->V = 1;
  g->nagg = 1;
  g->Va = 1;
  for (int mu = 0; mu < 4; ++mu) {
    g->L[mu] = dims[mu];
    g->a[mu] = agg[mu];
    if (dims[mu] <= 0 || agg[mu] <= 0 || dims[mu] % agg[mu] != 0) return -1;
    g->nb[mu] = dims[mu] / agg[mu];
    g->V *= dims[mu];
    g->nagg *= g->nb[mu];
    g->Va *= agg[mu];
  }
  return 0;
}

static void coords_of(const int* L, int s, int x[4]) {
  for (int mu = 0; mu < 4; ++mu) {
    x[mu] = s % L[mu];
    s /= L[mu];
  }
}

static int index_of(const int* L, const int x[4]) {
  return x[0] + L[0] * (x[1] + L[1] * (x[2] + L[2] * x[3]));
}

/* neighbour of s one step in direction mu, dir = +1 or -1; *flip = 1 when
 * the hop crosses the t boundary (the fermion picks up a factor -1 there) */
static int neighbour(const geom_t* g, int s, int mu, int dir, int* flip) {
  int x[4];
  coords_of(g->L, s, x);
  int v = x[mu] + dir;
  int f = 0;
  if (v < 0) { v += g->L[mu]; f = 1; }
  if (v >= g->L[mu]) { v -= g->L[mu]; f = 1; }
  x[mu] = v;
  if (flip) *flip = (mu == 3) ? f : 0;
  return index_of(g->L, x);
}

static int aggregate_of(const geom_t* g, int s, int* offset) {
  int x[4], bx[4], lx[4];
  coords_of(g->L, s, x);
  for (int mu = 0; mu < 4; ++mu) {
    bx[mu] = x[mu] / g->a[mu];
    lx[mu] = x[mu] % g->a[mu];
  }
  if (offset) *offset = index_of(g->a, lx);
  return index_of(g->nb, bx);
}

static int aggregate_colour(const geom_t* g, int A) {
  int b[4];
  coords_of(g->nb, A, b);
  return (b[0] + b[1] + b[2] + b[3]) & 1;
}

/* aggregate one step away in direction mu (periodic on the block lattice) */
static int aggregate_neighbour(const geom_t* g, int A, int mu, int dir) {
  int b[4];
  coords_of(g->nb, A, b);
  b[mu] = (b[mu] + dir + g->nb[mu]) % g->nb[mu];
  return index_of(g->nb, b);
}

/* Neighbour/aggregate tables in canonical order (the lattice blocks of
 * Sec. 2: aggregates of the coarse grid, which are also the Schwarz domains
 * of the smoother; domain size 4^4 in Sec. 7).
 *   nbr[s][k]    k = 0..3: s + mu_hat, k = 4..7: s - mu_hat; value = site
 *                index, with bit 30 set when the hop crosses the t boundary
 *   aggof[s][2]  (aggregate index, offset of s inside its aggregate)
 *   aggnbr[A][k] k = 0..3: A + mu_hat, 4..7: A - mu_hat on the block lattice */
int ora_tables(const int* dims, const int* agg, int* nbr, int* aggof, int* aggnbr) {
  geom_t g;
  if (geom_init(&g, dims, agg)) return -1;
  for (int s = 0; s < g.V; ++s) {
    for (int mu = 0; mu < 4; ++mu) {
      int f;
      int sp = neighbour(&g, s, mu, +1, &f);
      nbr[8 * s + mu] = sp | (f << 30);
      int sm = neighbour(&g, s, mu, -1, &f);
      nbr[8 * s + 4 + mu] = sm | (f << 30);
    }
    int off;
    aggof[2 * s] = aggregate_of(&g, s, &off);
    aggof[2 * s + 1] = off;
  }
  for (int A = 0; A < g.nagg; ++A)
    for (int mu = 0; mu < 4; ++mu) {
      aggnbr[8 * A + mu] = aggregate_neighbour(&g, A, mu, +1);
      aggnbr[8 * A + 4 + mu] = aggregate_neighbour(&g, A, mu, -1);
    }
  return 0;
}

/* ------------------------------------------------------------------ */
/* gamma matrices (chiral Euclidean basis)                              */
/* ------------------------------------------------------------------ */
static cplx GAMMA[4][4][4];
static cplx GAMMA5[4][4];
static cplx SIGMA[4][4][4][4]; /* sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu] */
static int gammas_ready = 0;

static void init_gammas(void) {
  if (gammas_ready) return;
  const cplx pauli[3][2][2] = {
      {{0, 1}, {1, 0}},
      {{0, -I}, {I, 0}},
      {{1, 0}, {0, -1}},
  };
  memset(GAMMA, 0, sizeof(GAMMA));
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        GAMMA[k][i][2 + j] = -I * pauli[k][i][j];
        GAMMA[k][2 + i][j] = I * pauli[k][i][j];
      }
  for (int i = 0; i < 2; ++i) {
    GAMMA[3][i][2 + i] = 1;
    GAMMA[3][2 + i][i] = 1;
  }
  /* gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 */
  cplx t1[4][4], t2[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      t1[i][j] = 0;
      for (int k = 0; k < 4; ++k) t1[i][j] += GAMMA[0][i][k] * GAMMA[1][k][j];
    }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      t2[i][j] = 0;
      for (int k = 0; k < 4; ++k) t2[i][j] += t1[i][k] * GAMMA[2][k][j];
    }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      GAMMA5[i][j] = 0;
      for (int k = 0; k < 4; ++k) GAMMA5[i][j] += t2[i][k] * GAMMA[3][k][j];
    }
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu)
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
          cplx c = 0;
          for (int k = 0; k < 4; ++k)
            c += GAMMA[mu][i][k] * GAMMA[nu][k][j] - GAMMA[nu][i][k] * GAMMA[mu][k][j];
          SIGMA[mu][nu][i][j] = 0.5 * I * c;
        }
  gammas_ready = 1;
}

/* out[0..3] = gamma_mu (mu = 0..3), out[4] = gamma_5; each 4x4 row-major */
void ora_gammas(cplx* out) {
  init_gammas();
  for (int mu = 0; mu < 4; ++mu) memcpy(out + 16 * mu, GAMMA[mu], 16 * sizeof(cplx));
  memcpy(out + 64, GAMMA5, 16 * sizeof(cplx));
}

/* ------------------------------------------------------------------ */
/* SU(3) helpers                                                        */
/* ------------------------------------------------------------------ */
typedef struct { cplx m[3][3]; } su3;

static su3 link_of(const cplx* U, int s, int mu) {
  su3 r;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) r.m[a][b] = U[((s * 4 + mu) * 3 + a) * 3 + b];
  return r;
}

static su3 mul(su3 x, su3 y) {
  su3 r;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      cplx c = 0;
      for (int k = 0; k < 3; ++k) c += x.m[a][k] * y.m[k][b];
      r.m[a][b] = c;
    }
  return r;
}

static su3 dag(su3 x) {
  su3 r;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) r.m[a][b] = conj(x.m[b][a]);
  return r;
}

static su3 add(su3 x, su3 y) {
  su3 r;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) r.m[a][b] = x.m[a][b] + y.m[a][b];
  return r;
}

/* site reached from s by steps (d1 along mu1) then (d2 along mu2) */
static int step2(const geom_t* g, int s, int mu1, int d1, int mu2, int d2) {
  int t = s;
  if (d1) t = neighbour(g, t, mu1, d1, NULL);
  if (d2) t = neighbour(g, t, mu2, d2, NULL);
  return t;
}

/* ------------------------------------------------------------------ */
/* clover term                                                          */
/* ------------------------------------------------------------------ */
/* Clover term of the Wilson-clover operator (Sec. 1-2; the paper takes the
 * operator from its references, this is the standard clover form):
 * A(x) = (4 + m0) 1 + (csw/2) sum_{mu<nu} i sigma_{mu nu} (x) Fhat_{mu nu}(x),
 * Fhat = (Q - Q^dag)/8 with Q the sum of the four plaquettes of the mu-nu
 * plane that touch x (clover leaf). Output: full 12x12 per site. */
int ora_clover(const int* dims, const cplx* U, double m0, double csw, cplx* A) {
  geom_t g;
  const int one[4] = {1, 1, 1, 1};
  if (geom_init(&g, dims, one)) return -1;
  init_gammas();
#pragma omp parallel for schedule(static)
  for (int s = 0; s < g.V; ++s) {
    cplx* a = A + (size_t)s * 144;
    for (int i = 0; i < 144; ++i) a[i] = 0;
    for (int i = 0; i < 12; ++i) a[i * 12 + i] = 4.0 + m0;
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu) {
        int xp_mu = step2(&g, s, mu, +1, nu, 0);
        int xp_nu = step2(&g, s, nu, +1, mu, 0);
        int xm_mu = step2(&g, s, mu, -1, nu, 0);
        int xm_nu = step2(&g, s, nu, -1, mu, 0);
        int xm_mu_p_nu = step2(&g, s, mu, -1, nu, +1);
        int xm_mu_m_nu = step2(&g, s, mu, -1, nu, -1);
        int xp_mu_m_nu = step2(&g, s, mu, +1, nu, -1);
        /* leaf 1: x -> x+mu -> x+mu+nu -> x+nu -> x */
        su3 q1 = mul(mul(link_of(U, s, mu), link_of(U, xp_mu, nu)),
                     mul(dag(link_of(U, xp_nu, mu)), dag(link_of(U, s, nu))));
        /* leaf 2: x -> x+nu -> x-mu+nu -> x-mu -> x */
        su3 q2 = mul(mul(link_of(U, s, nu), dag(link_of(U, xm_mu_p_nu, mu))),
                     mul(dag(link_of(U, xm_mu, nu)), link_of(U, xm_mu, mu)));
        /* leaf 3: x -> x-mu -> x-mu-nu -> x-nu -> x */
        su3 q3 = mul(mul(dag(link_of(U, xm_mu, mu)), dag(link_of(U, xm_mu_m_nu, nu))),
                     mul(link_of(U, xm_mu_m_nu, mu), link_of(U, xm_nu, nu)));
        /* leaf 4: x -> x-nu -> x+mu-nu -> x+mu -> x */
        su3 q4 = mul(mul(dag(link_of(U, xm_nu, nu)), link_of(U, xm_nu, mu)),
                     mul(link_of(U, xp_mu_m_nu, nu), dag(link_of(U, s, mu))));
        su3 Q = add(add(q1, q2), add(q3, q4));
        su3 Qd = dag(Q);
        for (int sp = 0; sp < 4; ++sp)
          for (int tp = 0; tp < 4; ++tp) {
            cplx sg = SIGMA[mu][nu][sp][tp];
            if (sg == 0) continue;
            for (int ca = 0; ca < 3; ++ca)
              for (int cb = 0; cb < 3; ++cb) {
                cplx F = (Q.m[ca][cb] - Qd.m[ca][cb]) / 8.0;
                a[(3 * sp + ca) * 12 + 3 * tp + cb] += 0.5 * csw * I * sg * F;
              }
          }
      }
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Wilson-clover operator                                               */
/* ------------------------------------------------------------------ */
/* The Wilson-clover operator D of the linear system that the solver of
 * Sec. 1-2 targets:
 * y(x) = A(x) psi(x)
 *      - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                   + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ]
 * with a factor -1 on hops across the t boundary. If block >= 0 only sites
 * of aggregate 'block' contribute as sources (Dirichlet restriction D_B). */
static void apply_D_site(const geom_t* g, const cplx* U, const cplx* A, const cplx* psi,
                         cplx* y, int s, int block) {
  const cplx* a = A + (size_t)s * 144;
  cplx out[12];
  for (int i = 0; i < 12; ++i) {
    cplx c = 0;
    for (int j = 0; j < 12; ++j) c += a[i * 12 + j] * psi[(size_t)s * 12 + j];
    out[i] = c;
  }
  for (int mu = 0; mu < 4; ++mu)
    for (int dir = +1; dir >= -1; dir -= 2) {
      int flip;
      int n = neighbour(g, s, mu, dir, &flip);
      if (block >= 0 && aggregate_of(g, n, NULL) != block) continue;
      su3 u = (dir > 0) ? link_of(U, s, mu) : dag(link_of(U, n, mu));
      double sgn = flip ? -1.0 : 1.0;
      /* U psi on colour, per spin */
      cplx up[12];
      for (int sp = 0; sp < 4; ++sp)
        for (int ca = 0; ca < 3; ++ca) {
          cplx c = 0;
          for (int cb = 0; cb < 3; ++cb) c += u.m[ca][cb] * psi[(size_t)n * 12 + 3 * sp + cb];
          up[3 * sp + ca] = c;
        }
      /* (1 -/+ gamma_mu) on spin */
      for (int sp = 0; sp < 4; ++sp)
        for (int ca = 0; ca < 3; ++ca) {
          cplx c = up[3 * sp + ca];
          for (int tp = 0; tp < 4; ++tp) c -= (double)dir * GAMMA[mu][sp][tp] * up[3 * tp + ca];
          out[3 * sp + ca] -= 0.5 * sgn * c;
        }
    }
  for (int i = 0; i < 12; ++i) y[(size_t)s * 12 + i] = out[i];
}

/* y = D psi on the whole lattice (single right-hand side) */
int ora_apply_D(const int* dims, const cplx* U, const cplx* A, const cplx* psi, cplx* y) {
  geom_t g;
  const int one[4] = {1, 1, 1, 1};
  if (geom_init(&g, dims, one)) return -1;
  init_gammas();
#pragma omp parallel for schedule(static)
  for (int s = 0; s < g.V; ++s) apply_D_site(&g, U, A, psi, y, s, -1);
  return 0;
}

/* y = D_B psi: D restricted to every aggregate (Dirichlet coupling between
 * aggregates), i.e. the block-diagonal part of D used by the Schwarz solves */
int ora_apply_D_block(const int* dims, const int* agg, const cplx* U, const cplx* A,
                      const cplx* psi, cplx* y) {
  geom_t g;
  if (geom_init(&g, dims, agg)) return -1;
  init_gammas();
#pragma omp parallel for schedule(static)
  for (int s = 0; s < g.V; ++s) apply_D_site(&g, U, A, psi, y, s, aggregate_of(&g, s, NULL));
  return 0;
}

/* ------------------------------------------------------------------ */
/* vector helpers                                                       */
/* ------------------------------------------------------------------ */
static cplx dotc(const cplx* a, const cplx* b, size_t n) {
  cplx c = 0;
  for (size_t i = 0; i < n; ++i) c += conj(a[i]) * b[i];
  return c;
}

static double norm2(const cplx* a, size_t n) {
  double c = 0;
  for (size_t i = 0; i < n; ++i) c += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
  return c;
}

/* list of the sites of every aggregate, in increasing site order */
static int* aggregate_sites(const geom_t* g) {
  int* list = (int*)malloc(sizeof(int) * (size_t)g->V);
  int* fill = (int*)calloc((size_t)g->nagg, sizeof(int));
  for (int s = 0; s < g->V; ++s) {
    int A = aggregate_of(g, s, NULL);
    list[(size_t)A * g->Va + fill[A]++] = s;
  }
  free(fill);
  return list;
}

/* ------------------------------------------------------------------ */
/* SAP smoother: red-black multiplicative Schwarz, MR block solves      */
/* ------------------------------------------------------------------ */
/* The domain-decomposition smoother of Sec. 2 (Schwarz alternating
 * procedure), used in the initial phase and in the V-cycle of Algorithm 1.
 * One sweep = colour 0 then colour 1 (colour = parity of the sum of the
 * aggregate coordinates). Per colour: r = b - D x; then for every aggregate
 * B of that colour, n_mr minimal-residual steps on D_B e = r_B from e = 0:
 *   q = D_B rho, alpha = <q,rho>/<q,q>, e += alpha rho, rho -= alpha q;
 * finally x_B += e. <a,b> = sum conj(a) b; alpha = 0 when q = 0. */
static void sap_rhs(const geom_t* g, const int* sites, const cplx* U, const cplx* A,
                    const cplx* b, cplx* x, int n_sweeps, int n_mr) {
  size_t n = (size_t)g->V * 12;
  cplx* r = (cplx*)malloc(sizeof(cplx) * n);
  /* rho and q are shared: blocks of one colour touch disjoint sites */
  cplx* rho = (cplx*)calloc(n, sizeof(cplx));
  cplx* q = (cplx*)calloc(n, sizeof(cplx));
  for (int sweep = 0; sweep < n_sweeps; ++sweep)
    for (int col = 0; col < 2; ++col) {
#pragma omp parallel for schedule(static)
      for (int s = 0; s < g->V; ++s) {
        apply_D_site(g, U, A, x, r, s, -1);
        for (int i = 0; i < 12; ++i) r[(size_t)s * 12 + i] = b[(size_t)s * 12 + i] - r[(size_t)s * 12 + i];
      }
#pragma omp parallel
      {
        cplx* e = (cplx*)malloc(sizeof(cplx) * (size_t)g->Va * 12);
#pragma omp for schedule(dynamic)
        for (int B = 0; B < g->nagg; ++B) {
          if (aggregate_colour(g, B) != col) continue;
          const int* bs = sites + (size_t)B * g->Va;
          for (int k = 0; k < g->Va; ++k)
            for (int i = 0; i < 12; ++i) {
              rho[(size_t)bs[k] * 12 + i] = r[(size_t)bs[k] * 12 + i];
              e[k * 12 + i] = 0;
            }
          for (int it = 0; it < n_mr; ++it) {
            cplx qr = 0;
            double qq = 0;
            for (int k = 0; k < g->Va; ++k) apply_D_site(g, U, A, rho, q, bs[k], B);
            for (int k = 0; k < g->Va; ++k) {
              qr += dotc(q + (size_t)bs[k] * 12, rho + (size_t)bs[k] * 12, 12);
              qq += norm2(q + (size_t)bs[k] * 12, 12);
            }
            cplx alpha = (qq > 0) ? qr / qq : 0;
            for (int k = 0; k < g->Va; ++k)
              for (int i = 0; i < 12; ++i) {
                e[k * 12 + i] += alpha * rho[(size_t)bs[k] * 12 + i];
                rho[(size_t)bs[k] * 12 + i] -= alpha * q[(size_t)bs[k] * 12 + i];
              }
          }
          for (int k = 0; k < g->Va; ++k)
            for (int i = 0; i < 12; ++i) x[(size_t)bs[k] * 12 + i] += e[k * 12 + i];
        }
        free(e);
      }
    }
  free(rho);
  free(q);
  free(r);
}

/* ------------------------------------------------------------------ */
/* even-odd preconditioned domain solves                                 */
/* ------------------------------------------------------------------ */
/* On a domain B (Dirichlet), D_B = [[A_EE, H_EO], [H_OE, A_OO]] with E and O
 * the sites of even and odd parity (x+y+z+t) and H the hopping terms, which
 * always change the parity. D_B e = r is solved through the Schur complement
 * on the even sites:
 *   S = A_EE - H_EO A_OO^-1 H_OE,   S e_E = r_E - H_EO A_OO^-1 r_O,
 *   e_O = A_OO^-1 (r_O - H_OE e_E),
 * with n_mr minimal-residual steps on S e_E = rhat from e_E = 0 (the same MR
 * as the plain smoother, inner products over the even sites). The result is
 * the exact domain solve in the limit of many steps, as for the plain form. */

/* 12 x 12 inverse by Gauss-Jordan elimination with partial pivoting */
static int invert12(const cplx* a, cplx* inv) {
  cplx m[12][24];
  for (int i = 0; i < 12; ++i)
    for (int j = 0; j < 24; ++j) m[i][j] = j < 12 ? a[i * 12 + j] : (j - 12 == i ? 1.0 : 0.0);
  for (int c = 0; c < 12; ++c) {
    int p = c;
    for (int i = c + 1; i < 12; ++i)
      if (cabs(m[i][c]) > cabs(m[p][c])) p = i;
    if (cabs(m[p][c]) == 0) return -1;
    if (p != c)
      for (int j = 0; j < 24; ++j) {
        cplx t = m[p][j];
        m[p][j] = m[c][j];
        m[c][j] = t;
      }
    cplx piv = m[c][c];
    for (int j = 0; j < 24; ++j) m[c][j] /= piv;
    for (int i = 0; i < 12; ++i) {
      if (i == c) continue;
      cplx f = m[i][c];
      if (f != 0)
        for (int j = 0; j < 24; ++j) m[i][j] -= f * m[c][j];
    }
  }
  for (int i = 0; i < 12; ++i)
    for (int j = 0; j < 12; ++j) inv[i * 12 + j] = m[i][j + 12];
  return 0;
}

static int site_parity(const geom_t* g, int s) {
  int x[4];
  coords_of(g->L, s, x);
  return (x[0] + x[1] + x[2] + x[3]) & 1;
}

/* y_s = (H psi)_s: the hopping terms of D at site s with sources in block B */
static void hop_site(const geom_t* g, const cplx* U, const cplx* psi, cplx* y, int s, int B) {
  cplx out[12] = {0};
  for (int mu = 0; mu < 4; ++mu)
    for (int dir = +1; dir >= -1; dir -= 2) {
      int flip;
      int n = neighbour(g, s, mu, dir, &flip);
      if (aggregate_of(g, n, NULL) != B) continue;
      su3 u = (dir > 0) ? link_of(U, s, mu) : dag(link_of(U, n, mu));
      double sgn = flip ? -1.0 : 1.0;
      cplx up[12];
      for (int sp = 0; sp < 4; ++sp)
        for (int ca = 0; ca < 3; ++ca) {
          cplx c = 0;
          for (int cb = 0; cb < 3; ++cb) c += u.m[ca][cb] * psi[(size_t)n * 12 + 3 * sp + cb];
          up[3 * sp + ca] = c;
        }
      for (int sp = 0; sp < 4; ++sp)
        for (int ca = 0; ca < 3; ++ca) {
          cplx c = up[3 * sp + ca];
          for (int tp = 0; tp < 4; ++tp) c -= (double)dir * GAMMA[mu][sp][tp] * up[3 * tp + ca];
          out[3 * sp + ca] -= 0.5 * sgn * c;
        }
    }
  for (int i = 0; i < 12; ++i) y[(size_t)s * 12 + i] = out[i];
}

/* y_s = M_s v_s for a 12 x 12 matrix per site */
static void site_mul(const cplx* M, const cplx* v, cplx* y, int s) {
  cplx out[12];
  for (int i = 0; i < 12; ++i) {
    cplx c = 0;
    for (int j = 0; j < 12; ++j) c += M[(size_t)s * 144 + i * 12 + j] * v[(size_t)s * 12 + j];
    out[i] = c;
  }
  for (int i = 0; i < 12; ++i) y[(size_t)s * 12 + i] = out[i];
}

/* the SAP sweeps of sap_rhs with every domain solve done on the Schur
 * complement of its even sites (Ainv: the inverse clover term per site) */
static void sap_rhs_eo(const geom_t* g, const int* sites, const cplx* U, const cplx* A, const cplx* Ainv,
                       const cplx* b, cplx* x, int n_sweeps, int n_mr) {
  size_t n = (size_t)g->V * 12;
  cplx* r = (cplx*)malloc(sizeof(cplx) * n);
  /* work vectors on the whole lattice; blocks of one colour touch disjoint
   * sites, and every hop reads only sites of the other parity */
  cplx* rho = (cplx*)calloc(n, sizeof(cplx));
  cplx* u = (cplx*)calloc(n, sizeof(cplx));
  cplx* q = (cplx*)calloc(n, sizeof(cplx));
  cplx* e = (cplx*)calloc(n, sizeof(cplx));
  cplx* t = (cplx*)calloc(n, sizeof(cplx));
  for (int sweep = 0; sweep < n_sweeps; ++sweep)
    for (int col = 0; col < 2; ++col) {
#pragma omp parallel for schedule(static)
      for (int s = 0; s < g->V; ++s) {
        apply_D_site(g, U, A, x, r, s, -1);
        for (int i = 0; i < 12; ++i) r[(size_t)s * 12 + i] = b[(size_t)s * 12 + i] - r[(size_t)s * 12 + i];
      }
#pragma omp parallel for schedule(dynamic)
      for (int B = 0; B < g->nagg; ++B) {
        if (aggregate_colour(g, B) != col) continue;
        const int* bs = sites + (size_t)B * g->Va;
        /* u_O = A_OO^-1 r_O; rho_E = rhat = r_E - H_EO u_O; e_E = 0 */
        for (int k = 0; k < g->Va; ++k)
          if (site_parity(g, bs[k]) == 1) site_mul(Ainv, r, u, bs[k]);
        for (int k = 0; k < g->Va; ++k) {
          const int s = bs[k];
          if (site_parity(g, s) != 0) continue;
          hop_site(g, U, u, t, s, B);
          for (int i = 0; i < 12; ++i) {
            rho[(size_t)s * 12 + i] = r[(size_t)s * 12 + i] - t[(size_t)s * 12 + i];
            e[(size_t)s * 12 + i] = 0;
          }
        }
        for (int it = 0; it < n_mr; ++it) {
          /* q_E = S rho_E = A_EE rho_E - H_EO A_OO^-1 H_OE rho_E */
          for (int k = 0; k < g->Va; ++k)
            if (site_parity(g, bs[k]) == 1) {
              hop_site(g, U, rho, t, bs[k], B);
              site_mul(Ainv, t, u, bs[k]);
            }
          cplx qr = 0;
          double qq = 0;
          for (int k = 0; k < g->Va; ++k) {
            const int s = bs[k];
            if (site_parity(g, s) != 0) continue;
            site_mul(A, rho, q, s);
            hop_site(g, U, u, t, s, B);
            for (int i = 0; i < 12; ++i) q[(size_t)s * 12 + i] -= t[(size_t)s * 12 + i];
            qr += dotc(q + (size_t)s * 12, rho + (size_t)s * 12, 12);
            qq += norm2(q + (size_t)s * 12, 12);
          }
          cplx alpha = (qq > 0) ? qr / qq : 0;
          for (int k = 0; k < g->Va; ++k) {
            const int s = bs[k];
            if (site_parity(g, s) != 0) continue;
            for (int i = 0; i < 12; ++i) {
              e[(size_t)s * 12 + i] += alpha * rho[(size_t)s * 12 + i];
              rho[(size_t)s * 12 + i] -= alpha * q[(size_t)s * 12 + i];
            }
          }
        }
        /* e_O = A_OO^-1 (r_O - H_OE e_E); x_B += e */
        for (int k = 0; k < g->Va; ++k) {
          const int s = bs[k];
          if (site_parity(g, s) != 1) continue;
          hop_site(g, U, e, t, s, B);
          for (int i = 0; i < 12; ++i) t[(size_t)s * 12 + i] = r[(size_t)s * 12 + i] - t[(size_t)s * 12 + i];
          site_mul(Ainv, t, e, s);
        }
        for (int k = 0; k < g->Va; ++k)
          for (int i = 0; i < 12; ++i) x[(size_t)bs[k] * 12 + i] += e[(size_t)bs[k] * 12 + i];
      }
    }
  free(rho);
  free(u);
  free(q);
  free(e);
  free(t);
  free(r);
}

/* the inverse clover term of every site (NULL if a block is singular) */
static cplx* clover_inverses(const geom_t* g, const cplx* A) {
  cplx* Ainv = (cplx*)malloc(sizeof(cplx) * (size_t)g->V * 144);
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int s = 0; s < g->V; ++s) bad |= invert12(A + (size_t)s * 144, Ainv + (size_t)s * 144) != 0;
  if (bad) {
    free(Ainv);
    return NULL;
  }
  return Ainv;
}

/* the smoother of the setup and of the V-cycle: plain (even_odd = 0) or
 * with even-odd preconditioned domain solves (even_odd = 1) */
static int smooth(const geom_t* g, const int* sites, const cplx* U, const cplx* A, const cplx* Ainv,
                  const cplx* b, cplx* x, int n_sweeps, int n_mr, int even_odd) {
  if (!even_odd) {
    sap_rhs(g, sites, U, A, b, x, n_sweeps, n_mr);
    return 0;
  }
  if (!Ainv) return -6;
  sap_rhs_eo(g, sites, U, A, Ainv, b, x, n_sweeps, n_mr);
  return 0;
}

/* x <- SAP^n_sweeps(b, x) with even-odd preconditioned domain solves */
int ora_sap_eo(const int* dims, const int* agg, const cplx* U, const cplx* A, const cplx* b, cplx* x, int nrhs,
               int n_sweeps, int n_mr) {
  geom_t g;
  if (geom_init(&g, dims, agg)) return -1;
  init_gammas();
  int* sites = aggregate_sites(&g);
  cplx* Ainv = clover_inverses(&g, A);
  size_t n = (size_t)g.V * 12;
  int st = 0;
  for (int j = 0; j < nrhs && !st; ++j) st = smooth(&g, sites, U, A, Ainv, b + j * n, x + j * n, n_sweeps, n_mr, 1);
  free(Ainv);
  free(sites);
  return st;
}

/* x <- SAP^n_sweeps(b, x) for nrhs right-hand sides, one after the other */
int ora_sap(const int* dims, const int* agg, const cplx* U, const cplx* A, const cplx* b,
            cplx* x, int nrhs, int n_sweeps, int n_mr) {
  geom_t g;
  if (geom_init(&g, dims, agg)) return -1;
  init_gammas();
  int* sites = aggregate_sites(&g);
  size_t n = (size_t)g.V * 12;
  for (int j = 0; j < nrhs; ++j) sap_rhs(&g, sites, U, A, b + j * n, x + j * n, n_sweeps, n_mr);
  free(sites);
  return 0;
}

/* ------------------------------------------------------------------ */
/* aggregate-wise Gram-Schmidt -> P = R^dag                              */
/* ------------------------------------------------------------------ */
/* P = R^dag from the test vectors (Sec. 2), aggregate by aggregate and
 * split by chirality as in Algorithm 3 (Sec. 5).
 * For every aggregate A and chirality h, the test vectors restricted to
 * (sites of A) x (components of chirality h) are orthonormalised in order
 * j = 0..ntv-1 by modified Gram-Schmidt, applied twice. Column j of P is the
 * orthonormalised vector j; within chirality h it is the column (h, j) of
 * the prolongation. Returns -6 if a vector becomes linearly dependent. */
int ora_gram_schmidt(const int* dims, const int* agg, int ntv, const cplx* tv, cplx* P) {
  geom_t g;
  if (geom_init(&g, dims, agg)) return -1;
  int* sites = aggregate_sites(&g);
  size_t n = (size_t)g.V * 12;
  int L = 6 * g.Va;
  int bad = 0;
#pragma omp parallel
  {
    cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)L * ntv);
#pragma omp for schedule(dynamic)
    for (int Ah = 0; Ah < 2 * g.nagg; ++Ah) {
      int A = Ah / 2, h = Ah % 2;
      const int* bs = sites + (size_t)A * g.Va;
      for (int j = 0; j < ntv; ++j)
        for (int k = 0; k < g.Va; ++k)
          for (int c = 0; c < 6; ++c) w[(size_t)j * L + 6 * k + c] = tv[j * n + (size_t)bs[k] * 12 + 6 * h + c];
      for (int j = 0; j < ntv; ++j) {
        cplx* wj = w + (size_t)j * L;
        for (int pass = 0; pass < 2; ++pass)
          for (int i = 0; i < j; ++i) {
            cplx* wi = w + (size_t)i * L;
            cplx c = dotc(wi, wj, L);
            for (int k = 0; k < L; ++k) wj[k] -= c * wi[k];
          }
        double nn = sqrt(norm2(wj, L));
        if (!(nn > 0) || !isfinite(nn)) {
#pragma omp atomic write
          bad = 1;
          nn = 1;
        }
        for (int k = 0; k < L; ++k) wj[k] /= nn;
      }
      for (int j = 0; j < ntv; ++j)
        for (int k = 0; k < g.Va; ++k)
          for (int c = 0; c < 6; ++c) P[j * n + (size_t)bs[k] * 12 + 6 * h + c] = w[(size_t)j * L + 6 * k + c];
    }
    free(w);
  }
  free(sites);
  return bad ? -6 : 0;
}

/* ------------------------------------------------------------------ */
/* restriction, prolongation (R = P^dag)                                */
/* ------------------------------------------------------------------ */
/* restriction R = P^dag (Sec. 2; the sum of Algorithm 3, Sec. 5):
 * vc[A][h*ntv + j] = sum_{s in A, c in h} conj(P_j(s,c)) v(s,c) */
static void restrict_one(const geom_t* g, int ntv, const cplx* P, const cplx* v, cplx* vc) {
  size_t n = (size_t)g->V * 12;
  for (int i = 0; i < g->nagg * 2 * ntv; ++i) vc[i] = 0;
  for (int s = 0; s < g->V; ++s) {
    int A = aggregate_of(g, s, NULL);
    for (int c = 0; c < 12; ++c) {
      int h = c / 6;
      for (int j = 0; j < ntv; ++j)
        vc[(size_t)A * 2 * ntv + h * ntv + j] += conj(P[j * n + (size_t)s * 12 + c]) * v[(size_t)s * 12 + c];
    }
  }
}

/* prolongation P (Sec. 2, Algorithm 1):
 * u(s,c) = sum_j P_j(s,c) uc[A(s)][h(c)*ntv + j] */
static void prolong_one(const geom_t* g, int ntv, const cplx* P, const cplx* uc, cplx* u) {
  size_t n = (size_t)g->V * 12;
  for (int s = 0; s < g->V; ++s) {
    int A = aggregate_of(g, s, NULL);
    for (int c = 0; c < 12; ++c) {
      int h = c / 6;
      cplx acc = 0;
      for (int j = 0; j < ntv; ++j) acc += P[j * n + (size_t)s * 12 + c] * uc[(size_t)A * 2 * ntv + h * ntv + j];
      u[(size_t)s * 12 + c] = acc;
    }
  }
}

int ora_restrict(const int* dims, const int* agg, int ntv, const cplx* P, const cplx* v,
                 cplx* vc, int nrhs) {
  geom_t g;
  if (geom_init(&g, dims, agg)) return -1;
  for (int r = 0; r < nrhs; ++r)
    restrict_one(&g, ntv, P, v + (size_t)r * g.V * 12, vc + (size_t)r * g.nagg * 2 * ntv);
  return 0;
}

int ora_prolong(const int* dims, const int* agg, int ntv, const cplx* P, const cplx* uc,
                cplx* u, int nrhs) {
  geom_t g;
  if (geom_init(&g, dims, agg)) return -1;
  for (int r = 0; r < nrhs; ++r)
    prolong_one(&g, ntv, P, uc + (size_t)r * g.nagg * 2 * ntv, u + (size_t)r * g.V * 12);
  return 0;
}

/* ------------------------------------------------------------------ */
/* coarse operator Dc = P^dag D P as a 9-point stencil                   */
/* ------------------------------------------------------------------ */
/* The coarse-grid operator of Sec. 2, D_c = R D P (Galerkin product with
 * R = P^dag), as a nearest-neighbour stencil on the aggregates.
 * The hopping terms of D are routed by the aggregate they connect:
 *   k = 0      A(x) psi(x) and hops with both ends in the same aggregate
 *   k = 1+mu   the +mu hop of x when x+mu lies in another aggregate
 *   k = 5+mu   the -mu hop of x when x-mu lies in another aggregate
 * Dc[A][k][(h,i)][(h',j)] = sum_{x in A} P_(h,i)(x)^dag (D_k P_(h',j))(x).
 * Column (h', j) is P_j restricted to the components of chirality h'. */
int ora_coarse_op(const int* dims, const int* agg, int ntv, const cplx* U, const cplx* A,
                  const cplx* P, cplx* Dc) {
  geom_t g;
  if (geom_init(&g, dims, agg)) return -1;
  init_gammas();
  size_t n = (size_t)g.V * 12;
  int nc = 2 * ntv;
  memset(Dc, 0, sizeof(cplx) * (size_t)g.nagg * 9 * nc * nc);
  int* sites = aggregate_sites(&g);
  cplx* col = (cplx*)malloc(sizeof(cplx) * n);
  cplx* part = (cplx*)malloc(sizeof(cplx) * n * 9); /* D_k col, k = 0..8 */
  for (int hp = 0; hp < 2; ++hp)
    for (int j = 0; j < ntv; ++j) {
      for (size_t i = 0; i < n; ++i) col[i] = ((i % 12) / 6 == (size_t)hp) ? P[j * n + i] : 0;
      memset(part, 0, sizeof(cplx) * n * 9);
#pragma omp parallel for schedule(static)
      for (int s = 0; s < g.V; ++s) {
        int As = aggregate_of(&g, s, NULL);
        const cplx* a = A + (size_t)s * 144;
        cplx* p0 = part + (size_t)s * 12;
        for (int i = 0; i < 12; ++i) {
          cplx c = 0;
          for (int jj = 0; jj < 12; ++jj) c += a[i * 12 + jj] * col[(size_t)s * 12 + jj];
          p0[i] += c;
        }
        for (int mu = 0; mu < 4; ++mu)
          for (int dir = +1; dir >= -1; dir -= 2) {
            int flip;
            int nn = neighbour(&g, s, mu, dir, &flip);
            int k = (aggregate_of(&g, nn, NULL) == As) ? 0 : (dir > 0 ? 1 + mu : 5 + mu);
            cplx* pk = part + (size_t)k * n + (size_t)s * 12;
            su3 u = (dir > 0) ? link_of(U, s, mu) : dag(link_of(U, nn, mu));
            double sgn = flip ? -1.0 : 1.0;
            cplx up[12];
            for (int sp = 0; sp < 4; ++sp)
              for (int ca = 0; ca < 3; ++ca) {
                cplx c = 0;
                for (int cb = 0; cb < 3; ++cb) c += u.m[ca][cb] * col[(size_t)nn * 12 + 3 * sp + cb];
                up[3 * sp + ca] = c;
              }
            for (int sp = 0; sp < 4; ++sp)
              for (int ca = 0; ca < 3; ++ca) {
                cplx c = up[3 * sp + ca];
                for (int tp = 0; tp < 4; ++tp) c -= (double)dir * GAMMA[mu][sp][tp] * up[3 * tp + ca];
                pk[3 * sp + ca] -= 0.5 * sgn * c;
              }
          }
      }
      /* project every part onto the rows (h, i) of the receiving aggregate */
#pragma omp parallel for schedule(static)
      for (int Ag = 0; Ag < g.nagg; ++Ag)
        for (int kk = 0; kk < g.Va; ++kk) {
          int s = sites[(size_t)Ag * g.Va + kk];
          for (int k = 0; k < 9; ++k) {
            const cplx* pk = part + (size_t)k * n + (size_t)s * 12;
            for (int c = 0; c < 12; ++c) {
              if (pk[c] == 0) continue;
              int h = c / 6;
              for (int i = 0; i < ntv; ++i)
                Dc[(((size_t)Ag * 9 + k) * nc + h * ntv + i) * nc + hp * ntv + j] +=
                    conj(P[i * n + (size_t)s * 12 + c]) * pk[c];
            }
          }
        }
    }
  free(col);
  free(part);
  free(sites);
  return 0;
}

/* yc(A) = sum_k Dc[A][k] xc(nbr_k(A)), nbr_0(A) = A */
static void apply_Dc_one(const geom_t* g, int ntv, const cplx* Dc, const cplx* xc, cplx* yc) {
  int nc = 2 * ntv;
  for (int A = 0; A < g->nagg; ++A) {
    int nb[9];
    nb[0] = A;
    for (int mu = 0; mu < 4; ++mu) {
      nb[1 + mu] = aggregate_neighbour(g, A, mu, +1);
      nb[5 + mu] = aggregate_neighbour(g, A, mu, -1);
    }
    for (int i = 0; i < nc; ++i) {
      cplx c = 0;
      for (int k = 0; k < 9; ++k)
        for (int j = 0; j < nc; ++j) c += Dc[(((size_t)A * 9 + k) * nc + i) * nc + j] * xc[(size_t)nb[k] * nc + j];
      yc[(size_t)A * nc + i] = c;
    }
  }
}

int ora_apply_Dc(const int* dims, const int* agg, int ntv, const cplx* Dc, const cplx* xc,
                 cplx* yc, int nrhs) {
  geom_t g;
  if (geom_init(&g, dims, agg)) return -1;
  size_t nc = (size_t)g.nagg * 2 * ntv;
  for (int r = 0; r < nrhs; ++r) apply_Dc_one(&g, ntv, Dc, xc + r * nc, yc + r * nc);
  return 0;
}

/* ------------------------------------------------------------------ */
/* GMRES(m) with Givens rotations (coarse solve and the two-level FGMRES) */
/* ------------------------------------------------------------------ */
typedef void (*op_fn)(void* ctx, const cplx* in, cplx* out);

/* The approximate coarse solve of Algorithm 1 (relative tolerance 0.05 in
 * Sec. 7) and the outer FGMRES of Sec. 2.
 * Solves op x = b from x = 0. Stops when the residual estimate falls to
 * tol*|b| or after maxit iterations in total (restarting every m). With
 * precond != NULL it is right-preconditioned flexible GMRES: z_k = M v_k is
 * stored and x is built from the z_k. Returns the iteration count. */
static int gmres(op_fn op, void* octx, op_fn precond, void* pctx, size_t n, const cplx* b,
                 cplx* x, double tol, int m, int maxit, double* relres) {
  cplx* Vb = (cplx*)malloc(sizeof(cplx) * n * (m + 1));
  cplx* Z = precond ? (cplx*)malloc(sizeof(cplx) * n * m) : NULL;
  cplx* w = (cplx*)malloc(sizeof(cplx) * n);
  cplx* H = (cplx*)calloc((size_t)(m + 1) * m, sizeof(cplx));
  cplx* cs = (cplx*)malloc(sizeof(cplx) * m);
  cplx* sn = (cplx*)malloc(sizeof(cplx) * m);
  cplx* gv = (cplx*)malloc(sizeof(cplx) * (m + 1));
  cplx* y = (cplx*)malloc(sizeof(cplx) * m);
  for (size_t i = 0; i < n; ++i) x[i] = 0;
  double bnorm = sqrt(norm2(b, n));
  int it = 0;
  double res = 0;
  if (bnorm == 0) {
    if (relres) *relres = 0;
    goto done;
  }
  res = 1;
  while (it < maxit) {
    /* r = b - op x */
    op(octx, x, w);
    for (size_t i = 0; i < n; ++i) w[i] = b[i] - w[i];
    double beta = sqrt(norm2(w, n));
    res = beta / bnorm;
    if (beta <= tol * bnorm) break;
    for (size_t i = 0; i < n; ++i) Vb[i] = w[i] / beta;
    for (int i = 0; i <= m; ++i) gv[i] = 0;
    gv[0] = beta;
    int kend = 0, conv = 0;
    for (int k = 0; k < m; ++k) {
      cplx* vk = Vb + (size_t)k * n;
      if (precond) {
        precond(pctx, vk, Z + (size_t)k * n);
        op(octx, Z + (size_t)k * n, w);
      } else {
        op(octx, vk, w);
      }
      for (int i = 0; i <= k; ++i) {
        cplx hik = dotc(Vb + (size_t)i * n, w, n);
        H[i * m + k] = hik;
        for (size_t l = 0; l < n; ++l) w[l] -= hik * Vb[(size_t)i * n + l];
      }
      double hk1 = sqrt(norm2(w, n));
      H[(k + 1) * m + k] = hk1;
      /* previous rotations */
      for (int i = 0; i < k; ++i) {
        cplx a = H[i * m + k], bb = H[(i + 1) * m + k];
        H[i * m + k] = conj(cs[i]) * a + conj(sn[i]) * bb;
        H[(i + 1) * m + k] = -sn[i] * a + cs[i] * bb;
      }
      /* new rotation zeroing H[k+1][k] */
      {
        cplx a = H[k * m + k], bb = H[(k + 1) * m + k];
        double nu = sqrt(creal(a * conj(a)) + creal(bb * conj(bb)));
        if (nu == 0) {
          cs[k] = 1;
          sn[k] = 0;
        } else {
          cs[k] = a / nu;
          sn[k] = bb / nu;
        }
        H[k * m + k] = nu;
        H[(k + 1) * m + k] = 0;
        cplx g0 = gv[k];
        gv[k] = conj(cs[k]) * g0;
        gv[k + 1] = -sn[k] * g0;
      }
      ++it;
      kend = k + 1;
      res = cabs(gv[k + 1]) / bnorm;
      if (hk1 > 0)
        for (size_t l = 0; l < n; ++l) Vb[(size_t)(k + 1) * n + l] = w[l] / hk1;
      if (cabs(gv[k + 1]) <= tol * bnorm || hk1 == 0) conv = 1;
      if (conv || it >= maxit) break;
    }
    /* back substitution H y = g on the leading kend x kend triangle */
    for (int i = kend - 1; i >= 0; --i) {
      cplx c = gv[i];
      for (int l = i + 1; l < kend; ++l) c -= H[i * m + l] * y[l];
      y[i] = c / H[i * m + i];
    }
    const cplx* basis = precond ? Z : Vb;
    for (int i = 0; i < kend; ++i)
      for (size_t l = 0; l < n; ++l) x[l] += y[i] * basis[(size_t)i * n + l];
    if (conv) break;
  }
done:
  if (relres) *relres = res;
  free(Vb);
  free(Z);
  free(w);
  free(H);
  free(cs);
  free(sn);
  free(gv);
  free(y);
  return it;
}

typedef struct {
  const geom_t* g;
  int ntv;
  const cplx* Dc;
} coarse_ctx;

static void coarse_op(void* c, const cplx* in, cplx* out) {
  coarse_ctx* cc = (coarse_ctx*)c;
  apply_Dc_one(cc->g, cc->ntv, cc->Dc, in, out);
}

/* coarse GMRES per right-hand side; iters[r] receives each count */
int ora_coarse_solve(const int* dims, const int* agg, int ntv, const cplx* Dc, const cplx* bc,
                     cplx* xc, int nrhs, double tol, int restart, int maxit, int* iters) {
  geom_t g;
  if (geom_init(&g, dims, agg)) return -1;
  coarse_ctx cc = {&g, ntv, Dc};
  size_t nc = (size_t)g.nagg * 2 * ntv;
  for (int r = 0; r < nrhs; ++r) {
    int it = gmres(coarse_op, &cc, NULL, NULL, nc, bc + r * nc, xc + r * nc, tol, restart, maxit, NULL);
    if (iters) iters[r] = it;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* even-odd preconditioned coarse solve                                  */
/* ------------------------------------------------------------------ */
/* The red-black colouring of the aggregates (the SAP domains) makes every
 * hop block of D_c join aggregates of different colour, so with e the
 * aggregates of colour 0 and o those of colour 1, D_c = [[D_ee, D_eo],
 * [D_oe, D_oo]] with D_ee and D_oo block-diagonal (the self blocks). The
 * coarse system is solved on the Schur complement of the even aggregates
 * (Sec. 4 names even-odd preconditioning of the coarse grid):
 *   S x_e = b_e - D_eo D_oo^-1 b_o,   S = D_ee - D_eo D_oo^-1 D_oe,
 *   x_o = D_oo^-1 (b_o - D_oe x_e),
 * GMRES(m) on S from x_e = 0 with the relative tolerance taken on the Schur
 * system's right-hand side. Vectors keep the full coarse layout with zeros on
 * the odd aggregates. */

/* n x n inverse by Gauss-Jordan elimination with partial pivoting */
static int invert_n(int n, const cplx* a, cplx* inv) {
  cplx* m = (cplx*)malloc(sizeof(cplx) * (size_t)n * 2 * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) m[(size_t)i * 2 * n + j] = j < n ? a[(size_t)i * n + j] : (j - n == i ? 1.0 : 0.0);
  int st = 0;
  for (int c = 0; c < n && !st; ++c) {
    int p = c;
    for (int i = c + 1; i < n; ++i)
      if (cabs(m[(size_t)i * 2 * n + c]) > cabs(m[(size_t)p * 2 * n + c])) p = i;
    if (cabs(m[(size_t)p * 2 * n + c]) == 0) {
      st = -6;
      break;
    }
    if (p != c)
      for (int j = 0; j < 2 * n; ++j) {
        cplx t = m[(size_t)p * 2 * n + j];
        m[(size_t)p * 2 * n + j] = m[(size_t)c * 2 * n + j];
        m[(size_t)c * 2 * n + j] = t;
      }
    cplx piv = m[(size_t)c * 2 * n + c];
    for (int j = 0; j < 2 * n; ++j) m[(size_t)c * 2 * n + j] /= piv;
    for (int i = 0; i < n; ++i) {
      if (i == c) continue;
      cplx f = m[(size_t)i * 2 * n + c];
      if (f != 0)
        for (int j = 0; j < 2 * n; ++j) m[(size_t)i * 2 * n + j] -= f * m[(size_t)c * 2 * n + j];
    }
  }
  for (int i = 0; i < n && !st; ++i)
    for (int j = 0; j < n; ++j) inv[(size_t)i * n + j] = m[(size_t)i * 2 * n + n + j];
  free(m);
  return st;
}

typedef struct {
  const geom_t* g;
  int ntv;
  const cplx* Dc;
  const cplx* Dinv; /* [nagg][nc][nc], the inverse self blocks of the odd aggregates */
  cplx *t, *u;      /* work vectors of the coarse size */
} coarse_eo_ctx;

/* y = D_oo^-1 x on the odd aggregates, 0 on the even ones */
static void odd_block_inverse(const coarse_eo_ctx* e, const cplx* x, cplx* y) {
  const int nc = 2 * e->ntv;
  for (int A = 0; A < e->g->nagg; ++A)
    for (int i = 0; i < nc; ++i) {
      cplx c = 0;
      if (aggregate_colour(e->g, A) == 1)
        for (int j = 0; j < nc; ++j) c += e->Dinv[((size_t)A * nc + i) * nc + j] * x[(size_t)A * nc + j];
      y[(size_t)A * nc + i] = c;
    }
}

/* out = S in (in zero on the odd aggregates; out likewise) */
static void coarse_schur_op(void* c, const cplx* in, cplx* out) {
  coarse_eo_ctx* e = (coarse_eo_ctx*)c;
  const int nc = 2 * e->ntv;
  apply_Dc_one(e->g, e->ntv, e->Dc, in, e->t);  /* even rows: D_ee in_e; odd rows: D_oe in_e */
  odd_block_inverse(e, e->t, e->u);              /* u_o = D_oo^-1 D_oe in_e */
  apply_Dc_one(e->g, e->ntv, e->Dc, e->u, out);  /* even rows: D_eo u_o */
  for (int A = 0; A < e->g->nagg; ++A)
    for (int i = 0; i < nc; ++i) {
      const size_t k = (size_t)A * nc + i;
      out[k] = aggregate_colour(e->g, A) == 0 ? e->t[k] - out[k] : 0;
    }
}

/* the inverse self blocks of the odd aggregates (NULL if one is singular) */
static cplx* odd_self_inverses(const geom_t* g, int ntv, const cplx* Dc) {
  const int nc = 2 * ntv;
  cplx* Dinv = (cplx*)calloc((size_t)g->nagg * nc * nc, sizeof(cplx));
  int bad = 0;
  for (int A = 0; A < g->nagg && !bad; ++A)
    if (aggregate_colour(g, A) == 1)
      bad = invert_n(nc, Dc + (size_t)A * 9 * nc * nc, Dinv + (size_t)A * nc * nc) != 0;
  if (bad) {
    free(Dinv);
    return NULL;
  }
  return Dinv;
}

/* x = D_c^-1 b approximately, on the Schur complement (one right-hand side);
 * returns the GMRES iteration count, or -1 when a self block is singular */
static int coarse_solve_eo_one(const geom_t* g, int ntv, const cplx* Dc, const cplx* Dinv, const cplx* b, cplx* x,
                               double tol, int restart, int maxit) {
  const int nc = 2 * ntv;
  const size_t n = (size_t)g->nagg * nc;
  cplx* t = (cplx*)malloc(sizeof(cplx) * n);
  cplx* u = (cplx*)malloc(sizeof(cplx) * n);
  cplx* bh = (cplx*)malloc(sizeof(cplx) * n);
  cplx* s = (cplx*)malloc(sizeof(cplx) * n);
  coarse_eo_ctx e = {g, ntv, Dc, Dinv, t, u};
  /* bhat_e = b_e - D_eo D_oo^-1 b_o */
  odd_block_inverse(&e, b, u);
  apply_Dc_one(g, ntv, Dc, u, s);
  for (int A = 0; A < g->nagg; ++A)
    for (int i = 0; i < nc; ++i) {
      const size_t k = (size_t)A * nc + i;
      bh[k] = aggregate_colour(g, A) == 0 ? b[k] - s[k] : 0;
    }
  int it = gmres(coarse_schur_op, &e, NULL, NULL, n, bh, x, tol, restart, maxit, NULL);
  /* x_o = D_oo^-1 (b_o - D_oe x_e) */
  apply_Dc_one(g, ntv, Dc, x, s);
  for (int A = 0; A < g->nagg; ++A)
    for (int i = 0; i < nc; ++i) {
      const size_t k = (size_t)A * nc + i;
      s[k] = aggregate_colour(g, A) == 1 ? b[k] - s[k] : 0;
    }
  odd_block_inverse(&e, s, u);
  for (int A = 0; A < g->nagg; ++A)
    if (aggregate_colour(g, A) == 1)
      for (int i = 0; i < nc; ++i) x[(size_t)A * nc + i] = u[(size_t)A * nc + i];
  free(t);
  free(u);
  free(bh);
  free(s);
  return it;
}

int ora_coarse_solve_eo(const int* dims, const int* agg, int ntv, const cplx* Dc, const cplx* bc, cplx* xc,
                        int nrhs, double tol, int restart, int maxit, int* iters) {
  geom_t g;
  if (geom_init(&g, dims, agg)) return -1;
  cplx* Dinv = odd_self_inverses(&g, ntv, Dc);
  if (!Dinv) return -6;
  size_t nc = (size_t)g.nagg * 2 * ntv;
  for (int r = 0; r < nrhs; ++r) {
    int it = coarse_solve_eo_one(&g, ntv, Dc, Dinv, bc + r * nc, xc + r * nc, tol, restart, maxit);
    if (iters) iters[r] = it;
  }
  free(Dinv);
  return 0;
}

/* ------------------------------------------------------------------ */
/* the setup (Algorithm 1 order, one test vector at a time)              */
/* ------------------------------------------------------------------ */
typedef struct {
  int init_mode;        /* 0: one smoother call of n_sweeps sweeps, b = v, x0 = 0
                           1: n_sweeps calls of one sweep, each v <- SAP(b = v, x0 = 0) */
  int n_init_sweeps, n_init_mr;
  int n_refine, n_smooth_sweeps, n_smooth_mr;
  double coarse_tol;
  int coarse_restart, coarse_maxit;
  int even_odd;         /* 1: even-odd preconditioned domain solves in the smoother */
  int coarse_even_odd;  /* 1: coarse solves on the Schur complement of the even aggregates */
} ora_setup_params;

static void normalise(cplx* v, size_t n) {
  double nn = sqrt(norm2(v, n));
  if (nn > 0)
    for (size_t i = 0; i < n; ++i) v[i] /= nn;
}

/* Initial phase of the setup (Sec. 2): the smoother on every test vector
 * from x0 = 0, normalise, then P (Gram-Schmidt) and Dc. tv is updated in
 * place. */
int ora_setup_init(const int* dims, const int* agg, int ntv, const cplx* U, const cplx* A,
                   cplx* tv, const ora_setup_params* p, cplx* P, cplx* Dc) {
  geom_t g;
  if (geom_init(&g, dims, agg)) return -1;
  init_gammas();
  int* sites = aggregate_sites(&g);
  cplx* Ainv = p->even_odd ? clover_inverses(&g, A) : NULL;
  size_t n = (size_t)g.V * 12;
  cplx* x = (cplx*)malloc(sizeof(cplx) * n);
  int sst = 0;
  for (int j = 0; j < ntv && !sst; ++j) {
    cplx* v = tv + j * n;
    if (p->init_mode == 0) {
      memset(x, 0, sizeof(cplx) * n);
      sst = smooth(&g, sites, U, A, Ainv, v, x, p->n_init_sweeps, p->n_init_mr, p->even_odd);
      memcpy(v, x, sizeof(cplx) * n);
    } else {
      for (int it = 0; it < p->n_init_sweeps && !sst; ++it) {
        memset(x, 0, sizeof(cplx) * n);
        sst = smooth(&g, sites, U, A, Ainv, v, x, 1, p->n_init_mr, p->even_odd);
        memcpy(v, x, sizeof(cplx) * n);
      }
    }
    normalise(v, n);
  }
  free(x);
  free(Ainv);
  free(sites);
  if (sst) return sst;
  int st = ora_gram_schmidt(dims, agg, ntv, tv, P);
  if (st) return st;
  return ora_coarse_op(dims, agg, ntv, U, A, P, Dc);
}

/* Iterative refinement, Algorithm 1: for each test vector j in turn,
 * v_c = R v_j, u_c ~ Dc^{-1} v_c (GMRES to coarse_tol), u = P u_c,
 * v_j <- SAP(b = v_j, x0 = u), normalised; after all j, rebuild P and Dc. */
int ora_setup_refine(const int* dims, const int* agg, int ntv, const cplx* U, const cplx* A,
                     cplx* tv, const ora_setup_params* p, cplx* P, cplx* Dc, int* coarse_iters) {
  geom_t g;
  if (geom_init(&g, dims, agg)) return -1;
  init_gammas();
  int* sites = aggregate_sites(&g);
  size_t n = (size_t)g.V * 12;
  size_t nc = (size_t)g.nagg * 2 * ntv;
  cplx* vc = (cplx*)malloc(sizeof(cplx) * nc);
  cplx* uc = (cplx*)malloc(sizeof(cplx) * nc);
  cplx* x = (cplx*)malloc(sizeof(cplx) * n);
  cplx* Ainv = p->even_odd ? clover_inverses(&g, A) : NULL;
  coarse_ctx cc = {&g, ntv, Dc};
  int st = 0;
  for (int i = 0; i < p->n_refine; ++i) {
    cplx* Dinv = NULL;
    if (p->coarse_even_odd) {
      Dinv = odd_self_inverses(&g, ntv, Dc);
      if (!Dinv) {
        st = -6;
        break;
      }
    }
    for (int j = 0; j < ntv; ++j) {
      cplx* v = tv + j * n;
      restrict_one(&g, ntv, P, v, vc);
      int it = p->coarse_even_odd
                   ? coarse_solve_eo_one(&g, ntv, Dc, Dinv, vc, uc, p->coarse_tol, p->coarse_restart,
                                         p->coarse_maxit)
                   : gmres(coarse_op, &cc, NULL, NULL, nc, vc, uc, p->coarse_tol, p->coarse_restart,
                           p->coarse_maxit, NULL);
      if (coarse_iters) coarse_iters[i * ntv + j] = it;
      prolong_one(&g, ntv, P, uc, x);
      st = smooth(&g, sites, U, A, Ainv, v, x, p->n_smooth_sweeps, p->n_smooth_mr, p->even_odd);
      if (st) break;
      memcpy(v, x, sizeof(cplx) * n);
      normalise(v, n);
    }
    free(Dinv);
    if (st) break;
    st = ora_gram_schmidt(dims, agg, ntv, tv, P);
    if (st) break;
    st = ora_coarse_op(dims, agg, ntv, U, A, P, Dc);
    if (st) break;
  }
  free(vc);
  free(uc);
  free(x);
  free(Ainv);
  free(sites);
  return st;
}

/* ------------------------------------------------------------------ */
/* two-level FGMRES (the quality check of a setup)                       */
/* ------------------------------------------------------------------ */
typedef struct {
  geom_t g;
  const int* sites;
  int ntv;
  const cplx *U, *A, *P, *Dc, *Ainv, *Dinv;
  int even_odd, coarse_even_odd;
  double coarse_tol;
  int coarse_restart, coarse_maxit, n_sweeps, n_mr;
  cplx *rc, *uc;
} mg_ctx;

static void fine_op(void* c, const cplx* in, cplx* out) {
  mg_ctx* m = (mg_ctx*)c;
#pragma omp parallel for schedule(static)
  for (int s = 0; s < m->g.V; ++s) apply_D_site(&m->g, m->U, m->A, in, out, s, -1);
}

/* V-cycle preconditioner of the outer FGMRES (Sec. 2), steps in the order
 * of the V-cycle of Algorithm 1: coarse-grid correction, then the smoother
 * from its result: z = SAP^nu(b = r, x0 = P GMRES_c(R r)) (post-smoothing
 * only) */
static void vcycle(void* c, const cplx* r, cplx* z) {
  mg_ctx* m = (mg_ctx*)c;
  coarse_ctx cc = {&m->g, m->ntv, m->Dc};
  size_t nc = (size_t)m->g.nagg * 2 * m->ntv;
  restrict_one(&m->g, m->ntv, m->P, r, m->rc);
  if (m->coarse_even_odd)
    coarse_solve_eo_one(&m->g, m->ntv, m->Dc, m->Dinv, m->rc, m->uc, m->coarse_tol, m->coarse_restart,
                        m->coarse_maxit);
  else
    gmres(coarse_op, &cc, NULL, NULL, nc, m->rc, m->uc, m->coarse_tol, m->coarse_restart, m->coarse_maxit, NULL);
  prolong_one(&m->g, m->ntv, m->P, m->uc, z);
  smooth(&m->g, m->sites, m->U, m->A, m->Ainv, r, z, m->n_sweeps, m->n_mr, m->even_odd);
}

int ora_fgmres(const int* dims, const int* agg, int ntv, const cplx* U, const cplx* A,
               const cplx* P, const cplx* Dc, const cplx* b, cplx* x, double tol, int restart,
               int maxit, double coarse_tol, int coarse_restart, int coarse_maxit, int n_sweeps,
               int n_mr, int even_odd, int coarse_even_odd, int* iters, double* relres) {
  mg_ctx m;
  if (geom_init(&m.g, dims, agg)) return -1;
  init_gammas();
  int* sites = aggregate_sites(&m.g);
  m.sites = sites;
  m.even_odd = even_odd;
  m.Ainv = even_odd ? clover_inverses(&m.g, A) : NULL;
  m.coarse_even_odd = coarse_even_odd;
  m.Dinv = coarse_even_odd ? odd_self_inverses(&m.g, ntv, Dc) : NULL;
  if ((even_odd && !m.Ainv) || (coarse_even_odd && !m.Dinv)) {
    free((void*)m.Ainv);
    free((void*)m.Dinv);
    free(sites);
    return -6;
  }
  m.ntv = ntv;
  m.U = U;
  m.A = A;
  m.P = P;
  m.Dc = Dc;
  m.coarse_tol = coarse_tol;
  m.coarse_restart = coarse_restart;
  m.coarse_maxit = coarse_maxit;
  m.n_sweeps = n_sweeps;
  m.n_mr = n_mr;
  size_t nc = (size_t)m.g.nagg * 2 * ntv;
  m.rc = (cplx*)malloc(sizeof(cplx) * nc);
  m.uc = (cplx*)malloc(sizeof(cplx) * nc);
  size_t n = (size_t)m.g.V * 12;
  int it = gmres(fine_op, &m, vcycle, &m, n, b, x, tol, restart, maxit, relres);
  if (iters) *iters = it;
  free(m.rc);
  free(m.uc);
  free((void*)m.Ainv);
  free((void*)m.Dinv);
  free(sites);
  return 0;
}

/* the smoother alone as a preconditioner-free solver check: x <- SAP(b, x) is
 * exported above; this returns the relative residual |b - D x| / |b|. */
double ora_relres(const int* dims, const cplx* U, const cplx* A, const cplx* b, const cplx* x) {
  geom_t g;
  const int one[4] = {1, 1, 1, 1};
  if (geom_init(&g, dims, one)) return -1;
  init_gammas();
  size_t n = (size_t)g.V * 12;
  cplx* r = (cplx*)malloc(sizeof(cplx) * n);
#pragma omp parallel for schedule(static)
  for (int s = 0; s < g.V; ++s) apply_D_site(&g, U, A, x, r, s, -1);
  double rr = 0, bb = 0;
  for (size_t i = 0; i < n; ++i) {
    cplx d = b[i] - r[i];
    rr += creal(d * conj(d));
    bb += creal(b[i] * conj(b[i]));
  }
  free(r);
  return sqrt(rr / bb);
}

/* ------------------------------------------------------------------ */
/* learned test-vector generator: gauge-covariant convolution network   */
/* ------------------------------------------------------------------ */
/* The paper has no learned part: this network is the project's learned
 * test-vector generator, replacing initial-phase smoother sweeps (Sec. 2).
 * Channels are colour triplets: a field of C channels is h[s][c][a],
 * a = colour. One layer maps C_in -> C_out channels:
 *   z(x)[c] = sum_{k=0..8} sum_c' W[k][c][c'] T_k(x) h(x + k)[c']
 * with k = 0 the site itself (T_0 = 1), k = 1+mu the +mu neighbour
 * (T = U_mu(x)), k = 5+mu the -mu neighbour (T = U_mu(x-mu)^dag) and the
 * fermion sign -1 on hops across the t boundary. W acts on the channel
 * index only, so the layer is gauge covariant. Between layers the
 * nonlinearity acts on every channel triplet:
 *   modrelu(z; b)[c] = z[c] * max(0, |z[c]| + b[c]) / |z[c]|  (0 if z[c] = 0),
 * which depends on |z[c]| only and is therefore gauge invariant.
 * The network is 3 layers, C0 -> C1 -> C2 -> C3, modrelu after layers 1 and 2
 * (skipped when linear != 0). Spinors enter as 4 channels (spin) x 3 colours.
 * Weights: W_l[9][C_{l+1}][C_l] complex for l = 0, 1, 2, then biases
 * b_1[C1], b_2[C2] (real), packed in that order in one array.
 * Gradients use G = dL/dRe(p) + i dL/dIm(p) for complex parameters p and
 * dL/db for the biases. */

/* x rounded to the nearest FP32 value and then to the nearest bfloat16
 * (8 significant bits; ties to the even bit pattern), real and imaginary
 * parts separately: the operand precision of a bf16 tensor-core product */
static double round_bf16(double x) {
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, sizeof u);
  u += 0x7fffu + ((u >> 16) & 1u);
  u &= 0xffff0000u;
  memcpy(&f, &u, sizeof f);
  return (double)f;
}

/* one layer; round_t != 0: every transported input triplet s_k T_k h(n_k)[c']
 * rounded to bfloat16 (part by part) before the channel mixing */
static void covconv_r(const geom_t* g, const cplx* U, int cin, int cout, const cplx* W, const cplx* h, cplx* z,
                      int round_t) {
#pragma omp parallel for schedule(static)
  for (int s = 0; s < g->V; ++s) {
    cplx* zs = z + (size_t)s * cout * 3;
    for (int i = 0; i < cout * 3; ++i) zs[i] = 0;
    for (int k = 0; k < 9; ++k) {
      int n = s, flip = 0;
      su3 T;
      if (k == 0) {
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) T.m[a][b] = (a == b);
      } else if (k <= 4) {
        n = neighbour(g, s, k - 1, +1, &flip);
        T = link_of(U, s, k - 1);
      } else {
        n = neighbour(g, s, k - 5, -1, &flip);
        T = dag(link_of(U, n, k - 5));
      }
      double sg = flip ? -1.0 : 1.0;
      const cplx* hn = h + (size_t)n * cin * 3;
      for (int cp = 0; cp < cin; ++cp) {
        cplx t[3];
        for (int a = 0; a < 3; ++a) {
          t[a] = 0;
          for (int b = 0; b < 3; ++b) t[a] += T.m[a][b] * hn[cp * 3 + b];
          t[a] *= sg;
          if (round_t) t[a] = round_bf16(creal(t[a])) + I * round_bf16(cimag(t[a]));
        }
        for (int c = 0; c < cout; ++c) {
          cplx w = W[((size_t)k * cout + c) * cin + cp];
          for (int a = 0; a < 3; ++a) zs[c * 3 + a] += w * t[a];
        }
      }
    }
  }
}

static void covconv(const geom_t* g, const cplx* U, int cin, int cout, const cplx* W, const cplx* h, cplx* z) {
  covconv_r(g, U, cin, cout, W, h, z, 0);
}

static void modrelu(int V, int C, const double* bias, const cplx* z, cplx* h) {
  for (int s = 0; s < V; ++s)
    for (int c = 0; c < C; ++c) {
      const cplx* zc = z + ((size_t)s * C + c) * 3;
      cplx* hc = h + ((size_t)s * C + c) * 3;
      double n = sqrt(norm2(zc, 3));
      double f = (n > 0 && n + bias[c] > 0) ? (n + bias[c]) / n : 0.0;
      for (int a = 0; a < 3; ++a) hc[a] = zc[a] * f;
    }
}

static size_t nn_wsize(int c0, int c1, int c2, int c3) {
  return (size_t)9 * ((size_t)c1 * c0 + (size_t)c2 * c1 + (size_t)c3 * c2);
}

static int nn_forward_impl(const int* dims, const cplx* U, int c0, int c1, int c2, int c3, const cplx* W,
                           const double* bias, int linear, int round_in, const cplx* in, cplx* out, int nrhs);

/* out = net(in) for nrhs right-hand sides; in [nrhs][V][c0*3], out [nrhs][V][c3*3] */
int ora_nn_forward(const int* dims, const cplx* U, int c0, int c1, int c2, int c3, const cplx* W,
                   const double* bias, int linear, const cplx* in, cplx* out, int nrhs) {
  return nn_forward_impl(dims, U, c0, c1, c2, c3, W, bias, linear, 0, in, out, nrhs);
}

/* the same with the operands of every layer's channel mixing in bfloat16:
 * each transported input triplet s_k T_k(x) h(n_k(x))[c'] (the transport in
 * full precision) rounded to bfloat16 before it is multiplied by the weights,
 * the arithmetic of an inference whose layer products take bf16 operands */
int ora_nn_forward_bf16act(const int* dims, const cplx* U, int c0, int c1, int c2, int c3, const cplx* W,
                           const double* bias, int linear, const cplx* in, cplx* out, int nrhs) {
  return nn_forward_impl(dims, U, c0, c1, c2, c3, W, bias, linear, 1, in, out, nrhs);
}

static int nn_forward_impl(const int* dims, const cplx* U, int c0, int c1, int c2, int c3, const cplx* W,
                           const double* bias, int linear, int round_in, const cplx* in, cplx* out, int nrhs) {
  geom_t g;
  const int one[4] = {1, 1, 1, 1};
  if (geom_init(&g, dims, one)) return -1;
  const cplx* W0 = W;
  const cplx* W1 = W0 + (size_t)9 * c1 * c0;
  const cplx* W2 = W1 + (size_t)9 * c2 * c1;
  const double* b1 = bias;
  const double* b2 = bias + c1;
  size_t V = g.V;
  cplx* z1 = (cplx*)malloc(sizeof(cplx) * V * c1 * 3);
  cplx* h1 = (cplx*)malloc(sizeof(cplx) * V * c1 * 3);
  cplx* z2 = (cplx*)malloc(sizeof(cplx) * V * c2 * 3);
  cplx* h2 = (cplx*)malloc(sizeof(cplx) * V * c2 * 3);
  for (int r = 0; r < nrhs; ++r) {
    covconv_r(&g, U, c0, c1, W0, in + (size_t)r * V * c0 * 3, z1, round_in);
    if (linear) memcpy(h1, z1, sizeof(cplx) * V * c1 * 3);
    else modrelu(g.V, c1, b1, z1, h1);
    covconv_r(&g, U, c1, c2, W1, h1, z2, round_in);
    if (linear) memcpy(h2, z2, sizeof(cplx) * V * c2 * 3);
    else modrelu(g.V, c2, b2, z2, h2);
    covconv_r(&g, U, c2, c3, W2, h2, out + (size_t)r * V * c3 * 3, round_in);
  }
  free(z1);
  free(h1);
  free(z2);
  free(h2);
  return 0;
}

/* dz = adjoint of covconv applied to dz_out (gradient with respect to h):
 * dh(y)[c'] = sum_k sum_c conj(W[k][c][c']) T_k(x)^dag dz(x)[c], x = y - k */
static void covconv_adjoint(const geom_t* g, const cplx* U, int cin, int cout, const cplx* W, const cplx* dz,
                            cplx* dh) {
  memset(dh, 0, sizeof(cplx) * (size_t)g->V * cin * 3);
  for (int s = 0; s < g->V; ++s) {
    const cplx* dzs = dz + (size_t)s * cout * 3;
    for (int k = 0; k < 9; ++k) {
      int n = s, flip = 0;
      su3 T;
      if (k == 0) {
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) T.m[a][b] = (a == b);
      } else if (k <= 4) {
        n = neighbour(g, s, k - 1, +1, &flip);
        T = link_of(U, s, k - 1);
      } else {
        n = neighbour(g, s, k - 5, -1, &flip);
        T = dag(link_of(U, n, k - 5));
      }
      double sg = flip ? -1.0 : 1.0;
      cplx* dhn = dh + (size_t)n * cin * 3;
      for (int cp = 0; cp < cin; ++cp) {
        cplx u[3] = {0, 0, 0};
        for (int c = 0; c < cout; ++c) {
          cplx w = conj(W[((size_t)k * cout + c) * cin + cp]);
          for (int a = 0; a < 3; ++a) u[a] += w * dzs[c * 3 + a];
        }
        for (int b = 0; b < 3; ++b) {
          cplx acc = 0;
          for (int a = 0; a < 3; ++a) acc += conj(T.m[a][b]) * u[a];
          dhn[cp * 3 + b] += sg * acc;
        }
      }
    }
  }
}

/* gW[k][c][c'] += sum_{x,a} dz(x)[c][a] conj((T_k h(x+k))[c'][a]) */
static void covconv_wgrad(const geom_t* g, const cplx* U, int cin, int cout, const cplx* dz, const cplx* h,
                          cplx* gW) {
  for (int s = 0; s < g->V; ++s) {
    const cplx* dzs = dz + (size_t)s * cout * 3;
    for (int k = 0; k < 9; ++k) {
      int n = s, flip = 0;
      su3 T;
      if (k == 0) {
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) T.m[a][b] = (a == b);
      } else if (k <= 4) {
        n = neighbour(g, s, k - 1, +1, &flip);
        T = link_of(U, s, k - 1);
      } else {
        n = neighbour(g, s, k - 5, -1, &flip);
        T = dag(link_of(U, n, k - 5));
      }
      double sg = flip ? -1.0 : 1.0;
      const cplx* hn = h + (size_t)n * cin * 3;
      for (int cp = 0; cp < cin; ++cp) {
        cplx t[3];
        for (int a = 0; a < 3; ++a) {
          t[a] = 0;
          for (int b = 0; b < 3; ++b) t[a] += T.m[a][b] * hn[cp * 3 + b];
          t[a] *= sg;
        }
        for (int c = 0; c < cout; ++c) {
          cplx acc = 0;
          for (int a = 0; a < 3; ++a) acc += dzs[c * 3 + a] * conj(t[a]);
          gW[((size_t)k * cout + c) * cin + cp] += acc;
        }
      }
    }
  }
}

/* backward of modrelu: given z, b and dh, returns dz and accumulates db */
static void modrelu_backward(int V, int C, const double* bias, const cplx* z, const cplx* dh, cplx* dz, double* db) {
  for (int s = 0; s < V; ++s)
    for (int c = 0; c < C; ++c) {
      const cplx* zc = z + ((size_t)s * C + c) * 3;
      const cplx* dhc = dh + ((size_t)s * C + c) * 3;
      cplx* dzc = dz + ((size_t)s * C + c) * 3;
      double n = sqrt(norm2(zc, 3));
      if (!(n > 0) || n + bias[c] <= 0) {
        for (int a = 0; a < 3; ++a) dzc[a] = 0;
        continue;
      }
      double zd = 0; /* real dot of z and dh */
      for (int a = 0; a < 3; ++a) zd += creal(zc[a]) * creal(dhc[a]) + cimag(zc[a]) * cimag(dhc[a]);
      double f = 1.0 + bias[c] / n;
      for (int a = 0; a < 3; ++a) dzc[a] = f * dhc[a] - bias[c] / (n * n * n) * zd * zc[a];
      db[c] += zd / n;
    }
}

/* Gradient of a real loss through the network: given dout = dL/dRe(out) +
 * i dL/dIm(out) [nrhs][V][c3*3], returns the weight gradients gW (same
 * packing as W), the bias gradients gb [c1 + c2] and (if din != NULL) the
 * gradient with respect to the input [nrhs][V][c0*3]. */
int ora_nn_backward(const int* dims, const cplx* U, int c0, int c1, int c2, int c3, const cplx* W,
                    const double* bias, int linear, const cplx* in, const cplx* dout, int nrhs, cplx* gW, double* gb,
                    cplx* din) {
  geom_t g;
  const int one[4] = {1, 1, 1, 1};
  if (geom_init(&g, dims, one)) return -1;
  const cplx* W0 = W;
  const cplx* W1 = W0 + (size_t)9 * c1 * c0;
  const cplx* W2 = W1 + (size_t)9 * c2 * c1;
  cplx* gW0 = gW;
  cplx* gW1 = gW0 + (size_t)9 * c1 * c0;
  cplx* gW2 = gW1 + (size_t)9 * c2 * c1;
  const double* b1 = bias;
  const double* b2 = bias + c1;
  memset(gW, 0, sizeof(cplx) * nn_wsize(c0, c1, c2, c3));
  memset(gb, 0, sizeof(double) * (size_t)(c1 + c2));
  size_t V = g.V;
  cplx* z1 = (cplx*)malloc(sizeof(cplx) * V * c1 * 3);
  cplx* h1 = (cplx*)malloc(sizeof(cplx) * V * c1 * 3);
  cplx* z2 = (cplx*)malloc(sizeof(cplx) * V * c2 * 3);
  cplx* h2 = (cplx*)malloc(sizeof(cplx) * V * c2 * 3);
  cplx* dh2 = (cplx*)malloc(sizeof(cplx) * V * c2 * 3);
  cplx* dz2 = (cplx*)malloc(sizeof(cplx) * V * c2 * 3);
  cplx* dh1 = (cplx*)malloc(sizeof(cplx) * V * c1 * 3);
  cplx* dz1 = (cplx*)malloc(sizeof(cplx) * V * c1 * 3);
  cplx* dh0 = (cplx*)malloc(sizeof(cplx) * V * c0 * 3);
  for (int r = 0; r < nrhs; ++r) {
    const cplx* h0 = in + (size_t)r * V * c0 * 3;
    const cplx* d3 = dout + (size_t)r * V * c3 * 3;
    covconv(&g, U, c0, c1, W0, h0, z1);
    if (linear) memcpy(h1, z1, sizeof(cplx) * V * c1 * 3);
    else modrelu(g.V, c1, b1, z1, h1);
    covconv(&g, U, c1, c2, W1, h1, z2);
    if (linear) memcpy(h2, z2, sizeof(cplx) * V * c2 * 3);
    else modrelu(g.V, c2, b2, z2, h2);
    /* layer 2 */
    covconv_wgrad(&g, U, c2, c3, d3, h2, gW2);
    covconv_adjoint(&g, U, c2, c3, W2, d3, dh2);
    if (linear) memcpy(dz2, dh2, sizeof(cplx) * V * c2 * 3);
    else modrelu_backward(g.V, c2, b2, z2, dh2, dz2, gb + c1);
    /* layer 1 */
    covconv_wgrad(&g, U, c1, c2, dz2, h1, gW1);
    covconv_adjoint(&g, U, c1, c2, W1, dz2, dh1);
    if (linear) memcpy(dz1, dh1, sizeof(cplx) * V * c1 * 3);
    else modrelu_backward(g.V, c1, b1, z1, dh1, dz1, gb);
    /* layer 0 */
    covconv_wgrad(&g, U, c0, c1, dz1, h0, gW0);
    if (din) {
      covconv_adjoint(&g, U, c0, c1, W0, dz1, dh0);
      memcpy(din + (size_t)r * V * c0 * 3, dh0, sizeof(cplx) * V * c0 * 3);
    }
  }
  free(z1);
  free(h1);
  free(z2);
  free(h2);
  free(dh2);
  free(dz2);
  free(dh1);
  free(dz1);
  free(dh0);
  return 0;
}

/* Training loss of the learned test vectors v (nrhs of them) and its
 * gradient dv = dL/dRe(v) + i dL/dIm(v):
 *   L = sum_r |D v_r|^2/|v_r|^2 + lambda |v_r - P P^dag v_r|^2/|v_r|^2
 * with P the prolongation of a plain setup (columns orthonormal per
 * aggregate and chirality, [ntv][V][12]). D^dag = gamma_5 D gamma_5. */
int ora_nn_loss(const int* dims, const int* agg, int ntv, const cplx* U, const cplx* A, const cplx* P,
                const cplx* v, int nrhs, double lambda, double* loss, cplx* dv) {
  geom_t g;
  if (geom_init(&g, dims, agg)) return -1;
  init_gammas();
  size_t n = (size_t)g.V * 12;
  size_t nc = (size_t)g.nagg * 2 * ntv;
  cplx* Dv = (cplx*)malloc(sizeof(cplx) * n);
  cplx* DDv = (cplx*)malloc(sizeof(cplx) * n);
  cplx* vc = (cplx*)malloc(sizeof(cplx) * nc);
  cplx* pv = (cplx*)malloc(sizeof(cplx) * n);
  double total = 0;
  for (int r = 0; r < nrhs; ++r) {
    const cplx* vr = v + r * n;
    cplx* dvr = dv ? dv + r * n : NULL;
    double vv = norm2(vr, n);
#pragma omp parallel for schedule(static)
    for (int s = 0; s < g.V; ++s) apply_D_site(&g, U, A, vr, Dv, s, -1);
    double dd = norm2(Dv, n);
    /* gamma_5 D gamma_5 (D v) */
    for (size_t i = 0; i < n; ++i) DDv[i] = (i % 12) < 6 ? Dv[i] : -Dv[i];
    cplx* tmp = pv;
#pragma omp parallel for schedule(static)
    for (int s = 0; s < g.V; ++s) apply_D_site(&g, U, A, DDv, tmp, s, -1);
    for (size_t i = 0; i < n; ++i) DDv[i] = (i % 12) < 6 ? tmp[i] : -tmp[i];
    /* q = v - P P^dag v */
    restrict_one(&g, ntv, P, vr, vc);
    prolong_one(&g, ntv, P, vc, pv);
    for (size_t i = 0; i < n; ++i) pv[i] = vr[i] - pv[i];
    double qq = norm2(pv, n);
    total += dd / vv + lambda * qq / vv;
    if (dvr)
      for (size_t i = 0; i < n; ++i)
        dvr[i] = 2.0 * (DDv[i] / vv - dd * vr[i] / (vv * vv)) + 2.0 * lambda * (pv[i] / vv - qq * vr[i] / (vv * vv));
  }
  *loss = total;
  free(Dv);
  free(DDv);
  free(vc);
  free(pv);
  return 0;
}
