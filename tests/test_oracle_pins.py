"""Pins of the FP64 CPU oracle against mathematics that does not come from the
oracle itself: closed forms, invariants, symmetries, special cases that reduce
to library routines (dense eigenvalues, QR, linear solves, least squares) and
brute-force dense constructions on tiny lattices.

The paper (arXiv:1601.03184) prints no worked numerical example for any
operator (its Sec. 7 gives only speed-up ratios), so every pin here is
mathematical.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1601_03184_gb300 import inputs
from lattice_helpers import (aggregate_of_sites, colour_rotate, coords, dense_coarse, dense_D,
                             dense_P, gamma5_fine, gauge_transform, shift_index, vol)

C1 = dict(dims=(4, 4, 4, 4), agg=(2, 2, 2, 2), ntv=8, eps=0.3, m0=-0.2, csw=1.0, gseed=1001, tvseed=2001)


def c1_field():
    U = inputs.gauge_field(C1["dims"], C1["eps"], C1["gseed"])
    A = oracle.clover(C1["dims"], U, C1["m0"], C1["csw"])
    return U, A


# ---------------------------------------------------------------- inputs ----
def test_gauge_field_is_su3():
    U = inputs.gauge_field((4, 4, 4, 4), 0.6, 7)
    Ud = np.conj(np.swapaxes(U, -1, -2))
    assert np.abs(Ud @ U - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    # eps -> 0 gives the unit field
    U0 = inputs.gauge_field((2, 2, 2, 2), 1e-13, 7)
    assert np.abs(U0 - np.eye(3)).max() < 1e-12


def test_gell_mann_algebra():
    lam = inputs.gell_mann()
    for a in range(8):
        assert np.allclose(lam[a], lam[a].conj().T)
        assert abs(np.trace(lam[a])) < 1e-15
        for b in range(8):
            assert abs(np.trace(lam[a] @ lam[b]) - 2 * (a == b)) < 1e-14


# ---------------------------------------------------------------- gammas ----
def test_gamma_clifford_and_chiral_basis():
    G = oracle.gammas()
    for mu in range(4):
        assert np.allclose(G[mu], G[mu].conj().T)
        for nu in range(4):
            assert np.allclose(G[mu] @ G[nu] + G[nu] @ G[mu], 2 * np.eye(4) * (mu == nu), atol=1e-15)
    assert np.allclose(G[4], np.diag([1, 1, -1, -1]))
    for mu in range(4):
        for nu in range(4):
            sig = 0.5j * (G[mu] @ G[nu] - G[nu] @ G[mu])
            assert np.allclose(sig @ G[4], G[4] @ sig)  # chirality block diagonal


# ------------------------------------------------------------ index tables --
@pytest.mark.parametrize("dims,agg", [((4, 4, 4, 4), (2, 2, 2, 2)), ((4, 6, 4, 8), (2, 3, 2, 2)),
                                      ((2, 4, 6, 2), (1, 2, 3, 1))],
                         ids=["4^4", "ragged", "extent-2"])
def test_index_tables_by_enumeration(dims, agg):
    """The oracle's neighbour and aggregate tables against a plain enumeration
    of the lattice: site s = x + Lx (y + Ly (z + Lz t)); entry k < 4 is
    s + mu_hat and k >= 4 is s - mu_hat, periodic, with bit 30 set when the
    hop wraps around in t (the fermion boundary sign); aggregates and offsets
    in the same lexicographic order on block and intra-block coordinates;
    aggregate neighbours periodic on the block lattice. Extent 2 makes the
    forward and backward neighbour the same site, with different t flags."""
    def lex(c, ext):
        return c[0] + ext[0] * (c[1] + ext[1] * (c[2] + ext[2] * c[3]))

    nb = [d // a for d, a in zip(dims, agg)]
    V, na = vol(dims), int(np.prod(nb))
    nbr = np.zeros((V, 8), np.int64)
    aggof = np.zeros((V, 2), np.int64)
    for t, z, y, x in itertools.product(*[range(d) for d in dims[::-1]]):
        c = [x, y, z, t]
        s = lex(c, dims)
        for mu in range(4):
            for k, step in ((mu, 1), (4 + mu, -1)):
                n = list(c)
                n[mu] = (c[mu] + step) % dims[mu]
                wraps = mu == 3 and not 0 <= c[mu] + step < dims[mu]
                nbr[s, k] = lex(n, dims) | (int(wraps) << 30)
        aggof[s] = (lex([c[m] // agg[m] for m in range(4)], nb), lex([c[m] % agg[m] for m in range(4)], agg))
    aggnbr = np.zeros((na, 8), np.int64)
    for bt, bz, by, bx in itertools.product(*[range(n) for n in nb[::-1]]):
        b = [bx, by, bz, bt]
        for mu in range(4):
            for k, step in ((mu, 1), (4 + mu, -1)):
                n = list(b)
                n[mu] = (b[mu] + step) % nb[mu]
                aggnbr[lex(b, nb), k] = lex(n, nb)
    onbr, oaggof, oaggnbr = oracle.tables(dims, agg)
    assert np.array_equal(onbr, nbr)
    assert np.array_equal(oaggof, aggof)
    assert np.array_equal(oaggnbr, aggnbr)


# ---------------------------------------------------------------- clover ----
def test_clover_unit_field():
    dims = (4, 4, 4, 4)
    A = oracle.clover(dims, inputs.unit_gauge_field(dims), -0.3, 1.7)
    assert np.abs(A - 3.7 * np.eye(12)).max() < 1e-15


@pytest.mark.parametrize("plane", [(0, 1), (0, 3), (1, 2), (2, 3)])
def test_clover_constant_abelian_field(plane):
    """U_nu(x) = diag(e^{i phi x_mu}, e^{-i phi x_mu}, 1), other links 1, with
    phi L_mu = 2 pi: every plaquette of the mu-nu plane equals
    diag(e^{i phi}, e^{-i phi}, 1), so Fhat = i sin(phi) diag(1,-1,0) and
    A = (4+m0) + (csw/2) i sigma_{mu nu} (x) Fhat in closed form."""
    mu, nu = plane
    dims = (4, 4, 4, 4)
    V = vol(dims)
    U = inputs.unit_gauge_field(dims)
    phi = 2 * np.pi / dims[mu]
    xm = coords(dims)[:, mu]
    U[:, nu, 0, 0] = np.exp(1j * phi * xm)
    U[:, nu, 1, 1] = np.exp(-1j * phi * xm)
    m0, csw = -0.4, 1.3
    A = oracle.clover(dims, U, m0, csw)
    G = oracle.gammas()
    sig = 0.5j * (G[mu] @ G[nu] - G[nu] @ G[mu])
    F = 1j * np.sin(phi) * np.diag([1, -1, 0])
    ref = (4 + m0) * np.eye(12) + 0.5 * csw * 1j * np.kron(sig, F)
    assert np.abs(A - ref[None]).max() < 1e-14
    assert V == A.shape[0]


def test_clover_hermitian_chiral_and_covariant():
    dims = (4, 4, 4, 4)
    U = inputs.gauge_field(dims, 0.6, 11)
    A = oracle.clover(dims, U, -0.2, 1.5)
    assert np.abs(A - np.conj(np.swapaxes(A, 1, 2))).max() < 1e-14
    assert np.abs(A[:, :6, 6:]).max() < 1e-15 and np.abs(A[:, 6:, :6]).max() < 1e-15
    Om = inputs.random_su3(vol(dims), 12)
    At = oracle.clover(dims, gauge_transform(dims, U, Om), -0.2, 1.5)
    O12 = np.einsum("ij,sab->siajb", np.eye(4), Om).reshape(-1, 12, 12)
    ref = O12 @ A @ np.conj(np.swapaxes(O12, 1, 2))
    assert np.abs(At - ref).max() < 1e-13


@pytest.mark.parametrize("plane", [(0, 1), (1, 3), (2, 3)])
def test_clover_covariant_under_a_lattice_rotation(plane):
    """Rotate a random gauge field by 90 degrees in the plane (mu, nu):
    x -> R x with R e_mu = e_nu and R e_nu = -e_mu. The clover term of the
    rotated field at R x is S A(x) S^dag for one fixed spin rotation
    S = cos(pi/4) + sin(pi/4) gamma_mu gamma_nu (either sense), the same at
    every site. This holds only if all six planes and the four leaves of each
    clover are oriented consistently."""
    mu, nu = plane
    dims = (4, 4, 4, 4)
    U = inputs.gauge_field(dims, 0.6, 13)
    A = oracle.clover(dims, U, -0.2, 1.5)
    X = coords(dims)
    Xr = X.copy()
    Xr[:, nu] = X[:, mu]
    Xr[:, mu] = (-X[:, nu]) % dims[mu]
    lex = lambda c: c[:, 0] + dims[0] * (c[:, 1] + dims[1] * (c[:, 2] + dims[2] * c[:, 3]))
    r = lex(Xr)
    Ur = np.empty_like(U)
    for rho in range(4):
        if rho not in plane:
            Ur[r, rho] = U[:, rho]
    # the link x -> x + e_mu becomes R x -> R x + e_nu
    Ur[r, nu] = U[:, mu]
    # the link x -> x - e_nu becomes R x -> R x + e_mu
    Ur[r, mu] = np.conj(np.swapaxes(U[shift_index(dims, nu, -1), nu], -1, -2))
    Ar = oracle.clover(dims, Ur, -0.2, 1.5)
    G = oracle.gammas()
    errs = []
    for sense in (1, -1):
        S = np.kron(np.cos(np.pi / 4) * np.eye(4) + sense * np.sin(np.pi / 4) * G[mu] @ G[nu], np.eye(3))
        errs.append(np.abs(Ar[r] - S @ A @ S.conj().T).max())
    assert min(errs) < 1e-13
    assert max(errs) > 1e-3  # the other sense is wrong: the check has teeth


# ---------------------------------------------------------- Dirac operator --
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
def test_free_field_spectrum(dims):
    """Unit gauge field: eigenvalues m0 + sum(1-cos p) +/- i sqrt(sum sin^2 p),
    6-fold each, p_k = 2 pi n/L_k (x,y,z), p_t = (2n+1) pi/L_t."""
    from scipy.optimize import linear_sum_assignment

    m0 = -0.2
    U = inputs.unit_gauge_field(dims)
    A = oracle.clover(dims, U, m0, 1.0)
    ev = np.linalg.eigvals(dense_D(dims, U, A))
    moms = [2 * np.pi * np.arange(dims[k]) / dims[k] for k in range(3)]
    moms.append((2 * np.arange(dims[3]) + 1) * np.pi / dims[3])
    ref = []
    for p in itertools.product(*moms):
        p = np.array(p)
        a = m0 + np.sum(1 - np.cos(p))
        b = np.sqrt(np.sum(np.sin(p) ** 2))
        ref += [a + 1j * b] * 6 + [a - 1j * b] * 6
    ref = np.array(ref)
    cost = np.abs(ev[:, None] - ref[None, :])
    r, c = linear_sum_assignment(cost)
    assert cost[r, c].max() < 1e-11


def test_plane_wave_fixes_sign_convention():
    """D e^{ipx} u = e^{ipx} (m0 + sum(1-cos p) + i sum gamma_mu sin p_mu) u"""
    dims = (4, 4, 4, 4)
    m0 = -0.2
    U = inputs.unit_gauge_field(dims)
    A = oracle.clover(dims, U, m0, 1.0)
    G = oracle.gammas()
    x = coords(dims)
    rng = np.random.default_rng(3)
    for n in [(1, 0, 0, 0), (0, 2, 1, 0), (3, 1, 2, 1)]:
        p = np.array([2 * np.pi * n[k] / dims[k] for k in range(3)] + [(2 * n[3] + 1) * np.pi / dims[3]])
        u = rng.standard_normal(12) + 1j * rng.standard_normal(12)
        ph = np.exp(1j * x @ p)
        Dp = (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(G[m] * np.sin(p[m]) for m in range(4))
        ref = ph[:, None] * (np.kron(Dp, np.eye(3)) @ u)[None, :]
        y = oracle.apply_D(dims, U, A, ph[:, None] * u[None, :])
        assert np.abs(y - ref).max() < 1e-13


def test_gamma5_hermiticity():
    U, A = c1_field()
    dims = C1["dims"]
    rng = np.random.default_rng(5)
    x = rng.standard_normal((vol(dims), 12)) + 1j * rng.standard_normal((vol(dims), 12))
    y = rng.standard_normal((vol(dims), 12)) + 1j * rng.standard_normal((vol(dims), 12))
    g5 = np.array([1] * 6 + [-1] * 6)
    lhs = np.vdot(x, g5 * oracle.apply_D(dims, U, A, g5 * y))
    rhs = np.vdot(oracle.apply_D(dims, U, A, x), y)
    assert abs(lhs - rhs) < 1e-13 * abs(rhs) * 100


def test_gauge_covariance_of_D():
    U, _ = c1_field()
    dims = C1["dims"]
    A = oracle.clover(dims, U, -0.2, 1.0)
    Om = inputs.random_su3(vol(dims), 21)
    Ut = gauge_transform(dims, U, Om)
    At = oracle.clover(dims, Ut, -0.2, 1.0)
    psi = inputs.gaussian_field((vol(dims), 12), 22)
    lhs = oracle.apply_D(dims, Ut, At, colour_rotate(Om, psi))
    rhs = colour_rotate(Om, oracle.apply_D(dims, U, A, psi))
    assert np.abs(lhs - rhs).max() < 1e-13


def test_block_D_is_D_with_cut_links():
    """D_B equals the full D on a field whose links crossing aggregate
    boundaries are set to zero (clover kept from the original field)."""
    U, A = c1_field()
    dims, agg = C1["dims"], C1["agg"]
    Ag = aggregate_of_sites(dims, agg)
    Ucut = U.copy()
    c = coords(dims)
    for mu in range(4):
        cp = c.copy()
        cp[:, mu] = (cp[:, mu] + 1) % dims[mu]
        xp = cp[:, 0] + dims[0] * (cp[:, 1] + dims[1] * (cp[:, 2] + dims[2] * cp[:, 3]))
        Ucut[Ag != Ag[xp], mu] = 0
    psi = inputs.gaussian_field((vol(dims), 12), 31)
    y1 = oracle.apply_D_block(dims, agg, U, A, psi)
    y2 = oracle.apply_D(dims, Ucut, A, psi)
    assert np.abs(y1 - y2).max() < 1e-14


# -------------------------------------------------------------------- SAP ----
def test_sap_many_mr_steps_is_block_gauss_seidel():
    """With many MR steps the block solves are exact, so one sweep is the
    multiplicative Schwarz step: x0 <- x0 + D_00^-1 (b - D x)_0, then colour 1."""
    U, A = c1_field()
    dims, agg = C1["dims"], C1["agg"]
    V = vol(dims)
    D = dense_D(dims, U, A)
    Ag = aggregate_of_sites(dims, agg)
    nb = [d // a for d, a in zip(dims, agg)]
    bc = np.stack(np.unravel_index(Ag, nb[::-1]), axis=1)[:, ::-1]
    colour = bc.sum(axis=1) % 2
    b = inputs.gaussian_field((V, 12), 41)
    x0 = inputs.gaussian_field((V, 12), 42) * 0.1
    x = x0.reshape(-1).copy()
    bb = b.reshape(-1)
    for col in (0, 1):
        r = bb - D @ x
        for Bk in np.unique(Ag[colour == col]):
            idx = np.concatenate([np.arange(s * 12, s * 12 + 12) for s in np.where(Ag == Bk)[0]])
            x[idx] += np.linalg.solve(D[np.ix_(idx, idx)], r[idx])
    xo = oracle.sap(dims, agg, U, A, b[None], x0[None], 1, 400)[0]
    assert np.abs(xo.reshape(-1) - x).max() / np.abs(x).max() < 1e-11


def _colours_and_parity(dims, agg):
    Ag = aggregate_of_sites(dims, agg)
    nb = [d // a for d, a in zip(dims, agg)]
    colour = np.stack(np.unravel_index(Ag, nb[::-1]), axis=1)[:, ::-1].sum(axis=1) % 2
    c = np.stack(np.unravel_index(np.arange(vol(dims)), tuple(dims[::-1])), axis=1)[:, ::-1]
    return Ag, colour, c.sum(axis=1) % 2


def test_sap_even_odd_many_mr_steps_is_block_gauss_seidel():
    """The even-odd form of the domain solve (MR on the Schur complement of
    the even sites, then the odd sites) solves D_B e = r exactly in the limit
    of many steps: one sweep is then the same multiplicative Schwarz step as
    for the plain form."""
    U, A = c1_field()
    dims, agg = C1["dims"], C1["agg"]
    V = vol(dims)
    D = dense_D(dims, U, A)
    Ag, colour, _ = _colours_and_parity(dims, agg)
    b = inputs.gaussian_field((V, 12), 43)
    x0 = inputs.gaussian_field((V, 12), 44) * 0.1
    x = x0.reshape(-1).copy()
    bb = b.reshape(-1)
    for col in (0, 1):
        r = bb - D @ x
        for Bk in np.unique(Ag[colour == col]):
            idx = np.concatenate([np.arange(s * 12, s * 12 + 12) for s in np.where(Ag == Bk)[0]])
            x[idx] += np.linalg.solve(D[np.ix_(idx, idx)], r[idx])
    xo = oracle.sap_eo(dims, agg, U, A, b[None], x0[None], 1, 200)[0]
    assert np.abs(xo.reshape(-1) - x).max() / np.abs(x).max() < 1e-11


def test_sap_even_odd_one_mr_step_is_the_schur_complement_step():
    """One sweep of one MR step from x0 = 0, written with dense matrices: on
    every domain D_B = [[A_EE, H_EO], [H_OE, A_OO]] (sites of even and odd
    parity), S = A_EE - H_EO A_OO^-1 H_OE, rhat = r_E - H_EO A_OO^-1 r_O,
    e_E = alpha rhat with alpha = <S rhat, rhat> / <S rhat, S rhat>, and
    e_O = A_OO^-1 (r_O - H_OE e_E). A dropped or misplaced A_OO^-1, a sign of
    the hopping part or the plain MR step in its place fails this."""
    U, A = c1_field()
    dims, agg = C1["dims"], C1["agg"]
    V = vol(dims)
    D = dense_D(dims, U, A)
    Ag, colour, par = _colours_and_parity(dims, agg)
    b = inputs.gaussian_field((V, 12), 45)
    x = np.zeros(V * 12, complex)
    bb = b.reshape(-1)
    rows = lambda sites: np.concatenate([np.arange(s * 12, s * 12 + 12) for s in sites])
    for col in (0, 1):
        r = bb - D @ x
        for Bk in np.unique(Ag[colour == col]):
            sB = np.where(Ag == Bk)[0]
            E, O = rows(sB[par[sB] == 0]), rows(sB[par[sB] == 1])
            Aoo_inv = np.linalg.inv(D[np.ix_(O, O)])
            S = D[np.ix_(E, E)] - D[np.ix_(E, O)] @ Aoo_inv @ D[np.ix_(O, E)]
            rhat = r[E] - D[np.ix_(E, O)] @ (Aoo_inv @ r[O])
            q = S @ rhat
            eE = (np.vdot(q, rhat) / np.vdot(q, q)) * rhat
            eO = Aoo_inv @ (r[O] - D[np.ix_(O, E)] @ eE)
            x[E] += eE
            x[O] += eO
    xo = oracle.sap_eo(dims, agg, U, A, b[None], np.zeros_like(b)[None], 1, 1)[0]
    assert np.abs(xo.reshape(-1) - x).max() / np.abs(x).max() < 1e-12
    # and it is not the plain one-step MR sweep
    xp = oracle.sap(dims, agg, U, A, b[None], np.zeros_like(b)[None], 1, 1)[0]
    assert np.abs(xp - xo).max() / np.abs(xo).max() > 1e-2


def test_sap_reduces_residual_and_is_gauge_covariant():
    U, A = c1_field()
    dims, agg = C1["dims"], C1["agg"]
    V = vol(dims)
    b = inputs.gaussian_field((1, V, 12), 43)
    res = [1.0]
    for ns in (1, 2, 4):
        x = oracle.sap(dims, agg, U, A, b, np.zeros_like(b), ns, 4)
        res.append(oracle.relres(dims, U, A, b[0], x[0]))
    assert all(res[i + 1] < res[i] for i in range(len(res) - 1))
    Om = inputs.random_su3(V, 44)
    Ut = gauge_transform(dims, U, Om)
    At = oracle.clover(dims, Ut, C1["m0"], C1["csw"])
    xt = oracle.sap(dims, agg, Ut, At, colour_rotate(Om, b), np.zeros_like(b), 2, 3)
    x = oracle.sap(dims, agg, U, A, b, np.zeros_like(b), 2, 3)
    assert np.abs(xt - colour_rotate(Om, x)).max() < 1e-12


# ------------------------------------------------------------ Gram-Schmidt --
def test_gram_schmidt_is_unique_thin_qr():
    dims, agg, ntv = C1["dims"], C1["agg"], C1["ntv"]
    tv = inputs.test_vectors(ntv, dims, 51)
    P = oracle.gram_schmidt(dims, agg, tv)
    Ag = aggregate_of_sites(dims, agg)
    for Ak in range(16):
        sites = np.where(Ag == Ak)[0]
        for h in range(2):
            Vm = tv[:, sites, 6 * h:6 * h + 6].reshape(ntv, -1).T
            Pm = P[:, sites, 6 * h:6 * h + 6].reshape(ntv, -1).T
            assert np.abs(Pm.conj().T @ Pm - np.eye(ntv)).max() < 1e-14
            Q, R = np.linalg.qr(Vm)  # Householder (LAPACK)
            ph = np.diag(R) / np.abs(np.diag(R))
            assert np.abs(Pm - Q * ph[None, :]).max() < 1e-13
    # columns outside the chirality are untouched: P restricted to (A, h) only
    assert P.shape == tv.shape


# ----------------------------------------------------------- coarse operator --
@pytest.mark.parametrize("case", ["c1", "tiny"])
def test_coarse_operator_brute_force(case):
    """Summed 9-point stencil == dense P^dag D P (P the dense prolongation)."""
    if case == "c1":
        dims, agg, ntv = C1["dims"], C1["agg"], C1["ntv"]
        U, A = c1_field()
    else:
        dims, agg, ntv = (2, 2, 2, 2), (1, 1, 1, 1), 4
        U = inputs.gauge_field(dims, 0.5, 61)
        A = oracle.clover(dims, U, 0.1, 1.2)
    tv = inputs.test_vectors(ntv, dims, 62)
    P = oracle.gram_schmidt(dims, agg, tv)
    Dc = oracle.coarse_op(dims, agg, U, A, P)
    Pd = dense_P(dims, agg, P)
    ref = Pd.conj().T @ dense_D(dims, U, A) @ Pd
    got = dense_coarse(dims, agg, Dc)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    # coarse gamma_5 hermiticity: Gamma5 Dc Gamma5 = Dc^dag
    nagg = Dc.shape[0]
    g5c = np.kron(np.eye(nagg), np.diag([1.0] * ntv + [-1.0] * ntv))
    assert np.abs(g5c @ got @ g5c - got.conj().T).max() < 1e-12 * np.abs(got).max()
    # R P = 1 on the coarse space, apply_Dc = R D P
    uc = inputs.gaussian_field((2, nagg, 2 * ntv), 63)
    u = oracle.prolong(dims, agg, P, uc)
    assert np.abs(oracle.restrict(dims, agg, P, u) - uc).max() < 1e-13
    yc = oracle.apply_Dc(dims, agg, Dc, uc)
    ref_yc = oracle.restrict(dims, agg, P, oracle.apply_D(dims, U, A, u))
    assert np.abs(yc - ref_yc).max() < 1e-12 * np.abs(ref_yc).max()


# ------------------------------------------------------------------ GMRES ----
def test_coarse_gmres_iterate_is_krylov_minimiser():
    dims, agg, ntv = C1["dims"], C1["agg"], C1["ntv"]
    U, A = c1_field()
    P = oracle.gram_schmidt(dims, agg, inputs.test_vectors(ntv, dims, 71))
    Dc = oracle.coarse_op(dims, agg, U, A, P)
    M = dense_coarse(dims, agg, Dc)
    bc = inputs.gaussian_field((1, Dc.shape[0], 2 * ntv), 72)
    b = bc.reshape(-1)
    for k in (1, 3, 6):
        xc, its = oracle.coarse_solve(dims, agg, Dc, bc, 0.0, 20, k)
        assert its[0] == k
        K = np.stack([np.linalg.matrix_power(M, i) @ b for i in range(k)], axis=1)
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(M @ Q, b, rcond=None)
        ref = Q @ y
        assert np.abs(xc.reshape(-1) - ref).max() < 1e-10 * np.abs(ref).max()
    # to tolerance: the true residual meets it
    xc, its = oracle.coarse_solve(dims, agg, Dc, bc, 1e-9, 10, 1000)
    assert np.linalg.norm(b - M @ xc.reshape(-1)) <= 1.01e-9 * np.linalg.norm(b)


def test_setup_and_fgmres_c1():
    """The C1 setup (3 SAP sweeps x 4 MR, 1 refinement) gives an orthonormal
    P and a D_c equal to P^dag D P; two-level FGMRES then solves D x = b to
    1e-10 and agrees with the dense solve."""
    dims, agg, ntv = C1["dims"], C1["agg"], C1["ntv"]
    U, A = c1_field()
    tv0 = inputs.test_vectors(ntv, dims, C1["tvseed"])
    prm = oracle.make_params(n_init_sweeps=3, n_init_mr=4, n_refine=1)
    tv, P, Dc = oracle.setup_init(dims, agg, U, A, tv0, prm)
    tv, P, Dc, its = oracle.setup_refine(dims, agg, U, A, tv, P, Dc, prm)
    assert (its >= 1).all()
    Pd = dense_P(dims, agg, P)
    assert np.abs(Pd.conj().T @ Pd - np.eye(Pd.shape[1])).max() < 1e-13
    D = dense_D(dims, U, A)
    assert np.abs(dense_coarse(dims, agg, Dc) - Pd.conj().T @ D @ Pd).max() < 1e-12 * 10
    b = inputs.gaussian_field((vol(dims), 12), 3001)
    x, it, rr = oracle.fgmres(dims, agg, U, A, P, Dc, b, tol=1e-10)
    assert rr <= 1e-10 and it < 100
    xd = np.linalg.solve(D, b.reshape(-1))
    assert np.abs(x.reshape(-1) - xd).max() < 1e-8 * np.abs(xd).max()


def _dense_sap_exact(D, Ag, colour, b, x, n_sweeps):
    """Red-black multiplicative Schwarz with exact domain solves: the SAP
    sweep of Sec. 2 in the limit of many MR steps."""
    x = x.copy()
    for _ in range(n_sweeps):
        for col in (0, 1):
            r = b - D @ x
            for Bk in np.unique(Ag[colour == col]):
                idx = np.concatenate([np.arange(s * 12, s * 12 + 12) for s in np.where(Ag == Bk)[0]])
                x[idx] += np.linalg.solve(D[np.ix_(idx, idx)], r[idx])
    return x


def test_setup_phases_with_exact_domain_and_coarse_solves():
    """Initial phase: v_j <- SAP^n(b = v_j, x0 = 0), normalised. Refinement
    (Alg. 1 order, P and D_c fixed while the vectors are visited):
    v_j <- SAP^nu(b = v_j, x0 = P D_c^-1 R v_j), normalised, then P and D_c
    rebuilt. With 400 MR steps per domain and a coarse tolerance of 1e-13 the
    oracle must reproduce these phases written with dense block solves, a
    dense coarse solve and the dense P^dag D P."""
    dims, agg, ntv = C1["dims"], C1["agg"], 4
    U, A = c1_field()
    D = dense_D(dims, U, A)
    Ag = aggregate_of_sites(dims, agg)
    nb = [d // a for d, a in zip(dims, agg)]
    bc = np.stack(np.unravel_index(Ag, nb[::-1]), axis=1)[:, ::-1]
    colour = bc.sum(axis=1) % 2
    tv0 = inputs.test_vectors(ntv, dims, 95)
    prm = oracle.make_params(n_init_sweeps=2, n_init_mr=400, n_refine=1, n_smooth_sweeps=2, n_smooth_mr=400,
                             coarse_tol=1e-13, coarse_restart=40, coarse_maxit=4000)
    tv, P, Dc = oracle.setup_init(dims, agg, U, A, tv0, prm)
    ref = []
    for j in range(ntv):
        v = _dense_sap_exact(D, Ag, colour, tv0[j].reshape(-1), np.zeros(D.shape[0], complex), 2)
        ref.append(v / np.linalg.norm(v))
    ref = np.array(ref).reshape(tv.shape)
    assert np.abs(tv - ref).max() < 1e-10

    tv1, P1, Dc1, _ = oracle.setup_refine(dims, agg, U, A, tv, P, Dc, prm)
    Pd = dense_P(dims, agg, P)
    Dcd = Pd.conj().T @ D @ Pd
    ref = []
    for j in range(ntv):
        v = tv[j].reshape(-1)
        x0 = Pd @ np.linalg.solve(Dcd, Pd.conj().T @ v)
        x = _dense_sap_exact(D, Ag, colour, v, x0, 2)
        ref.append(x / np.linalg.norm(x))
    ref = np.array(ref).reshape(tv.shape)
    assert np.abs(tv1 - ref).max() < 1e-9
    Pd1 = dense_P(dims, agg, P1)
    assert np.abs(Pd1.conj().T @ Pd1 - np.eye(Pd1.shape[1])).max() < 1e-13
    assert np.abs(dense_coarse(dims, agg, Dc1) - Pd1.conj().T @ D @ Pd1).max() < 1e-11


def test_fgmres_first_step_is_the_preconditioned_minimal_residual_step():
    """Right-preconditioned FGMRES from x0 = 0: after one iteration
    x = alpha z with z = M b the V-cycle of Sec. 2 (coarse correction
    x0 = P D_c^-1 R b, then nu SAP sweeps on D x = b) and alpha minimising
    |b - alpha D z|. With exact domain and coarse solves, M is written here
    with dense linear algebra; a smoother-first or coarse-only V-cycle fails."""
    dims, agg, ntv = C1["dims"], C1["agg"], 4
    U, A = c1_field()
    D = dense_D(dims, U, A)
    Ag = aggregate_of_sites(dims, agg)
    nb = [d // a for d, a in zip(dims, agg)]
    colour = np.stack(np.unravel_index(Ag, nb[::-1]), axis=1)[:, ::-1].sum(axis=1) % 2
    tv, P, Dc = oracle.setup_init(dims, agg, U, A, inputs.test_vectors(ntv, dims, 96), oracle.make_params())
    b = inputs.gaussian_field((vol(dims), 12), 97)
    x, it, rr = oracle.fgmres(dims, agg, U, A, P, Dc, b, tol=1e-30, restart=25, maxit=1, coarse_tol=1e-13,
                              coarse_restart=40, coarse_maxit=4000, n_sweeps=2, n_mr=400)
    assert it == 1
    Pd = dense_P(dims, agg, P)
    bb = b.reshape(-1)
    x0 = Pd @ np.linalg.solve(Pd.conj().T @ D @ Pd, Pd.conj().T @ bb)
    z = _dense_sap_exact(D, Ag, colour, bb, x0, 2)
    Dz = D @ z
    ref = (np.vdot(Dz, bb) / np.vdot(Dz, Dz)) * z
    assert np.abs(x.reshape(-1) - ref).max() < 1e-9 * np.abs(ref).max()
    assert abs(rr - np.linalg.norm(bb - D @ ref) / np.linalg.norm(bb)) < 1e-9


def _coarse_c1():
    dims, agg, ntv = C1["dims"], C1["agg"], 4
    U, A = c1_field()
    _, P, Dc = oracle.setup_init(dims, agg, U, A, inputs.test_vectors(ntv, dims, 98), oracle.make_params())
    Dd = dense_coarse(dims, agg, Dc)
    nb = [d // a for d, a in zip(dims, agg)]
    nagg = int(np.prod(nb))
    colour = np.stack(np.unravel_index(np.arange(nagg), nb[::-1]), axis=1)[:, ::-1].sum(axis=1) % 2
    row_colour = np.repeat(colour, 2 * ntv)
    return dims, agg, ntv, Dc, Dd, row_colour


def test_coarse_even_odd_solve_converges_to_the_dense_solve():
    """The coarse solve on the Schur complement of the even aggregates, then
    the odd ones, reaches D_c^-1 b (the hop blocks join aggregates of
    different colour, so the even-odd split is exact)."""
    dims, agg, ntv, Dc, Dd, _ = _coarse_c1()
    bc = inputs.gaussian_field((2, Dd.shape[0] // (2 * ntv), 2 * ntv), 99)
    xc, its = oracle.coarse_solve_eo(dims, agg, Dc, bc, 1e-13, 40, 4000)
    for r in range(2):
        xd = np.linalg.solve(Dd, bc[r].reshape(-1))
        assert np.abs(xc[r].reshape(-1) - xd).max() < 1e-10 * np.abs(xd).max()
    assert (its > 0).all()


def test_coarse_even_odd_one_iteration_is_the_schur_minimal_residual_step():
    """One GMRES iteration from zero on S = D_ee - D_eo D_oo^-1 D_oe with the
    right side bhat = b_e - D_eo D_oo^-1 b_o gives x_e = alpha bhat, alpha
    minimising |bhat - alpha S bhat|; then x_o = D_oo^-1 (b_o - D_oe x_e).
    Written with the dense D_c split by aggregate colour."""
    dims, agg, ntv, Dc, Dd, rc = _coarse_c1()
    E, O = np.where(rc == 0)[0], np.where(rc == 1)[0]
    assert np.abs(Dd[np.ix_(E, E)] - np.diag(np.diag(Dd[np.ix_(E, E)]))).max() > 0  # self blocks are dense
    bc = inputs.gaussian_field((1, Dd.shape[0] // (2 * ntv), 2 * ntv), 100)
    b = bc[0].reshape(-1)
    Doo_inv = np.linalg.inv(Dd[np.ix_(O, O)])
    S = Dd[np.ix_(E, E)] - Dd[np.ix_(E, O)] @ Doo_inv @ Dd[np.ix_(O, E)]
    bh = b[E] - Dd[np.ix_(E, O)] @ (Doo_inv @ b[O])
    q = S @ bh
    xE = (np.vdot(q, bh) / np.vdot(q, q)) * bh
    xO = Doo_inv @ (b[O] - Dd[np.ix_(O, E)] @ xE)
    xc, its = oracle.coarse_solve_eo(dims, agg, Dc, bc, 0.0, 10, 1)
    x = xc[0].reshape(-1)
    assert its[0] == 1
    assert np.abs(x[E] - xE).max() < 1e-12 * np.abs(xE).max()
    assert np.abs(x[O] - xO).max() < 1e-12 * np.abs(xO).max()


def test_setup_gauge_invariance():
    """U -> U^Om and tv -> Om tv leave D_c unchanged and map P -> Om P."""
    dims, agg, ntv = C1["dims"], C1["agg"], 4
    U, A = c1_field()
    tv0 = inputs.test_vectors(ntv, dims, 81)
    Om = inputs.random_su3(vol(dims), 82)
    Ut = gauge_transform(dims, U, Om)
    At = oracle.clover(dims, Ut, C1["m0"], C1["csw"])
    prm = oracle.make_params(n_init_sweeps=2, n_init_mr=3, n_refine=1, n_smooth_sweeps=2, n_smooth_mr=3,
                             coarse_tol=0.0, coarse_maxit=6)
    tv, P, Dc = oracle.setup_init(dims, agg, U, A, tv0, prm)
    tv, P, Dc, _ = oracle.setup_refine(dims, agg, U, A, tv, P, Dc, prm)
    tvt, Pt, Dct = oracle.setup_init(dims, agg, Ut, At, colour_rotate(Om, tv0), prm)
    tvt, Pt, Dct, _ = oracle.setup_refine(dims, agg, Ut, At, tvt, Pt, Dct, prm)
    assert np.abs(Dct - Dc).max() < 1e-11 * np.abs(Dc).max()
    assert np.abs(Pt - colour_rotate(Om, P)).max() < 1e-11


def test_init_modes_agree_for_one_sweep():
    dims, agg, ntv = C1["dims"], C1["agg"], 3
    U, A = c1_field()
    tv0 = inputs.test_vectors(ntv, dims, 91)
    a = oracle.setup_init(dims, agg, U, A, tv0, oracle.make_params(init_mode=0, n_init_sweeps=1))
    b = oracle.setup_init(dims, agg, U, A, tv0, oracle.make_params(init_mode=1, n_init_sweeps=1))
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_init_mode_1_is_repeated_single_sweep_calls():
    """The second reading of the initial phase (Sec. 2, 'a few iterations with
    starting guess 0'): n_sweeps calls of ONE sweep, each v <- SAP(b = v,
    x0 = 0), the result of a call becoming the right-hand side of the next,
    normalised once at the end. With 400 MR steps per domain the oracle at
    three sweeps must equal that composition written with dense block solves;
    it must also differ from the one-call reading (init_mode 0), which a
    carried-over starting guess or a reused right-hand side would reproduce."""
    dims, agg, ntv = C1["dims"], C1["agg"], 3
    U, A = c1_field()
    D = dense_D(dims, U, A)
    Ag = aggregate_of_sites(dims, agg)
    nb = [d // a for d, a in zip(dims, agg)]
    colour = np.stack(np.unravel_index(Ag, nb[::-1]), axis=1)[:, ::-1].sum(axis=1) % 2
    tv0 = inputs.test_vectors(ntv, dims, 93)
    prm1 = oracle.make_params(init_mode=1, n_init_sweeps=3, n_init_mr=400)
    prm0 = oracle.make_params(init_mode=0, n_init_sweeps=3, n_init_mr=400)
    tv1, _, _ = oracle.setup_init(dims, agg, U, A, tv0, prm1)
    tv0m, _, _ = oracle.setup_init(dims, agg, U, A, tv0, prm0)
    ref, ref0 = [], []
    zero = np.zeros(D.shape[0], complex)
    for j in range(ntv):
        v = tv0[j].reshape(-1)
        for _ in range(3):
            v = _dense_sap_exact(D, Ag, colour, v, zero, 1)
        ref.append(v / np.linalg.norm(v))
        w = _dense_sap_exact(D, Ag, colour, tv0[j].reshape(-1), zero, 3)
        ref0.append(w / np.linalg.norm(w))
    ref = np.array(ref).reshape(tv1.shape)
    ref0 = np.array(ref0).reshape(tv1.shape)
    assert np.abs(tv1 - ref).max() < 1e-10
    assert np.abs(tv0m - ref0).max() < 1e-10
    assert np.abs(ref - ref0).max() > 1e-2  # the two readings are different maps


def test_gamma5_fine_helper_consistent():
    g = gamma5_fine(2)
    assert g.shape == (24, 24) and np.allclose(np.diag(g)[:12], [1] * 6 + [-1] * 6)


def test_mr_block_solve_minimises_the_block_residual():
    """Right-hand side on one colour-0 domain B and x0 = 0: after one sweep,
    x on B is the MR iterate for D_B e = b_B, since the colour-1 phase does not
    touch B. Each MR step minimises the residual along D_B rho. So the block
    residual never grows with n_mr. After one step the residual is orthogonal
    to D_B b_B (a conjugated alpha breaks this) and x_B is parallel to b_B.
    Many steps reach the dense block solve."""
    U, A = c1_field()
    dims, agg = C1["dims"], C1["agg"]
    V = vol(dims)
    sites = np.where(aggregate_of_sites(dims, agg) == 0)[0]
    idx = (sites[:, None] * 12 + np.arange(12)[None, :]).reshape(-1)
    DB = dense_D(dims, U, A)[np.ix_(idx, idx)]
    b = np.zeros((1, V, 12), complex)
    b[0, sites] = inputs.gaussian_field((len(sites), 12), 45)
    bB = b.reshape(-1)[idx]
    res = []
    for n_mr in (1, 2, 3, 4, 8, 16):
        xB = oracle.sap(dims, agg, U, A, b, np.zeros_like(b), 1, n_mr)[0].reshape(-1)[idx]
        rB = bB - DB @ xB
        res.append(np.linalg.norm(rB))
        if n_mr == 1:
            q = DB @ bB
            assert abs(np.vdot(q, rB)) < 1e-13 * np.linalg.norm(q) * np.linalg.norm(bB)
            alpha = np.vdot(bB, xB) / np.vdot(bB, bB)
            assert np.abs(xB - alpha * bB).max() < 1e-14 * np.abs(xB).max()
    assert res[0] < np.linalg.norm(bB)
    assert all(res[i + 1] <= res[i] * (1 + 1e-13) for i in range(len(res) - 1))
    xB = oracle.sap(dims, agg, U, A, b, np.zeros_like(b), 1, 400)[0].reshape(-1)[idx]
    ref = np.linalg.solve(DB, bB)
    assert np.abs(xB - ref).max() / np.abs(ref).max() < 1e-11


def test_m0_tuning_on_the_free_field():
    """The m0 tuning (tests/golden/tune_m0.py: ARPACK on the oracle's D) on the
    unit gauge field against the closed-form free spectrum
    lambda(p) = sum_mu (1 - cos p_mu) +/- i sqrt(sum_mu sin^2 p_mu) at m0 = 0,
    with the antiperiodic p_t. The tuned m0 puts the leftmost real part at
    1e-3 of the largest |lambda + m0|."""
    import importlib.util
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tune_m0.py")
    spec = importlib.util.spec_from_file_location("tune_m0", path)
    tune_m0 = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(tune_m0)
    dims = (4, 4, 4, 4)
    r = tune_m0.tune(dims, 0.0, 1.0, 7)
    moms = [2 * np.pi * np.arange(dims[k]) / dims[k] for k in range(3)]
    moms.append((2 * np.arange(dims[3]) + 1) * np.pi / dims[3])
    lam = []
    for p in itertools.product(*moms):
        p = np.array(p)
        a, b = np.sum(1 - np.cos(p)), np.sqrt(np.sum(np.sin(p) ** 2))
        lam += [a + 1j * b, a - 1j * b]
    lam = np.array(lam)
    m0 = -lam.real.min()
    for _ in range(50):
        m0 = -lam.real.min() + tune_m0.RATIO * np.abs(lam + m0).max()
    assert abs(r["m0"] - m0) < 1e-10
    assert abs(r["lambda_max_at_m0"] - np.abs(lam + m0).max()) < 1e-8
