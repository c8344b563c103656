"""Test-side helpers: dense matrices built column by column from the oracle,
gauge transformations and coarse-stencil densification. Used only by tests."""
import numpy as np

import oracle


def vol(dims):
    return int(np.prod(dims))


def coords(dims):
    V = vol(dims)
    s = np.arange(V)
    x = s % dims[0]
    y = (s // dims[0]) % dims[1]
    z = (s // (dims[0] * dims[1])) % dims[2]
    t = s // (dims[0] * dims[1] * dims[2])
    return np.stack([x, y, z, t], axis=1)


def shift_index(dims, mu, d):
    """index of x + d*mu_hat for every site x (periodic)"""
    c = coords(dims).copy()
    c[:, mu] = (c[:, mu] + d) % dims[mu]
    return c[:, 0] + dims[0] * (c[:, 1] + dims[1] * (c[:, 2] + dims[2] * c[:, 3]))


def dense_D(dims, U, A, block_agg=None):
    """Dense 12V x 12V matrix of D (or of D_B when block_agg is given)."""
    n = vol(dims) * 12
    E = np.eye(n, dtype=np.complex128).reshape(n, vol(dims), 12)
    if block_agg is None:
        cols = oracle.apply_D(dims, U, A, E)
    else:
        cols = oracle.apply_D_block(dims, block_agg, U, A, E)
    return cols.reshape(n, n).T


def gauge_transform(dims, U, Om):
    """U^Om_mu(x) = Om(x) U_mu(x) Om(x+mu)^dag"""
    Ut = np.empty_like(U)
    for mu in range(4):
        xp = shift_index(dims, mu, +1)
        Ut[:, mu] = Om @ U[:, mu] @ np.conj(np.transpose(Om[xp], (0, 2, 1)))
    return Ut


def colour_rotate(Om, psi):
    """(Om psi)(x) = Om(x) psi(x) on the colour index; psi [..., V, 12]"""
    p = psi.reshape(psi.shape[:-1] + (4, 3))
    out = np.einsum("sab,...sib->...sia", Om, p)
    return out.reshape(psi.shape)


def aggregate_of_sites(dims, agg):
    c = coords(dims)
    b = c // np.array(agg)
    nb = [d // a for d, a in zip(dims, agg)]
    return b[:, 0] + nb[0] * (b[:, 1] + nb[1] * (b[:, 2] + nb[2] * b[:, 3]))


def dense_P(dims, agg, P):
    """Dense prolongation 12V x (nagg*2ntv): column (A, h*ntv+j) = P_j on A x h."""
    ntv = P.shape[0]
    V = vol(dims)
    nagg = int(np.prod([d // a for d, a in zip(dims, agg)]))
    Ag = aggregate_of_sites(dims, agg)
    M = np.zeros((V * 12, nagg * 2 * ntv), np.complex128)
    for s in range(V):
        for c in range(12):
            h = c // 6
            for j in range(ntv):
                M[s * 12 + c, Ag[s] * 2 * ntv + h * ntv + j] = P[j, s, c]
    return M


def dense_coarse(dims, agg, Dc):
    """Sum the 9-point coarse stencil into a dense (nagg*2ntv)^2 matrix."""
    _, _, aggnbr = oracle.tables(dims, agg)
    nagg, _, nc, _ = Dc.shape
    M = np.zeros((nagg * nc, nagg * nc), np.complex128)
    for A in range(nagg):
        nb = [A] + list(aggnbr[A])
        for k in range(9):
            B = nb[k]
            M[A * nc:(A + 1) * nc, B * nc:(B + 1) * nc] += Dc[A, k]
    return M


def gamma5_fine(V):
    g = np.kron(np.diag([1, 1, -1, -1]), np.eye(3))
    return np.kron(np.eye(V), g)


# ----------------------------------------------------- sampled full-size checks
# The operator, the clover term and one SAP sweep from x0 = 0 are local: the
# result at one site (or on one colour-0 domain) depends only on the fields in
# a few lattice spacings around it. So the oracle can produce single outputs of
# a full-size lattice from a small cut-out of its fields.

def lex(c, ext):
    """canonical index of coordinates c (..., 4), x fastest"""
    c = np.asarray(c)
    return c[..., 0] + ext[0] * (c[..., 1] + ext[1] * (c[..., 2] + ext[2] * c[..., 3]))


def cutout(dims, corner, ext):
    """The ext^4 block of sites whose local coordinate 0 is the global site
    `corner` (any integers; periodic). Returns the global canonical index of
    every local site (local lexicographic order, x fastest) and whether its
    unwrapped t coordinate lies outside [0, L_t)."""
    loc = np.stack(np.unravel_index(np.arange(ext ** 4), (ext,) * 4)[::-1], axis=1)  # (n, 4): x fastest
    raw = loc + np.asarray(corner)[None, :]
    glob = raw % np.asarray(dims)[None, :]
    return lex(glob, dims), (raw[:, 3] < 0) | (raw[:, 3] >= dims[3])


def device_site(dims, agg, s):
    """the library's device site index of canonical sites s (aggregate-major:
    aggregate index times sites per aggregate, plus the offset inside it)"""
    s = np.asarray(s)
    c = np.stack(np.unravel_index(s, tuple(dims[::-1])), axis=-1)[..., ::-1]
    nb = [d // a for d, a in zip(dims, agg)]
    a = np.asarray(agg)
    return lex(c // a, nb) * int(np.prod(agg)) + lex(c % a, agg)


def stencil_at_site(dims, U, m0, csw, psi_at, site):
    """(D psi)(site) for all right-hand sides from the oracle on the 4^4
    cut-out whose local site (1,1,1,1) is `site`. U: the full gauge field
    [V, 4, 3, 3]; psi_at(global_sites) -> [nrhs, n, 12] gives psi there.
    Hops of the site across the global t boundary carry -1: the cut-out's
    psi is negated on the sites reached that way (only the centre's output
    is read)."""
    x = np.stack(np.unravel_index(site, tuple(dims[::-1])))[::-1]
    glob, wrapped = cutout(dims, x - 1, 4)
    Uc = U[glob]
    Ac = oracle.clover((4, 4, 4, 4), Uc, m0, csw)
    psi = psi_at(glob).astype(np.complex128)
    psi[:, wrapped] *= -1
    y = oracle.apply_D((4, 4, 4, 4), Uc, Ac, psi)
    return y[:, lex([1, 1, 1, 1], (4, 4, 4, 4))]


def sap_sweep_on_domain(dims, agg, U, m0, csw, b_at, block, n_mr):
    """x on the colour-0 domain `block` (block coordinates) after one SAP
    sweep from x0 = 0, from the oracle. From x0 = 0 the colour-0 phase solves
    D_B e = b_B on the domain alone and the colour-1 phase does not touch it,
    so the oracle's sweep on an 8^4 lattice whose domain 0 carries this
    domain's links, clover and right-hand side (b = 0 elsewhere, unit links,
    diagonal clover) gives the same values there. Returns [nrhs, |B|, 12] in
    the domain's local lexicographic order; b_at as in stencil_at_site."""
    a = agg[0]
    assert all(e == a for e in agg), "cubic domains"
    origin = np.asarray(block) * np.asarray(agg)
    # the clover of the domain's sites needs their neighbours: (a+2)^4 cut-out
    g6, _ = cutout(dims, origin - 1, a + 2)
    A6 = oracle.clover((a + 2,) * 4, U[g6], m0, csw)
    inner = np.stack(np.unravel_index(np.arange(a ** 4), (a,) * 4)[::-1], axis=1)
    A_dom = A6[lex(inner + 1, (a + 2,) * 4)]
    g_dom = lex((inner + origin[None, :]) % np.asarray(dims)[None, :], dims)
    d8 = (2 * a,) * 4
    V8 = int(np.prod(d8))
    s8 = lex(inner, d8)
    U8 = np.zeros((V8, 4, 3, 3), np.complex128)
    U8[:] = np.eye(3)
    U8[s8] = U[g_dom]
    A8 = np.zeros((V8, 12, 12), np.complex128)
    A8[:] = (4 + m0) * np.eye(12)
    A8[s8] = A_dom
    b_dom = b_at(g_dom).astype(np.complex128)
    b8 = np.zeros((b_dom.shape[0], V8, 12), np.complex128)
    b8[:, s8] = b_dom
    x8 = oracle.sap(d8, agg, U8, A8, b8, np.zeros_like(b8), 1, n_mr)
    return x8[:, s8], g_dom
