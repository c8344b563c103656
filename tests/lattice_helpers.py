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
