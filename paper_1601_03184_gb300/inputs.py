"""Seeded synthetic inputs: SU(3) gauge fields, complex Gaussian test vectors
and random gauge transformations.

This module holds none of the method's arithmetic (no Dirac operator, no
smoother, no projection). Both the CUDA library's tests and the CPU oracle's
tests draw their inputs from here, so that both sides see identical data.

Layouts are the canonical host layouts of the library's C ABI:
  gauge field   U[s][mu][a][b], complex128, s = x + Lx*(y + Ly*(z + Lz*t))
  fields        psi[rhs][s][c], complex128, c = 3*spin + colour

Gauge links follow U = exp(i*eps*H), H = sum_a h_a lambda_a / 2 with
h_a ~ N(0, 1) (lambda_a the Gell-Mann matrices), so H is Hermitian and
traceless; the exponential is taken through the eigen-decomposition of H
and the result is projected back onto SU(3) (normalise row 0,
Gram-Schmidt row 1 against it, row 2 = conj(row0 x row1)). The normal
draws come from numpy's PCG64 stream seeded with `seed`, drawn as one array
of shape [V][4][8] in C order (Gell-Mann index fastest, then direction,
then site).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "volume",
    "gell_mann",
    "gauge_field",
    "unit_gauge_field",
    "random_su3",
    "test_vectors",
    "gaussian_field",
]


def volume(dims) -> int:
    v = 1
    for d in dims:
        v *= int(d)
    return v


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape [8, 3, 3]."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def _project_su3(m: np.ndarray) -> np.ndarray:
    r0 = m[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = m[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def _exp_i_eps_h(h: np.ndarray, eps: float) -> np.ndarray:
    """exp(i eps H) for H = sum_a h_a lambda_a / 2; h has shape [..., 8]."""
    H = np.einsum("...a,aij->...ij", h, gell_mann() / 2)
    w, Q = np.linalg.eigh(H)
    ph = np.exp(1j * eps * w)
    U = np.einsum("...ik,...k,...jk->...ij", Q, ph, np.conj(Q))
    return _project_su3(U)


def _exp_i_eps_h_torch(h: np.ndarray, eps: float, device) -> np.ndarray:
    """The same map as _exp_i_eps_h, evaluated with torch on `device` (used to
    generate large fields quickly; equal to the numpy path up to rounding)."""
    import torch

    lam = torch.as_tensor(gell_mann() / 2, device=device)
    ht = torch.as_tensor(h, device=device).to(torch.complex128)
    H = torch.einsum("...a,aij->...ij", ht, lam)
    U = torch.linalg.matrix_exp(1j * eps * H)
    r0 = U[..., 0, :]
    r0 = r0 / torch.linalg.vector_norm(r0, dim=-1, keepdim=True)
    r1 = U[..., 1, :]
    r1 = r1 - torch.sum(r0.conj() * r1, dim=-1, keepdim=True) * r0
    r1 = r1 / torch.linalg.vector_norm(r1, dim=-1, keepdim=True)
    r2 = torch.linalg.cross(r0, r1).conj()
    return torch.stack([r0, r1, r2], dim=-2).cpu().numpy()


def gauge_field(dims, eps: float, seed: int, chunk_sites: int = 1 << 18, device=None) -> np.ndarray:
    """Seeded SU(3) gauge field, complex128 [V, 4, 3, 3]. With device (e.g.
    "cuda") the exponential is evaluated there with torch; the random draws
    are the same."""
    V = volume(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    U = np.empty((V, 4, 3, 3), dtype=np.complex128)
    for s0 in range(0, V, chunk_sites):
        s1 = min(V, s0 + chunk_sites)
        h = rng.standard_normal((s1 - s0, 4, 8))
        U[s0:s1] = _exp_i_eps_h(h, eps) if device is None else _exp_i_eps_h_torch(h, eps, device)
    return U


def unit_gauge_field(dims) -> np.ndarray:
    V = volume(dims)
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[:, :, 0, 0] = U[:, :, 1, 1] = U[:, :, 2, 2] = 1
    return U


def random_su3(n: int, seed: int, eps: float = 2.0) -> np.ndarray:
    """n seeded SU(3) matrices (a gauge transformation Omega(x)), [n, 3, 3]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return _exp_i_eps_h(rng.standard_normal((n, 8)), eps)


def gaussian_field(shape, seed: int) -> np.ndarray:
    """Complex Gaussian array with Re, Im ~ N(0, 1), complex128."""
    rng = np.random.Generator(np.random.PCG64(seed))
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return re + 1j * im


def test_vectors(ntv: int, dims, seed: int) -> np.ndarray:
    """ntv complex Gaussian test vectors, complex128 [ntv, V, 12]."""
    return gaussian_field((ntv, volume(dims), 12), seed)
