"""ctypes binding of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline may use it; the product path (the CUDA library) never does.

All arrays are numpy complex128 in the canonical host layout described at the
top of oracle.c. Functions return new arrays; inputs are not modified unless
stated.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
SRC = os.path.join(HERE, "oracle.c")

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (plain C11 + OpenMP)."""
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC):
        tmp = LIB_PATH + ".tmp.%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
        )
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(LIB_PATH)
        _lib.ora_relres.restype = ctypes.c_double
    return _lib


class SetupParams(ctypes.Structure):
    _fields_ = [
        ("init_mode", ctypes.c_int),
        ("n_init_sweeps", ctypes.c_int),
        ("n_init_mr", ctypes.c_int),
        ("n_refine", ctypes.c_int),
        ("n_smooth_sweeps", ctypes.c_int),
        ("n_smooth_mr", ctypes.c_int),
        ("coarse_tol", ctypes.c_double),
        ("coarse_restart", ctypes.c_int),
        ("coarse_maxit", ctypes.c_int),
        ("even_odd", ctypes.c_int),
        ("coarse_even_odd", ctypes.c_int),
    ]


def _i4(v):
    return (ctypes.c_int * 4)(*[int(x) for x in v])


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _vol(dims):
    return int(np.prod(dims))


def _nagg(dims, agg):
    return int(np.prod([d // a for d, a in zip(dims, agg)]))


def _check(st, what):
    if st != 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, st))


def tables(dims, agg):
    V, na = _vol(dims), _nagg(dims, agg)
    nbr = np.zeros((V, 8), np.int32)
    aggof = np.zeros((V, 2), np.int32)
    aggnbr = np.zeros((na, 8), np.int32)
    _check(lib().ora_tables(_i4(dims), _i4(agg), _p(nbr), _p(aggof), _p(aggnbr)), "tables")
    return nbr, aggof, aggnbr


def gammas():
    out = np.zeros((5, 4, 4), np.complex128)
    lib().ora_gammas(_p(out))
    return out


def clover(dims, U, m0, csw):
    U = _c(U)
    A = np.zeros((_vol(dims), 12, 12), np.complex128)
    _check(lib().ora_clover(_i4(dims), _p(U), ctypes.c_double(m0), ctypes.c_double(csw), _p(A)), "clover")
    return A


def apply_D(dims, U, A, psi):
    """y = D psi; psi is [V, 12] or [nrhs, V, 12] (one oracle call per vector)."""
    U, A, psi = _c(U), _c(A), _c(psi)
    y = np.zeros_like(psi)
    flat_in = psi.reshape(-1, _vol(dims), 12)
    flat_out = y.reshape(-1, _vol(dims), 12)
    for r in range(flat_in.shape[0]):
        _check(lib().ora_apply_D(_i4(dims), _p(U), _p(A), _p(flat_in[r]), _p(flat_out[r])), "apply_D")
    return y


def apply_D_block(dims, agg, U, A, psi):
    """y = D_B psi (D with the couplings between aggregates removed)."""
    U, A, psi = _c(U), _c(A), _c(psi)
    y = np.zeros_like(psi)
    flat_in = psi.reshape(-1, _vol(dims), 12)
    flat_out = y.reshape(-1, _vol(dims), 12)
    for r in range(flat_in.shape[0]):
        _check(lib().ora_apply_D_block(_i4(dims), _i4(agg), _p(U), _p(A), _p(flat_in[r]), _p(flat_out[r])),
               "apply_D_block")
    return y


def sap(dims, agg, U, A, b, x0, n_sweeps, n_mr):
    """x = SAP^n_sweeps(b, x0) for every right-hand side; b, x0: [nrhs, V, 12]."""
    U, A, b = _c(U), _c(A), _c(b)
    x = _c(x0).copy()
    nrhs = b.shape[0]
    _check(lib().ora_sap(_i4(dims), _i4(agg), _p(U), _p(A), _p(b), _p(x), nrhs, n_sweeps, n_mr), "sap")
    return x


def sap_eo(dims, agg, U, A, b, x0, n_sweeps, n_mr):
    """x <- SAP^n_sweeps(b, x0) with even-odd preconditioned domain solves."""
    U, A, b = _c(U), _c(A), _c(b)
    x = _c(x0).copy()
    nrhs = b.shape[0] if b.ndim == 3 else 1
    _check(lib().ora_sap_eo(_i4(dims), _i4(agg), _p(U), _p(A), _p(b), _p(x), nrhs, n_sweeps, n_mr), "sap_eo")
    return x


def gram_schmidt(dims, agg, tv):
    tv = _c(tv)
    P = np.zeros_like(tv)
    _check(lib().ora_gram_schmidt(_i4(dims), _i4(agg), tv.shape[0], _p(tv), _p(P)), "gram_schmidt")
    return P


def coarse_op(dims, agg, U, A, P):
    U, A, P = _c(U), _c(A), _c(P)
    ntv = P.shape[0]
    Dc = np.zeros((_nagg(dims, agg), 9, 2 * ntv, 2 * ntv), np.complex128)
    _check(lib().ora_coarse_op(_i4(dims), _i4(agg), ntv, _p(U), _p(A), _p(P), _p(Dc)), "coarse_op")
    return Dc


def restrict(dims, agg, P, v):
    P, v = _c(P), _c(v)
    ntv, nrhs = P.shape[0], v.shape[0]
    vc = np.zeros((nrhs, _nagg(dims, agg), 2 * ntv), np.complex128)
    _check(lib().ora_restrict(_i4(dims), _i4(agg), ntv, _p(P), _p(v), _p(vc), nrhs), "restrict")
    return vc


def prolong(dims, agg, P, uc):
    P, uc = _c(P), _c(uc)
    nrhs = uc.shape[0]
    u = np.zeros((nrhs, _vol(dims), 12), np.complex128)
    _check(lib().ora_prolong(_i4(dims), _i4(agg), P.shape[0], _p(P), _p(uc), _p(u), nrhs), "prolong")
    return u


def apply_Dc(dims, agg, Dc, xc):
    Dc, xc = _c(Dc), _c(xc)
    ntv = Dc.shape[-1] // 2
    yc = np.zeros_like(xc)
    _check(lib().ora_apply_Dc(_i4(dims), _i4(agg), ntv, _p(Dc), _p(xc), _p(yc), xc.shape[0]), "apply_Dc")
    return yc


def coarse_solve(dims, agg, Dc, bc, tol, restart, maxit):
    Dc, bc = _c(Dc), _c(bc)
    ntv = Dc.shape[-1] // 2
    xc = np.zeros_like(bc)
    its = np.zeros(bc.shape[0], np.int32)
    _check(
        lib().ora_coarse_solve(_i4(dims), _i4(agg), ntv, _p(Dc), _p(bc), _p(xc), bc.shape[0],
                               ctypes.c_double(tol), restart, maxit, _p(its)),
        "coarse_solve",
    )
    return xc, its


def coarse_solve_eo(dims, agg, Dc, bc, tol, restart, maxit):
    """Coarse solve on the Schur complement of the even aggregates. Returns (xc, iterations)."""
    Dc, bc = _c(Dc), _c(bc)
    nrhs = bc.shape[0]
    xc = np.zeros_like(bc)
    its = np.zeros(nrhs, np.int32)
    _check(lib().ora_coarse_solve_eo(_i4(dims), _i4(agg), Dc.shape[2] // 2, _p(Dc), _p(bc), _p(xc), nrhs,
                                     ctypes.c_double(tol), restart, maxit, _p(its)), "coarse_solve_eo")
    return xc, its


def make_params(init_mode=0, n_init_sweeps=3, n_init_mr=4, n_refine=1, n_smooth_sweeps=4,
                n_smooth_mr=4, coarse_tol=0.05, coarse_restart=20, coarse_maxit=200, even_odd=0,
                coarse_even_odd=0):
    return SetupParams(init_mode, n_init_sweeps, n_init_mr, n_refine, n_smooth_sweeps, n_smooth_mr,
                       float(coarse_tol), coarse_restart, coarse_maxit, int(even_odd), int(coarse_even_odd))


def setup_init(dims, agg, U, A, tv0, params):
    """Initial phase. Returns (tv, P, Dc)."""
    U, A = _c(U), _c(A)
    tv = _c(tv0).copy()
    ntv = tv.shape[0]
    P = np.zeros_like(tv)
    Dc = np.zeros((_nagg(dims, agg), 9, 2 * ntv, 2 * ntv), np.complex128)
    _check(lib().ora_setup_init(_i4(dims), _i4(agg), ntv, _p(U), _p(A), _p(tv), ctypes.byref(params),
                                _p(P), _p(Dc)), "setup_init")
    return tv, P, Dc


def setup_refine(dims, agg, U, A, tv, P, Dc, params):
    """Refinement phase (Algorithm 1 order). Returns (tv, P, Dc, coarse_iters)."""
    U, A = _c(U), _c(A)
    tv, P, Dc = _c(tv).copy(), _c(P).copy(), _c(Dc).copy()
    ntv = tv.shape[0]
    its = np.zeros((max(params.n_refine, 1), ntv), np.int32)
    _check(lib().ora_setup_refine(_i4(dims), _i4(agg), ntv, _p(U), _p(A), _p(tv), ctypes.byref(params),
                                  _p(P), _p(Dc), _p(its)), "setup_refine")
    return tv, P, Dc, its


def fgmres(dims, agg, U, A, P, Dc, b, tol=1e-10, restart=25, maxit=500, coarse_tol=0.05,
           coarse_restart=20, coarse_maxit=200, n_sweeps=4, n_mr=4, even_odd=0, coarse_even_odd=0):
    """Two-level FGMRES on D x = b. Returns (x, iterations, relative residual estimate)."""
    U, A, P, Dc, b = _c(U), _c(A), _c(P), _c(Dc), _c(b)
    x = np.zeros_like(b)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0)
    _check(
        lib().ora_fgmres(_i4(dims), _i4(agg), P.shape[0], _p(U), _p(A), _p(P), _p(Dc), _p(b), _p(x),
                         ctypes.c_double(tol), restart, maxit, ctypes.c_double(coarse_tol), coarse_restart,
                         coarse_maxit, n_sweeps, n_mr, int(even_odd), int(coarse_even_odd), ctypes.byref(it),
                         ctypes.byref(rr)),
        "fgmres",
    )
    return x, it.value, rr.value


def relres(dims, U, A, b, x):
    return lib().ora_relres(_i4(dims), _p(_c(U)), _p(_c(A)), _p(_c(b)), _p(_c(x)))


# ------------------------------------------------------ learned generator --
def nn_sizes(widths):
    c0, c1, c2, c3 = widths
    return 9 * (c1 * c0 + c2 * c1 + c3 * c2), c1 + c2


def nn_forward(dims, U, widths, W, bias, x, linear=False):
    """x: [nrhs, V, c0*3] complex -> [nrhs, V, c3*3]."""
    c0, c1, c2, c3 = widths
    U, W, x = _c(U), _c(W), _c(x)
    bias = np.ascontiguousarray(bias, dtype=np.float64)
    nrhs = x.shape[0]
    out = np.zeros((nrhs, _vol(dims), c3 * 3), np.complex128)
    _check(lib().ora_nn_forward(_i4(dims), _p(U), c0, c1, c2, c3, _p(W), _p(bias), int(linear), _p(x), _p(out),
                                nrhs), "nn_forward")
    return out


def nn_forward_bf16act(dims, U, widths, W, bias, x, linear=False):
    """nn_forward with the operands of every layer's channel mixing in
    bfloat16: each transported input triplet rounded (via FP32, ties to even)
    before it meets the weights."""
    c0, c1, c2, c3 = widths
    U, W, x = _c(U), _c(W), _c(x)
    bias = np.ascontiguousarray(bias, dtype=np.float64)
    nrhs = x.shape[0]
    out = np.zeros((nrhs, _vol(dims), c3 * 3), np.complex128)
    _check(lib().ora_nn_forward_bf16act(_i4(dims), _p(U), c0, c1, c2, c3, _p(W), _p(bias), int(linear), _p(x),
                                        _p(out), nrhs), "nn_forward_bf16act")
    return out


def nn_backward(dims, U, widths, W, bias, x, dout, linear=False, want_din=False):
    """Returns (gW, gb, din) with g = dL/dRe + i dL/dIm for complex parameters."""
    c0, c1, c2, c3 = widths
    U, W, x, dout = _c(U), _c(W), _c(x), _c(dout)
    bias = np.ascontiguousarray(bias, dtype=np.float64)
    nw, nb = nn_sizes(widths)
    gW = np.zeros(nw, np.complex128)
    gb = np.zeros(nb, np.float64)
    din = np.zeros_like(x) if want_din else None
    _check(lib().ora_nn_backward(_i4(dims), _p(U), c0, c1, c2, c3, _p(W), _p(bias), int(linear), _p(x), _p(dout),
                                 x.shape[0], _p(gW), _p(gb), _p(din) if want_din else None), "nn_backward")
    return gW, gb, din


def nn_loss(dims, agg, U, A, P, v, lam):
    """(loss, dv) of sum_r |D v_r|^2/|v_r|^2 + lam |(1 - P P^dag) v_r|^2/|v_r|^2."""
    U, A, P, v = _c(U), _c(A), _c(P), _c(v)
    dv = np.zeros_like(v)
    loss = ctypes.c_double(0)
    _check(lib().ora_nn_loss(_i4(dims), _i4(agg), P.shape[0], _p(U), _p(A), _p(P), _p(v), v.shape[0],
                             ctypes.c_double(lam), ctypes.byref(loss), _p(dv)), "nn_loss")
    return loss.value, dv
