"""Parity of the CUDA library (through its C ABI) with the FP64 CPU oracle.

FP64 paths: relative error <= 1e-12 in the 2-norm of every output (the
oracle and the kernels evaluate the same sums in different orders; rounding
differences stay at a few ulps times the operator norm, far below 1e-12).
FP32 stencil: <= 1e-5 relative (each output is a sum of ~130 products of
FP32-rounded inputs, unit roundoff 6e-8, giving a worst-case bound of about
1e-5 and a typical error of about 1e-7).
Index tables: bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_1601_03184_gb300 import (MRHS_ERR_NONFINITE, MRHS_ERR_SHAPE, MRHS_ERR_STATE, MRHS_F32, MRHS_F64,
                                    MRHS_PREC_FP32, MRHS_PREC_FP64, Lattice, MrhsError, inputs)

pytestmark = pytest.mark.gpu

C1 = dict(dims=(4, 4, 4, 4), agg=(2, 2, 2, 2), ntv=8, eps=0.3, m0=-0.2, csw=1.0, gseed=1001, tvseed=2001)
# a lattice whose extents and aggregates differ per direction (ragged), still
# with an even number of aggregates per direction
RAGGED = dict(dims=(4, 6, 4, 8), agg=(2, 3, 2, 2), ntv=5, eps=0.5, m0=0.1, csw=1.3, gseed=1101, tvseed=2101)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def make(cfg, prec=MRHS_PREC_FP64):
    U = inputs.gauge_field(cfg["dims"], cfg["eps"], cfg["gseed"])
    A = oracle.clover(cfg["dims"], U, cfg["m0"], cfg["csw"])
    lat = Lattice(cfg["dims"], cfg["agg"], cfg["ntv"], prec)
    lat.set_gauge(U)
    lat.build_clover(cfg["m0"], cfg["csw"])
    return lat, U, A


@pytest.fixture(scope="module")
def c1():
    return make(C1)


@pytest.fixture(scope="module")
def ragged():
    return make(RAGGED)


# ------------------------------------------------------------------ tables --
@pytest.mark.parametrize("cfg", [C1, RAGGED], ids=["c1", "ragged"])
def test_tables_bit_exact(cfg):
    lat = Lattice(cfg["dims"], cfg["agg"], cfg["ntv"], MRHS_PREC_FP64)
    nbr, aggof, aggnbr = lat.tables()
    onbr, oaggof, oaggnbr = oracle.tables(cfg["dims"], cfg["agg"])
    assert np.array_equal(nbr, onbr)
    assert np.array_equal(aggof, oaggof)
    assert np.array_equal(aggnbr, oaggnbr)


def test_clover_matches_oracle(c1, ragged):
    for lat, U, A in (c1, ragged):
        got = lat.clover()
        assert np.abs(got[:, 0] - A[:, :6, :6]).max() < 1e-13
        assert np.abs(got[:, 1] - A[:, 6:, 6:]).max() < 1e-13


# ---------------------------------------------------------------- stencil --
@pytest.mark.parametrize("nrhs", [1, 3, 8])
def test_apply_D_fp64(c1, nrhs):
    lat, U, A = c1
    x = inputs.gaussian_field((nrhs, lat.V, 12), 500 + nrhs)
    xd = lat.to_device(x, MRHS_F64)
    yd = lat.field(nrhs, MRHS_F64)
    lat.apply_D(xd, yd, nrhs, MRHS_F64)
    y = lat.to_host(yd, nrhs, MRHS_F64)
    assert rel(y, oracle.apply_D(lat.dims, U, A, x)) < 1e-13


def test_apply_D_ragged_fp64_and_fp32(ragged):
    lat, U, A = ragged
    nrhs = 7
    x = inputs.gaussian_field((nrhs, lat.V, 12), 601)
    ref = oracle.apply_D(lat.dims, U, A, x)
    for dt, tol in ((MRHS_F64, 1e-13), (MRHS_F32, 1e-5)):
        xd = lat.to_device(x, dt)
        yd = lat.field(nrhs, dt)
        lat.apply_D(xd, yd, nrhs, dt)
        assert rel(lat.to_host(yd, nrhs, dt), ref) < tol


@pytest.mark.parametrize("nrhs", [6, 8, 12])
def test_apply_D_fp32_multi_rhs_per_thread(ragged, nrhs):
    """FP32 stencil with 2 or 4 right-hand sides per thread (nrhs even)."""
    lat, U, A = ragged
    x = inputs.gaussian_field((nrhs, lat.V, 12), 620 + nrhs)
    xd = lat.to_device(x, MRHS_F32)
    yd = lat.field(nrhs, MRHS_F32)
    lat.apply_D(xd, yd, nrhs, MRHS_F32)
    assert rel(lat.to_host(yd, nrhs, MRHS_F32), oracle.apply_D(lat.dims, U, A, x)) < 1e-5


def test_apply_D_block_fp64(c1, ragged):
    for lat, U, A in (c1, ragged):
        x = inputs.gaussian_field((4, lat.V, 12), 611)
        xd = lat.to_device(x, MRHS_F64)
        yd = lat.field(4, MRHS_F64)
        lat.apply_D_block(xd, yd, 4, MRHS_F64)
        assert rel(lat.to_host(yd, 4, MRHS_F64), oracle.apply_D_block(lat.dims, lat.agg, U, A, x)) < 1e-13


# -------------------------------------------------------------------- SAP --
@pytest.mark.parametrize("cfg_name", ["c1", "ragged"])
def test_sap_fp64(c1, ragged, cfg_name):
    lat, U, A = c1 if cfg_name == "c1" else ragged
    nrhs = lat.ntv
    b = inputs.gaussian_field((nrhs, lat.V, 12), 701)
    x0 = 0.1 * inputs.gaussian_field((nrhs, lat.V, 12), 702)
    bd = lat.to_device(b, MRHS_F64)
    xd = lat.to_device(x0, MRHS_F64)
    lat.sap(bd, xd, nrhs, MRHS_F64, 3, 4)
    ref = oracle.sap(lat.dims, lat.agg, U, A, b, x0, 3, 4)
    assert rel(lat.to_host(xd, nrhs, MRHS_F64), ref) < 1e-12


def test_sap_fp32(c1):
    lat32 = make(C1, MRHS_PREC_FP32)[0]
    _, U, A = c1
    nrhs = 8
    b = inputs.gaussian_field((nrhs, lat32.V, 12), 711)
    bd = lat32.to_device(b, MRHS_F32)
    xd = lat32.field(nrhs, MRHS_F32)
    lat32.sap(bd, xd, nrhs, MRHS_F32, 3, 4)
    ref = oracle.sap(C1["dims"], C1["agg"], U, A, b, np.zeros_like(b), 3, 4)
    assert rel(lat32.to_host(xd, nrhs, MRHS_F32), ref) < 1e-5


# the paper's 4^4 domains (256 sites: two items per thread in the on-chip
# SAP kernel) and a ragged 2x3x2x2 domain (24 sites, partial warpgroup), with
# one and several chunks of four right-hand sides and a nonzero start vector
P4 = dict(dims=(8, 8, 8, 8), agg=(4, 4, 4, 4), ntv=8, eps=0.4, m0=-0.1, csw=1.2, gseed=1301, tvseed=2301)


@pytest.mark.parametrize("cfg,nrhs", [(P4, 4), (P4, 12), (RAGGED, 8)], ids=["4^4-n4", "4^4-n12", "ragged-n8"])
def test_sap_fp32_domains(cfg, nrhs):
    lat, U, A = make(cfg, MRHS_PREC_FP32)
    b = inputs.gaussian_field((nrhs, lat.V, 12), 721)
    x0 = 0.1 * inputs.gaussian_field((nrhs, lat.V, 12), 722)
    bd = lat.to_device(b, MRHS_F32)
    xd = lat.to_device(x0, MRHS_F32)
    lat.sap(bd, xd, nrhs, MRHS_F32, 2, 4)
    ref = oracle.sap(cfg["dims"], cfg["agg"], U, A, b, x0, 2, 4)
    assert rel(lat.to_host(xd, nrhs, MRHS_F32), ref) < 1e-5


# ------------------------------------------------------------ GS, Dc, R/P --
@pytest.mark.parametrize("cfg_name", ["c1", "ragged"])
def test_gram_schmidt_and_coarse_op_fp64(c1, ragged, cfg_name):
    lat, U, A = c1 if cfg_name == "c1" else ragged
    tv = inputs.test_vectors(lat.ntv, lat.dims, 801)
    lat.set_tv(lat.to_device(tv, MRHS_F64), MRHS_F64)
    lat.build_P()
    P = lat.get_P()
    Pref = oracle.gram_schmidt(lat.dims, lat.agg, tv)
    assert rel(P, Pref) < 1e-12
    lat.build_Dc()
    Dref = oracle.coarse_op(lat.dims, lat.agg, U, A, Pref)
    assert rel(lat.get_Dc(), Dref) < 1e-12
    # restriction / prolongation / coarse stencil on the same P
    nrhs = 3
    v = inputs.gaussian_field((nrhs, lat.V, 12), 802)
    vd = lat.to_device(v, MRHS_F64)
    vc = lat.field(nrhs, MRHS_F64, coarse=True)
    lat.restrict(vd, vc, nrhs, MRHS_F64)
    assert rel(lat.to_host(vc, nrhs, MRHS_F64, coarse=True), oracle.restrict(lat.dims, lat.agg, Pref, v)) < 1e-12
    uc = inputs.gaussian_field((nrhs, lat.nagg, 2 * lat.ntv), 803)
    ucd = lat.to_device(uc, MRHS_F64, coarse=True)
    ud = lat.field(nrhs, MRHS_F64)
    lat.prolong(ucd, ud, nrhs, MRHS_F64)
    assert rel(lat.to_host(ud, nrhs, MRHS_F64), oracle.prolong(lat.dims, lat.agg, Pref, uc)) < 1e-12
    yc = lat.field(nrhs, MRHS_F64, coarse=True)
    lat.apply_Dc(ucd, yc, nrhs, MRHS_F64)
    assert rel(lat.to_host(yc, nrhs, MRHS_F64, coarse=True), oracle.apply_Dc(lat.dims, lat.agg, Dref, uc)) < 1e-12


def test_gram_schmidt_dependent_vectors_flagged(c1):
    lat, _, _ = c1
    tv = inputs.test_vectors(lat.ntv, lat.dims, 811)
    tv[3] = tv[1] * (2 - 1j)  # v_3 is a multiple of v_1 on every aggregate
    lat.set_tv(lat.to_device(tv, MRHS_F64), MRHS_F64)
    with pytest.raises(MrhsError) as e:
        lat.build_P()
    assert e.value.status == MRHS_ERR_NONFINITE


# ------------------------------------------------------------ coarse GMRES --
@pytest.mark.parametrize("maxit", [1, 5, 13, 30])
def test_coarse_solve_fixed_iterations_fp64(c1, maxit):
    """tol = 0: exactly maxit iterations (restart 10, so 13 and 30 restart)."""
    lat, U, A = c1
    tv = inputs.test_vectors(lat.ntv, lat.dims, 821)
    lat.set_tv(lat.to_device(tv, MRHS_F64), MRHS_F64)
    lat.build_P()
    lat.build_Dc()
    Dc = lat.get_Dc()
    nrhs = 4
    bc = inputs.gaussian_field((nrhs, lat.nagg, 2 * lat.ntv), 822)
    bcd = lat.to_device(bc, MRHS_F64, coarse=True)
    xcd = lat.field(nrhs, MRHS_F64, coarse=True)
    its = lat.coarse_solve(bcd, xcd, nrhs, MRHS_F64, 0.0, 10, maxit)
    ref, rits = oracle.coarse_solve(lat.dims, lat.agg, Dc, bc, 0.0, 10, maxit)
    assert list(its) == list(rits) == [maxit] * nrhs
    assert rel(lat.to_host(xcd, nrhs, MRHS_F64, coarse=True), ref) < 1e-11


def test_coarse_solve_tolerance_fp64(c1):
    lat, U, A = c1
    tv = inputs.test_vectors(lat.ntv, lat.dims, 831)
    lat.set_tv(lat.to_device(tv, MRHS_F64), MRHS_F64)
    lat.build_P()
    lat.build_Dc()
    Dc = lat.get_Dc()
    nrhs = 5
    bc = inputs.gaussian_field((nrhs, lat.nagg, 2 * lat.ntv), 832)
    bc[2] = 0  # a zero right-hand side stops at once with x = 0
    bcd = lat.to_device(bc, MRHS_F64, coarse=True)
    xcd = lat.field(nrhs, MRHS_F64, coarse=True)
    its = lat.coarse_solve(bcd, xcd, nrhs, MRHS_F64, 1e-6, 8, 200)
    ref, rits = oracle.coarse_solve(lat.dims, lat.agg, Dc, bc, 1e-6, 8, 200)
    assert list(its) == list(rits)
    assert its[2] == 0
    xc = lat.to_host(xcd, nrhs, MRHS_F64, coarse=True)
    assert np.abs(xc[2]).max() == 0
    assert rel(xc, ref) < 1e-10
    res = bc - oracle.apply_Dc(lat.dims, lat.agg, Dc, xc)
    for r in (0, 1, 3, 4):
        assert np.linalg.norm(res[r]) <= 1.0001e-6 * np.linalg.norm(bc[r])


# ------------------------------------------------------------------ setup --
def _oracle_setup(cfg, U, A, prm):
    tv0 = inputs.test_vectors(cfg["ntv"], cfg["dims"], cfg["tvseed"])
    tv, P, Dc = oracle.setup_init(cfg["dims"], cfg["agg"], U, A, tv0, prm)
    tv, P, Dc, its = oracle.setup_refine(cfg["dims"], cfg["agg"], U, A, tv, P, Dc, prm)
    return tv0, tv, P, Dc, its


@pytest.mark.parametrize("init_mode", [0, 1])
def test_setup_c1_fp64_fixed_coarse_iterations(c1, init_mode):
    """The whole C1 setup (3 sweeps x 4 MR, 1 refinement), all test vectors at
    once on the GPU, equals the oracle's one-vector-at-a-time setup."""
    lat, U, A = c1
    prm = oracle.make_params(init_mode=init_mode, n_init_sweeps=3, n_init_mr=4, n_refine=1, n_smooth_sweeps=4,
                             n_smooth_mr=4, coarse_tol=0.0, coarse_restart=10, coarse_maxit=12)
    tv0, tv, P, Dc, its = _oracle_setup(C1, U, A, prm)
    lat.setup_init(lat.to_device(tv0, MRHS_F64), MRHS_F64, init_mode, 3, 4)
    gits = lat.setup_refine(1, 4, 4, 0.0, 10, 12)
    assert np.array_equal(gits, its)
    assert rel(lat.get_tv(), tv) < 1e-12
    assert rel(lat.get_P(), P) < 1e-12
    assert rel(lat.get_Dc(), Dc) < 1e-12


def test_setup_c1_fp64_coarse_tolerance_and_fgmres(c1):
    """C1 with the paper's coarse tolerance 0.05, then the two-level FGMRES
    solve to 1e-10: identical coarse iteration counts and FGMRES count."""
    lat, U, A = c1
    prm = oracle.make_params(n_init_sweeps=3, n_init_mr=4, n_refine=1, coarse_tol=0.05, coarse_restart=20,
                             coarse_maxit=200)
    tv0, tv, P, Dc, its = _oracle_setup(C1, U, A, prm)
    lat.setup_init(lat.to_device(tv0, MRHS_F64), MRHS_F64, 0, 3, 4)
    gits = lat.setup_refine(1, 4, 4, 0.05, 20, 200)
    assert np.array_equal(gits, its)
    assert rel(lat.get_P(), P) < 1e-12
    assert rel(lat.get_Dc(), Dc) < 1e-12
    b = inputs.gaussian_field((lat.V, 12), 3001)
    x, it, rr = lat.solve_fgmres(b, tol=1e-10, restart=25, maxit=200)
    xo, ito, rro = oracle.fgmres(lat.dims, lat.agg, U, A, P, Dc, b, tol=1e-10)
    assert rr <= 1e-10 and abs(it - ito) <= 1
    assert rel(x, xo) < 1e-8


def test_setup_ragged_fp64(ragged):
    lat, U, A = ragged
    prm = oracle.make_params(n_init_sweeps=2, n_init_mr=3, n_refine=2, n_smooth_sweeps=2, n_smooth_mr=3,
                             coarse_tol=0.0, coarse_restart=6, coarse_maxit=9)
    tv0, tv, P, Dc, its = _oracle_setup(RAGGED, U, A, prm)
    lat.setup_init(lat.to_device(tv0, MRHS_F64), MRHS_F64, 0, 2, 3)
    gits = lat.setup_refine(2, 2, 3, 0.0, 6, 9)
    assert np.array_equal(gits, its)
    assert rel(lat.get_P(), P) < 1e-12
    assert rel(lat.get_Dc(), Dc) < 1e-12


def test_setup_is_deterministic(c1):
    lat, U, A = c1
    tv0 = inputs.test_vectors(lat.ntv, lat.dims, 901)
    out = []
    for _ in range(2):
        lat.setup_init(lat.to_device(tv0, MRHS_F64), MRHS_F64, 0, 2, 3)
        lat.setup_refine(1, 2, 3, 0.05, 20, 100)
        out.append((lat.get_P(), lat.get_Dc()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


# ----------------------------------------------------------- error paths --
def test_shape_and_state_errors():
    with pytest.raises(MrhsError) as e:
        Lattice((4, 4, 4, 4), (4, 2, 2, 2), 4)  # one aggregate along x: no red-black colouring
    assert e.value.status == MRHS_ERR_SHAPE
    with pytest.raises(MrhsError) as e:
        Lattice((4, 4, 4, 4), (2, 2, 2, 2), 97)  # ntv > 6 |aggregate|
    assert e.value.status == MRHS_ERR_SHAPE
    lat = Lattice((4, 4, 4, 4), (2, 2, 2, 2), 4)
    x = lat.field(1, MRHS_F64)
    with pytest.raises(MrhsError) as e:
        lat.apply_D(x, lat.field(1, MRHS_F64), 1, MRHS_F64)
    assert e.value.status == MRHS_ERR_STATE
    with pytest.raises(MrhsError) as e:
        lat.setup_refine(1)
    assert e.value.status == MRHS_ERR_STATE
