"""Even-odd preconditioned coarse solve (mrhs_set_coarse_solver(ctx, 1)):
GMRES on the Schur complement of the even aggregates, then the odd ones by
back-substitution, against the oracle's form of the same (coarse_solve_eo,
itself pinned against a dense solve in tests/test_oracle_pins.py). The oracle
builds its D_c from the same test vectors (gram_schmidt, coarse_op); the GPU
builds its own. FP64 to 1e-10 (D_c agrees to ~1e-14, GMRES amplifies that by
the condition number of the few iterations), FP32 to 2e-5; the FP64 setup
with fixed coarse iteration counts and the two-level FGMRES with this coarse
solver against the oracle's."""
import numpy as np
import pytest

import oracle
from paper_1601_03184_gb300 import (MRHS_ERR_ARG, MRHS_F32, MRHS_F64, MRHS_PREC_FP32, MRHS_PREC_FP64, Lattice,
                                    MrhsError, inputs, mrhs_coarse_solve_noalloc)

pytestmark = pytest.mark.gpu

C1 = dict(dims=(4, 4, 4, 4), agg=(2, 2, 2, 2), ntv=8, eps=0.3, m0=-0.2, csw=1.0, gseed=1001, tvseed=2001)
RAGGED = dict(dims=(4, 6, 4, 8), agg=(2, 3, 2, 2), ntv=5, eps=0.5, m0=0.1, csw=1.3, gseed=1101, tvseed=2101)
P4 = dict(dims=(8, 8, 8, 16), agg=(4, 4, 4, 4), ntv=12, eps=0.4, m0=-0.1, csw=1.2, gseed=1301, tvseed=2301)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def make(cfg, prec, dt, tvseed):
    U = inputs.gauge_field(cfg["dims"], cfg["eps"], cfg["gseed"])
    A = oracle.clover(cfg["dims"], U, cfg["m0"], cfg["csw"])
    lat = Lattice(cfg["dims"], cfg["agg"], cfg["ntv"], prec)
    lat.set_gauge(U)
    lat.build_clover(cfg["m0"], cfg["csw"])
    tv = inputs.test_vectors(cfg["ntv"], cfg["dims"], tvseed)
    lat.set_tv(lat.to_device(tv, dt), dt)
    lat.build_P()
    lat.build_Dc()
    lat.set_coarse_solver(1)
    Dc = oracle.coarse_op(cfg["dims"], cfg["agg"], U, A, oracle.gram_schmidt(cfg["dims"], cfg["agg"], tv))
    return lat, U, A, Dc


@pytest.mark.parametrize("cfg", [C1, RAGGED], ids=["c1", "ragged"])
@pytest.mark.parametrize("maxit", [1, 7, 23])
def test_coarse_eo_fixed_iterations_fp64(cfg, maxit):
    """tol = 0: exactly maxit iterations on S (restart 10: 23 restarts twice)."""
    lat, U, A, Dc = make(cfg, MRHS_PREC_FP64, MRHS_F64, 4101)
    nrhs = 3
    bc = inputs.gaussian_field((nrhs, lat.nagg, 2 * lat.ntv), 4102)
    bcd = lat.to_device(bc, MRHS_F64, coarse=True)
    xcd = lat.field(nrhs, MRHS_F64, coarse=True)
    its = lat.coarse_solve(bcd, xcd, nrhs, MRHS_F64, 0.0, 10, maxit)
    ref, rits = oracle.coarse_solve_eo(cfg["dims"], cfg["agg"], Dc, bc, 0.0, 10, maxit)
    assert list(its) == list(rits) == [maxit] * nrhs
    assert rel(lat.to_host(xcd, nrhs, MRHS_F64, coarse=True), ref) < 1e-10
    if maxit == 1:  # one step on S is not one step on D_c (both reach the solution by 23)
        plain, _ = oracle.coarse_solve(cfg["dims"], cfg["agg"], Dc, bc, 0.0, 10, maxit)
        assert rel(plain, ref) > 1e-2
    lat.close()


def test_coarse_eo_tolerance_and_residual_fp64():
    """tol 1e-8: the same iteration counts as the oracle, and the residual of
    the full system equals that of the Schur system (the odd rows are solved
    exactly), so |b - D_c x| <= tol |bhat| with bhat_e = b_e - D_eo D_oo^-1 b_o."""
    lat, U, A, Dc = make(C1, MRHS_PREC_FP64, MRHS_F64, 4201)
    nrhs = 4
    bc = inputs.gaussian_field((nrhs, lat.nagg, 2 * lat.ntv), 4202)
    bc[1] = 0  # a zero right-hand side stops at once with x = 0
    bcd = lat.to_device(bc, MRHS_F64, coarse=True)
    xcd = lat.field(nrhs, MRHS_F64, coarse=True)
    its = lat.coarse_solve(bcd, xcd, nrhs, MRHS_F64, 1e-8, 10, 300)
    ref, rits = oracle.coarse_solve_eo(C1["dims"], C1["agg"], Dc, bc, 1e-8, 10, 300)
    assert list(its) == list(rits)
    assert its[1] == 0
    xc = lat.to_host(xcd, nrhs, MRHS_F64, coarse=True)
    assert np.abs(xc[1]).max() == 0
    assert rel(xc, ref) < 1e-9
    res = bc - oracle.apply_Dc(C1["dims"], C1["agg"], Dc, xc)
    for r in (0, 2, 3):
        assert np.linalg.norm(res[r]) <= 1.0001e-8 * np.linalg.norm(bc[r])
    # fewer iterations than GMRES on D_c for the same tolerance
    _, pits = oracle.coarse_solve(C1["dims"], C1["agg"], Dc, bc, 1e-8, 10, 300)
    assert all(its[r] < pits[r] for r in (0, 2, 3))
    lat.close()


@pytest.mark.parametrize("nrhs", [8, 16], ids=["cuda-cores", "tensor-cores"])
def test_coarse_eo_fp32_and_dc_rebuild(nrhs):
    """FP32 context, 2ntv = 24, 32 aggregates; 8 right-hand sides take the
    CUDA-core stencil, 16 the tensor-core one (split tf32). Then new test
    vectors and a new D_c: the inverse self blocks follow the new D_c."""
    lat, U, A, Dc = make(P4, MRHS_PREC_FP32, MRHS_F32, 4301)
    bc = inputs.gaussian_field((nrhs, lat.nagg, 2 * lat.ntv), 4302)
    bcd = lat.to_device(bc, MRHS_F32, coarse=True)
    xcd = lat.field(nrhs, MRHS_F32, coarse=True)
    its = lat.coarse_solve(bcd, xcd, nrhs, MRHS_F32, 0.0, 12, 20)
    ref, _ = oracle.coarse_solve_eo(P4["dims"], P4["agg"], Dc, bc, 0.0, 12, 20)
    assert list(its) == [20] * nrhs
    assert rel(lat.to_host(xcd, nrhs, MRHS_F32, coarse=True), ref) < 2e-5
    tv2 = inputs.test_vectors(P4["ntv"], P4["dims"], 4303)
    lat.set_tv(lat.to_device(tv2, MRHS_F32), MRHS_F32)
    lat.build_P()
    lat.build_Dc()
    Dc2 = oracle.coarse_op(P4["dims"], P4["agg"], U, A, oracle.gram_schmidt(P4["dims"], P4["agg"], tv2))
    lat.coarse_solve(bcd, xcd, nrhs, MRHS_F32, 0.0, 12, 20)
    ref2, _ = oracle.coarse_solve_eo(P4["dims"], P4["agg"], Dc2, bc, 0.0, 12, 20)
    assert rel(lat.to_host(xcd, nrhs, MRHS_F32, coarse=True), ref2) < 2e-5
    assert rel(ref2, ref) > 1e-3
    lat.close()


def test_noalloc_ignores_the_coarse_solver_setting():
    lat, U, A, Dc = make(C1, MRHS_PREC_FP64, MRHS_F64, 4401)
    nrhs = 2
    bc = inputs.gaussian_field((nrhs, lat.nagg, 2 * lat.ntv), 4402)
    bcd = lat.to_device(bc, MRHS_F64, coarse=True)
    xcd = lat.field(nrhs, MRHS_F64, coarse=True)
    mrhs_coarse_solve_noalloc(lat.ctx, bcd, xcd, nrhs, MRHS_F64, 0.0, 10, 9)
    ref, _ = oracle.coarse_solve(C1["dims"], C1["agg"], Dc, bc, 0.0, 10, 9)
    assert rel(lat.to_host(xcd, nrhs, MRHS_F64, coarse=True), ref) < 1e-10
    with pytest.raises(MrhsError) as e:
        lat.set_coarse_solver(2)
    assert e.value.status == MRHS_ERR_ARG
    lat.close()


def test_setup_and_fgmres_with_coarse_eo_fp64():
    """The C1 setup (3 sweeps x 4 MR, 2 refinements, 12 coarse iterations on S
    per refinement) and the FGMRES solve with the even-odd coarse solver."""
    U = inputs.gauge_field(C1["dims"], C1["eps"], C1["gseed"])
    A = oracle.clover(C1["dims"], U, C1["m0"], C1["csw"])
    lat = Lattice(C1["dims"], C1["agg"], C1["ntv"], MRHS_PREC_FP64)
    lat.set_gauge(U)
    lat.build_clover(C1["m0"], C1["csw"])
    lat.set_coarse_solver(1)
    tv0 = inputs.test_vectors(C1["ntv"], C1["dims"], C1["tvseed"])
    prm = oracle.make_params(n_init_sweeps=3, n_init_mr=4, n_refine=2, n_smooth_sweeps=3, n_smooth_mr=4,
                             coarse_tol=0.0, coarse_restart=10, coarse_maxit=12, coarse_even_odd=1)
    tv, P, Dc = oracle.setup_init(C1["dims"], C1["agg"], U, A, tv0, prm)
    tv, P, Dc, its = oracle.setup_refine(C1["dims"], C1["agg"], U, A, tv, P, Dc, prm)
    lat.setup_init(lat.to_device(tv0, MRHS_F64), MRHS_F64, 0, 3, 4)
    gits = lat.setup_refine(2, 3, 4, 0.0, 10, 12)
    assert np.array_equal(gits, its)
    assert rel(lat.get_P(), P) < 1e-11
    assert rel(lat.get_Dc(), Dc) < 1e-11
    b = inputs.gaussian_field((lat.V, 12), 4501)
    x, it, rr = lat.solve_fgmres(b, tol=1e-10, restart=25, maxit=200, n_sweeps=3, n_mr=4)
    xo, ito, rro = oracle.fgmres(C1["dims"], C1["agg"], U, A, P, Dc, b, tol=1e-10, n_sweeps=3, n_mr=4,
                                 coarse_even_odd=1)
    assert rr <= 1e-10 and abs(it - ito) <= 1
    assert rel(x, xo) < 1e-8
    lat.close()
