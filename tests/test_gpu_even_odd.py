"""Even-odd preconditioned SAP domain solves (mrhs_set_smoother(ctx, 1)):
MR on the Schur complement of the even sites of every domain, then the odd
sites, against the oracle's form of the same (sap_eo, itself pinned against
dense linear algebra in tests/test_oracle_pins.py): FP64 to 1e-12 (the same
sums in another order), FP32 to 1e-5; the whole FP64 setup with fixed coarse
iteration counts and the two-level FGMRES solve with this smoother against
the oracle's."""
import numpy as np
import pytest

import oracle
from paper_1601_03184_gb300 import (MRHS_ERR_ARG, MRHS_F32, MRHS_F64, MRHS_PREC_FP32, MRHS_PREC_FP64, Lattice,
                                    MrhsError, inputs)

pytestmark = pytest.mark.gpu

C1 = dict(dims=(4, 4, 4, 4), agg=(2, 2, 2, 2), ntv=8, eps=0.3, m0=-0.2, csw=1.0, gseed=1001, tvseed=2001)
RAGGED = dict(dims=(4, 6, 4, 8), agg=(2, 3, 2, 2), ntv=5, eps=0.5, m0=0.1, csw=1.3, gseed=1101, tvseed=2101)
P4 = dict(dims=(8, 8, 8, 8), agg=(4, 4, 4, 4), ntv=8, eps=0.4, m0=-0.1, csw=1.2, gseed=1301, tvseed=2301)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def make(cfg, prec):
    U = inputs.gauge_field(cfg["dims"], cfg["eps"], cfg["gseed"])
    A = oracle.clover(cfg["dims"], U, cfg["m0"], cfg["csw"])
    lat = Lattice(cfg["dims"], cfg["agg"], cfg["ntv"], prec)
    lat.set_gauge(U)
    lat.build_clover(cfg["m0"], cfg["csw"])
    lat.set_smoother(1)
    return lat, U, A


@pytest.mark.parametrize("cfg,prec,dt,tol", [(C1, MRHS_PREC_FP64, MRHS_F64, 1e-12),
                                             (RAGGED, MRHS_PREC_FP64, MRHS_F64, 1e-12),
                                             (P4, MRHS_PREC_FP32, MRHS_F32, 1e-5)], ids=["c1", "ragged", "4^4-fp32"])
def test_sap_even_odd(cfg, prec, dt, tol):
    lat, U, A = make(cfg, prec)
    nrhs = 3
    b = inputs.gaussian_field((nrhs, lat.V, 12), 7701)
    x0 = 0.1 * inputs.gaussian_field((nrhs, lat.V, 12), 7702)
    xd = lat.to_device(x0, dt)
    lat.sap(lat.to_device(b, dt), xd, nrhs, dt, 2, 4)
    ref = oracle.sap_eo(cfg["dims"], cfg["agg"], U, A, b, x0, 2, 4)
    assert rel(lat.to_host(xd, nrhs, dt), ref) < tol
    # the plain smoother gives something else
    assert rel(oracle.sap(cfg["dims"], cfg["agg"], U, A, b, x0, 2, 4), ref) > 1e-3
    lat.close()


def test_setup_and_fgmres_even_odd_fp64():
    lat, U, A = make(C1, MRHS_PREC_FP64)
    tv0 = inputs.test_vectors(C1["ntv"], C1["dims"], C1["tvseed"])
    prm = oracle.make_params(n_init_sweeps=3, n_init_mr=4, n_refine=1, n_smooth_sweeps=3, n_smooth_mr=4,
                             coarse_tol=0.0, coarse_restart=10, coarse_maxit=12, even_odd=1)
    tv, P, Dc = oracle.setup_init(C1["dims"], C1["agg"], U, A, tv0, prm)
    tv, P, Dc, its = oracle.setup_refine(C1["dims"], C1["agg"], U, A, tv, P, Dc, prm)
    lat.setup_init(lat.to_device(tv0, MRHS_F64), MRHS_F64, 0, 3, 4)
    gits = lat.setup_refine(1, 3, 4, 0.0, 10, 12)
    assert np.array_equal(gits, its)
    assert rel(lat.get_P(), P) < 1e-12
    assert rel(lat.get_Dc(), Dc) < 1e-12
    b = inputs.gaussian_field((lat.V, 12), 7703)
    x, it, rr = lat.solve_fgmres(b, tol=1e-10, restart=25, maxit=200, n_sweeps=3, n_mr=4)
    xo, ito, rro = oracle.fgmres(C1["dims"], C1["agg"], U, A, P, Dc, b, tol=1e-10, n_sweeps=3, n_mr=4, even_odd=1)
    assert rr <= 1e-10 and abs(it - ito) <= 1
    assert rel(x, xo) < 1e-8
    with pytest.raises(MrhsError) as e:
        lat.set_smoother(2)
    assert e.value.status == MRHS_ERR_ARG
    lat.close()
