"""Setup update after a change of the gauge field (HMC renews the setup every
few solves, Sec. 1): D_c rebuilt from the kept P with the new operator, then
refinement iterations from the kept test vectors (mrhs_setup_update).

- FP64 parity with the oracle composed of its own steps: D_c' = P^dag D' P,
  then Algorithm 1's refinement on D' from the kept vectors (1e-12, identical
  coarse iteration counts).
- Quality: after a small change of the field (every link multiplied by a
  random SU(3) matrix exp(i 0.05 H)), one update iteration gives a two-level
  FGMRES iteration count within 10 % (+1) of a whole new setup on the new
  field, and no worse than keeping the old P with only D_c rebuilt.
"""
import numpy as np
import pytest

import oracle
from paper_1601_03184_gb300 import (MRHS_ERR_STATE, MRHS_F32, MRHS_F64, MRHS_PREC_FP32, MRHS_PREC_FP64, Lattice,
                                    MrhsError, inputs)

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def moved_field(dims, U, delta, seed):
    """U_mu(x) -> R_mu(x) U_mu(x), R = exp(i delta H) random SU(3) (one HMC-like step)"""
    R = inputs.gauge_field(dims, delta, seed)
    return np.einsum("smab,smbc->smac", R, U)


def test_update_fp64_matches_oracle():
    dims, agg, ntv, m0, csw = (4, 4, 4, 4), (2, 2, 2, 2), 8, -0.2, 1.0
    U = inputs.gauge_field(dims, 0.3, 1001)
    A = oracle.clover(dims, U, m0, csw)
    tv0 = inputs.test_vectors(ntv, dims, 2001)
    prm = oracle.make_params(n_init_sweeps=3, n_init_mr=4, n_refine=1, n_smooth_sweeps=3, n_smooth_mr=4,
                             coarse_tol=0.0, coarse_restart=10, coarse_maxit=12)
    tv, P, Dc = oracle.setup_init(dims, agg, U, A, tv0, prm)
    tv, P, Dc, _ = oracle.setup_refine(dims, agg, U, A, tv, P, Dc, prm)
    U2 = moved_field(dims, U, 0.05, 1002)
    A2 = oracle.clover(dims, U2, m0, csw)
    Dc2 = oracle.coarse_op(dims, agg, U2, A2, P)
    tv2, P2, Dc2, its = oracle.setup_refine(dims, agg, U2, A2, tv, P, Dc2, prm)

    lat = Lattice(dims, agg, ntv, MRHS_PREC_FP64)
    with pytest.raises(MrhsError) as e:
        lat.setup_update(1)
    assert e.value.status == MRHS_ERR_STATE
    lat.set_gauge(U)
    lat.build_clover(m0, csw)
    lat.setup_init(lat.to_device(tv0, MRHS_F64), MRHS_F64, 0, 3, 4)
    lat.setup_refine(1, 3, 4, 0.0, 10, 12)
    lat.set_gauge(U2)
    with pytest.raises(MrhsError) as e:  # the new field's clover term first
        lat.setup_update(1, 3, 4, 0.0, 10, 12)
    assert e.value.status == MRHS_ERR_STATE
    lat.build_clover(m0, csw)
    gits = lat.setup_update(1, 3, 4, 0.0, 10, 12)
    assert np.array_equal(gits, its)
    assert rel(lat.get_tv(), tv2) < 1e-12
    assert rel(lat.get_P(), P2) < 1e-12
    assert rel(lat.get_Dc(), Dc2) < 1e-12
    lat.close()


def test_update_quality_fp32():
    import json
    import os

    dims, agg, ntv, csw, eps = (16, 16, 16, 16), (4, 4, 4, 4), 16, 1.5, 0.6
    m0 = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "m0.json")))[
        "proxy_12x12x12x12_eps0.6_csw1.5_seed1002"]["m0"]
    U = inputs.gauge_field(dims, eps, 1401)
    U2 = moved_field(dims, U, 0.05, 1402)
    b = inputs.gaussian_field((int(np.prod(dims)), 12), 1403)
    tv0 = inputs.test_vectors(ntv, dims, 1404).astype(np.complex64)
    sched = dict(n_sweeps=4, n_mr=4, coarse_tol=0.05, coarse_restart=20, coarse_maxit=100)

    def fgmres(lat):
        return lat.solve_fgmres(b, tol=1e-10, restart=10, maxit=300, coarse_tol=0.05, coarse_restart=20,
                                coarse_maxit=100, n_sweeps=4, n_mr=4, allow_noconv=True)[1]

    lat = Lattice(dims, agg, ntv, MRHS_PREC_FP32)
    # a whole new setup on the new field
    lat.set_gauge(U2)
    lat.build_clover(m0, csw)
    lat.setup_init(lat.to_device(tv0, MRHS_F32), MRHS_F32, 0, 5, 4)
    lat.setup_refine(3, **sched)
    it_fresh = fgmres(lat)
    # the setup of the old field, then the new field with only D_c rebuilt
    lat.set_gauge(U)
    lat.build_clover(m0, csw)
    lat.setup_init(lat.to_device(tv0, MRHS_F32), MRHS_F32, 0, 5, 4)
    lat.setup_refine(3, **sched)
    lat.set_gauge(U2)
    lat.build_clover(m0, csw)
    lat.build_Dc()
    it_stale = fgmres(lat)
    # ... and updated by one refinement iteration on the new field
    lat.setup_update(1, **sched)
    it_update = fgmres(lat)
    print("FGMRES iterations: new setup %d, stale P %d, updated %d" % (it_fresh, it_stale, it_update))
    assert it_update <= 1.1 * it_fresh + 1
    assert it_update <= it_stale
    lat.close()
