"""Block length N_b of Algorithm 2 (the single-right-hand-side order of
Algorithm 1 at N_b = 1): every block length, including one that leaves a
remainder block (the footnote to Algorithm 2), gives the setup of the
all-at-once order, because R, P and D_c stay fixed while the test vectors are
visited and only the order of the work changes (Sec. 3). Checked through the
C ABI against the oracle (which runs Algorithm 1, one vector at a time) and
against the GPU's own N_b = N_tv run: FP64 to 1e-12 with identical coarse
iteration counts; FP32 to 1e-5 (the kernels for 1, 3 and 4 right-hand sides
differ from those for 8).
"""
import numpy as np
import pytest

import oracle
from paper_1601_03184_gb300 import (MRHS_ERR_ARG, MRHS_F32, MRHS_F64, MRHS_PREC_FP32, MRHS_PREC_FP64, Lattice,
                                    MrhsError, inputs)

pytestmark = pytest.mark.gpu

C1 = dict(dims=(4, 4, 4, 4), agg=(2, 2, 2, 2), ntv=8, eps=0.3, m0=-0.2, csw=1.0, gseed=1001, tvseed=2001)
P4 = dict(dims=(8, 8, 8, 8), agg=(4, 4, 4, 4), ntv=8, eps=0.4, m0=-0.1, csw=1.2, gseed=1301, tvseed=2301)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def make(cfg, prec):
    U = inputs.gauge_field(cfg["dims"], cfg["eps"], cfg["gseed"])
    A = oracle.clover(cfg["dims"], U, cfg["m0"], cfg["csw"])
    lat = Lattice(cfg["dims"], cfg["agg"], cfg["ntv"], prec)
    lat.set_gauge(U)
    lat.build_clover(cfg["m0"], cfg["csw"])
    return lat, U, A


@pytest.mark.parametrize("init_mode,ctol", [(0, 0.0), (1, 0.0), (0, 0.05)])
def test_block_lengths_fp64_equal_the_oracle(init_mode, ctol):
    lat, U, A = make(C1, MRHS_PREC_FP64)
    tv0 = inputs.test_vectors(C1["ntv"], C1["dims"], C1["tvseed"])
    maxit = 12 if ctol == 0 else 200
    prm = oracle.make_params(init_mode=init_mode, n_init_sweeps=3, n_init_mr=4, n_refine=2, n_smooth_sweeps=3,
                             n_smooth_mr=4, coarse_tol=ctol, coarse_restart=10, coarse_maxit=maxit)
    tv, P, Dc = oracle.setup_init(C1["dims"], C1["agg"], U, A, tv0, prm)
    tv, P, Dc, its = oracle.setup_refine(C1["dims"], C1["agg"], U, A, tv, P, Dc, prm)
    for nb in (1, 3, 5, 0):
        lat.set_block_length(nb)
        lat.setup_init(lat.to_device(tv0, MRHS_F64), MRHS_F64, init_mode, 3, 4)
        gits = lat.setup_refine(2, 3, 4, ctol, 10, maxit)
        assert np.array_equal(gits, its), nb
        assert rel(lat.get_tv(), tv) < 1e-12, nb
        assert rel(lat.get_P(), P) < 1e-12, nb
        assert rel(lat.get_Dc(), Dc) < 1e-12, nb
    lat.close()


def test_block_lengths_fp32_agree():
    lat, U, A = make(P4, MRHS_PREC_FP32)
    tv0 = inputs.test_vectors(P4["ntv"], P4["dims"], P4["tvseed"]).astype(np.complex64)
    out = {}
    for nb in (0, 1, 3, 4):
        lat.set_block_length(nb)
        lat.setup_init(lat.to_device(tv0, MRHS_F32), MRHS_F32, 0, 2, 4)
        its = lat.setup_refine(1, 2, 4, 0.0, 10, 15)
        out[nb] = (lat.get_P(), lat.get_Dc(), its)
    P0, D0, i0 = out[0]
    for nb in (1, 3, 4):
        P, D, its = out[nb]
        assert np.array_equal(its, i0)
        assert rel(P, P0) < 1e-5, (nb, rel(P, P0))
        assert rel(D, D0) < 1e-5, (nb, rel(D, D0))
    lat.close()


def test_block_length_argument():
    lat = Lattice((4, 4, 4, 4), (2, 2, 2, 2), 4, MRHS_PREC_FP64)
    with pytest.raises(MrhsError) as e:
        lat.set_block_length(-1)
    assert e.value.status == MRHS_ERR_ARG
    lat.set_block_length(100)  # >= ntv: all at once
    lat.close()
