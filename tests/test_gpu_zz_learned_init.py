"""The learned initial phase (mrhs_setup_init_learned) against the oracle,
step by step: x = SAP^1(b = v, x0 = 0), then v <- net(x), each vector
normalised, then P by the aggregate-wise Gram-Schmidt and D_c = P^dag D P. On
an 8^4 lattice with 4^4 domains and 8 test vectors, FP32, with the
bf16-rounded weights the kernels use given to the oracle as well.

Bounds: the test vectors within 3e-4 relative (the FP32 network's own bound
against FP64 is 1e-4, the smoother's 1e-5). P and D_c within 1e-3: the
Gram-Schmidt here passes a perturbation of the vectors to P about one to one,
and to D_c reduced (measured with the oracle on these inputs: 1e-5 on the
vectors gives 1.4e-5 on P and 9e-7 on D_c)."""
import numpy as np
import pytest

import oracle
from paper_1601_03184_gb300 import (MRHS_F32, MRHS_PREC_FP32, Lattice, inputs, mrhs_nn_create, mrhs_nn_get_weights,
                                    mrhs_nn_set_weights, mrhs_setup_init_learned)

pytestmark = pytest.mark.gpu

DIMS, AGG, NTV, WIDTHS = (8, 8, 8, 8), (4, 4, 4, 4), 8, (4, 8, 6, 4)
M0, CSW, N_MR = -0.3, 1.5, 4


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def test_learned_initial_phase_matches_oracle():
    U = inputs.gauge_field(DIMS, 0.4, 5501)
    A = oracle.clover(DIMS, U, M0, CSW)
    lat = Lattice(DIMS, AGG, NTV, MRHS_PREC_FP32)
    lat.set_gauge(U)
    lat.build_clover(M0, CSW)
    mrhs_nn_create(lat.ctx, WIDTHS, 1)
    nw, nb = oracle.nn_sizes(WIDTHS)
    rng = np.random.default_rng(5502)
    mrhs_nn_set_weights(lat.ctx, np.concatenate([0.3 * rng.standard_normal(2 * nw),
                                                 0.2 * rng.standard_normal(nb)]).astype(np.float32))
    used = mrhs_nn_get_weights(lat.ctx, 1)  # the bf16-rounded weights the kernels compute with
    W = used[0:2 * nw:2].astype(np.float64) + 1j * used[1:2 * nw:2].astype(np.float64)
    b = used[2 * nw:].astype(np.float64)
    tv0 = inputs.test_vectors(NTV, DIMS, 5503).astype(np.complex64)
    mrhs_setup_init_learned(lat.ctx, lat.to_device(tv0, MRHS_F32), MRHS_F32, 1, N_MR)

    x = oracle.sap(DIMS, AGG, U, A, tv0.astype(np.complex128), np.zeros(tv0.shape, np.complex128), 1, N_MR)
    y = oracle.nn_forward(DIMS, U, WIDTHS, W, b, x)
    v = y / np.linalg.norm(y.reshape(NTV, -1), axis=1)[:, None, None]
    P = oracle.gram_schmidt(DIMS, AGG, v)
    Dc = oracle.coarse_op(DIMS, AGG, U, A, P)
    e_tv, e_P, e_Dc = rel(lat.get_tv(), v), rel(lat.get_P(), P), rel(lat.get_Dc(), Dc)
    print("learned initial phase vs oracle: tv %.2e, P %.2e, D_c %.2e" % (e_tv, e_P, e_Dc))
    assert e_tv < 3e-4
    assert e_P < 1e-3
    assert e_Dc < 1e-3
    lat.close()
