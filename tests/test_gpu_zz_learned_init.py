"""The learned initial phase (mrhs_setup_init_learned) against the oracle,
step by step: x = SAP^1(b = v, x0 = 0), then v <- net(x), each vector
normalised, then P by the aggregate-wise Gram-Schmidt and D_c = P^dag D P. On
an 8^4 lattice with 4^4 domains and 8 test vectors, FP32, with the
bf16-rounded weights the kernels use given to the oracle as well.

Two forms of the network. FP32 weights: the CUDA-core layers with FP32
activations, against the oracle's forward. Bounds: the test vectors within
3e-4 relative (the FP32 network's own bound against FP64 is 1e-4, the
smoother's 1e-5). P and D_c within 1e-3: the Gram-Schmidt here passes a
perturbation of the vectors to P about one to one, and to D_c reduced
(measured with the oracle on these inputs: 1e-5 on the vectors gives 1.4e-5 on
P and 9e-7 on D_c).
bf16 weights: the tensor-core layers with bf16 operands, against the oracle's
forward with bf16-rounded operands. The network input is the FP32 smoother
output, which differs from the oracle's by up to 1e-5 relative, and that
moves some bf16 rounding decisions: measured with the oracle on these inputs,
1e-6 and 1e-5 relative noise on the network input move the vectors by 5.8e-4
and 1.4e-3, P by 5.8e-4 and 1.4e-3, D_c by 3.9e-5 and 9.5e-5. Bounds: 3e-3 on
the vectors and P, 3e-4 on D_c. (The tensor-core layer itself is checked bit
for bit in tests/test_gpu_nn_tc.py.)"""
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


@pytest.mark.parametrize("bf16", [0, 1], ids=["fp32-weights", "bf16-tensor-cores"])
def test_learned_initial_phase_matches_oracle(bf16):
    U = inputs.gauge_field(DIMS, 0.4, 5501)
    A = oracle.clover(DIMS, U, M0, CSW)
    lat = Lattice(DIMS, AGG, NTV, MRHS_PREC_FP32)
    lat.set_gauge(U)
    lat.build_clover(M0, CSW)
    mrhs_nn_create(lat.ctx, WIDTHS, bf16)
    nw, nb = oracle.nn_sizes(WIDTHS)
    rng = np.random.default_rng(5502)
    mrhs_nn_set_weights(lat.ctx, np.concatenate([0.3 * rng.standard_normal(2 * nw),
                                                 0.2 * rng.standard_normal(nb)]).astype(np.float32))
    used = mrhs_nn_get_weights(lat.ctx, 1)  # the weights the kernels compute with (bf16-rounded if bf16)
    W = used[0:2 * nw:2].astype(np.float64) + 1j * used[1:2 * nw:2].astype(np.float64)
    b = used[2 * nw:].astype(np.float64)
    tv0 = inputs.test_vectors(NTV, DIMS, 5503).astype(np.complex64)
    mrhs_setup_init_learned(lat.ctx, lat.to_device(tv0, MRHS_F32), MRHS_F32, 1, N_MR)

    x = oracle.sap(DIMS, AGG, U, A, tv0.astype(np.complex128), np.zeros(tv0.shape, np.complex128), 1, N_MR)
    y = (oracle.nn_forward_bf16act if bf16 else oracle.nn_forward)(DIMS, U, WIDTHS, W, b, x)
    v = y / np.linalg.norm(y.reshape(NTV, -1), axis=1)[:, None, None]
    P = oracle.gram_schmidt(DIMS, AGG, v)
    Dc = oracle.coarse_op(DIMS, AGG, U, A, P)
    e_tv, e_P, e_Dc = rel(lat.get_tv(), v), rel(lat.get_P(), P), rel(lat.get_Dc(), Dc)
    print("learned initial phase vs oracle: tv %.2e, P %.2e, D_c %.2e" % (e_tv, e_P, e_Dc))
    bounds = (3e-3, 3e-3, 3e-4) if bf16 else (3e-4, 1e-3, 1e-3)
    assert e_tv < bounds[0]
    assert e_P < bounds[1]
    assert e_Dc < bounds[2]
    lat.close()
