"""Learned test-vector generator on the GPU: forward, backward (weight, bias
and input gradients) and training loss against the FP64 oracle, and what a
trained network gains over the same SAP budget without it.

Bounds: FP32 kernels against FP64 with bf16-rounded weights shared by both
sides: outputs and gradients within 1e-4 relative (sums of up to
9 x 32 x 3 FP32 products per output and a site reduction for the weight
gradients, unit roundoff 6e-8)."""
import numpy as np
import pytest

import oracle
from paper_1601_03184_gb300 import (MRHS_F32, MRHS_PREC_FP32, Lattice, inputs, learned, mrhs_nn_backward,
                                    mrhs_nn_create, mrhs_nn_forward, mrhs_nn_get_grads, mrhs_nn_get_weights,
                                    mrhs_nn_loss, mrhs_nn_set_weights, mrhs_nn_zero_grads)

pytestmark = pytest.mark.gpu

DIMS, AGG = (4, 4, 4, 8), (2, 2, 2, 2)
WIDTHS = (4, 8, 6, 4)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def unpack(flat, widths):
    nw, nb = oracle.nn_sizes(widths)
    W = flat[0:2 * nw:2].astype(np.float64) + 1j * flat[1:2 * nw:2].astype(np.float64)
    return W, flat[2 * nw:].astype(np.float64)


@pytest.fixture(scope="module")
def net():
    U = inputs.gauge_field(DIMS, 0.4, 5101)
    lat = Lattice(DIMS, AGG, 6, MRHS_PREC_FP32)
    lat.set_gauge(U)
    lat.build_clover(-0.1, 1.2)
    mrhs_nn_create(lat.ctx, WIDTHS, 1)
    rng = np.random.default_rng(5102)
    nw, nb = oracle.nn_sizes(WIDTHS)
    flat = np.concatenate([0.4 * rng.standard_normal(2 * nw), 0.3 * rng.standard_normal(nb)]).astype(np.float32)
    mrhs_nn_set_weights(lat.ctx, flat)
    W, b = unpack(mrhs_nn_get_weights(lat.ctx, 1), WIDTHS)  # the bf16-rounded weights the kernels use
    return lat, U, W, b


def test_nn_forward_matches_oracle(net):
    lat, U, W, b = net
    nrhs = 5
    x = inputs.gaussian_field((nrhs, lat.V, 12), 5103)
    y = lat.field(nrhs, MRHS_F32)
    mrhs_nn_forward(lat.ctx, lat.to_device(x, MRHS_F32), y, nrhs)
    ref = oracle.nn_forward(DIMS, U, WIDTHS, W, b, x)
    assert rel(lat.to_host(y, nrhs, MRHS_F32), ref) < 1e-4


def test_nn_backward_matches_oracle(net):
    lat, U, W, b = net
    nrhs = 3
    x = inputs.gaussian_field((nrhs, lat.V, 12), 5104)
    dout = inputs.gaussian_field((nrhs, lat.V, 12), 5105)
    y = lat.field(nrhs, MRHS_F32)
    din = lat.field(nrhs, MRHS_F32)
    mrhs_nn_forward(lat.ctx, lat.to_device(x, MRHS_F32), y, nrhs)
    mrhs_nn_zero_grads(lat.ctx)
    mrhs_nn_backward(lat.ctx, lat.to_device(dout, MRHS_F32), din, nrhs)
    gW, gb = unpack(mrhs_nn_get_grads(lat.ctx), WIDTHS)
    rW, rb, rdin = oracle.nn_backward(DIMS, U, WIDTHS, W, b, x, dout, want_din=True)
    assert rel(gW, rW) < 1e-4
    assert rel(gb, rb) < 1e-4
    assert rel(lat.to_host(din, nrhs, MRHS_F32), rdin) < 1e-4


def test_nn_loss_matches_oracle(net):
    lat, U, W, b = net
    A = oracle.clover(DIMS, U, -0.1, 1.2)
    tv = inputs.test_vectors(6, DIMS, 5106)
    lat.set_tv(lat.to_device(tv, MRHS_F32), MRHS_F32)
    lat.build_P()
    P = lat.get_P()  # the FP32 P the loss uses, as FP64 for the oracle
    nrhs = 4
    v = inputs.gaussian_field((nrhs, lat.V, 12), 5107)
    gv = lat.field(nrhs, MRHS_F32)
    loss, per = mrhs_nn_loss(lat.ctx, lat.to_device(v, MRHS_F32), gv, nrhs, 0.8)
    rloss, rdv = oracle.nn_loss(DIMS, AGG, U, A, P, v, 0.8)
    assert abs(loss - rloss) < 1e-5 * rloss
    assert rel(lat.to_host(gv, nrhs, MRHS_F32), rdv) < 1e-4


def rayleigh(lat, P_or_tv):
    """|D v| / |v| per vector, from host vectors [n, V, 12]"""
    import torch

    n = P_or_tv.shape[0]
    xd = lat.to_device(P_or_tv.astype(np.complex64), MRHS_F32)
    yd = lat.field(n, MRHS_F32)
    lat.apply_D(xd, yd, n, MRHS_F32)
    y = lat.to_host(yd, n, MRHS_F32)
    return np.linalg.norm(y.reshape(n, -1), axis=1) / np.linalg.norm(P_or_tv.reshape(n, -1), axis=1)


def test_training_gain():
    """Train on 3 seeded fields (8^4 lattice, 4^4 domains, 8 test vectors),
    then on an unseen field: the network's vectors after one SAP sweep have a
    lower Rayleigh quotient |Dv|/|v| than the same sweep without the network
    (the gain), and the setup built from them (1 sweep + network, then the
    refinement) needs the plain setup's FGMRES iteration count within +-10%
    (the plain setup uses 5 initial sweeps)."""
    import torch

    dims, agg, ntv = (8, 8, 8, 8), (4, 4, 4, 4), 8
    sched = dict(init_sweeps=5, init_mr=4, n_refine=1, sweeps=4, mr=4, ctol=0.05, crestart=20, cmaxit=200)
    lat = Lattice(dims, agg, ntv, MRHS_PREC_FP32)
    learned.attach(lat, (4, 16, 16, 4), seed=11, noise=0.01, bf16=True)
    step = 1
    first, last = [], []
    for f in range(3):
        U = inputs.gauge_field(dims, 0.4, 5200 + f)
        lat.set_gauge(U)
        lat.build_clover(-0.3, 1.5)
        losses = learned.train_on_field(lat, sched, 40, seed=5300 + f, lr=3e-3, first_step=step)
        step += len(losses)
        first.append(losses[0])
        last.append(losses[-1])
    assert last[-1] < first[0]
    # unseen field
    U = inputs.gauge_field(dims, 0.4, 5250)
    lat.set_gauge(U)
    lat.build_clover(-0.3, 1.5)
    b, x1 = learned.sap_vectors(lat, 5400, 1, 4)
    v_sap = lat.to_host(x1, ntv, MRHS_F32)
    y = lat.field(ntv, MRHS_F32)
    mrhs_nn_forward(lat.ctx, x1, y, ntv)
    v_net = lat.to_host(y, ntv, MRHS_F32)
    r_sap, r_net = rayleigh(lat, v_sap).mean(), rayleigh(lat, v_net).mean()
    print("Rayleigh quotient: 1 SAP sweep %.4f, + network %.4f" % (r_sap, r_net))
    assert r_net < r_sap
    rhs = inputs.gaussian_field((lat.V, 12), 5401)
    learned.learned_setup(lat, b, sched, n_sweeps=1)
    _, it_learned, _ = lat.solve_fgmres(rhs, tol=1e-10, maxit=500)
    lat.setup_init(b, MRHS_F32, 0, 1, 4)
    lat.setup_refine(sched["n_refine"], sched["sweeps"], sched["mr"], sched["ctol"], sched["crestart"], sched["cmaxit"])
    _, it_same_budget, _ = lat.solve_fgmres(rhs, tol=1e-10, maxit=500)
    lat.setup_init(b, MRHS_F32, 0, 5, 4)
    lat.setup_refine(sched["n_refine"], sched["sweeps"], sched["mr"], sched["ctol"], sched["crestart"], sched["cmaxit"])
    _, it_plain, _ = lat.solve_fgmres(rhs, tol=1e-10, maxit=500)
    print("FGMRES iterations: learned %d, same SAP budget %d, plain 5 sweeps %d" % (it_learned, it_same_budget, it_plain))
    assert abs(it_learned - it_plain) <= max(1, 0.1 * it_plain)
    # against the same SAP budget (one sweep) without the network the
    # iteration count stays within 10 % (+1): on this small case the gain is
    # in the Rayleigh quotient (measured on a GB300: 3.17 -> 1.44), not in
    # the FGMRES count (measured: learned 25, one sweep alone 23, plain 24)
    assert it_learned <= 1.1 * it_same_budget + 1
