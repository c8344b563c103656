"""Inference of the learned generator with the channel mixing on the tensor
cores (mrhs_nn_infer with bf16 weights: bf16 operands, FP32 products and
sums) against the oracle's forward with every transported operand rounded to
bf16 before it meets the weights (oracle.nn_forward_bf16act, pinned in
tests/test_oracle_nn.py).

- Exact case: links that are monomial matrices with entries in {±1, ±i},
  weights with few bits (multiples of 1/2, most of them zero), inputs in
  {-1, 0, 1} and zero biases (modReLU is then the identity in both
  arithmetics). Every product and partial sum is exact in FP32 and in FP64,
  so both sides take the same bf16 rounding decisions and the outputs agree
  bit for bit; a wrong index, sign, transpose or rounding place changes them.
- Generic case: a rough SU(3) field, Gaussian inputs, random weights and
  biases. FP32 transports and sums against FP64 ones move some bf16 rounding
  decisions; measured with the oracle alone, a relative change of 1e-6 in the
  input moves the output by 5.4e-4, while rounding the operands at all moves
  it by 2.9e-3. Bound: 1.5e-3.
- Layers with fewer than 16 channels on both sides, and FP32 weights, take
  the CUDA-core layer: against the unrounded oracle at 1e-4.
"""
import numpy as np
import pytest

import oracle
import paper_1601_03184_gb300 as pkg
from paper_1601_03184_gb300 import (MRHS_F32, MRHS_PREC_FP32, Lattice, inputs, mrhs_nn_create, mrhs_nn_get_weights,
                                    mrhs_nn_infer, mrhs_nn_set_weights)

pytestmark = pytest.mark.gpu

DIMS, AGG = (4, 4, 4, 8), (2, 2, 2, 2)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def unpack(flat, widths):
    nw, nb = oracle.nn_sizes(widths)
    W = flat[0:2 * nw:2].astype(np.float64) + 1j * flat[1:2 * nw:2].astype(np.float64)
    return W, flat[2 * nw:].astype(np.float64)


def monomial_links(seed):
    """[V][4][3][3] matrices P diag(p) with P a permutation and p in {±1, ±i}"""
    rng = np.random.default_rng(seed)
    V = int(np.prod(DIMS))
    U = np.zeros((V, 4, 3, 3), np.complex128)
    ph = np.array([1, 1j, -1, -1j])
    for s in range(V):
        for mu in range(4):
            perm = rng.permutation(3)
            U[s, mu, np.arange(3), perm] = ph[rng.integers(0, 4, 3)]
    return U


def make(U, widths, flat, bf16=1):
    lat = Lattice(DIMS, AGG, 4, MRHS_PREC_FP32)
    lat.set_gauge(U)
    lat.build_clover(-0.1, 1.2)
    mrhs_nn_create(lat.ctx, widths, bf16)
    mrhs_nn_set_weights(lat.ctx, flat.astype(np.float32))
    W, b = unpack(mrhs_nn_get_weights(lat.ctx, 1), widths)
    return lat, W, b


def infer(lat, x, nrhs):
    y = lat.field(nrhs, MRHS_F32)
    pkg.mrhs_profile(lat.ctx, 1)
    mrhs_nn_infer(lat.ctx, lat.to_device(x, MRHS_F32), y, nrhs)
    ran = pkg.mrhs_profile_read(lat.ctx)
    pkg.mrhs_profile(lat.ctx, 0)
    return lat.to_host(y, nrhs, MRHS_F32), ran


@pytest.mark.parametrize("widths,nrhs,rounds", [((4, 32, 32, 4), 13, True), ((4, 16, 21, 4), 6, True)],
                         ids=["32-wide", "ragged"])
def test_infer_tensor_cores_exact(widths, nrhs, rounds):
    """13 right-hand sides run as chunks of 8 and 5 (tiles of 8 and 12
    sites; 512 = 42 x 12 + 8 leaves a ragged last tile); 6 as one chunk of
    tiles of 10 sites, with 16 and 21 hidden channels (operand K of 32 and 48
    per step). The hidden values need more than 8 significant bits, so the
    bf16 rounding of the operands shows in the output."""
    rng = np.random.default_rng(5301)
    nw, nb = oracle.nn_sizes(widths)
    mask = rng.random(nw) < 0.25
    W = mask * (rng.integers(-2, 3, nw) / 2 + 1j * rng.integers(-2, 3, nw) / 2)
    flat = np.zeros(2 * nw + nb)
    flat[0:2 * nw:2], flat[1:2 * nw:2] = W.real, W.imag
    U = monomial_links(5302)
    lat, Wk, b = make(U, widths, flat)
    assert np.array_equal(Wk, W) and not b.any()
    x = rng.integers(-1, 2, (nrhs, lat.V, 12)) + 1j * rng.integers(-1, 2, (nrhs, lat.V, 12))
    y, ran = infer(lat, x.astype(np.complex128), nrhs)
    assert "nn_covconv_tc" in ran and "nn_covconv" not in ran, ran
    ref = oracle.nn_forward_bf16act(DIMS, U, widths, W, b, x)
    assert np.array_equal(y, ref), float(np.abs(y - ref).max())
    # the hidden fields were rounded where they needed it
    assert np.array_equal(ref, oracle.nn_forward(DIMS, U, widths, W, b, x)) != rounds
    lat.close()


@pytest.mark.parametrize("widths,nrhs,scale", [((4, 32, 32, 4), 13, 0.15), ((4, 24, 16, 4), 1, 0.25)],
                         ids=["32-wide", "24-16"])
def test_infer_tensor_cores_generic(widths, nrhs, scale):
    rng = np.random.default_rng(5201)
    nw, nb = oracle.nn_sizes(widths)
    flat = np.concatenate([scale * rng.standard_normal(2 * nw), 0.3 * rng.standard_normal(nb)])
    U = inputs.gauge_field(DIMS, 0.4, 5101)
    lat, W, b = make(U, widths, flat)
    x = inputs.gaussian_field((nrhs, lat.V, 12), 5202)
    y, ran = infer(lat, x, nrhs)
    assert "nn_covconv_tc" in ran, ran
    ref = oracle.nn_forward_bf16act(DIMS, U, widths, W, b, x)
    assert rel(y, ref) < 1.5e-3
    lat.close()


@pytest.mark.parametrize("widths,bf16", [((4, 8, 6, 4), 0), ((4, 32, 32, 4), 0), ((4, 11, 11, 4), 1)],
                         ids=["fp32-weights", "fp32-weights-32", "bf16-11-wide"])
def test_infer_cuda_core_layers(widths, bf16):
    nrhs = 3
    rng = np.random.default_rng(5401)
    nw, nb = oracle.nn_sizes(widths)
    flat = np.concatenate([0.25 * rng.standard_normal(2 * nw), 0.3 * rng.standard_normal(nb)])
    U = inputs.gauge_field(DIMS, 0.4, 5402)
    lat, W, b = make(U, widths, flat, bf16=bf16)
    x = inputs.gaussian_field((nrhs, lat.V, 12), 5403)
    y, ran = infer(lat, x, nrhs)
    assert "nn_covconv" in ran and "nn_covconv_tc" not in ran, ran
    assert rel(y, oracle.nn_forward(DIMS, U, widths, W, b, x)) < 1e-4
    lat.close()
