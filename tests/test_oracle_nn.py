"""Pins of the oracle's learned test-vector generator (gauge-covariant
convolution network) and of its training loss: central finite differences of
every parameter class and of the input, gauge covariance, and the identity
network."""
import numpy as np
import pytest

import oracle
from paper_1601_03184_gb300 import inputs
from lattice_helpers import colour_rotate, gauge_transform, vol

DIMS = (2, 2, 2, 4)
WIDTHS = (4, 3, 2, 4)


def params(seed, widths=WIDTHS, scale=0.3):
    nw, nb = oracle.nn_sizes(widths)
    rng = np.random.default_rng(seed)
    W = scale * (rng.standard_normal(nw) + 1j * rng.standard_normal(nw))
    b = 0.2 * rng.standard_normal(nb)
    return W, b


def net_loss(U, W, b, x, dout_weights, linear=False):
    out = oracle.nn_forward(DIMS, U, WIDTHS, W, b, x, linear)
    # a real loss with a known gradient: L = sum Re(conj(c) out) + |out|^2
    return float(np.sum((np.conj(dout_weights) * out).real) + np.sum(np.abs(out) ** 2)), out


@pytest.mark.parametrize("linear", [False, True])
def test_nn_gradients_by_central_differences(linear):
    U = inputs.gauge_field(DIMS, 0.5, 11)
    W, b = params(12)
    x = inputs.gaussian_field((2, vol(DIMS), 12), 13)
    cw = inputs.gaussian_field((2, vol(DIMS), 12), 14)
    L0, out = net_loss(U, W, b, x, cw, linear)
    dout = cw + 2 * out  # dL/dRe(out) + i dL/dIm(out)
    gW, gb, din = oracle.nn_backward(DIMS, U, WIDTHS, W, b, x, dout, linear, want_din=True)
    h = 1e-6
    rng = np.random.default_rng(15)
    for i in rng.choice(len(W), 12, replace=False):
        for part, unit in ((gW[i].real, 1.0), (gW[i].imag, 1j)):
            Wp, Wm = W.copy(), W.copy()
            Wp[i] += h * unit
            Wm[i] -= h * unit
            fd = (net_loss(U, Wp, b, x, cw, linear)[0] - net_loss(U, Wm, b, x, cw, linear)[0]) / (2 * h)
            assert abs(fd - part) <= 1e-6 * max(1.0, abs(fd))
    if not linear:
        for i in range(len(b)):
            bp, bm = b.copy(), b.copy()
            bp[i] += h
            bm[i] -= h
            fd = (net_loss(U, W, bp, x, cw)[0] - net_loss(U, W, bm, x, cw)[0]) / (2 * h)
            assert abs(fd - gb[i]) <= 1e-6 * max(1.0, abs(fd))
    for (r, s, c) in [(0, 0, 0), (1, 7, 5), (0, 15, 11)]:
        for unit, part in ((1.0, din[r, s, c].real), (1j, din[r, s, c].imag)):
            xp, xm = x.copy(), x.copy()
            xp[r, s, c] += h * unit
            xm[r, s, c] -= h * unit
            fd = (net_loss(U, W, b, xp, cw, linear)[0] - net_loss(U, W, b, xm, cw, linear)[0]) / (2 * h)
            assert abs(fd - part) <= 1e-6 * max(1.0, abs(fd))


def test_nn_is_gauge_covariant():
    dims = (4, 4, 4, 4)
    U = inputs.gauge_field(dims, 0.5, 21)
    widths = (4, 5, 5, 4)
    W, b = params(22, widths)
    x = inputs.gaussian_field((1, vol(dims), 12), 23)
    Om = inputs.random_su3(vol(dims), 24)
    y = oracle.nn_forward(dims, U, widths, W, b, x)
    yt = oracle.nn_forward(dims, gauge_transform(dims, U, Om), widths, W, b, colour_rotate(Om, x))
    assert np.abs(yt - colour_rotate(Om, y)).max() < 1e-12 * np.abs(y).max()


def test_identity_network():
    """Linear net with W_0 = identity on channels at k = 0 and every other
    weight zero returns its input."""
    widths = (4, 4, 4, 4)
    nw, nb = oracle.nn_sizes(widths)
    W = np.zeros(nw, np.complex128)
    for layer in range(3):
        off = layer * 9 * 16
        for c in range(4):
            W[off + c * 4 + c] = 1.0  # k = 0 block of layer `layer`
    U = inputs.gauge_field(DIMS, 0.5, 31)
    x = inputs.gaussian_field((2, vol(DIMS), 12), 32)
    y = oracle.nn_forward(DIMS, U, widths, W, np.zeros(nb), x, linear=True)
    assert np.abs(y - x).max() < 1e-15


def test_modrelu_closed_form():
    """The nonlinearity between layers written out: every colour triplet z
    of a hidden channel c becomes z max(0, |z| + b_c) / |z| (|z| the norm of
    the triplet, 0 for z = 0). Network: layer 1 mixes the four input channels
    at the site only (k = 0), layers 2 and 3 are the identity, the second
    bias is 0 (so the second modReLU is the identity), the first has both
    signs, with magnitudes that switch some triplets off and leave others
    shrunk or grown. A bias entering as |z| - b, a norm over the wrong index
    or a missing division by |z| fails this."""
    widths = (4, 4, 4, 4)
    nw, nb = oracle.nn_sizes(widths)
    rng = np.random.default_rng(51)
    W1 = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    W = np.zeros(nw, np.complex128)
    W[:16] = W1.reshape(-1)  # layer 1, k = 0, [c_out][c_in]
    for layer in (1, 2):
        off = layer * 9 * 16
        for c in range(4):
            W[off + c * 4 + c] = 1.0
    x = inputs.gaussian_field((2, vol(DIMS), 12), 52)
    z = np.einsum("oi,rsic->rsoc", W1, x.reshape(2, vol(DIMS), 4, 3))
    mag = np.linalg.norm(z, axis=-1)
    b1 = np.array([-0.8, 0.5, -0.3 * np.median(mag), -1.5 * np.median(mag)])
    bias = np.concatenate([b1, np.zeros(4)])
    U = inputs.gauge_field(DIMS, 0.5, 53)
    y = oracle.nn_forward(DIMS, U, widths, W, bias, x)
    gain = np.maximum(0.0, mag + b1[None, None, :]) / mag
    ref = (z * gain[..., None]).reshape(x.shape)
    assert np.abs(y - ref).max() < 1e-13 * np.abs(ref).max()
    # the chosen biases exercise every regime
    assert (gain[..., 3] == 0).any() and (gain[..., 3] > 0).any() and (gain[..., 1] > 1).all()


def test_loss_gradient_by_central_differences():
    dims, agg, ntv = (4, 4, 4, 4), (2, 2, 2, 2), 4
    U = inputs.gauge_field(dims, 0.3, 41)
    A = oracle.clover(dims, U, -0.2, 1.0)
    P = oracle.gram_schmidt(dims, agg, inputs.test_vectors(ntv, dims, 42))
    v = inputs.gaussian_field((2, vol(dims), 12), 43)
    lam = 0.7
    L, dv = oracle.nn_loss(dims, agg, U, A, P, v, lam)
    # the loss itself from its definition with dense operators
    from lattice_helpers import dense_D, dense_P
    Dm = dense_D(dims, U, A)
    Pm = dense_P(dims, agg, P)
    ref = 0.0
    for r in range(2):
        vr = v[r].reshape(-1)
        q = vr - Pm @ (Pm.conj().T @ vr)
        ref += np.linalg.norm(Dm @ vr) ** 2 / np.linalg.norm(vr) ** 2 + lam * np.linalg.norm(q) ** 2 / np.linalg.norm(vr) ** 2
    assert abs(L - ref) < 1e-12 * ref
    h = 1e-6
    for (r, s, c) in [(0, 3, 2), (1, 100, 7), (1, 255, 11)]:
        for unit, part in ((1.0, dv[r, s, c].real), (1j, dv[r, s, c].imag)):
            vp, vm = v.copy(), v.copy()
            vp[r, s, c] += h * unit
            vm[r, s, c] -= h * unit
            fd = (oracle.nn_loss(dims, agg, U, A, P, vp, lam)[0] - oracle.nn_loss(dims, agg, U, A, P, vm, lam)[0]) / (2 * h)
            assert abs(fd - part) <= 1e-6 * max(1.0, abs(fd))


def _bf16(a):
    """complex array rounded part by part to FP32 and then to bfloat16 by
    torch (round to nearest, ties to even)"""
    import torch
    re = torch.from_numpy(np.ascontiguousarray(a.real)).float().to(torch.bfloat16).double().numpy()
    im = torch.from_numpy(np.ascontiguousarray(a.imag)).float().to(torch.bfloat16).double().numpy()
    return re + 1j * im


def _identity_weights(widths=(4, 4, 4, 4), first=None):
    nw, nb = oracle.nn_sizes(widths)
    W = np.zeros(nw, np.complex128)
    for layer in range(3):
        off = layer * 9 * 16
        if layer == 0 and first is not None:
            W[:first.size] = first
            continue
        for c in range(4):
            W[off + c * 4 + c] = 1.0
    return W, nb


def test_bf16_activation_rounding_is_round_to_nearest_even():
    """The identity network with bf16 operands returns its input
    rounded once to bfloat16 (rounding is idempotent), equal bit for bit to
    torch's conversion, on Gaussian values and on exact ties between two
    bfloat16 numbers (FP32 values whose low 16 bits are 0x8000, with even
    and odd upper halves)."""
    torch = pytest.importorskip("torch")
    W, nb = _identity_weights()
    U = inputs.gauge_field(DIMS, 0.5, 61)
    x = inputs.gaussian_field((1, vol(DIMS), 12), 62)
    rng = np.random.default_rng(63)
    hi = rng.integers(0x3f00, 0x4100, size=x.size).astype(np.uint32)
    ties = ((hi << 16) | 0x8000).astype(np.uint32).view(np.float32).astype(np.float64)
    x = x.copy()
    x.real.reshape(-1)[::2] = ties[::2]  # half of the real parts exact ties
    y = oracle.nn_forward_bf16act(DIMS, U, (4, 4, 4, 4), W, np.zeros(nb), x, linear=True)
    assert np.array_equal(y, _bf16(x))
    assert not np.array_equal(y, x)
    del torch


def _monomial_links(seed):
    """[V][4][3][3] matrices P diag(p), P a permutation, p in {±1, ±i}: the
    transport by them is exact and commutes with any rounding"""
    rng = np.random.default_rng(seed)
    U = np.zeros((vol(DIMS), 4, 3, 3), np.complex128)
    ph = np.array([1, 1j, -1, -1j])
    for s in range(vol(DIMS)):
        for mu in range(4):
            U[s, mu, np.arange(3), rng.permutation(3)] = ph[rng.integers(0, 4, 3)]
    return U


def test_bf16_rounding_after_the_transport():
    """The rounded operand is the transported triplet s_k T_k h(n_k), not the
    layer input: with layer 1 the identity on the +x hop only (k = 1) and
    layers 2 and 3 the identity at the site, a rough SU(3) field gives
    bf16(layer1(x)) bit for bit, which differs from rounding x first."""
    pytest.importorskip("torch")
    first = np.zeros(9 * 16, np.complex128)
    for c in range(4):
        first[1 * 16 + c * 4 + c] = 1.0  # k = 1 block of layer 1
    W, nb = _identity_weights(first=first)
    U = inputs.gauge_field(DIMS, 0.5, 91)
    x = inputs.gaussian_field((2, vol(DIMS), 12), 92)
    y = oracle.nn_forward_bf16act(DIMS, U, (4, 4, 4, 4), W, np.zeros(nb), x, linear=True)
    hop = oracle.nn_forward(DIMS, U, (4, 4, 4, 4), W, np.zeros(nb), x, linear=True)
    assert np.array_equal(y, _bf16(hop))
    before = _bf16(oracle.nn_forward(DIMS, U, (4, 4, 4, 4), W, np.zeros(nb), _bf16(x), linear=True))
    assert not np.array_equal(y, before)


def test_bf16_activation_rounding_placement():
    """With layers 2 and 3 the identity, a random first layer (all nine
    blocks) and links whose transport commutes with rounding, the
    bf16-operand forward equals bf16(layer1(bf16(x))) bit for bit: the
    operands of layer 1 and of layers 2 and 3 are rounded, and nothing else
    is."""
    pytest.importorskip("torch")
    rng = np.random.default_rng(71)
    first = rng.standard_normal(9 * 16) + 1j * rng.standard_normal(9 * 16)
    W, nb = _identity_weights(first=first)
    U = _monomial_links(72)
    x = inputs.gaussian_field((2, vol(DIMS), 12), 73)
    y = oracle.nn_forward_bf16act(DIMS, U, (4, 4, 4, 4), W, np.zeros(nb), x, linear=True)
    ref = _bf16(oracle.nn_forward(DIMS, U, (4, 4, 4, 4), W, np.zeros(nb), _bf16(x), linear=True))
    assert np.array_equal(y, ref)
    # and it differs from the unrounded forward by bf16-sized amounts only
    plain = oracle.nn_forward(DIMS, U, (4, 4, 4, 4), W, np.zeros(nb), x, linear=True)
    assert 1e-5 < np.linalg.norm(y - plain) / np.linalg.norm(plain) < 2 ** -7


def test_bf16_activation_output_not_rounded():
    """Layers 1 and 2 the identity, layer 3 random, links whose transport
    commutes with rounding: the bf16-operand forward is the plain forward of
    bf16(x) bit for bit, so the output of the last layer is not rounded."""
    pytest.importorskip("torch")
    rng = np.random.default_rng(81)
    last = rng.standard_normal(9 * 16) + 1j * rng.standard_normal(9 * 16)
    W, nb = _identity_weights()
    W[2 * 9 * 16:] = last
    U = _monomial_links(82)
    x = inputs.gaussian_field((2, vol(DIMS), 12), 83)
    y = oracle.nn_forward_bf16act(DIMS, U, (4, 4, 4, 4), W, np.zeros(nb), x, linear=True)
    assert np.array_equal(y, oracle.nn_forward(DIMS, U, (4, 4, 4, 4), W, np.zeros(nb), _bf16(x), linear=True))
    assert not np.array_equal(y, _bf16(y))
