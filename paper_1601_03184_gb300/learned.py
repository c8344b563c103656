"""Training and use of the learned test-vector generator through the C ABI
(orchestration only: every step runs in the library's kernels).

Initial weights: the identity network (k = 0, channel c -> c for the first
four channels of every layer, biases 0, so modReLU passes its input through)
plus seeded complex Gaussian noise of size `noise`.
"""
from __future__ import annotations

import numpy as np

from . import (MRHS_F32, mrhs_nn_create, mrhs_nn_num_params, mrhs_nn_set_weights, mrhs_nn_train_step,
               mrhs_sap, mrhs_setup_init, mrhs_setup_init_learned, mrhs_setup_refine)

# 4 -> 11 -> 11 -> 4 colour triplets: 12 -> 33 -> 33 -> 12 complex channels
# per site, the gauge-covariant width closest to 32 complex channels
WIDTHS = (4, 11, 11, 4)


def initial_weights(widths=WIDTHS, seed=7, noise=0.01):
    c0, c1, c2, c3 = widths
    sizes = [9 * c1 * c0, 9 * c2 * c1, 9 * c3 * c2]
    rng = np.random.Generator(np.random.PCG64(seed))
    w = []
    for (cin, cout), n in zip(((c0, c1), (c1, c2), (c2, c3)), sizes):
        W = noise * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
        W = W.reshape(9, cout, cin)
        for c in range(min(cin, cout, 4)):
            W[0, c, c] += 1.0
        w.append(W.reshape(-1))
    W = np.concatenate(w)
    flat = np.empty(2 * W.size + c1 + c2, np.float32)
    flat[0:2 * W.size:2] = W.real
    flat[1:2 * W.size:2] = W.imag
    flat[2 * W.size:] = 0.0
    return flat


def attach(lat, widths=WIDTHS, seed=7, noise=0.01, bf16=True):
    mrhs_nn_create(lat.ctx, widths, 1 if bf16 else 0)
    mrhs_nn_set_weights(lat.ctx, initial_weights(widths, seed, noise))


def sap_vectors(lat, seed, n_sweeps=1, n_mr=4):
    """Gaussian vectors (drawn on the device, seeded) after n_sweeps SAP sweeps from x0 = 0."""
    import torch

    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    b = torch.randn(lat.field(lat.ntv, MRHS_F32).numel() // 4, generator=g, device="cuda")
    x = torch.zeros_like(b)
    mrhs_sap(lat.ctx, b, x, lat.ntv, MRHS_F32, n_sweeps, n_mr)
    return b, x


def train_on_field(lat, plain_schedule, steps, seed, lr=1e-3, lam=1.0, first_step=1):
    """Plain setup on the context's current gauge field (its P is the target
    span), then `steps` Adam steps on fresh 1-sweep vectors. Returns losses."""
    import torch

    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    tv0 = torch.randn(lat.field(lat.ntv, MRHS_F32).numel() // 4, generator=g, device="cuda")
    s = plain_schedule
    mrhs_setup_init(lat.ctx, tv0, MRHS_F32, 0, s["init_sweeps"], s["init_mr"])
    mrhs_setup_refine(lat.ctx, s["n_refine"], s["sweeps"], s["mr"], s["ctol"], s["crestart"], s["cmaxit"])
    losses = []
    for i in range(steps):
        _, x = sap_vectors(lat, seed * 1000 + i, 1, s["init_mr"])
        losses.append(mrhs_nn_train_step(lat.ctx, x, lat.ntv, lam, lr, first_step + i))
    return losses


def learned_setup(lat, tv0, schedule, n_sweeps=1):
    """Initial phase with one SAP sweep and the network, then the refinement."""
    s = schedule
    mrhs_setup_init_learned(lat.ctx, tv0, MRHS_F32, n_sweeps, s["init_mr"])
    mrhs_setup_refine(lat.ctx, s["n_refine"], s["sweeps"], s["mr"], s["ctol"], s["crestart"], s["cmaxit"])
