"""Every kernel form that a supported right-hand-side count, storage type or
environment switch selects, against the FP64 oracle through the C ABI:

- the SAP smoother (Sec. 2) with 2 right-hand sides per on-chip chunk
  (k_sap_tm2: nrhs = 2 mod 4), with an odd count (k_sap_fused, one per
  thread), and the forms the switches MRHS_SAP_KERNEL=smem (k_sap_fused8 /
  k_sap_fused), MRHS_SAP_CHUNK=2 and MRHS_SAP_CPB=1 select;
- the stencil D with bf16 and fp16 storage (FP32 arithmetic) and in several
  passes over the right-hand sides (MRHS_STENCIL_PASSES);
- the coarse stencil on the CUDA cores (MRHS_DC_APPLY=alu);
- the Adam step of the learned generator against the update written out.

Switch-selected forms run in a child process (tests/variant_check.py): the
library reads its switches once per process.

Bounds: FP32 work 1e-5 relative (as for the default forms). Reduced storage:
every output entry is the FP32 result rounded once to the storage type, so
|y - y_ref| <= u |y_ref| + 1e-5 max|y_ref| entrywise, u = 2^-8 (bf16) or
2^-11 (fp16) the unit roundoff, with the oracle applied to the same rounded
input.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
import paper_1601_03184_gb300 as pkg
from paper_1601_03184_gb300 import MRHS_BF16, MRHS_F16, MRHS_F32, MRHS_PREC_FP32, Lattice, inputs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
P4 = dict(dims=(8, 8, 8, 8), agg=(4, 4, 4, 4), eps=0.4, m0=-0.1, csw=1.2, gseed=1301)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def make(cfg, ntv=8):
    U = inputs.gauge_field(cfg["dims"], cfg["eps"], cfg["gseed"])
    A = oracle.clover(cfg["dims"], U, cfg["m0"], cfg["csw"])
    lat = Lattice(cfg["dims"], cfg["agg"], ntv, MRHS_PREC_FP32)
    lat.set_gauge(U)
    lat.build_clover(cfg["m0"], cfg["csw"])
    return lat, U, A


@pytest.mark.parametrize("nrhs,kernel", [(4, "sap_pk"), (8, "sap_pk"), (6, "sap_tm2"), (10, "sap_tm2"),
                                          (5, "sap_fused"), (1, "sap_fused")])
def test_sap_fp32_other_widths(nrhs, kernel):
    """nrhs = 2 mod 4 takes the two-per-chunk on-chip kernel, an odd nrhs the
    one-per-thread form; two sweeps from a nonzero start on 4^4 domains."""
    lat, U, A = make(P4)
    b = inputs.gaussian_field((nrhs, lat.V, 12), 761)
    x0 = 0.1 * inputs.gaussian_field((nrhs, lat.V, 12), 762)
    xd = lat.to_device(x0, MRHS_F32)
    pkg.mrhs_profile(lat.ctx, 1)
    lat.sap(lat.to_device(b, MRHS_F32), xd, nrhs, MRHS_F32, 2, 4)
    ran = pkg.mrhs_profile_read(lat.ctx)
    assert kernel in ran, ran
    ref = oracle.sap(P4["dims"], P4["agg"], U, A, b, x0, 2, 4)
    assert rel(lat.to_host(xd, nrhs, MRHS_F32), ref) < 1e-5
    lat.close()


def _round_to(x, dt):
    """x (complex128) rounded to bf16 or fp16 part by part (round to nearest even)"""
    t = torch.from_numpy(np.stack([x.real, x.imag])).float()
    t = t.to(torch.bfloat16 if dt == MRHS_BF16 else torch.float16).double().numpy()
    return t[0] + 1j * t[1]


@pytest.mark.parametrize("dt,u", [(MRHS_BF16, 2.0 ** -8), (MRHS_F16, 2.0 ** -11)], ids=["bf16", "fp16"])
@pytest.mark.parametrize("nrhs", [4, 7])
def test_apply_D_reduced_storage(dt, u, nrhs):
    lat, U, A = make(P4)
    x = _round_to(inputs.gaussian_field((nrhs, lat.V, 12), 771), dt)
    xd = lat.to_device(x, dt)
    # the device field holds exactly the rounded values
    assert np.array_equal(lat.to_host(xd, nrhs, dt), x)
    yd = lat.field(nrhs, dt)
    lat.apply_D(xd, yd, nrhs, dt)
    y = lat.to_host(yd, nrhs, dt)
    ref = oracle.apply_D(P4["dims"], U, A, x)
    bound = u * np.abs(ref) + 1e-5 * np.abs(ref).max()
    assert (np.abs(y - ref) <= bound).all(), float((np.abs(y - ref) / bound).max())
    assert rel(y, ref) < u
    lat.close()


def _child(env, kind, nrhs):
    out = subprocess.run([sys.executable, os.path.join(HERE, "variant_check.py"), kind, str(nrhs)],
                         env=dict(os.environ, **env), capture_output=True, text=True, timeout=600,
                         cwd=os.path.dirname(HERE))
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("env,kind,nrhs,kernel,tol", [
    ({"MRHS_SAP_KERNEL": "smem"}, "sap", 8, "sap_fused8", 1e-5),
    ({"MRHS_SAP_KERNEL": "smem"}, "sap", 6, "sap_fused", 1e-5),
    ({"MRHS_SAP_KERNEL": "tm", "MRHS_SAP_CHUNK": "2"}, "sap", 8, "sap_tm2", 1e-5),
    ({"MRHS_SAP_KERNEL": "tm"}, "sap", 8, "sap_tm", 1e-5),
    ({"MRHS_SAP_KERNEL": "tm", "MRHS_SAP_CPB": "1"}, "sap", 8, "sap_tm", 1e-5),
    ({"MRHS_STENCIL_PASSES": "2"}, "apply_D", 8, "dslash_full", 1e-5),
    ({"MRHS_DC_APPLY": "alu"}, "apply_Dc", 16, "apply_dc", 1e-5),
    ({"MRHS_SAP_PK": "1g"}, "sap", 8, "sap_pk", 1e-5),
    ({"MRHS_SAP_PK": "1g"}, "sap", 6, "sap_pk", 1e-5),
    ({"MRHS_SAP_PK": "1g", "MRHS_SAP_CPB": "2"}, "sap", 8, "sap_pk", 1e-5),
    ({"MRHS_SAP_PK": "2s"}, "sap", 8, "sap_pk", 1e-5),
    ({"MRHS_SAP_PK": "2s", "MRHS_SAP_CPB": "1"}, "sap", 8, "sap_pk", 1e-5),
    ({}, "restrict", 8, "restrict", 1e-5),
    ({}, "restrict", 6, "restrict", 1e-5),
    ({"MRHS_RESTRICT": "tiled"}, "restrict", 8, "restrict", 1e-5),
    ({}, "prolong", 8, "prolong", 1e-5),
    ({}, "prolong", 6, "prolong", 1e-5),
], ids=["smem-fused8", "smem-fused2", "chunk2", "tm", "tm-cpb1", "passes2", "dc-alu", "pk1g", "pk1g-6", "pk1g-cpb2",
        "pk2s", "pk2s-cpb1", "restrict-stream", "restrict-tiled-6", "restrict-tiled", "prolong-4", "prolong-6"])
def test_switch_selected_forms(env, kind, nrhs, kernel, tol):
    r = _child(env, kind, nrhs)
    assert kernel in r["kernels"], r
    assert r["rel"] < tol, r


def test_adam_step_written_out():
    """Three Adam steps (gradients from three backward passes) against the
    update restated on the host in FP64: per real parameter
    m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
    w -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)."""
    lat, U, A = make(P4)
    widths = (4, 6, 6, 4)
    pkg.mrhs_nn_create(lat.ctx, widths, 0)
    nc, nr = pkg.mrhs_nn_num_params(lat.ctx)
    rng = np.random.default_rng(781)
    w = (0.2 * rng.standard_normal(2 * nc + nr)).astype(np.float32)
    pkg.mrhs_nn_set_weights(lat.ctx, w)
    nrhs = 2
    x = lat.to_device(inputs.gaussian_field((nrhs, lat.V, 12), 782), MRHS_F32)
    y = lat.field(nrhs, MRHS_F32)
    go = lat.to_device(inputs.gaussian_field((nrhs, lat.V, 12), 783), MRHS_F32)
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-8
    W = w.astype(np.float64)
    m = np.zeros_like(W)
    v = np.zeros_like(W)
    for t in (1, 2, 3):
        pkg.mrhs_nn_zero_grads(lat.ctx)
        pkg.mrhs_nn_forward(lat.ctx, x, y, nrhs)
        pkg.mrhs_nn_backward(lat.ctx, go, None, nrhs)
        g = pkg.mrhs_nn_get_grads(lat.ctx).astype(np.float64)
        assert np.abs(g).max() > 0
        pkg.mrhs_nn_adam(lat.ctx, lr, b1, b2, eps, t)
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        W = W - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
        got = pkg.mrhs_nn_get_weights(lat.ctx, 0).astype(np.float64)
        # FP32 arithmetic on the device: a few ulps of w plus of the step
        assert np.abs(got - W).max() <= 1e-6 * (np.abs(W).max() + lr), (t, float(np.abs(got - W).max()))
        W = got  # continue from the device's weights (its rounding)
    lat.close()
