"""The 16^3 x 32 workload end to end on the GPU against the oracle's stored
result (tests/golden/c2_fgmres.json, written by tests/golden/c2_fgmres.py
from the FP64 oracle only): the FP32 setup and the bf16 / fp16 mixed setups,
each followed by the two-level FGMRES solve on the same Gaussian right-hand
side to relative residual 1e-10. The iteration count must match the
oracle's within +-10% (at least +-1): the GPU runs Algorithm 2 (all test
vectors at once) where the oracle runs Algorithm 1 (one at a time), the same
computation in a different order, in reduced precision.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1601_03184_gb300 import (MRHS_F32, MRHS_PREC_FP32, MRHS_PREC_MIX_BF16, MRHS_PREC_MIX_FP16, Lattice,
                                    inputs)

pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c2_fgmres.json")))


@pytest.fixture(scope="module")
def problem():
    c = GOLDEN["case"]
    dims = tuple(c["dims"])
    U = inputs.gauge_field(dims, c["eps"], c["gseed"])
    tv0 = inputs.test_vectors(c["ntv"], dims, c["tvseed"]).astype(np.complex64)
    b = inputs.gaussian_field((int(np.prod(dims)), 12), c["bseed"])
    return dims, U, tv0, b


@pytest.mark.parametrize("prec", [MRHS_PREC_FP32, MRHS_PREC_MIX_BF16, MRHS_PREC_MIX_FP16],
                         ids=["fp32", "bf16", "fp16"])
def test_c2_setup_fgmres_iterations(problem, prec):
    dims, U, tv0, b = problem
    c, s, j = GOLDEN["case"], GOLDEN["schedule"], GOLDEN["solve"]
    lat = Lattice(dims, tuple(c["agg"]), c["ntv"], prec)
    lat.set_gauge(U)
    lat.build_clover(GOLDEN["m0"], c["csw"])
    lat.setup_init(lat.to_device(tv0, MRHS_F32), MRHS_F32, 0, s["init_sweeps"], s["init_mr"])
    lat.setup_refine(s["n_refine"], s["smooth_sweeps"], s["smooth_mr"], s["coarse_tol"], s["coarse_restart"],
                     s["coarse_maxit"])
    x, its, rr = lat.solve_fgmres(b, tol=j["tol"], restart=j["restart"], maxit=j["maxit"],
                                  coarse_tol=s["coarse_tol"], coarse_restart=s["coarse_restart"],
                                  coarse_maxit=s["coarse_maxit"], n_sweeps=s["smooth_sweeps"], n_mr=s["smooth_mr"])
    true_rr = oracle.relres(dims, U, oracle.clover(dims, U, GOLDEN["m0"], c["csw"]), b, x)
    ref = GOLDEN["iterations"]
    print("prec %d: FGMRES %d iterations (oracle %d), residual %.2e" % (prec, its, ref, true_rr))
    assert true_rr <= 1e-10 * 1.05
    assert abs(its - ref) <= max(1, 0.1 * ref)
