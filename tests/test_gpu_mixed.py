"""Reduced-precision setups (FP32, and bf16 / fp16 test-vector storage with
FP32 work) against the FP64 CPU oracle, on an 8^4 lattice with the paper's
4^4 domains.

Per-result errors (the stated bounds):
  P:   sine of the largest principal angle between the ranges of P_gpu and
       P_oracle on every aggregate x chirality (P is determined up to its
       range by the test vectors, which carry the rounding of the storage);
  D_c: Frobenius norm of D_c,gpu - D_c,oracle relative to that of D_c,oracle;
  FGMRES: two-level FGMRES on D x = b to 1e-10 with the GPU setup needs
  the oracle's iteration count within +-10% (at least +-1).
The errors scale with the storage unit roundoff u (fp32 6e-8, fp16 4.9e-4,
bf16 3.9e-3) carried through the smoother iterations of the setup; there is
no a-priori bound for an iterative procedure with tolerance-based coarse
solves, so the bounds are the values measured on a GB300 (the setup is
deterministic: the same inputs give the same bits) times 3:
  P sine  9.7e-7 (fp32, 16u), 1.07e-3 (fp16, 2.2u), 7.8e-3 (bf16, 2.0u)
          -> bounds 3e-6, 3.5e-3, 2.5e-2;
  D_c     8.5e-7, 1.9e-4, 1.5e-3 -> bounded by the same numbers.
"""
import numpy as np
import pytest

import oracle
from paper_1601_03184_gb300 import (MRHS_F32, MRHS_PREC_FP32, MRHS_PREC_MIX_BF16, MRHS_PREC_MIX_FP16, Lattice,
                                    inputs)
from lattice_helpers import aggregate_of_sites

pytestmark = pytest.mark.gpu

CFG = dict(dims=(8, 8, 8, 8), agg=(4, 4, 4, 4), ntv=8, eps=0.3, m0=-0.2, csw=1.0, gseed=1201, tvseed=2201)
SCHED = dict(init_sweeps=3, init_mr=4, n_refine=2, sweeps=4, mr=4, ctol=0.05, crestart=20, cmaxit=200)
BOUNDS = {MRHS_PREC_FP32: 3e-6, MRHS_PREC_MIX_FP16: 3.5e-3, MRHS_PREC_MIX_BF16: 2.5e-2}


@pytest.fixture(scope="module")
def reference():
    dims, agg, ntv = CFG["dims"], CFG["agg"], CFG["ntv"]
    U = inputs.gauge_field(dims, CFG["eps"], CFG["gseed"])
    A = oracle.clover(dims, U, CFG["m0"], CFG["csw"])
    tv0 = inputs.test_vectors(ntv, dims, CFG["tvseed"])
    prm = oracle.make_params(n_init_sweeps=SCHED["init_sweeps"], n_init_mr=SCHED["init_mr"],
                             n_refine=SCHED["n_refine"], n_smooth_sweeps=SCHED["sweeps"], n_smooth_mr=SCHED["mr"],
                             coarse_tol=SCHED["ctol"], coarse_restart=SCHED["crestart"], coarse_maxit=SCHED["cmaxit"])
    tv, P, Dc = oracle.setup_init(dims, agg, U, A, tv0, prm)
    tv, P, Dc, _ = oracle.setup_refine(dims, agg, U, A, tv, P, Dc, prm)
    b = inputs.gaussian_field((int(np.prod(dims)), 12), 3201)
    _, its, _ = oracle.fgmres(dims, agg, U, A, P, Dc, b, tol=1e-10)
    return dict(U=U, tv0=tv0, P=P, Dc=Dc, b=b, its=its)


def max_subspace_sine(Pa, Pb, dims, agg):
    Ag = aggregate_of_sites(dims, agg)
    worst = 0.0
    for a in np.unique(Ag):
        sites = np.where(Ag == a)[0]
        for h in range(2):
            Qa = Pa[:, sites, 6 * h:6 * h + 6].reshape(Pa.shape[0], -1).T
            Qb = Pb[:, sites, 6 * h:6 * h + 6].reshape(Pb.shape[0], -1).T
            Qa, _ = np.linalg.qr(Qa)  # re-orthonormalise (reduced-precision P is orthonormal only to ~u)
            Qb, _ = np.linalg.qr(Qb)
            worst = max(worst, np.linalg.norm(Qa - Qb @ (Qb.conj().T @ Qa), 2))
    return worst


@pytest.mark.parametrize("prec", [MRHS_PREC_FP32, MRHS_PREC_MIX_FP16, MRHS_PREC_MIX_BF16],
                         ids=["fp32", "fp16", "bf16"])
def test_reduced_precision_setup(reference, prec):
    dims, agg, ntv = CFG["dims"], CFG["agg"], CFG["ntv"]
    lat = Lattice(dims, agg, ntv, prec)
    lat.set_gauge(reference["U"])
    lat.build_clover(CFG["m0"], CFG["csw"])
    lat.setup_init(lat.to_device(reference["tv0"].astype(np.complex64), MRHS_F32), MRHS_F32, 0,
                   SCHED["init_sweeps"], SCHED["init_mr"])
    lat.setup_refine(SCHED["n_refine"], SCHED["sweeps"], SCHED["mr"], SCHED["ctol"], SCHED["crestart"],
                     SCHED["cmaxit"])
    P = lat.get_P()
    Dc = lat.get_Dc()
    sine = max_subspace_sine(P, reference["P"], dims, agg)
    dc_err = np.linalg.norm(Dc - reference["Dc"]) / np.linalg.norm(reference["Dc"])
    x, its, rr = lat.solve_fgmres(reference["b"], tol=1e-10, restart=25, maxit=400)
    print("prec %d: P sine %.3e, Dc rel %.3e, FGMRES %d (oracle %d)" % (prec, sine, dc_err, its, reference["its"]))
    assert sine <= BOUNDS[prec]
    assert dc_err <= BOUNDS[prec]
    assert rr <= 1e-10
    assert abs(its - reference["its"]) <= max(1, 0.1 * reference["its"])
