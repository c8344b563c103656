"""The mixed-precision workload: 32^3 x 64 lattice, N_tv = 24, 4^4
aggregates, roughness 0.6, c_sw 1.5, the setup schedule of the 16^3 x 32
workload. Test vectors stored in bf16 and in fp16 (two runs), the smoother
and the coarse grid in FP32, the D_c contraction on bf16 (bf16 run) or tf32
(fp16 run) tensor cores with FP32 accumulation, Gram-Schmidt reductions and
the FGMRES residual in FP64; beside them the plain FP32 setup.

Against the FP64 oracle's setup of the same inputs (tests/golden/c3_mixed.json
and .npz, written by tests/golden/c3_mixed.py from the oracle only):
  - the FGMRES iteration count at relative residual 1e-10 (the measure of setup quality):
    FP32 within +-10 % (at least +-1) of the oracle's count, bf16 and fp16
    within +-10 % of the plain FP32 GPU setup's count;
  - per-result errors on the stored aggregates (the first, one inside, the
    last): the largest principal-angle sine between range(P) and the
    oracle's range per aggregate and chirality, and the relative Frobenius
    error of the nine D_c blocks. A reduced-precision setup drifts from the
    FP64 one through many smoother and coarse iterations and the
    tolerance-based coarse solves, so no a-priori bound exists; the setup is
    deterministic, and the bounds are the values measured on a GB300 times 3:
      FP32  P sine 2.6e-6, D_c 1.3e-6            -> 8e-6
      bf16  P sine 1.47e-2 (3.8u), D_c 2.5e-3    -> 4.5e-2
      fp16  P sine 1.87e-3 (3.8u), D_c 3.0e-4    -> 6e-3
    (u the storage unit roundoff); FGMRES: 25 iterations in all three, as
    the oracle's setup.
Needs about 30 GB of device memory and 30 GB of host memory.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1601_03184_gb300 import (MRHS_F32, MRHS_PREC_FP32, MRHS_PREC_MIX_BF16, MRHS_PREC_MIX_FP16, Lattice,
                                    inputs)

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = json.load(open(os.path.join(HERE, "golden", "c3_mixed.json")))
STORED = np.load(os.path.join(HERE, "golden", "c3_mixed.npz"))
RESULTS = {}


def aggregate_rows(dims, agg, A):
    """canonical sites of aggregate A in lexicographic order inside it"""
    nb = [d // a for d, a in zip(dims, agg)]
    bc = np.array(np.unravel_index(A, nb[::-1])[::-1])
    loc = np.stack(np.unravel_index(np.arange(int(np.prod(agg))), tuple(agg[::-1]))[::-1], axis=1)
    c = loc + bc[None, :] * np.asarray(agg)[None, :]
    return c[:, 0] + dims[0] * (c[:, 1] + dims[1] * (c[:, 2] + dims[2] * c[:, 3]))


def subspace_sine(Pa, Pb):
    """largest principal-angle sine between the column ranges of [n, L] x ntv
    blocks, per chirality"""
    worst = 0.0
    for h in range(2):
        Qa = Pa[:, :, 6 * h:6 * h + 6].reshape(Pa.shape[0], -1).T.astype(np.complex128)
        Qb = Pb[:, :, 6 * h:6 * h + 6].reshape(Pb.shape[0], -1).T.astype(np.complex128)
        Qa, _ = np.linalg.qr(Qa)
        Qb, _ = np.linalg.qr(Qb)
        worst = max(worst, np.linalg.norm(Qa - Qb @ (Qb.conj().T @ Qa), 2))
    return worst


@pytest.fixture(scope="module")
def problem():
    c = GOLDEN["case"]
    dims = tuple(c["dims"])
    U = inputs.gauge_field(dims, c["eps"], c["gseed"], device="cuda")
    tv0 = inputs.test_vectors(c["ntv"], dims, c["tvseed"]).astype(np.complex64)
    b = inputs.gaussian_field((int(np.prod(dims)), 12), c["bseed"])
    return dims, U, tv0, b


def run_setup(problem, prec):
    import torch

    dims, U, tv0, b = problem
    c, s, j = GOLDEN["case"], GOLDEN["schedule"], GOLDEN["solve"]
    agg = tuple(c["agg"])
    lat = Lattice(dims, agg, c["ntv"], prec)
    lat.set_gauge(U)
    lat.build_clover(GOLDEN["m0"], c["csw"])
    lat.setup_init(lat.to_device(tv0, MRHS_F32), MRHS_F32, 0, s["init_sweeps"], s["init_mr"])
    lat.setup_refine(s["n_refine"], s["smooth_sweeps"], s["smooth_mr"], s["coarse_tol"], s["coarse_restart"],
                     s["coarse_maxit"])
    P = lat.get_P(MRHS_F32)
    Dc = lat.get_Dc(MRHS_F32)
    sines, dcerr = [], []
    for i, A in enumerate(STORED["aggregates"]):
        rows = aggregate_rows(dims, agg, int(A))
        sines.append(subspace_sine(P[:, rows, :], STORED["P"][i]))
        ref = STORED["Dc"][i].astype(np.complex128)
        dcerr.append(float(np.linalg.norm(Dc[int(A)] - ref) / np.linalg.norm(ref)))
    del P, Dc
    x, its, rr = lat.solve_fgmres(b, tol=j["tol"], restart=j["restart"], maxit=j["maxit"],
                                  coarse_tol=s["coarse_tol"], coarse_restart=s["coarse_restart"],
                                  coarse_maxit=s["coarse_maxit"], n_sweeps=s["smooth_sweeps"], n_mr=s["smooth_mr"],
                                  allow_noconv=True)
    lat.close()
    torch.cuda.empty_cache()
    res = {"fgmres": int(its), "relres": float(rr), "P_sine": float(max(sines)), "Dc_rel": float(max(dcerr))}
    print("prec %d: %s (oracle FGMRES %d)" % (prec, json.dumps(res), GOLDEN["iterations"]))
    return res


def test_c3_fp32_setup_against_oracle(problem):
    r = run_setup(problem, MRHS_PREC_FP32)
    RESULTS[MRHS_PREC_FP32] = r
    ref = GOLDEN["iterations"]
    assert r["relres"] <= 1e-10
    assert abs(r["fgmres"] - ref) <= max(1, 0.1 * ref)
    assert r["P_sine"] < 8e-6 and r["Dc_rel"] < 8e-6


@pytest.mark.parametrize("prec", [MRHS_PREC_MIX_BF16, MRHS_PREC_MIX_FP16], ids=["bf16", "fp16"])
def test_c3_mixed_setup_against_fp32_and_oracle(problem, prec):
    if MRHS_PREC_FP32 not in RESULTS:
        RESULTS[MRHS_PREC_FP32] = run_setup(problem, MRHS_PREC_FP32)
    plain = RESULTS[MRHS_PREC_FP32]["fgmres"]
    r = run_setup(problem, prec)
    assert r["relres"] <= 1e-10
    assert abs(r["fgmres"] - plain) <= max(1, 0.1 * plain)
    bound = {MRHS_PREC_MIX_BF16: 4.5e-2, MRHS_PREC_MIX_FP16: 6e-3}[prec]
    assert r["P_sine"] < bound and r["Dc_rel"] < bound
