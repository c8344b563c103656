"""Iteration count of the two-level FGMRES solve after the plain FP64 setup,
computed by the CPU oracle only, on the 16^3 x 32 workload: roughness 0.6,
c_sw 1.5, m0 near critical (tests/golden/m0.json), 4^4 aggregates (= Schwarz
domains), N_tv = 20 Gaussian test vectors; initial phase of 5 SAP sweeps
(4 MR steps), then 3 refinement iterations (4 sweeps, 4 MR steps, coarse
GMRES(20) to relative residual 0.05, at most 100 iterations), in the order of
Algorithm 1. The solve: FGMRES(10) on D x = b for a Gaussian b to relative
residual 1e-10, preconditioned by the V-cycle of the same setup.

Writes tests/golden/c2_fgmres.json. Run: python tests/golden/c2_fgmres.py
(about 10-30 minutes on 16 cores).
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
from paper_1601_03184_gb300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "c2_fgmres.json")

CASE = dict(dims=(16, 16, 16, 32), agg=(4, 4, 4, 4), ntv=20, eps=0.6, csw=1.5, gseed=1002, tvseed=2002,
            bseed=3005, m0_keys=["c2_16x16x16x32_eps0.6_csw1.5_seed1002", "proxy_12x12x12x12_eps0.6_csw1.5_seed1002"])
SCHEDULE = dict(init_sweeps=5, init_mr=4, n_refine=3, smooth_sweeps=4, smooth_mr=4, coarse_tol=0.05,
                coarse_restart=20, coarse_maxit=100)
SOLVE = dict(tol=1e-10, restart=10, maxit=300)


def m0_of(keys):
    d = json.load(open(os.path.join(HERE, "m0.json")))
    for k in keys:
        if k in d:
            return float(d[k]["m0"]), k
    raise KeyError("no tuned m0 for %s" % keys)


def main():
    c = CASE
    m0, key = m0_of(c["m0_keys"])
    t0 = time.time()
    U = inputs.gauge_field(c["dims"], c["eps"], c["gseed"])
    A = oracle.clover(c["dims"], U, m0, c["csw"])
    tv0 = inputs.test_vectors(c["ntv"], c["dims"], c["tvseed"])
    s = SCHEDULE
    prm = oracle.make_params(n_init_sweeps=s["init_sweeps"], n_init_mr=s["init_mr"], n_refine=s["n_refine"],
                             n_smooth_sweeps=s["smooth_sweeps"], n_smooth_mr=s["smooth_mr"],
                             coarse_tol=s["coarse_tol"], coarse_restart=s["coarse_restart"],
                             coarse_maxit=s["coarse_maxit"])
    tv, P, Dc = oracle.setup_init(c["dims"], c["agg"], U, A, tv0, prm)
    print("initial phase %.1f s" % (time.time() - t0), flush=True)
    tv, P, Dc, cits = oracle.setup_refine(c["dims"], c["agg"], U, A, tv, P, Dc, prm)
    print("refinement %.1f s" % (time.time() - t0), flush=True)
    b = inputs.gaussian_field((int(np.prod(c["dims"])), 12), c["bseed"])
    x, its, rr = oracle.fgmres(c["dims"], c["agg"], U, A, P, Dc, b, tol=SOLVE["tol"], restart=SOLVE["restart"],
                               maxit=SOLVE["maxit"], coarse_tol=s["coarse_tol"], coarse_restart=s["coarse_restart"],
                               coarse_maxit=s["coarse_maxit"], n_sweeps=s["smooth_sweeps"], n_mr=s["smooth_mr"])
    true_rr = oracle.relres(c["dims"], U, A, b, x)
    out = dict(case={k: v for k, v in c.items() if k != "m0_keys"}, m0=m0, m0_key=key, schedule=SCHEDULE,
               solve=SOLVE, iterations=int(its), relres=float(true_rr),
               last_coarse_iterations=[int(v) for v in cits[-1]], seconds=round(time.time() - t0, 1))
    json.dump(out, open(OUT, "w"), indent=1, sort_keys=True)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
