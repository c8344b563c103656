"""Reference results of the plain FP64 setup on the 32^3 x 64 mixed-precision
workload, computed by the CPU oracle only: roughness 0.6, c_sw 1.5, m0 of the
12^4 proxy field of the same roughness and c_sw (tests/golden/m0.json), 4^4
aggregates (= Schwarz domains), N_tv = 24 Gaussian test vectors; initial
phase of 5 SAP sweeps (4 MR steps), then 3 refinement iterations (4 sweeps,
4 MR steps, coarse GMRES(20) to relative residual 0.05, at most 100
iterations), in the order of Algorithm 1. Then FGMRES(10) on D x = b for a
Gaussian b to relative residual 1e-10, preconditioned by the V-cycle of the
same setup (Sec. 2).

Stored (tests/golden/c3_mixed.json and c3_mixed.npz):
- the FGMRES iteration count and the true relative residual;
- the coarse iteration counts of the last refinement;
- P on a fixed set of aggregates (complex64, [n][ntv][256 sites][12], sites
  of an aggregate in lexicographic order inside it) and the nine D_c blocks
  of the same aggregates (complex64), for per-result errors of the reduced
  precision setups.

Run: python tests/golden/c3_mixed.py (one to three hours on 8 cores, about
40 GB of host memory).
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
OUT = os.path.join(HERE, "c3_mixed.json")
OUT_NPZ = os.path.join(HERE, "c3_mixed.npz")

CASE = dict(dims=(32, 32, 32, 64), agg=(4, 4, 4, 4), ntv=24, eps=0.6, csw=1.5, gseed=1003, tvseed=2003,
            bseed=3003, m0_keys=["c3_32x32x32x64_eps0.6_csw1.5_seed1003", "proxy_12x12x12x12_eps0.6_csw1.5_seed1002"])
SCHEDULE = dict(init_sweeps=5, init_mr=4, n_refine=3, smooth_sweeps=4, smooth_mr=4, coarse_tol=0.05,
                coarse_restart=20, coarse_maxit=100)
SOLVE = dict(tol=1e-10, restart=10, maxit=300)
# aggregates whose P and D_c are stored: the first, one in the middle of the
# lattice, the last (the t = L_t - 1 boundary)
AGGREGATES = [0, 4100, 8191]


def m0_of(keys):
    d = json.load(open(os.path.join(HERE, "m0.json")))
    for k in keys:
        if k in d:
            return float(d[k]["m0"]), k
    raise KeyError("no tuned m0 for %s" % keys)


def aggregate_rows(dims, agg, A):
    """canonical site indices of aggregate A, in lexicographic order inside it"""
    nb = [d // a for d, a in zip(dims, agg)]
    bc = [0] * 4
    r = A
    for mu in range(4):
        bc[mu] = r % nb[mu]
        r //= nb[mu]
    out = []
    for t in range(agg[3]):
        for z in range(agg[2]):
            for y in range(agg[1]):
                for x in range(agg[0]):
                    c = [bc[0] * agg[0] + x, bc[1] * agg[1] + y, bc[2] * agg[2] + z, bc[3] * agg[3] + t]
                    out.append(c[0] + dims[0] * (c[1] + dims[1] * (c[2] + dims[2] * c[3])))
    return np.array(out, np.int64)


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
    del tv0
    print("initial phase %.1f s" % (time.time() - t0), flush=True)
    tv, P, Dc, cits = oracle.setup_refine(c["dims"], c["agg"], U, A, tv, P, Dc, prm)
    del tv
    print("refinement %.1f s" % (time.time() - t0), flush=True)
    Psel = np.stack([P[:, aggregate_rows(c["dims"], c["agg"], a), :] for a in AGGREGATES]).astype(np.complex64)
    Dsel = Dc[AGGREGATES].astype(np.complex64)
    np.savez(OUT_NPZ, aggregates=np.array(AGGREGATES, np.int32), P=Psel, Dc=Dsel)
    b = inputs.gaussian_field((int(np.prod(c["dims"])), 12), c["bseed"])
    x, its, rr = oracle.fgmres(c["dims"], c["agg"], U, A, P, Dc, b, tol=SOLVE["tol"], restart=SOLVE["restart"],
                               maxit=SOLVE["maxit"], coarse_tol=s["coarse_tol"], coarse_restart=s["coarse_restart"],
                               coarse_maxit=s["coarse_maxit"], n_sweeps=s["smooth_sweeps"], n_mr=s["smooth_mr"])
    true_rr = oracle.relres(c["dims"], U, A, b, x)
    out = dict(case={k: v for k, v in c.items() if k != "m0_keys"}, m0=m0, m0_key=key, schedule=SCHEDULE,
               solve=SOLVE, iterations=int(its), relres=float(true_rr), aggregates=AGGREGATES,
               last_coarse_iterations=[int(v) for v in cits[-1]], seconds=round(time.time() - t0, 1))
    json.dump(out, open(OUT, "w"), indent=1, sort_keys=True)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
