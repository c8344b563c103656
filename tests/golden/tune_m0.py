"""Tune the bare mass m0 of a seeded synthetic gauge field so that the
smallest-magnitude eigenvalue of the Wilson-clover operator D is about 1e-3 of
the largest-magnitude one (the "m0 tuned" / "near critical" configurations).

Calls only the CPU oracle. D(m0) = D(0) + m0 * 1, so every eigenvalue moves
rigidly with m0: one Arnoldi solve (ARPACK via scipy) for the eigenvalues of
D(0) with the smallest real parts and one for the largest magnitude fix m0:
    min_i |lambda_i(0) + m0| = ratio * max_i |lambda_i(0) + m0|.
The chosen m0 places the leftmost real eigenvalue at +ratio*|lambda_max|.
Writes tests/golden/m0.json. Run: python tests/golden/tune_m0.py [name ...]
"""
import json
import os
import sys
import time

import numpy as np
from scipy.sparse.linalg import LinearOperator, eigs

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
from paper_1601_03184_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "m0.json")

# name -> (dims, roughness eps, csw, gauge seed)
CASES = {
    "c2_16x16x16x32_eps0.6_csw1.5_seed1002": ((16, 16, 16, 32), 0.6, 1.5, 1002),
    "c3_32x32x32x64_eps0.6_csw1.5_seed1003": ((32, 32, 32, 64), 0.6, 1.5, 1003),
    "c5proxy_16x16x16x32_eps0.6_csw1.7_seed1005": ((16, 16, 16, 32), 0.6, 1.7, 1005),
    # small-volume proxies (same roughness and c_sw), used while the full-size
    # solves above are not available
    "proxy_12x12x12x12_eps0.6_csw1.5_seed1002": ((12, 12, 12, 12), 0.6, 1.5, 1002),
    "proxy_12x12x12x12_eps0.6_csw1.7_seed1005": ((12, 12, 12, 12), 0.6, 1.7, 1005),
    # the ends of the roughness range of the learned generator's training
    # fields (m0 interpolated in between)
    "proxy_12x12x12x12_eps0.4_csw1.5_seed4000": ((12, 12, 12, 12), 0.4, 1.5, 4000),
    "proxy_12x12x12x12_eps0.7_csw1.5_seed4001": ((12, 12, 12, 12), 0.7, 1.5, 4001),
}
RATIO = 1e-3


def tune(dims, eps, csw, seed):
    U = inputs.gauge_field(dims, eps, seed)
    A0 = oracle.clover(dims, U, 0.0, csw)
    n = int(np.prod(dims)) * 12
    count = [0]
    t = time.time()

    def mv(v):
        count[0] += 1
        if count[0] % 200 == 0:
            print("  matvecs", count[0], round(time.time() - t, 1), "s", flush=True)
        return oracle.apply_D(dims, U, A0, v.reshape(-1, 12)).reshape(-1)

    op = LinearOperator((n, n), matvec=mv, dtype=np.complex128)
    lmax = eigs(op, k=1, which="LM", tol=1e-4, return_eigenvectors=False)
    low = eigs(op, k=4, which="SR", tol=1e-4, ncv=40, maxiter=4000, return_eigenvectors=False)
    low = low[np.argsort(low.real)]
    lam_c = low[0]
    # m0 with |lambda_c + m0| = RATIO * |lambda_max + m0| (leftmost eigenvalue put at +RATIO*|lmax|)
    m0 = -lam_c.real
    for _ in range(20):
        m0 = -lam_c.real + RATIO * abs(lmax[0] + m0)
    spec = low + m0
    return dict(dims=list(dims), eps=eps, csw=csw, seed=seed, m0=float(m0), ratio=RATIO,
                lambda_max_at_m0=float(abs(lmax[0] + m0)), lowest_at_m0=[[float(z.real), float(z.imag)] for z in spec],
                min_abs_ratio=float(np.min(np.abs(spec)) / abs(lmax[0] + m0)), matvecs=count[0],
                seconds=round(time.time() - t, 1))


if __name__ == "__main__":
    names = sys.argv[1:] or list(CASES)
    for nm in names:
        r = tune(*CASES[nm])
        res = json.load(open(OUT)) if os.path.exists(OUT) else {}
        res[nm] = r
        print(nm, json.dumps(r), flush=True)
        json.dump(res, open(OUT, "w"), indent=1, sort_keys=True)
