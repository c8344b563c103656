"""One parity check of a kernel form that an environment switch or a
right-hand-side count selects, run in a child process (the library reads its
switches once per process). Prints one JSON line {"rel": ..., "kernels": [...]}
with the relative 2-norm error against the FP64 oracle and the kernel classes
the library timed, so that the caller can also see which form ran.

Usage: python tests/variant_check.py sap|apply_D|apply_Dc|restrict|prolong NRHS
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import paper_1601_03184_gb300 as pkg  # noqa: E402
from paper_1601_03184_gb300 import MRHS_F32, MRHS_PREC_FP32, Lattice, inputs  # noqa: E402

# the paper's 4^4 domains on an 8^4 lattice
P4 = dict(dims=(8, 8, 8, 8), agg=(4, 4, 4, 4), eps=0.4, m0=-0.1, csw=1.2, gseed=1301)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def main(kind, nrhs):
    cfg = P4
    U = inputs.gauge_field(cfg["dims"], cfg["eps"], cfg["gseed"])
    A = oracle.clover(cfg["dims"], U, cfg["m0"], cfg["csw"])
    ntv = 8
    lat = Lattice(cfg["dims"], cfg["agg"], ntv, MRHS_PREC_FP32)
    lat.set_gauge(U)
    lat.build_clover(cfg["m0"], cfg["csw"])
    pkg.mrhs_profile(lat.ctx, 1)
    if kind == "sap":
        b = inputs.gaussian_field((nrhs, lat.V, 12), 731)
        x0 = 0.1 * inputs.gaussian_field((nrhs, lat.V, 12), 732)
        xd = lat.to_device(x0, MRHS_F32)
        lat.sap(lat.to_device(b, MRHS_F32), xd, nrhs, MRHS_F32, 2, 4)
        err = rel(lat.to_host(xd, nrhs, MRHS_F32), oracle.sap(cfg["dims"], cfg["agg"], U, A, b, x0, 2, 4))
    elif kind == "apply_D":
        x = inputs.gaussian_field((nrhs, lat.V, 12), 741)
        yd = lat.field(nrhs, MRHS_F32)
        lat.apply_D(lat.to_device(x, MRHS_F32), yd, nrhs, MRHS_F32)
        err = rel(lat.to_host(yd, nrhs, MRHS_F32), oracle.apply_D(cfg["dims"], U, A, x))
    elif kind == "apply_Dc":
        tv = inputs.test_vectors(ntv, cfg["dims"], 751)
        lat.set_tv(lat.to_device(tv, MRHS_F32), MRHS_F32)
        lat.build_P()
        lat.build_Dc()
        Dc = lat.get_Dc()
        xc = inputs.gaussian_field((nrhs, lat.nagg, 2 * ntv), 752)
        yd = lat.field(nrhs, MRHS_F32, coarse=True)
        lat.apply_Dc(lat.to_device(xc, MRHS_F32, coarse=True), yd, nrhs, MRHS_F32)
        err = rel(lat.to_host(yd, nrhs, MRHS_F32, coarse=True), oracle.apply_Dc(cfg["dims"], cfg["agg"], Dc, xc))
    elif kind == "restrict":
        tv = inputs.test_vectors(ntv, cfg["dims"], 761)
        lat.set_tv(lat.to_device(tv, MRHS_F32), MRHS_F32)
        lat.build_P()
        P = oracle.gram_schmidt(cfg["dims"], cfg["agg"], tv)
        v = inputs.gaussian_field((nrhs, lat.V, 12), 762)
        vc = lat.field(nrhs, MRHS_F32, coarse=True)
        lat.restrict(lat.to_device(v, MRHS_F32), vc, nrhs, MRHS_F32)
        err = rel(lat.to_host(vc, nrhs, MRHS_F32, coarse=True), oracle.restrict(cfg["dims"], cfg["agg"], P, v))
    elif kind == "prolong":
        tv = inputs.test_vectors(ntv, cfg["dims"], 771)
        lat.set_tv(lat.to_device(tv, MRHS_F32), MRHS_F32)
        lat.build_P()
        P = oracle.gram_schmidt(cfg["dims"], cfg["agg"], tv)
        uc = inputs.gaussian_field((nrhs, lat.nagg, 2 * ntv), 772)
        u = lat.field(nrhs, MRHS_F32)
        lat.prolong(lat.to_device(uc, MRHS_F32, coarse=True), u, nrhs, MRHS_F32)
        err = rel(lat.to_host(u, nrhs, MRHS_F32), oracle.prolong(cfg["dims"], cfg["agg"], P, uc))
    else:
        raise SystemExit("unknown check " + kind)
    kernels = sorted(pkg.mrhs_profile_read(lat.ctx))
    lat.close()
    print(json.dumps({"rel": err, "kernels": kernels}))


if __name__ == "__main__":
    main(sys.argv[1], int(sys.argv[2]))
