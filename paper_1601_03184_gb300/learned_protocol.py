"""Training and judging protocol of the learned test-vector generator on the
16^3 x 32 workload (a project form beside the paper's method; the paper's
setup, Sec. 2, is its fallback and its reference).

Training data: n_train seeded gauge fields (roughness drawn uniformly in
[0.4, 0.7], m0 near critical for that roughness), each with the N_tv = 20
test vectors of the plain full setup (initial phase of 5 SAP sweeps, then 3
refinement iterations) as the target span. The network (4 -> 32 -> 32 -> 4
colour triplets, bf16 weights, FP32 accumulation) is trained on one-sweep
vectors of every field in turn (Adam on |Dv|^2/|v|^2 + lambda |v - P P^dag
v|^2/|v|^2). Judging: on n_test unseen fields the learned initial phase (one
SAP sweep + the network) against the plain one (5 sweeps), both followed by
the same refinement: the Rayleigh quotients |Dv|/|v| of the test vectors after
the initial phase and after the refinement, and the two-level FGMRES iteration
count to 1e-10. Every coarse solve (refinement and FGMRES) runs on the
Schur complement of the even aggregates unless coarse_eo = 0.

Orchestration only: every step runs in the library's kernels through the C
ABI; torch provides device memory and the norms of the Rayleigh quotients.
Run: python -m paper_1601_03184_gb300.learned_protocol [--fields 64 --test 8]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import MRHS_F32, MRHS_PREC_FP32, Lattice, inputs, learned, mrhs_nn_get_weights, mrhs_nn_set_weights

TRAIN_SEED0, TEST_SEED0, EPS_SEED = 4000, 4100, 4999
SCHEDULE = dict(init_sweeps=5, init_mr=4, n_refine=3, sweeps=4, mr=4, ctol=0.05, crestart=20, cmaxit=100)


def roughness(seed0, n):
    """field roughness of fields seed0 .. seed0+n-1: uniform in [0.4, 0.7]"""
    u = np.random.Generator(np.random.PCG64(EPS_SEED + seed0)).random(n)
    return 0.4 + 0.3 * u


def m0_for(eps, table):
    """m0 near critical for roughness eps: linear interpolation (constant
    outside) in the tuned (eps, m0) points of table"""
    e = np.array(sorted(table))
    return float(np.interp(eps, e, [table[k] for k in e]))


def rayleigh(lat, dev_tv):
    """|D v_r| / |v_r| for every test vector of a device FP32 field"""
    import torch

    y = torch.empty_like(dev_tv)
    lat.apply_D(dev_tv, y, lat.ntv, MRHS_F32)
    N = lat.ntv
    a = dev_tv.view(torch.float32).view(-1, N).double().pow(2).sum(0).sqrt()
    b = y.view(torch.float32).view(-1, N).double().pow(2).sum(0).sqrt()
    return (b / a).cpu().numpy()


def tv_rayleigh(lat):
    return rayleigh(lat, lat.to_device(lat.get_tv(MRHS_F32), MRHS_F32))


def run(n_train=64, n_test=8, dims=(16, 16, 16, 32), agg=(4, 4, 4, 4), ntv=20, widths=(4, 32, 32, 4),
        steps=25, lr=2e-3, lam=1.0, csw=1.5, m0_table=None, schedule=None, coarse_eo=1, log=print):
    import torch

    s = dict(SCHEDULE, **(schedule or {}))
    m0_table = m0_table or {0.6: -0.6278459331791598}
    t0 = time.perf_counter()
    lat = Lattice(dims, agg, ntv, MRHS_PREC_FP32)
    lat.set_coarse_solver(coarse_eo)
    learned.attach(lat, widths, seed=17, noise=0.01, bf16=True)
    step = 1
    first = last = None
    for f, eps in enumerate(roughness(TRAIN_SEED0, n_train)):
        lat.set_gauge(inputs.gauge_field(dims, float(eps), TRAIN_SEED0 + f, device="cuda"))
        lat.build_clover(m0_for(eps, m0_table), csw)
        losses = learned.train_on_field(lat, s, steps, seed=TRAIN_SEED0 * 10 + f, lr=lr, lam=lam, first_step=step)
        step += len(losses)
        first = losses[0] if first is None else first
        last = losses[-1]
        log("train field %d eps %.3f loss %.4f -> %.4f" % (f, eps, losses[0], losses[-1]))
    train_s = time.perf_counter() - t0
    weights = mrhs_nn_get_weights(lat.ctx, 0)
    tests = []
    for f, eps in enumerate(roughness(TEST_SEED0, n_test)):
        seed = TEST_SEED0 + f
        lat.set_gauge(inputs.gauge_field(dims, float(eps), seed, device="cuda"))
        m0 = m0_for(eps, m0_table)
        lat.build_clover(m0, csw)
        gen = torch.Generator(device="cuda")
        gen.manual_seed(seed)
        tv0 = torch.randn(lat.field(ntv, MRHS_F32).numel() // 4, generator=gen, device="cuda")
        rhs = inputs.gaussian_field((lat.V, 12), seed + 50)
        row = {"seed": seed, "eps": round(float(eps), 4), "m0": round(m0, 5)}
        for form in ("plain", "learned"):
            torch.cuda.synchronize()
            ta = time.perf_counter()
            if form == "plain":
                lat.setup_init(tv0, MRHS_F32, 0, s["init_sweeps"], s["init_mr"])
            else:
                # the network's input alone (one sweep, normalised) for comparison
                lat.setup_init(tv0, MRHS_F32, 0, 1, s["init_mr"])
                rq_one = tv_rayleigh(lat)
                torch.cuda.synchronize()
                ta = time.perf_counter()
                mrhs_nn_set_weights(lat.ctx, weights)
                learned.learned_setup(lat, tv0, dict(s, n_refine=0), n_sweeps=1)
            torch.cuda.synchronize()
            tb = time.perf_counter()
            rq_init = tv_rayleigh(lat)
            torch.cuda.synchronize()
            tc = time.perf_counter()
            lat.setup_refine(s["n_refine"], s["sweeps"], s["mr"], s["ctol"], s["crestart"], s["cmaxit"])
            torch.cuda.synchronize()
            td = time.perf_counter()
            rq_final = tv_rayleigh(lat)
            _, its, rr = lat.solve_fgmres(rhs, tol=1e-10, restart=10, maxit=300, coarse_tol=s["ctol"],
                                          coarse_restart=s["crestart"], coarse_maxit=s["cmaxit"],
                                          n_sweeps=s["sweeps"], n_mr=s["mr"], allow_noconv=True)
            row[form] = {"rq_init": round(float(rq_init.mean()), 5), "rq_final": round(float(rq_final.mean()), 5),
                         "fgmres": int(its), "relres": float(rr), "setup_ms": round(1e3 * (tb - ta + td - tc), 1)}
            if form == "learned":
                row[form]["rq_one_sweep"] = round(float(rq_one.mean()), 5)
        log("test field %d: %s" % (f, json.dumps(row)))
        tests.append(row)
    lat.close()
    agg_its = [(t["plain"]["fgmres"], t["learned"]["fgmres"]) for t in tests]
    return {"widths": list(widths), "coarse_solver": "even-odd" if coarse_eo else "plain",
            "train_fields": n_train, "test_fields": n_test, "steps_per_field": steps,
            "loss_first": first, "loss_last": last, "train_s": round(train_s, 1), "tests": tests,
            "fgmres_plain_mean": float(np.mean([a for a, _ in agg_its])),
            "fgmres_learned_mean": float(np.mean([b for _, b in agg_its])),
            "rq_init_plain_mean": float(np.mean([t["plain"]["rq_init"] for t in tests])),
            "rq_init_learned_mean": float(np.mean([t["learned"]["rq_init"] for t in tests]))}


def load_m0_table(csw=1.5):
    """(roughness -> m0) of the tuned 12^4 proxy fields at this c_sw
    (tests/golden/m0.json, written by tests/golden/tune_m0.py from the oracle)"""
    p = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden", "m0.json")
    d = json.load(open(p))
    return {float(v["eps"]): float(v["m0"]) for k, v in d.items()
            if k.startswith("proxy_12x12x12x12") and abs(float(v["csw"]) - csw) < 1e-12}


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--fields", type=int, default=64)
    ap.add_argument("--test", type=int, default=8)
    ap.add_argument("--steps", type=int, default=25)
    ap.add_argument("--width", type=int, default=32)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res = run(n_train=a.fields, n_test=a.test, steps=a.steps, widths=(4, a.width, a.width, 4),
              m0_table=load_m0_table())
    print(json.dumps(res))
    if a.out:
        json.dump(res, open(a.out, "w"), indent=1)
