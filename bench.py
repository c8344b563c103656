"""Benchmark of the multiple-right-hand-side DD-alpha-AMG setup on GB300.

One step = the whole setup on one lattice: initial phase (SAP on all N_tv
test vectors from x0 = 0, normalisation, P by aggregate-wise Gram-Schmidt,
D_c = P^dag D P) followed by the refinement iterations of Algorithm 2 with
block length N_b = N_tv (restriction, coarse GMRES to 0.05 on the Schur
complement of the even aggregates, prolongation, SAP, normalisation, P, D_c),
all in the library's CUDA kernels through its C ABI. Inputs (gauge field, clover, test vectors) are resident in HBM when the
timed region starts.

Prints one JSON line. `--impl reference` times the FP64 CPU oracle (the
single-RHS order of Algorithm 1) on a bounded sub-volume of the same
workload and scales it linearly in the volume.

Under torchrun (N > 1) every rank runs an independent replica of the whole
setup on its own GPU (the setup of one lattice does not shard here); there is
no collective in the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MRHS setup wall time (s) at Ntv; stencil HBM GB/s % peak; learned/mixed vs plain"

# workloads: lattice, aggregate (= Schwarz domain), N_tv, roughness, csw, seeds, setup schedule
CONFIGS = {
    "48x48x48x96_ntv32": dict(dims=(48, 48, 48, 96), agg=(4, 4, 4, 4), ntv=32, eps=0.6, csw=1.7, gseed=1005,
                              tvseed=2005, m0_keys=["c5proxy_16x16x16x32_eps0.6_csw1.7_seed1005",
                                                    "proxy_12x12x12x12_eps0.6_csw1.7_seed1005"]),
    "32x32x32x64_ntv24": dict(dims=(32, 32, 32, 64), agg=(4, 4, 4, 4), ntv=24, eps=0.6, csw=1.5, gseed=1003,
                              tvseed=2003, m0_keys=["c3_32x32x32x64_eps0.6_csw1.5_seed1003",
                                                    "proxy_12x12x12x12_eps0.6_csw1.5_seed1002"]),
    "16x16x16x32_ntv20": dict(dims=(16, 16, 16, 32), agg=(4, 4, 4, 4), ntv=20, eps=0.6, csw=1.5, gseed=1002,
                              tvseed=2002, m0_keys=["c2_16x16x16x32_eps0.6_csw1.5_seed1002",
                                                    "proxy_12x12x12x12_eps0.6_csw1.5_seed1002"]),
    # the 48^3x96 workload's physics and N_tv on a small volume (profiler captures)
    "16x16x16x32_ntv32": dict(dims=(16, 16, 16, 32), agg=(4, 4, 4, 4), ntv=32, eps=0.6, csw=1.7, gseed=1005,
                              tvseed=2005, m0_keys=["c5proxy_16x16x16x32_eps0.6_csw1.7_seed1005",
                                                    "proxy_12x12x12x12_eps0.6_csw1.7_seed1005"]),
}
DEFAULT_CONFIG = "48x48x48x96_ntv32"
SCHEDULE = dict(init_sweeps=5, init_mr=4, n_refine=3, smooth_sweeps=4, smooth_mr=4, coarse_tol=0.05,
                coarse_restart=20, coarse_maxit=100)
M0_FALLBACK = -0.45
# bounded CPU sample of the same setup (oracle): 8^3 x 32 lattice (two 4^4
# domains per spatial direction, eight in time), same aggregates and schedule;
# about 20 s on 16 Grace cores (53 s on 8 x86 cores)
CPU_SAMPLE_DIMS = (8, 8, 8, 32)


def reduce_max_over_ranks(x, dist=None, device="cuda"):
    """The largest of the ranks' values of x, returned on every rank (x
    itself when the run is not distributed). Times are reduced this way so
    that the job is as slow as its slowest replica."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_seconds_per_setup(ms_per_step, world):
    """Each of the `world` replicas completes one whole setup per step, so
    the job delivers `world` setups in the slowest rank's step time."""
    return ms_per_step / 1000.0 / world


def load_m0(keys):
    """m0 from tests/golden/m0.json (written by tests/golden/tune_m0.py from the
    oracle), first key present wins."""
    p = os.path.join(ROOT, "tests", "golden", "m0.json")
    if os.path.exists(p):
        d = json.load(open(p))
        for key in keys:
            if key in d:
                return float(d[key]["m0"]), "tuned: " + key
    return M0_FALLBACK, "fallback"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured", d
    return 6800.0, "fallback", {}


# ---------------------------------------------------------------- clocks ---
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------- algorithmic work ---
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch from
# the ncu captures summarised in profiles/ (16x16x16x32, N_tv = 32), scaled by
# the number of sites; None for a kernel whose code changed since its capture
NCU_TRAFFIC = {
    "sap_tm": {"bytes": 903.34e6, "sites": 16 * 16 * 16 * 32, "ntv": 32,
               "profile": "profiles/k_sap_tm_16x16x16x32_ntv32.md"},
    "sap_pk": {"bytes": 917.06e6, "sites": 16 * 16 * 16 * 32, "ntv": 32,
               "profile": "profiles/k_sap_pk_16x16x16x32_ntv32.md"},
}


def ncu_traffic(name, cfg):
    t = NCU_TRAFFIC.get(name)
    if t is None or t["ntv"] != cfg["ntv"]:
        return None
    return t["bytes"] * int(np.prod(cfg["dims"])) / t["sites"]


def kernel_work(name, cfg, launches_per_step, bytes_f=4):
    """Algorithmic bytes and flops of ONE launch of a kernel class for the
    benchmark workload (each operand touched once)."""
    V = int(np.prod(cfg["dims"]))
    N = cfg["ntv"]
    spin = 24 * bytes_f           # one spinor, one rhs
    link4 = 4 * 18 * bytes_f      # the four forward links of a site
    clov = 72 * bytes_f           # two packed Hermitian 6x6 blocks
    flop_site_rhs = 1872          # Wilson-clover D per site and rhs
    Va = int(np.prod(cfg["agg"]))
    if name == "dslash_full":
        return V * (link4 + clov + 2 * N * spin), V * N * flop_site_rhs
    if name == "dslash_resid":  # one colour: r = b - D x on half of the sites
        return V / 2 * (link4 + clov + 3 * N * spin), V / 2 * N * flop_site_rhs
    if name in ("sap_pk", "sap_tm", "sap_tm2", "sap_fused8", "sap_fused"):  # one colour: residual + n_mr MR steps, on chip
        nmr = SCHEDULE["smooth_mr"]
        flops = V / 2 * N * (flop_site_rhs + nmr * (flop_site_rhs + 336))
        byt = V / 2 * (link4 + clov + 3 * N * spin)  # b in, x in and out, links and clover once
        return byt, flops
    if name == "sap_block_mr":  # one colour, n_mr MR steps of D_B, two dots and two updates
        nmr = SCHEDULE["smooth_mr"]
        flops = V / 2 * N * nmr * (flop_site_rhs + 4 * 96)
        byt = V / 2 * (link4 + clov + 3 * N * spin)  # x, rho in and out once, links once
        return byt, flops
    if name == "apply_dc_tc" or name == "apply_dc":  # D_c read once, x_c of 9 neighbours (L2), y_c written
        nagg = V // Va
        nc = 2 * N
        byt = nagg * (9 * nc * nc * 2 * bytes_f + 2 * nc * 2 * N * bytes_f)
        fl = nagg * 9 * nc * nc * 8 * N
        return byt, fl
    if name in ("coarse_op", "coarse_op_tc"):  # P read once, U, A once, D_c written once
        nagg = V // Va
        nc = 2 * N
        byt = V * (N * spin + link4 + clov) + nagg * 9 * nc * nc * 2 * bytes_f
        fl = nagg * 9 * 0 + V * 2 * N * flop_site_rhs / 2 + nagg * (4 * 8 * N * N * 6 * Va + 8 * 4 * 8 * N * N * 6 * Va / 4)
        return byt, fl
    if name == "gs_cholqr2":
        byt = 4 * V * N * spin  # two passes: read V, read V + write Q, read Q, read Q + write P -> ~ 3 reads 2 writes
        fl = 2 * 2 * (8 * N * N * 6 * V / 2)  # two passes x (Gram + triangular solve), per chirality
        return byt, fl
    return None, None


# ------------------------------------------------------------ reference ----
def cpu_sample(cfg, m0, coarse_eo=1):
    """Oracle (FP64, single right-hand side at a time) full setup on the
    bounded sub-volume CPU_SAMPLE_DIMS with the workload's aggregates, N_tv and
    schedule. Returns (seconds, scaled seconds, threads, description)."""
    import oracle
    from paper_1601_03184_gb300 import inputs

    oracle.build()
    dims = CPU_SAMPLE_DIMS
    agg = cfg["agg"]
    U = inputs.gauge_field(dims, cfg["eps"], cfg["gseed"])
    A = oracle.clover(dims, U, m0, cfg["csw"])
    tv0 = inputs.test_vectors(cfg["ntv"], dims, cfg["tvseed"])
    prm = oracle.make_params(n_init_sweeps=SCHEDULE["init_sweeps"], n_init_mr=SCHEDULE["init_mr"],
                             n_refine=SCHEDULE["n_refine"], n_smooth_sweeps=SCHEDULE["smooth_sweeps"],
                             n_smooth_mr=SCHEDULE["smooth_mr"], coarse_tol=SCHEDULE["coarse_tol"],
                             coarse_restart=SCHEDULE["coarse_restart"], coarse_maxit=SCHEDULE["coarse_maxit"],
                             coarse_even_odd=coarse_eo)
    t0 = time.perf_counter()
    tv, P, Dc = oracle.setup_init(dims, agg, U, A, tv0, prm)
    oracle.setup_refine(dims, agg, U, A, tv, P, Dc, prm)
    dt = time.perf_counter() - t0
    scale = np.prod(cfg["dims"]) / np.prod(dims)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    desc = ("oracle FP64 full setup (Algorithm 1 order, same N_tv, aggregates, schedule and coarse solver) on a "
            "%s sub-volume, %.2f s, scaled linearly by the volume ratio %.0f" % ("x".join(map(str, dims)), dt, scale))
    return dt, dt * scale, threads, desc


def run_reference(args, cfg, cfg_name, m0, m0_src, rank, world):
    if rank != 0:
        return
    if world > 1:
        # torchrun limits every rank to one OpenMP thread; the other ranks do
        # no work in this arm, so the oracle on rank 0 takes every host core
        # (read by the OpenMP runtime when the oracle library is loaded)
        os.environ["OMP_NUM_THREADS"] = str(os.cpu_count() or 1)
    times = []
    threads = 1
    desc = ""
    for i in range(args.warmup + args.steps):
        dt, scaled, threads, desc = cpu_sample(cfg, m0, args.coarse_eo)
        if i >= args.warmup:
            times.append(scaled)
    v = float(np.mean(times))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": v * 1000, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg_name, "dims": cfg["dims"], "agg": cfg["agg"], "ntv": cfg["ntv"],
                   "m0": m0, "m0_source": m0_src, "csw": cfg["csw"], "schedule": SCHEDULE},
        "cpu_baseline": {"value": v, "unit": "s", "cores": threads, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- ours ----
def run_ours(args, cfg, cfg_name, m0, m0_src, rank, world, local_rank):
    import torch

    import paper_1601_03184_gb300 as pkg
    from paper_1601_03184_gb300 import MRHS_F32, MRHS_PREC_FP32, Lattice, inputs

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    dims, agg, N = cfg["dims"], cfg["agg"], cfg["ntv"]
    V = int(np.prod(dims))
    stream = torch.cuda.current_stream()
    t_gen = time.perf_counter()
    U = inputs.gauge_field(dims, cfg["eps"], cfg["gseed"], device="cuda")
    lat = Lattice(dims, agg, N, MRHS_PREC_FP32, stream.cuda_stream)
    lat.set_gauge(U)
    lat.build_clover(m0, cfg["csw"])
    lat.set_smoother(args.smoother_eo)
    lat.set_coarse_solver(args.coarse_eo)
    lat.set_dc_engine(args.dc_engine)
    # test vectors: complex Gaussian, drawn on the device directly in the library layout
    gen = torch.Generator(device="cuda")
    gen.manual_seed(cfg["tvseed"] + rank)
    nb = pkg.mrhs_field_bytes(lat.ctx, N, MRHS_F32)
    tv0 = torch.randn(nb // 4, generator=gen, device="cuda", dtype=torch.float32)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t_gen

    hbm_peak, hbm_src, peak_json = peaks()

    # ---- stencil alone (FP32, all N_tv right-hand sides), before the setup allocates its work fields
    y = torch.empty_like(tv0)
    for _ in range(3):
        lat.apply_D(tv0, y, N, MRHS_F32)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(reps):
        lat.apply_D(tv0, y, N, MRHS_F32)
    ev1.record(stream)
    torch.cuda.synchronize()
    st_ms = ev0.elapsed_time(ev1) / reps
    st_bytes, st_flops = kernel_work("dslash_full", cfg, 1)
    stencil = {"ms": round(st_ms, 3), "gbs": round(st_bytes / st_ms / 1e6, 1),
               "frac": round(st_bytes / st_ms / 1e6 / hbm_peak, 4), "peak_gbs": hbm_peak,
               "peak_source": hbm_src, "bytes_per_launch": st_bytes, "tflops": round(st_flops / st_ms / 1e9, 2),
               "nrhs": N}
    # ---- the same stencil with bf16 storage (FP32 arithmetic): FP32-ALU-bound,
    # reported against the FP32 peak
    xb = tv0.to(torch.bfloat16)
    yb = torch.empty_like(xb)
    for _ in range(3):
        lat.apply_D(xb, yb, N, pkg.MRHS_BF16)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(reps):
        lat.apply_D(xb, yb, N, pkg.MRHS_BF16)
    ev1.record(stream)
    torch.cuda.synchronize()
    sb_ms = ev0.elapsed_time(ev1) / reps
    sb_bytes = V * (288 + 288 + 2 * 48 * N)
    stencil_bf16 = {"ms": round(sb_ms, 3), "gbs": round(sb_bytes / sb_ms / 1e6, 1),
                    "tflops": round(st_flops / sb_ms / 1e9, 2), "nrhs": N}
    del y, xb, yb
    torch.cuda.empty_cache()

    def step():
        lat.setup_init(tv0, MRHS_F32, 0, SCHEDULE["init_sweeps"], SCHEDULE["init_mr"])
        return lat.setup_refine(SCHEDULE["n_refine"], SCHEDULE["smooth_sweeps"], SCHEDULE["smooth_mr"],
                                SCHEDULE["coarse_tol"], SCHEDULE["coarse_restart"], SCHEDULE["coarse_maxit"])

    for _ in range(args.warmup):
        its = step()
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    pkg.mrhs_profile(lat.ctx, 1)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        its = step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    prof = pkg.mrhs_profile_read(lat.ctx)
    pkg.mrhs_profile(lat.ctx, 0)
    clk = clocks.stop()
    ms = reduce_max_over_ranks(ms, dist)
    value = whole_job_seconds_per_setup(ms, world)

    # ---- per-kernel profile and the roofline of the dominant kernel
    total = sum(v[1] for v in prof.values())
    kernels = {k: {"launches": v[0] // args.steps, "ms_per_step": v[1] / args.steps,
                   "share": v[1] / total if total else 0.0} for k, v in prof.items()}
    top = max(prof, key=lambda k: prof[k][1]) if prof else None
    roof = None
    if top is not None:
        launches, tot_ms = prof[top]
        avg_ms = tot_ms / max(launches, 1)
        byt, fl = kernel_work(top, cfg, launches // args.steps)
        alu_peak = None
        if byt is not None:
            ai = fl / byt
            sms = lat.info()[6]
            clock = (clk.get("sm_mhz") or peak_json.get("clocks_under_load", {}).get("sm_mhz_median", 1432.0))
            alu_peak = sms * 128 * 2 * clock * 1e6 / 1e12  # FP32 FMA lanes x 2 flops x clock, TFLOP/s
            hbm_ach = byt / avg_ms / 1e6
            alu_ach = fl / avg_ms / 1e9
            if hbm_ach / hbm_peak >= alu_ach / alu_peak:
                roof = {"kernel": top, "bound": "hbm", "achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s",
                        "frac": hbm_ach / hbm_peak, "traffic": ncu_traffic(top, cfg), "peak_source": hbm_src,
                        "alu_frac": alu_ach / alu_peak, "avg_launch_ms": avg_ms, "bytes_per_launch": byt,
                        "flops_per_launch": fl}
            else:
                roof = {"kernel": top, "bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "TFLOP/s",
                        "frac": alu_ach / alu_peak, "traffic": ncu_traffic(top, cfg),
                        "traffic_source": NCU_TRAFFIC.get(top, {}).get("profile"),
                        "peak_source": "FP32: SMs x 128 lanes x 2 flop x median SM clock under load",
                        "hbm_frac": hbm_ach / hbm_peak, "avg_launch_ms": avg_ms, "bytes_per_launch": byt,
                        "flops_per_launch": fl, "arith_intensity": ai}
        else:
            roof = {"kernel": top, "bound": None, "avg_launch_ms": avg_ms}

    # ---- the quality check of the timed setup (the state the last timed step
    # left): two-level FGMRES to 1e-10
    fg_plain = None
    if not args.no_fgmres:
        pkg.mrhs_trim(lat.ctx)
        fg_plain = fgmres_check(lat, cfg)
    # ---- end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, lat, U, tv0, cfg, m0, stream, barrier)
        e2e["value"] = whole_job_seconds_per_setup(1000.0 * reduce_max_over_ranks(e2e["value"], dist), world)

    # ---- the order of Algorithm 1 (one vector at a time) against Algorithm 2
    # with N_b = N_tv on this GPU: one refinement iteration per block length
    srhs = None
    if not args.no_srhs:
        srhs = run_block_lengths(lat, tv0, stream, (N, 8, 1) if N > 8 else (N, 1))
    gpu_launches = int(sum(v[0] for v in prof.values()) / args.steps)
    sms = lat.info()[6]
    clock = clk.get("sm_mhz") or peak_json.get("clocks_under_load", {}).get("sm_mhz_median", 1432.0)
    fp32_peak = sms * 128 * 2 * clock * 1e6 / 1e12
    stencil_bf16["frac_fp32_peak"] = round(stencil_bf16["tflops"] / fp32_peak, 4)
    if roof is not None:
        roof = {k: (round(v, 6) if isinstance(v, float) else v) for k, v in roof.items()}
    line = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": cfg_name, "ntv": N, "precision": "fp32 (plain setup)", "m0": round(m0, 6),
                   "m0_source": m0_src, "csw": cfg["csw"], "roughness": cfg["eps"],
                   "smoother": "even-odd" if args.smoother_eo else "plain",
                   "coarse_solver": "even-odd" if args.coarse_eo else "plain",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (test vectors %.1f GB)" % (nb / 1e9)},
        "roofline": roof,
        "stencil": stencil,
        "stencil_bf16": stencil_bf16,
        "clocks": clk,
        "gpu_launches": gpu_launches,
        "e2e": e2e,
    }
    if srhs is not None:
        line["srhs_over_mrhs"] = srhs["srhs_over_mrhs"]
    # per-kernel tables and the rest of the detail go to stderr, so that the
    # one JSON line on stdout stays short
    detail = {"kernels": kernels, "dims": dims, "agg": agg, "schedule": SCHEDULE,
              "last_coarse_iterations": [int(x) for x in np.asarray(its).reshape(-1)[-N:]],
              "input_generation_s": round(gen_s, 1), "stencil_fp32": stencil, "block_lengths": srhs}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, scaled, threads, desc = cpu_sample(cfg, m0, args.coarse_eo)
        line["cpu_baseline"] = {"value": scaled, "unit": "s", "cores": threads, "kind": "oracle", "sample": desc}
    line["fgmres_plain"] = fg_plain
    # ---- learned + mixed-precision setup, wall-time ratio against the plain one
    if not args.no_learned:
        lat.close()
        del tv0
        torch.cuda.empty_cache()
        lm = run_learned_mixed(args, cfg, U, m0, stream, ms, barrier, dist, world)
        detail["learned_mixed"] = lm
        line["learned_mixed"] = {"value": round(lm["value"], 4), "unit": "s",
                                 "ratio_vs_plain": round(lm["ratio_vs_plain"], 4),
                                 "fgmres_iterations": (lm["fgmres"] or {}).get("iterations"),
                                 "widths": lm["widths"], "storage": "bf16"}
    if rank == 0:
        print("bench detail: " + json.dumps(detail), file=sys.stderr, flush=True)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# kernel classes of the library's profile grouped into the phases the paper
# times separately (Sec. 7): smoother, coarse grid, projections, setup of R
# and D_c, and the copies that move a block of test vectors in and out
PHASES = {"smoother": ("sap_pk", "sap_tm", "sap_tm2", "sap_fused", "sap_fused8", "sap_block_mr", "dslash_resid"),
          "coarse_grid": ("apply_dc_tc", "apply_dc", "multi_dot", "multi_axpy", "inverse_apply", "self_inverse"),
          "projections": ("restrict", "prolong", "normalise", "norms"),
          "R_and_Dc": ("gs_cholqr2", "coarse_op", "coarse_op_tc", "format_dc"),
          "block_copies": ("block_gather",)}


def phase_times(prof):
    out = {k: 0.0 for k in PHASES}
    out["other"] = 0.0
    for name, (_, ms) in prof.items():
        ph = next((p for p, names in PHASES.items() if name in names), "other")
        out[ph] += ms
    return out


def run_block_lengths(lat, tv0, stream, block_lengths=(32, 8, 1)):
    """One refinement iteration (Algorithm 2) of the plain FP32 setup with
    block length N_b = each of block_lengths, the setup state reset to the
    same initial phase before each: total and per-phase device time (CUDA
    events around every launch), and the N_b = 1 / N_b = N_tv ratios, the
    single- over multiple-right-hand-side speed-up of Sec. 7 on this GPU."""
    import torch

    import paper_1601_03184_gb300 as pkg
    from paper_1601_03184_gb300 import MRHS_F32

    res = {}
    for nb in block_lengths:
        lat.set_block_length(0)
        lat.setup_init(tv0, MRHS_F32, 0, SCHEDULE["init_sweeps"], SCHEDULE["init_mr"])
        lat.set_block_length(nb)
        torch.cuda.synchronize()
        pkg.mrhs_profile(lat.ctx, 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.setup_refine(1, SCHEDULE["smooth_sweeps"], SCHEDULE["smooth_mr"], SCHEDULE["coarse_tol"],
                         SCHEDULE["coarse_restart"], SCHEDULE["coarse_maxit"])
        e1.record(stream)
        torch.cuda.synchronize()
        prof = pkg.mrhs_profile_read(lat.ctx)
        pkg.mrhs_profile(lat.ctx, 0)
        ph = phase_times(prof)
        res[nb] = {"ms": round(e0.elapsed_time(e1), 1), **{k: round(v, 1) for k, v in ph.items()}}
    lat.set_block_length(0)
    lo, hi = min(block_lengths), max(block_lengths)
    ratio = {k: round(res[lo][k] / res[hi][k], 2) for k in res[hi] if res[hi][k] > 0}
    return {"per_block_length_ms": {str(k): v for k, v in res.items()}, "srhs_over_mrhs": ratio,
            "what": "one refinement iteration; N_b = %d vs N_b = %d" % (lo, hi)}


def fgmres_check(lat, cfg, seed=3005):
    """Two-level FGMRES (FP64 outer, restart 10) on a Gaussian right-hand side to
    relative residual 1e-10 with the context's current setup."""
    b = None
    from paper_1601_03184_gb300 import inputs

    b = inputs.gaussian_field((lat.V, 12), seed)
    t0 = time.perf_counter()
    x, it, rr = lat.solve_fgmres(b, tol=1e-10, restart=10, maxit=300, coarse_tol=SCHEDULE["coarse_tol"],
                                 coarse_restart=SCHEDULE["coarse_restart"], coarse_maxit=SCHEDULE["coarse_maxit"],
                                 n_sweeps=SCHEDULE["smooth_sweeps"], n_mr=SCHEDULE["smooth_mr"], allow_noconv=True)
    return {"iterations": int(it), "relres": float(rr), "seconds": round(time.perf_counter() - t0, 2),
            "tol": 1e-10, "restart": 10}


def run_learned_mixed(args, cfg, U, m0, stream, plain_ms, barrier, dist=None, world=1):
    """Train the network on small seeded lattices of the same roughness and
    csw (16^4, 8 fields x 50 Adam steps on 8 vectors), then time the learned
    initial phase (1 SAP sweep + network) and the refinement with bf16 test
    vectors on the benchmark lattice."""
    import torch

    import paper_1601_03184_gb300 as pkg
    from paper_1601_03184_gb300 import (MRHS_F32, MRHS_PREC_FP32, MRHS_PREC_MIX_BF16, Lattice, inputs, learned)

    t0 = time.perf_counter()
    widths = (4, args.learned_width, args.learned_width, 4) if args.learned_width else learned.WIDTHS
    small = Lattice((16, 16, 16, 16), cfg["agg"], 8, MRHS_PREC_FP32, stream.cuda_stream)
    learned.attach(small, widths, seed=17, noise=0.01, bf16=True)
    sched = dict(init_sweeps=SCHEDULE["init_sweeps"], init_mr=SCHEDULE["init_mr"], n_refine=1,
                 sweeps=SCHEDULE["smooth_sweeps"], mr=SCHEDULE["smooth_mr"], ctol=SCHEDULE["coarse_tol"],
                 crestart=SCHEDULE["coarse_restart"], cmaxit=SCHEDULE["coarse_maxit"])
    step = 1
    losses = []
    for f in range(8):
        small.set_gauge(inputs.gauge_field((16, 16, 16, 16), cfg["eps"], 6000 + f, device="cuda"))
        small.build_clover(m0, cfg["csw"])
        ls = learned.train_on_field(small, sched, 50, seed=6100 + f, lr=3e-3, first_step=step)
        step += len(ls)
        losses += ls
    weights = pkg.mrhs_nn_get_weights(small.ctx, 0)
    small.close()
    train_s = time.perf_counter() - t0
    dims, N = cfg["dims"], cfg["ntv"]
    lat = Lattice(dims, cfg["agg"], N, MRHS_PREC_MIX_BF16, stream.cuda_stream)
    lat.set_coarse_solver(args.coarse_eo)
    lat.set_gauge(U)
    lat.build_clover(m0, cfg["csw"])
    pkg.mrhs_nn_create(lat.ctx, widths, 1)
    pkg.mrhs_nn_set_weights(lat.ctx, weights)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(cfg["tvseed"])
    tv0 = torch.randn(pkg.mrhs_field_bytes(lat.ctx, N, MRHS_F32) // 4, generator=gen, device="cuda",
                      dtype=torch.float32)

    def step_fn():
        pkg.mrhs_setup_init_learned(lat.ctx, tv0, MRHS_F32, 1, SCHEDULE["init_mr"])
        lat.setup_refine(SCHEDULE["n_refine"], SCHEDULE["smooth_sweeps"], SCHEDULE["smooth_mr"],
                         SCHEDULE["coarse_tol"], SCHEDULE["coarse_restart"], SCHEDULE["coarse_maxit"])

    for _ in range(args.warmup):
        step_fn()
    torch.cuda.synchronize()
    barrier()
    pkg.mrhs_profile(lat.ctx, 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step_fn()
    e1.record(stream)
    torch.cuda.synchronize()
    lm_ms = e0.elapsed_time(e1) / args.steps
    prof = pkg.mrhs_profile_read(lat.ctx)
    pkg.mrhs_profile(lat.ctx, 0)
    kernels = {k: {"launches": n // args.steps, "ms_per_step": t / args.steps, "share": t / args.steps / lm_ms}
               for k, (n, t) in prof.items()}
    barrier()
    lm_ms = reduce_max_over_ranks(lm_ms, dist)
    fg = None
    if not args.no_fgmres:
        pkg.mrhs_trim(lat.ctx)
        fg = fgmres_check(lat, cfg)
    lat.close()
    return {"value": whole_job_seconds_per_setup(lm_ms, world), "unit": "s", "ratio_vs_plain": lm_ms / plain_ms,
            "widths": list(widths),
            "form": "1 SAP sweep + network (widths %s, bf16 weights) for the initial phase, bf16 test vectors and P, "
                    "FP32 smoother, D_c contraction on bf16 tensor cores with FP32 accumulation (D_c stored FP32), "
                    "tf32 tensor-core coarse stencil, then the same refinement" % (list(widths),),
            "kernels": kernels,
            "training": {"lattice": [16, 16, 16, 16], "fields": 8, "steps": step - 1, "loss_first": losses[0],
                         "loss_last": losses[-1], "seconds": round(train_s, 1)},
            "fgmres": fg}


def run_e2e(args, lat, U, tv0, cfg, m0, stream, barrier=lambda: None):
    """Setup through the public C ABI from host buffers: gauge field in,
    clover, test vectors packed from host, setup, P and D_c copied out."""
    import torch

    import paper_1601_03184_gb300 as pkg
    from paper_1601_03184_gb300 import MRHS_F32

    N = lat.ntv
    V = lat.V
    nc = 2 * N
    try:
        tv_host = torch.empty((N, V, 12), dtype=torch.complex64, pin_memory=True)
        p_host = torch.empty((N, V, 12), dtype=torch.complex64, pin_memory=True)
        dc_host = torch.empty((lat.nagg, 9, nc, nc), dtype=torch.complex64, pin_memory=True)
        U_host = torch.from_numpy(U).pin_memory()
    except RuntimeError:
        tv_host = torch.empty((N, V, 12), dtype=torch.complex64)
        p_host = torch.empty((N, V, 12), dtype=torch.complex64)
        dc_host = torch.empty((lat.nagg, 9, nc, nc), dtype=torch.complex64)
        U_host = torch.from_numpy(U)
    pkg.mrhs_unpack(lat.ctx, tv0, MRHS_F32, tv_host, MRHS_F32, N)
    dev_tv = tv0  # the device field the host test vectors are packed into

    def step():
        pkg.mrhs_set_gauge(lat.ctx, U_host)
        pkg.mrhs_build_clover(lat.ctx, m0, cfg["csw"])
        pkg.mrhs_pack(lat.ctx, tv_host, MRHS_F32, dev_tv, MRHS_F32, N)
        pkg.mrhs_setup_init(lat.ctx, dev_tv, MRHS_F32, 0, SCHEDULE["init_sweeps"], SCHEDULE["init_mr"])
        lat.setup_refine(SCHEDULE["n_refine"], SCHEDULE["smooth_sweeps"], SCHEDULE["smooth_mr"],
                         SCHEDULE["coarse_tol"], SCHEDULE["coarse_restart"], SCHEDULE["coarse_maxit"])
        pkg.mrhs_get_P(lat.ctx, p_host, MRHS_F32)
        pkg.mrhs_get_Dc(lat.ctx, dc_host, MRHS_F32)

    step()
    torch.cuda.synchronize()
    barrier()
    steps = max(1, min(args.steps, args.e2e_steps))
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    barrier()
    h2d = U.nbytes + tv_host.numel() * 8
    d2h = p_host.numel() * 8 + dc_host.numel() * 8
    return {"value": dt, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "steps": steps, "pinned": bool(tv_host.is_pinned())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=DEFAULT_CONFIG, choices=sorted(CONFIGS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fgmres", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-srhs", action="store_true", help="skip the block-length (N_b) comparison")
    ap.add_argument("--smoother-eo", type=int, default=0, choices=[0, 1],
                    help="1: even-odd preconditioned SAP domain solves")
    ap.add_argument("--coarse-eo", type=int, default=1, choices=[0, 1],
                    help="1 (default): coarse GMRES on the Schur complement of the even aggregates (Sec. 4); "
                         "0: GMRES on D_c")
    ap.add_argument("--dc-engine", type=int, default=0,
                    help="D_c contraction engine of the FP32 setup (mrhs_set_dc_engine; 0 = auto)")
    ap.add_argument("--learned-width", type=int, default=0,
                    help="hidden width of the learned generator (0: the library default)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus if args.gpus else 1))
    if "WORLD_SIZE" not in os.environ:
        world = 1
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    cfg = CONFIGS[args.config]
    m0, m0_src = load_m0(cfg["m0_keys"])
    if args.impl == "reference":
        run_reference(args, cfg, args.config, m0, m0_src, rank, world)
    else:
        run_ours(args, cfg, args.config, m0, m0_src, rank, world, local_rank)


if __name__ == "__main__":
    main()
