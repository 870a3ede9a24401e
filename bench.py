#!/usr/bin/env python3
"""RMTR seconds per load step on the 3D 129^3 four-level workload (20
penny-shaped fractures, pressure ramp p_t = 5e-4 t), plus the Hessian-vector
product's throughput and roofline, on one GB300.

One "step" is one pseudo-time load step: pressure_set + rmtr_load_step (all
of the hot path: energy, gradient, hessvec, projected CG, TR control,
transfers, coarse feasible set, level model, V-cycles).  Inputs are seeded
synthetic fracture networks (no dataset); the state lives in HBM.

  python bench.py [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference      # the FP64 CPU oracle, bounded sample

Multi-GPU: the path does not shard across GPUs here, so N ranks run N
independent replicas (one workload each; no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import pfinputs as PI  # noqa: E402

WORKLOAD = {
    "workload": "3d_129^3_q1_4level_20discs_ramp",
    "dim": 3, "n_coarse": [17, 17, 17], "levels": 4, "h_coarse": 1.0 / 16,
    "E": 1.0, "nu": 0.25, "Gc": 1.0, "ls_over_h": 2.0,
    "fractures": 20, "seed": PI.SEED_3D_PLAIN, "dp": 5e-4,
}
METRIC = "RMTR s/load-step & hessvec GDoF/s: mixed+learned vs FP64 plain, same GB300"

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# roofline kernels on this workload, from one ncu capture of
# `bench.py --kernels-only`; to be re-captured whenever those kernels change.
TRAFFIC_HESSVEC_FP32 = (68.733e6 + 16.743e6) + (47.790e6 + 1.079e6)  # element pass + gather
TRAFFIC_HESSVEC_FP64 = 7595.291e6 + 86.475e6
UNIT = "s/load-step"
# FP32 flops of one element of the 3D FP32 Hessian product (the paired-FMA
# element algebra and its corner sums), from the FP32 instruction counts of
# one ncu capture (FFMA2 x4, FFMA x2, FADD2/FMUL2 x2, FADD/FMUL x1): 6,135 M
# flop over the 144^3 element evaluations of an owner-computes launch.
FLOP32_PER_ELEMENT = 2055
# FP32 peak of one GB300 from its unit counts and clock: 152 SMs x 128 FP32
# lanes x 2 flop (FMA) x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12

# Finest-level-equivalent element passes per load step of the CUDA path on
# this workload (default configuration: mixed precision, extrapolated
# start), measured by this script's GPU arm (printed as "work_model"); they
# scale the oracle's per-pass seconds to seconds per load step for the
# reference arm.
REF_WORK_MODEL = {"fe_hessvec": 228.4, "fe_gradient": 9.18, "fe_energy": 8.17}



def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--start", choices=["plain", "extrapolate"], default="extrapolate",
                    help="starting iterate of each load step (plain = x_{t-1})")
    ap.add_argument("--compare-fp64", action="store_true",
                    help="also time the same K load steps in plain FP64")
    ap.add_argument("--kernels-only", action="store_true",
                    help="set up the workload state, launch the element kernels and exit")
    ap.add_argument("--coarse-n", type=int, default=17,
                    help="coarsest nodes per axis (17 = the 129^3 workload)")
    ap.add_argument("--coarse-model", choices=["first_order", "galerkin"], default="first_order")
    ap.add_argument("--batched", action="store_true",
                    help="the uneven 2D batch (64 instances, 129^2 .. 1025^2) instead of the 3D workload")
    ap.add_argument("--batch-threads", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def rank_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def job_seconds_per_load_step(rank_seconds, dist=None, device="cpu"):
    """Seconds per load step of N replicas (one per rank): each rank times its
    own load steps, the job lasts as long as its slowest rank, and in that
    time the N replicas complete N load steps.  Returns (the slowest rank's
    seconds per step, the whole job's seconds per load step); a collective
    call, made by every rank."""
    if dist is None:
        return rank_seconds, rank_seconds
    import torch
    t = torch.tensor([float(rank_seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    slowest = float(t.item())
    return slowest, slowest / dist.get_world_size()


# ---------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle timing
def oracle_pass_seconds(budget_s=20.0):
    """Seconds per finest-level hessvec / gradient / energy-difference pass of
    the FP64 oracle on the 129^3 workload state (one call each, repeated
    while the budget lasts)."""
    from oracle import pf_oracle as O
    W = WORKLOAD
    H = O.Hierarchy(3, W["n_coarse"], W["h_coarse"], W["levels"],
                    O.Params(E=W["E"], nu=W["nu"], Gc=W["Gc"], p=W["dp"]))
    g = H.fine
    x = np.zeros(4 * g.N)
    x[3 * g.N:] = O.rasterize(g, O.DISC3D, PI.disc_network_3d(W["seed"], W["fractures"]), g.h)
    x[:3 * g.N] = PI.random_direction(5, 3 * g.N, 1e-4)
    v = PI.random_direction(6, x.size, 1e-4)
    times = {"hessvec": [], "gradient": [], "energy": []}
    t_end = time.perf_counter() + budget_s
    while True:
        t = time.perf_counter(); O.hessvec(g, H.prm, x, v); times["hessvec"].append(time.perf_counter() - t)
        t = time.perf_counter(); O.gradient(g, H.prm, x); times["gradient"].append(time.perf_counter() - t)
        t = time.perf_counter(); O.energy_diff(g, H.prm, x, v); times["energy"].append(time.perf_counter() - t)
        if time.perf_counter() > t_end:
            break
    return {k: min(v) for k, v in times.items()}, g


def workload_config(W, args, world):
    """The workload both arms report: grid, sizes, the timed pressures and the
    GPU arm's solver settings."""
    n = [(c - 1) * (1 << (W["levels"] - 1)) + 1 for c in W["n_coarse"]]
    return {"workload": W["workload"], "grid": n, "levels": W["levels"],
            "dofs": (W["dim"] + 1) * int(np.prod(n)), "fractures": W["fractures"],
            "pressure_steps": [W["dp"] * t
                               for t in range(args.warmup + 1, args.warmup + args.steps + 1)],
            "precision": args.precision, "coarse_model": args.coarse_model, "start": args.start,
            "parallelism": f"replicas{world}",
            "l2": "working set > L2 (FP64 vectors 69 MB each, >20 resident)"}


def oracle_seconds_per_load_step(pass_s, work):
    return (pass_s["hessvec"] * work["fe_hessvec"] + pass_s["gradient"] * work["fe_gradient"]
            + pass_s["energy"] * work["fe_energy"])


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return 0
    vals = []
    sample = None
    for _ in range(args.warmup):
        oracle_pass_seconds(budget_s=0.0)
    for _ in range(args.steps):
        pass_s, g = oracle_pass_seconds(budget_s=0.0)
        vals.append(oracle_seconds_per_load_step(pass_s, REF_WORK_MODEL))
        sample = pass_s
    v = statistics.median(vals)
    out = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(WORKLOAD, args, world),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                         "sample": ("one FP64 numpy oracle pass each of hessvec, gradient and energy "
                                    "difference on the full 129^3 state per step, scaled by the CUDA path's "
                                    f"finest-equivalent passes per load step {REF_WORK_MODEL}"),
                         "pass_seconds": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


# ---------------------------------------------------------------- our arm
def kernels_only(pf, B, H, x, W):
    """One launch each of the FP64 hessvec, FP32 hessvec and FP64 gradient
    on the workload state (the launches an ncu capture takes), then their
    event-timed averages."""
    import torch
    pf.pressure_set(H, W["dp"])
    level = W["levels"] - 1
    ndof = H.ndof()
    v = torch.from_numpy(PI.random_direction(77, ndof, 1e-3)).cuda()
    out = torch.empty_like(v)
    x32, v32 = x.float(), v.float()
    o32 = torch.empty_like(v32)
    pf.hessvec_lag_set(H, level, x)
    pf.hessvec_lagged(H, level, v, out)
    pf.hessvec(H, level, x32, v32, o32)
    pf.gradient(H, level, x, out)
    pf.gradient_df(H, level, x, out)
    torch.cuda.synchronize()
    res = {}
    for name, fn in (("hessvec_fp64", lambda: pf.hessvec_lagged(H, level, v, out)),
                     ("hessvec_fp32", lambda: pf.hessvec(H, level, x32, v32, o32)),
                     ("gradient_fp64", lambda: pf.gradient(H, level, x, out)),
                     ("gradient_df", lambda: pf.gradient_df(H, level, x, out)),
                     ("energy_df", lambda: pf.energy_df(H, level, x)),
                     ("gradient_step_fp32", lambda: pf.gradient_step(H, level, x, v, out)),
                     ("energy_diff_mixed", lambda: pf.energy_diff_mixed(H, level, x, v, out)),
                     ("energy_diff_fp64", lambda: pf.energy_diff(H, level, x, v)),
                     ("energy_fp64", lambda: pf.energy(H, level, x))):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(10):
            fn()
        b.record()
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / 10 * 1e-3
        res[name] = {"us": t * 1e6, "gdofs": ndof / t / 1e9}
    print(json.dumps({"kernels": res, "dofs": ndof, "workload": W["workload"]}))
    return 0


def nvtx_range(name):
    """An NVTX range around the timed region (a no-op where torch has no NVTX)."""
    import contextlib
    import torch
    try:
        return torch.cuda.nvtx.range(name)
    except Exception:
        return contextlib.nullcontext()


def run_ours(args):
    import torch
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2007_12908_gb300 import build
    build.build()
    import paper_2007_12908_gb300 as pf
    from paper_2007_12908_gb300 import _binding as B

    W = dict(WORKLOAD)
    if args.coarse_n != 17:
        W["n_coarse"] = [args.coarse_n] * 3
        W["h_coarse"] = 1.0 / (args.coarse_n - 1)
        W["workload"] = f"3d_{8 * (args.coarse_n - 1) + 1}^3_q1_4level_20discs_ramp"
    prm = pf.default_params(
        precision=pf.PF_FP32 if args.precision == "mixed" else pf.PF_FP64,
        coarse_model=pf.PF_GALERKIN if args.coarse_model == "galerkin" else pf.PF_FIRST_ORDER,
        start=pf.PF_START_EXTRAPOLATE if args.start == "extrapolate" else pf.PF_START_PLAIN)
    H = pf.mesh_hierarchy_create(3, W["n_coarse"], W["levels"], W["h_coarse"], E=W["E"],
                                 nu=W["nu"], Gc=W["Gc"], ls_over_h=W["ls_over_h"])
    g_n, g_h, N = H.levels[-1]
    ndof = H.ndof()
    x = torch.zeros(ndof, dtype=torch.float64, device="cuda")
    rows = PI.disc_network_3d(W["seed"], W["fractures"])
    pf.fractures_set(H, pf.PF_DISC3D, rows, g_h, x)
    stream = torch.cuda.current_stream()

    if args.kernels_only:
        return kernels_only(pf, B, H, x, W)

    def load_step(t, xx):
        pf.pressure_set(H, W["dp"] * t)
        return pf.rmtr_load_step(H, xx, prm, check=False)

    for t in range(1, args.warmup + 1):
        st = load_step(t, x)
    x_after_warmup = x.clone()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stats = []
    e0.record(stream)
    with nvtx_range("timed_load_steps"):  # ncu --nvtx-include "timed_load_steps/"
        for t in range(args.warmup + 1, args.warmup + args.steps + 1):
            stats.append(load_step(t, x))
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    slowest_s, job_s = job_seconds_per_load_step(e0.elapsed_time(e1) / args.steps / 1e3, dist,
                                                 "cuda")
    ms = slowest_s * 1e3
    if dist:
        dist.barrier()

    # ---- dominant kernel: Hessian-vector product at the finest level
    v = torch.from_numpy(PI.random_direction(77, ndof, 1e-3)).cuda()
    out = torch.empty_like(v)

    def time_kernel(fn, reps=20):
        for _ in range(3):
            fn()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps * 1e-3

    level = W["levels"] - 1
    pf.hessvec_lag_set(H, level, x)  # the solver's FP64 operator: stored lagged coefficients
    t64 = time_kernel(lambda: pf.hessvec_lagged(H, level, v, out))
    x32, v32 = x.float(), v.float()
    o32 = torch.empty_like(v32)
    t32 = time_kernel(lambda: pf.hessvec(H, level, x32, v32, o32))
    t_grad = time_kernel(lambda: pf.gradient(H, level, x, out))
    fma64 = B.probe_fma(pf.PF_FP64)
    fma32 = B.probe_fma(pf.PF_FP32)
    hbm = None
    try:
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
        hbm_src = "measured"
    except (OSError, KeyError, ValueError):
        hbm, hbm_src = 6800.0, "fallback"
    # FP64 lagged Hessian = the assembled 27-point block stencil: it reads the
    # stencil (27 x 4 x 4 doubles per node) and v, and writes Hv
    bytes64 = (27 * 16 * 8 + 2 * 4 * 8) * N
    bytes32 = 12.0 * ndof
    roof64 = {"kernel": "hessvec_fp64 (assembled stencil apply)", "bound": "hbm",
              "achieved": bytes64 / t64 / 1e9, "peak": hbm, "unit": "GB/s",
              "frac": bytes64 / t64 / 1e9 / hbm, "traffic": TRAFFIC_HESSVEC_FP64,
              "fp64_pipe_active": 0.984,
              "peak_source": f"{hbm_src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
              "flop_per_node": 864, "fp64_fma_peak_tflops": fma64 / 1e12,
              "gdofs": ndof / t64 / 1e9, "us_per_launch": t64 * 1e6}
    # The FP32 product is bound by FP32 issue (FMA pipe ~67 % busy, DRAM ~10 %):
    # ALU roofline, algorithmic flops = FLOP32_PER_ELEMENT x elements
    ne = (g_n[0] - 1) * (g_n[1] - 1) * (g_n[2] - 1)
    flops32 = FLOP32_PER_ELEMENT * ne
    roof32 = {"kernel": "hessvec_fp32", "bound": "alu", "achieved": flops32 / t32 / 1e12,
              "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
              "frac": flops32 / t32 / 1e12 / FP32_PEAK_TFLOPS,
              # dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of
              # the product's two kernels
              "traffic": TRAFFIC_HESSVEC_FP32,
              "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz",
              "fp32_fma_probe_tflops": fma32 / 1e12,
              "flop_per_element": FLOP32_PER_ELEMENT,
              "hbm_achieved_gbs": bytes32 / t32 / 1e9, "hbm_peak_gbs": hbm,
              "gdofs": ndof / t32 / 1e9, "us_per_launch": t32 * 1e6}
    roofline = roof64 if args.precision == "fp64" else roof32

    def with_p_prev(p_src, t):
        """Parameters of timed step t: the first one names the warm-up's last
        pressure so an extrapolated start scales as in the timed run."""
        q = pf.default_params(**{k: getattr(p_src, k) for k, _ in p_src._fields_})
        if t == args.warmup + 1:
            q.p_prev = W["dp"] * args.warmup
        return q

    def compare(p_cmp):
        """The same K timed load steps from the same warmed-up state with
        other parameters."""
        xc = x_after_warmup.clone()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sc = []
        for t in range(args.warmup + 1, args.warmup + args.steps + 1):
            pf.pressure_set(H, W["dp"] * t)
            sc.append(pf.rmtr_load_step(H, xc, with_p_prev(p_cmp, t), check=False))
        b.record(stream)
        torch.cuda.synchronize()
        ec = [s["energy"] for s in sc]
        eh = [s["energy"] for s in stats]
        return {"value": a.elapsed_time(b) / args.steps / 1e3, "unit": UNIT,
                "speedup_of_headline": a.elapsed_time(b) / args.steps / ms,
                "energy_rel_diff": max(abs(p - q) / abs(q) for p, q in zip(eh, ec)),
                "cycles": [s["cycles"] for s in sc], "status": [s["status"] for s in sc]}

    fp64_cmp = mixed_plain = None
    if args.compare_fp64:
        fp64_cmp = compare(pf.default_params(precision=pf.PF_FP64, coarse_model=prm.coarse_model,
                                             start=pf.PF_START_PLAIN))
        if args.precision == "mixed" and args.start != "plain":
            mixed_plain = compare(pf.default_params(precision=pf.PF_FP32, coarse_model=prm.coarse_model,
                                                    start=pf.PF_START_PLAIN))

    # ---- end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        xh = torch.empty(ndof, dtype=torch.float64, pin_memory=True)
        xh.copy_(x_after_warmup.cpu())
        xn = xh.numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for t in range(args.warmup + 1, args.warmup + args.steps + 1):
            pf.pressure_set(H, W["dp"] * t)
            pf.rmtr_load_step_host(H, xn, with_p_prev(prm, t), check=False)
        _, e2e_s = job_seconds_per_load_step((time.perf_counter() - t0) / args.steps, dist, "cuda")
        e2e = {"value": e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * ndof,
               "d2h_bytes_per_step": 8 * ndof}

    work = {k: statistics.mean(s[k] for s in stats) for k in ("fe_hessvec", "fe_gradient", "fe_energy")}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pass_s, _ = oracle_pass_seconds(budget_s=10.0)
        cpu = {"value": oracle_seconds_per_load_step(pass_s, work), "unit": UNIT,
               "cores": cpu_cores(), "kind": "oracle",
               "sample": ("FP64 numpy oracle: one hessvec, gradient and energy-difference pass on the "
                          "full 129^3 state (best of repeats within 10 s), scaled by this run's "
                          "finest-equivalent passes per load step"),
               "pass_seconds": pass_s}

    launches = int(sum(s["launches"] for s in stats))
    value = job_s
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f64+f32",
            "data": "synthetic",
            "config": workload_config(W, args, world),
            "roofline": roofline,
            "roofline_other": roof32 if roofline is roof64 else roof64,
            "hessvec_gdofs": {"fp64": ndof / t64 / 1e9, "fp32": ndof / t32 / 1e9},
            "gradient_fp64_us": t_grad * 1e6,
            "fp64_plain": fp64_cmp,
            "mixed_plain_start": mixed_plain,
            "clocks": clk,
            "e2e": e2e,
            "gpu_launches": launches,
            "cpu_baseline": cpu,
            "work_model": work,
            "solver": {k: [s[k] for s in stats] for k in ("cycles", "converged", "cg", "tr_its",
                                                          "tr_rejected", "coarse_rejected", "status",
                                                          "hv_cauchy", "hv_search", "cg_restarts",
                                                          "fe_hessvec", "fe_gradient", "fe_energy")},
            "solver_levels": {k: [list(s[k])[:W["levels"]] for s in stats]
                              for k in ("cg_level", "tr_level", "rej_level")},
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """Load steps of 64 uneven 2D instances (16 each of 129^2, 257^2, 513^2,
    1025^2 nodes; 10-1000 line fractures, +-30 deg families) run
    concurrently, each on its own stream, by the library's host workers."""
    import torch
    from paper_2007_12908_gb300 import build
    build.build()
    import paper_2007_12908_gb300 as pf
    sizes, counts = PI.batched_grid_draw(PI.SEED_2D_BATCHED, 64)
    prm = pf.default_params(precision=pf.PF_FP32 if args.precision == "mixed" else pf.PF_FP64,
                            start=pf.PF_START_EXTRAPOLATE if args.start == "extrapolate" else pf.PF_START_PLAIN)
    Hs, xs = [], []
    for i, (n, nf) in enumerate(zip(sizes, counts)):
        levels = int(round(np.log2((n - 1) / 16))) + 1
        st = torch.cuda.Stream()
        H = pf.mesh_hierarchy_create(2, (17, 17), levels, 1 / 16, E=1.0, nu=0.3, Gc=1.0, stream=st)
        x = torch.zeros(H.ndof(), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        pf.fractures_set(H, pf.PF_LINE2D, PI.line_network_2d(PI.SEED_2D_BATCHED + 1 + i, nf),
                         H.levels[-1][1], x)
        Hs.append(H)
        xs.append(x)
    dofs = sum(H.ndof() for H in Hs)

    def step(t, threads):
        for H in Hs:
            pf.pressure_set(H, 1e-3 * t)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = pf.rmtr_load_step_batch(Hs, xs, prm, n_threads=threads, check=False)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, out

    for t in range(1, args.warmup + 1):
        step(t, args.batch_threads)
    clocks = Clocks(0)
    clocks.start()
    times, outs = [], []
    for t in range(args.warmup + 1, args.warmup + args.steps + 1):
        dt, out = step(t, args.batch_threads)
        times.append(dt)
        outs.append(out)
    clk = clocks.stop()
    sec = statistics.mean(times)
    line = {
        "metric": "batched RMTR load steps: GDoF/s over 64 uneven 2D instances",
        "value": dofs / sec / 1e9, "unit": "GDoF/s (load steps)", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f64+f32", "data": "synthetic",
        "config": {"workload": "2d_batched_64_uneven_129-1025", "instances": len(Hs), "dofs": dofs,
                   "sizes": sizes, "fractures": counts, "precision": args.precision,
                   "start": args.start, "threads": args.batch_threads or len(Hs)},
        "instances_per_s": len(Hs) / sec,
        "converged": [sum(o["converged"] for o in out) for out in outs],
        "cycles_mean": [statistics.mean(o["cycles"] for o in out) for out in outs],
        "clocks": clk,
    }
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.batched:
        return run_batched(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
